"""GB300 library for Localized Topological Simplification (LTS).

Thin ctypes binding over ``liblts.so`` (declared in ``include/lts.h``): the
names mirror the C ABI (``lts_create``, ``lts_simplify``, ``lts_destroy``,
``lts_workspace_bytes``, ``lts_last_error``).  Arguments are marshalled here
and every step of the method runs in the library's CUDA kernels; PyTorch is
used only for device memory and streams.  There is no fallback: if the
library is missing, importing the binding raises.
"""
from __future__ import annotations

import ctypes
import os

__all__ = [
    "LtsGrid", "LtsStats", "LtsError", "Context", "lts_create", "lts_simplify", "lts_destroy",
    "lts_workspace_bytes", "lts_last_error", "lts_order_field_static", "lts_simplify_batch", "lts_submit",
    "lts_poll", "lts_simplify_persistence", "lts_simplify_f64", "lts_classify", "lts_serve_config", "library_path",
    "LtsTuning", "lts_set_tuning", "lts_get_tuning",
    "load", "simplify",
    "simplify_persistence",
    "MODE_MIN", "MODE_MAX", "MODE_BOTH", "ORDER_STATIC_MAX_VERTICES",
]

_HERE = os.path.dirname(os.path.abspath(__file__))
library_path = os.path.join(_HERE, "liblts.so")

MODE_MIN, MODE_MAX, MODE_BOTH = 1, 2, 3
ORDER_STATIC_MAX_VERTICES = 1 << 20   # LTS_ORDER_STATIC_MAX_VERTICES
MODE_RESTORE = 4   # LTS_MODE_RESTORE, or-ed into a mode
_MODES = {"min": MODE_MIN, "max": MODE_MAX, "both": MODE_BOTH, 1: 1, 2: 2, 3: 3,
          "min+restore": MODE_MIN | MODE_RESTORE, "max+restore": MODE_MAX | MODE_RESTORE,
          "both+restore": MODE_BOTH | MODE_RESTORE, 5: 5, 6: 6, 7: 7}
STATUS = {0: "LTS_OK", 1: "LTS_ERR_ARG", 2: "LTS_ERR_NAN", 3: "LTS_ERR_NO_AUTHORIZED", 4: "LTS_ERR_OOM",
          5: "LTS_ERR_CUDA", 6: "LTS_ERR_TIMEOUT", 7: "LTS_ERR_INTERNAL"}


class LtsGrid(ctypes.Structure):
    _fields_ = [("ndim", ctypes.c_int32), ("dims", ctypes.c_int64 * 3)]


class LtsTuning(ctypes.Structure):
    _fields_ = [("engine_blocks_per_sm", ctypes.c_int32), ("team_blocks_per_sm", ctypes.c_int32),
                ("batch_workspaces", ctypes.c_int32), ("reserved", ctypes.c_int32 * 5)]

    def as_dict(self):
        return {"engine_blocks_per_sm": self.engine_blocks_per_sm, "team_blocks_per_sm": self.team_blocks_per_sm,
                "batch_workspaces": self.batch_workspaces}


class LtsStats(ctypes.Structure):
    _fields_ = [
        ("n_vertices", ctypes.c_int64),
        ("removed", ctypes.c_int64 * 2),
        ("regions", ctypes.c_int64 * 2),
        ("region_vertices", ctypes.c_int64 * 2),
        ("max_region", ctypes.c_int64 * 2),
        ("max_local_floods", ctypes.c_int32 * 2),
        ("total_local_floods", ctypes.c_int64 * 2),
        ("heap_spills", ctypes.c_int64 * 2),
        ("stage_us", ctypes.c_float * 8),
        ("kernel_launches", ctypes.c_int64),
        ("fallback_regions", ctypes.c_int64 * 2),
        ("restored", ctypes.c_int64 * 2),
    ]

    def as_dict(self):
        return {
            "n_vertices": self.n_vertices,
            "removed": list(self.removed), "regions": list(self.regions),
            "region_vertices": list(self.region_vertices), "max_region": list(self.max_region),
            "max_local_floods": list(self.max_local_floods),
            "total_local_floods": list(self.total_local_floods),
            "heap_spills": list(self.heap_spills),
            "launches": int(self.kernel_launches),
            "fallback_regions": list(self.fallback_regions),
            "restored": list(self.restored),
            "stage_us": {k: round(float(v), 2) for k, v in zip(
                ["order_field", "classify", "propagate", "regions", "local_order", "reorder", "total"],
                list(self.stage_us)[:7])},
        }


class LtsError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code


_lib = None


def load():
    """Loads liblts.so; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(library_path):
            raise RuntimeError(f"liblts.so is missing at {library_path}: build it with "
                               "`python -c 'import __graft_entry__ as g; g.build()'`")
        lib = ctypes.CDLL(library_path)
        P = ctypes.c_void_p
        lib.lts_create.argtypes = [ctypes.POINTER(P), ctypes.c_int, ctypes.c_int64, P]
        lib.lts_create.restype = ctypes.c_int
        lib.lts_workspace_bytes.argtypes = [ctypes.POINTER(LtsGrid)]
        lib.lts_workspace_bytes.restype = ctypes.c_size_t
        lib.lts_simplify.argtypes = [P, ctypes.POINTER(LtsGrid), P, P, ctypes.c_int64, ctypes.c_int, P, P,
                                     ctypes.POINTER(LtsStats)]
        lib.lts_simplify.restype = ctypes.c_int
        lib.lts_classify.argtypes = [P, ctypes.POINTER(LtsGrid), P, P, P, ctypes.POINTER(ctypes.c_int64)]
        lib.lts_classify.restype = ctypes.c_int
        lib.lts_simplify_f64.argtypes = [P, ctypes.POINTER(LtsGrid), P, P, ctypes.c_int64, ctypes.c_int, P, P,
                                         ctypes.POINTER(LtsStats)]
        lib.lts_simplify_f64.restype = ctypes.c_int
        lib.lts_simplify_persistence.argtypes = [P, ctypes.POINTER(LtsGrid), P, ctypes.c_double, ctypes.c_int, P, P,
                                                 ctypes.POINTER(LtsStats)]
        lib.lts_simplify_persistence.restype = ctypes.c_int
        lib.lts_last_error.argtypes = [P]
        lib.lts_last_error.restype = ctypes.c_char_p
        lib.lts_destroy.argtypes = [P]
        lib.lts_destroy.restype = None
        lib.lts_order_field_static.argtypes = [ctypes.c_int, ctypes.POINTER(LtsGrid), P, P, P, ctypes.c_char_p,
                                               ctypes.c_size_t]
        lib.lts_order_field_static.restype = ctypes.c_int
        PP = ctypes.POINTER(P)
        lib.lts_simplify_batch.argtypes = [P, ctypes.c_int32, ctypes.POINTER(LtsGrid), PP, PP,
                                           ctypes.POINTER(ctypes.c_int64), ctypes.c_int, PP, PP,
                                           ctypes.POINTER(LtsStats)]
        lib.lts_simplify_batch.restype = ctypes.c_int
        lib.lts_submit.argtypes = [P, ctypes.POINTER(LtsGrid), P, P, ctypes.c_int64, ctypes.c_int, P, P,
                                   ctypes.POINTER(ctypes.c_uint64)]
        lib.lts_submit.restype = ctypes.c_int
        lib.lts_poll.argtypes = [P, ctypes.c_uint64, ctypes.POINTER(ctypes.c_int)]
        lib.lts_poll.restype = ctypes.c_int
        lib.lts_serve_config.argtypes = [P, ctypes.c_int32, ctypes.c_int64]
        lib.lts_serve_config.restype = ctypes.c_int
        lib.lts_set_tuning.argtypes = [P, ctypes.POINTER(LtsTuning)]
        lib.lts_set_tuning.restype = ctypes.c_int
        lib.lts_get_tuning.argtypes = [P, ctypes.POINTER(LtsTuning)]
        lib.lts_get_tuning.restype = ctypes.c_int
        _lib = lib
    return _lib


def grid_of_shape(shape):
    """LtsGrid for a C-ordered (Z, Y, X) or (Y, X) field shape."""
    g = LtsGrid()
    if len(shape) == 2:
        g.ndim = 2
        g.dims[0], g.dims[1], g.dims[2] = shape[1], shape[0], 1
    elif len(shape) == 3:
        g.ndim = 3
        g.dims[0], g.dims[1], g.dims[2] = shape[2], shape[1], shape[0]
    else:
        raise ValueError("field must be 2D or 3D")
    return g


# ---- the C ABI, one Python function per entry point ----

def lts_create(device: int, max_vertices: int, cuda_stream: int = 0):
    ctx = ctypes.c_void_p()
    code = load().lts_create(ctypes.byref(ctx), int(device), int(max_vertices), ctypes.c_void_p(cuda_stream))
    if code != 0:
        raise LtsError(code, "lts_create failed")
    return ctx


def lts_workspace_bytes(grid: LtsGrid) -> int:
    return int(load().lts_workspace_bytes(ctypes.byref(grid)))


def lts_simplify(ctx, grid: LtsGrid, d_field: int, d_authorized: int, n_authorized: int, mode,
                 d_out_field: int, d_out_order: int, stats: LtsStats | None = None) -> int:
    return load().lts_simplify(ctx, ctypes.byref(grid), ctypes.c_void_p(d_field), ctypes.c_void_p(d_authorized),
                               int(n_authorized), _MODES[mode], ctypes.c_void_p(d_out_field),
                               ctypes.c_void_p(d_out_order), ctypes.byref(stats) if stats is not None else None)


def lts_classify(ctx, grid: LtsGrid, d_order: int, d_lower: int = 0, d_upper: int = 0):
    """Returns (status, counts): minima, maxima, regular, saddles, join and
    split saddle multiplicities."""
    counts = (ctypes.c_int64 * 6)()
    code = load().lts_classify(ctx, ctypes.byref(grid), ctypes.c_void_p(d_order), ctypes.c_void_p(d_lower or None),
                               ctypes.c_void_p(d_upper or None), counts)
    return int(code), list(counts)


def lts_simplify_f64(ctx, grid: LtsGrid, d_field: int, d_authorized: int, n_authorized: int, mode,
                     d_out_field: int, d_out_order: int, stats: LtsStats | None = None) -> int:
    return load().lts_simplify_f64(ctx, ctypes.byref(grid), ctypes.c_void_p(d_field), ctypes.c_void_p(d_authorized),
                                   int(n_authorized), _MODES[mode], ctypes.c_void_p(d_out_field),
                                   ctypes.c_void_p(d_out_order), ctypes.byref(stats) if stats is not None else None)


def lts_simplify_persistence(ctx, grid: LtsGrid, d_field: int, epsilon: float, mode, d_out_field: int,
                             d_out_order: int, stats: LtsStats | None = None) -> int:
    return load().lts_simplify_persistence(ctx, ctypes.byref(grid), ctypes.c_void_p(d_field), float(epsilon),
                                           _MODES[mode], ctypes.c_void_p(d_out_field), ctypes.c_void_p(d_out_order),
                                           ctypes.byref(stats) if stats is not None else None)


def lts_last_error(ctx) -> str:
    return load().lts_last_error(ctx).decode()


def lts_destroy(ctx) -> None:
    load().lts_destroy(ctx)


def lts_simplify_batch(ctx, grids, d_fields, d_authorized, n_authorized, mode, d_out_fields, d_out_orders,
                       stats=None) -> int:
    """grids: list of LtsGrid; the others: lists of device addresses / counts (one per field);
    stats: a ctypes array of LtsStats of the same length, or None."""
    nf = len(grids)
    P = ctypes.c_void_p
    ga = (LtsGrid * max(nf, 1))(*grids)
    arr = lambda xs: (P * max(nf, 1))(*[P(x) for x in xs])
    na = (ctypes.c_int64 * max(nf, 1))(*[int(x) for x in n_authorized])
    return load().lts_simplify_batch(ctx, nf, ga, arr(d_fields), arr(d_authorized), na, _MODES[mode],
                                     arr(d_out_fields), arr(d_out_orders), stats)


def lts_submit(ctx, grid: LtsGrid, d_field: int, d_authorized: int, n_authorized: int, mode, d_out_field: int,
               d_out_order: int):
    """Returns (status, ticket)."""
    t = ctypes.c_uint64(0)
    code = load().lts_submit(ctx, ctypes.byref(grid), ctypes.c_void_p(d_field), ctypes.c_void_p(d_authorized),
                             int(n_authorized), _MODES[mode], ctypes.c_void_p(d_out_field),
                             ctypes.c_void_p(d_out_order), ctypes.byref(t))
    return int(code), int(t.value)


def lts_poll(ctx, ticket: int):
    """Returns (status, done)."""
    d = ctypes.c_int(0)
    code = load().lts_poll(ctx, ctypes.c_uint64(ticket), ctypes.byref(d))
    return int(code), bool(d.value)


def lts_serve_config(ctx, max_concurrent: int, hbm_budget_bytes: int) -> int:
    return load().lts_serve_config(ctx, int(max_concurrent), int(hbm_budget_bytes))


def lts_set_tuning(ctx, tuning: dict | None) -> int:
    """Sets the context's launch tuning from a dict of LtsTuning fields (None: defaults)."""
    if tuning is None:
        return load().lts_set_tuning(ctx, None)
    t = LtsTuning()
    for k, v in tuning.items():
        if k not in ("engine_blocks_per_sm", "team_blocks_per_sm", "batch_workspaces"):
            raise KeyError(k)
        setattr(t, k, int(v))
    return load().lts_set_tuning(ctx, ctypes.byref(t))


def lts_get_tuning(ctx) -> dict:
    t = LtsTuning()
    code = load().lts_get_tuning(ctx, ctypes.byref(t))
    if code != 0:
        raise LtsError(code, "lts_get_tuning")
    return t.as_dict()


def lts_order_field_static(device: int, grid: LtsGrid, d_field: int, d_order: int, cuda_stream: int = 0):
    """Order field with the library's static scratch (no allocation); returns (status, message)."""
    buf = ctypes.create_string_buffer(256)
    code = load().lts_order_field_static(int(device), ctypes.byref(grid), ctypes.c_void_p(d_field),
                                         ctypes.c_void_p(d_order), ctypes.c_void_p(cuda_stream), buf, len(buf))
    return int(code), buf.value.decode()


# ---- convenience wrapper over torch tensors ----

class Context:
    """Owns an lts_ctx bound to a device and a CUDA stream."""

    def __init__(self, max_vertices: int, device=None, stream=None):
        import torch

        self.device = torch.device("cuda", torch.cuda.current_device() if device is None else device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self.max_vertices = int(max_vertices)
        self._ctx = lts_create(self.device.index, self.max_vertices, self.stream.cuda_stream)

    def close(self):
        if getattr(self, "_ctx", None) is not None:
            lts_destroy(self._ctx)
            self._ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def simplify(self, field, authorized, mode="both", out_field=None, out_order=None, with_stats=True):
        """field: CUDA float32 or float64 tensor (Y, X) or (Z, Y, X);
        authorized: CUDA int32 tensor of vertex ids.  Returns (g, order, stats
        dict or None); g has the field's dtype."""
        import torch

        if field.dtype not in (torch.float32, torch.float64) or not field.is_cuda or not field.is_contiguous():
            raise ValueError("field must be a contiguous CUDA float32 or float64 tensor")
        if authorized.dtype != torch.int32 or not authorized.is_cuda:
            raise ValueError("authorized must be a CUDA int32 tensor")
        authorized = authorized.contiguous()
        grid = grid_of_shape(tuple(field.shape))
        g = out_field if out_field is not None else torch.empty_like(field)
        o = out_order if out_order is not None else torch.empty(field.shape, dtype=torch.int32, device=field.device)
        st = LtsStats() if with_stats else None
        call = lts_simplify_f64 if field.dtype == torch.float64 else lts_simplify
        code = call(self._ctx, grid, field.data_ptr(), authorized.data_ptr() if authorized.numel() else 0,
                    authorized.numel(), mode, g.data_ptr(), o.data_ptr(), st)
        if code != 0:
            raise LtsError(code, lts_last_error(self._ctx))
        return g, o, (st.as_dict() if st is not None else None)

    def simplify_persistence(self, field, epsilon, mode="both", out_field=None, out_order=None, with_stats=True):
        """Persistence-driven simplification (Sec. 4.5): removes the extrema
        whose persistence is at most epsilon.  Returns (g, order, stats or None)."""
        import torch

        if field.dtype != torch.float32 or not field.is_cuda or not field.is_contiguous():
            raise ValueError("field must be a contiguous CUDA float32 tensor")
        grid = grid_of_shape(tuple(field.shape))
        g = out_field if out_field is not None else torch.empty_like(field)
        o = out_order if out_order is not None else torch.empty(field.shape, dtype=torch.int32, device=field.device)
        st = LtsStats() if with_stats else None
        code = lts_simplify_persistence(self._ctx, grid, field.data_ptr(), epsilon, mode, g.data_ptr(), o.data_ptr(),
                                        st)
        if code != 0:
            raise LtsError(code, lts_last_error(self._ctx))
        return g, o, (st.as_dict() if st is not None else None)

    def simplify_batch(self, fields, authorized, mode="both", with_stats=True):
        """fields: list of CUDA float32 tensors; authorized: list of CUDA int32
        tensors.  Returns (list of (g, order), list of stats dicts or None)."""
        import torch

        if len(fields) != len(authorized):
            raise ValueError("one authorized list per field")
        outs, grids = [], []
        auth = [a.contiguous() for a in authorized]
        for f in fields:
            if f.dtype != torch.float32 or not f.is_cuda or not f.is_contiguous():
                raise ValueError("fields must be contiguous CUDA float32 tensors")
            grids.append(grid_of_shape(tuple(f.shape)))
            outs.append((torch.empty_like(f), torch.empty(f.shape, dtype=torch.int32, device=f.device)))
        st = (LtsStats * max(len(fields), 1))() if with_stats else None
        code = lts_simplify_batch(self._ctx, grids, [f.data_ptr() for f in fields],
                                  [a.data_ptr() if a.numel() else 0 for a in auth], [a.numel() for a in auth], mode,
                                  [o[0].data_ptr() for o in outs], [o[1].data_ptr() for o in outs], st)
        if code != 0:
            raise LtsError(code, lts_last_error(self._ctx))
        return outs, ([st[i].as_dict() for i in range(len(fields))] if st is not None else None)

    def set_tuning(self, tuning: dict | None = None):
        """Launch tuning (see lts_set_tuning); None restores the defaults."""
        code = lts_set_tuning(self._ctx, tuning)
        if code != 0:
            raise LtsError(code, lts_last_error(self._ctx))

    def tuning(self) -> dict:
        return lts_get_tuning(self._ctx)

    def serve_config(self, max_concurrent: int, hbm_budget_bytes: int = 120 << 30):
        code = lts_serve_config(self._ctx, max_concurrent, hbm_budget_bytes)
        if code != 0:
            raise LtsError(code, lts_last_error(self._ctx))

    def submit(self, field, authorized, mode="both"):
        """Queues a simplification; returns a ticket.  The tensors are kept
        alive until the ticket is polled done."""
        import torch

        if field.dtype != torch.float32 or not field.is_cuda or not field.is_contiguous():
            raise ValueError("field must be a contiguous CUDA float32 tensor")
        authorized = authorized.contiguous()
        g = torch.empty_like(field)
        o = torch.empty(field.shape, dtype=torch.int32, device=field.device)
        code, t = lts_submit(self._ctx, grid_of_shape(tuple(field.shape)), field.data_ptr(),
                             authorized.data_ptr() if authorized.numel() else 0, authorized.numel(), mode,
                             g.data_ptr(), o.data_ptr())
        if code != 0:
            raise LtsError(code, lts_last_error(self._ctx))
        if not hasattr(self, "_pending"):
            self._pending = {}
        self._pending[t] = (field, authorized, g, o)
        return t

    def poll(self, ticket):
        """None while the request runs; (g, order) once it is done; raises
        LtsError if it failed."""
        code, done = lts_poll(self._ctx, ticket)
        if not done:
            if code != 0:
                raise LtsError(code, lts_last_error(self._ctx))
            return None
        _, _, g, o = getattr(self, "_pending", {}).pop(ticket, (None, None, None, None))
        if code != 0:
            raise LtsError(code, lts_last_error(self._ctx))
        return g, o


def simplify(field, authorized, mode="both"):
    """One-shot: creates a context sized for this field, simplifies, frees it."""
    ctx = Context(field.numel(), device=field.device.index)
    try:
        return ctx.simplify(field, authorized, mode)
    finally:
        ctx.close()


def simplify_persistence(field, epsilon, mode="both"):
    """One-shot persistence-driven simplification (Sec. 4.5)."""
    ctx = Context(field.numel(), device=field.device.index)
    try:
        return ctx.simplify_persistence(field, epsilon, mode)
    finally:
        ctx.close()
