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
    "lts_workspace_bytes", "lts_last_error", "lts_order_field_static", "library_path", "load", "simplify",
    "MODE_MIN", "MODE_MAX", "MODE_BOTH", "ORDER_STATIC_MAX_VERTICES",
]

_HERE = os.path.dirname(os.path.abspath(__file__))
library_path = os.path.join(_HERE, "liblts.so")

MODE_MIN, MODE_MAX, MODE_BOTH = 1, 2, 3
ORDER_STATIC_MAX_VERTICES = 1 << 20   # LTS_ORDER_STATIC_MAX_VERTICES
_MODES = {"min": MODE_MIN, "max": MODE_MAX, "both": MODE_BOTH, 1: 1, 2: 2, 3: 3}
STATUS = {0: "LTS_OK", 1: "LTS_ERR_ARG", 2: "LTS_ERR_NAN", 3: "LTS_ERR_NO_AUTHORIZED", 4: "LTS_ERR_OOM",
          5: "LTS_ERR_CUDA", 6: "LTS_ERR_TIMEOUT", 7: "LTS_ERR_INTERNAL"}


class LtsGrid(ctypes.Structure):
    _fields_ = [("ndim", ctypes.c_int32), ("dims", ctypes.c_int64 * 3)]


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
        lib.lts_last_error.argtypes = [P]
        lib.lts_last_error.restype = ctypes.c_char_p
        lib.lts_destroy.argtypes = [P]
        lib.lts_destroy.restype = None
        lib.lts_order_field_static.argtypes = [ctypes.c_int, ctypes.POINTER(LtsGrid), P, P, P, ctypes.c_char_p,
                                               ctypes.c_size_t]
        lib.lts_order_field_static.restype = ctypes.c_int
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


def lts_last_error(ctx) -> str:
    return load().lts_last_error(ctx).decode()


def lts_destroy(ctx) -> None:
    load().lts_destroy(ctx)


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
        """field: CUDA float32 tensor (Y, X) or (Z, Y, X); authorized: CUDA int32
        tensor of vertex ids.  Returns (g, order, stats dict or None)."""
        import torch

        if field.dtype != torch.float32 or not field.is_cuda or not field.is_contiguous():
            raise ValueError("field must be a contiguous CUDA float32 tensor")
        if authorized.dtype != torch.int32 or not authorized.is_cuda:
            raise ValueError("authorized must be a CUDA int32 tensor")
        authorized = authorized.contiguous()
        grid = grid_of_shape(tuple(field.shape))
        g = out_field if out_field is not None else torch.empty_like(field)
        o = out_order if out_order is not None else torch.empty(field.shape, dtype=torch.int32, device=field.device)
        st = LtsStats() if with_stats else None
        code = lts_simplify(self._ctx, grid, field.data_ptr(), authorized.data_ptr() if authorized.numel() else 0,
                            authorized.numel(), mode, g.data_ptr(), o.data_ptr(), st)
        if code != 0:
            raise LtsError(code, lts_last_error(self._ctx))
        return g, o, (st.as_dict() if st is not None else None)


def simplify(field, authorized, mode="both"):
    """One-shot: creates a context sized for this field, simplifies, frees it."""
    ctx = Context(field.numel(), device=field.device.index)
    try:
        return ctx.simplify(field, authorized, mode)
    finally:
        ctx.close()
