// C ABI of the library (include/lts.h): context and workspace management,
// argument checks, and the sequence of stages of one simplification.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <string>

#include "lts_internal.cuh"

namespace lts {
int propagate_lanes(int sms);
long long propagate_log_slack(int lanes);
long long propagate_spill_slack(int lanes);
long long propagate_heap_slack(int lanes);
int scan_tiles_for(long long max_count);
}  // namespace lts

using namespace lts;

struct lts_ctx {
    int device = 0;
    int sms = 0;
    cudaStream_t stream = nullptr;
    Work w{};
    bool dirty = false;          // workspace may hold state of an aborted call
    std::string err;
    cudaEvent_t ev[16];
    bool events = false;
    void* allocs[64];
    int nallocs = 0;
};

namespace {

struct Sizes {
    long long n, half, lanes, tiles, log_cap, spill_cap, heap_cap, lo_cap, nblk, scan_tiles;
};

Sizes sizes_for(long long n, int sms) {
    Sizes z;
    z.n = n;
    z.half = n / 2 + 1;
    z.lanes = propagate_lanes(sms);
    z.tiles = (n + 4095) / 4096;
    z.log_cap = n + z.half + propagate_log_slack((int)z.lanes);
    z.spill_cap = std::min<long long>(4 * n + propagate_spill_slack((int)z.lanes), (1LL << 31) - 1);
    z.heap_cap = 2 * n + propagate_heap_slack((int)z.lanes);
    z.lo_cap = n + z.half;
    z.nblk = (n + 31) / 32;
    z.scan_tiles = std::max<long long>(scan_tiles_for(z.half + 1), (z.nblk + 4095) / 4096 + 1);
    return z;
}

size_t bytes_for(const Sizes& z) {
    size_t b = 0;
    b += 4 * 4 * (size_t)z.n;                       // sort key/value double buffers
    b += (size_t)z.tiles * 256 * 8 + 4096 * 3;      // look-back words, histograms
    b += ((size_t)z.n + 31) / 32 * 4;               // authorized bitmap
    b += 2 * 4 * (size_t)z.n + 8 * (size_t)z.n;     // owner, loc, qmark
    b += 8 * 4 * (size_t)z.half;                    // U and class records
    b += 16 * (size_t)z.half;                       // task records
    b += 4 * (size_t)z.n;                           // saddle arrival counters
    b += 4 * (size_t)z.spill_cap + 8 * (size_t)z.heap_cap + 4 * (size_t)z.log_cap;
    b += 11 * 4 * (size_t)z.half;                   // region records
    b += 2 * 4 * (size_t)z.n;                       // members, lhat
    b += 17 * (size_t)z.lo_cap;                     // local-order scratch
    b += sizeof(RankBlk) * (size_t)z.nblk + 2 * 4 * (size_t)z.half;
    b += 8 * (size_t)z.scan_tiles + sizeof(DevCounters) + 2 * sizeof(PassStats);
    return b;
}

template <typename T>
bool dev_alloc(lts_ctx* c, T** p, size_t count) {
    void* q = nullptr;
    if (cudaMalloc(&q, std::max<size_t>(count, 1) * sizeof(T)) != cudaSuccess) return false;
    c->allocs[c->nallocs++] = q;
    *p = static_cast<T*>(q);
    return true;
}

void free_all(lts_ctx* c) {
    for (int i = 0; i < c->nallocs; ++i) cudaFree(c->allocs[i]);
    c->nallocs = 0;
    if (c->w.h_ctr) cudaFreeHost(c->w.h_ctr);
    c->w.h_ctr = nullptr;
    if (c->events)
        for (auto& e : c->ev) cudaEventDestroy(e);
    c->events = false;
}

bool grid_ok(const lts_grid* g, long long* n_out) {
    if (!g || (g->ndim != 2 && g->ndim != 3)) return false;
    if (g->dims[0] < 2 || g->dims[1] < 2) return false;
    if (g->ndim == 3 && g->dims[2] < 2) return false;
    if (g->ndim == 2 && g->dims[2] != 1) return false;
    long long n = g->dims[0] * g->dims[1] * g->dims[2];
    if (g->dims[0] >= (1LL << 31) || g->dims[1] >= (1LL << 31) || g->dims[2] >= (1LL << 31)) return false;
    if (n >= (1LL << 31) || n < 4) return false;
    *n_out = n;
    return true;
}

lts_status fail(lts_ctx* c, lts_status s, const char* msg) {
    c->err = msg;
    return s;
}

lts_status cuda_fail(lts_ctx* c, cudaError_t e, const char* where) {
    c->err = std::string(where) + ": " + cudaGetErrorString(e);
    c->dirty = true;
    return LTS_ERR_CUDA;
}

// reset the per-vertex state after an aborted call
cudaError_t clean_workspace(lts_ctx* c) {
    Work& w = c->w;
    cudaMemsetAsync(w.owner, 0xff, sizeof(int) * (size_t)w.nmax, c->stream);
    cudaMemsetAsync(w.cnt, 0, sizeof(int) * (size_t)w.nmax, c->stream);
    cudaMemsetAsync(w.sort_status, 0, (size_t)w.max_tiles * 256 * sizeof(unsigned long long), c->stream);
    w.epoch = 0;
    return cudaGetLastError();
}

}  // namespace

namespace lts {
cudaError_t pass_reset(Work& w, cudaStream_t s) {
    // every counter but the status word
    cudaMemsetAsync(reinterpret_cast<char*>(w.ctr) + sizeof(int), 0, sizeof(DevCounters) - sizeof(int), s);
    cudaMemsetAsync(w.rblk, 0, sizeof(RankBlk) * (size_t)w.nblk_cur, s);
    return cudaGetLastError();
}

namespace {
__global__ void save_pass_kernel(const DevCounters* ctr, const int* reg_start, PassStats* ps) {
    ps->removed = ctr->n_unauth;
    ps->regions = ctr->n_regions;
    ps->region_vertices = ctr->n_regions > 0 ? reg_start[ctr->n_regions] : 0;
    ps->max_region = ctr->max_region;
    ps->max_floods = ctr->max_floods;
    ps->total_floods = ctr->total_floods;
    ps->heap_spills = ctr->heap_spills;
}
}  // namespace
}  // namespace lts

extern "C" {

size_t lts_workspace_bytes(const lts_grid* g) {
    long long n;
    if (!grid_ok(g, &n)) return 0;
    int dev = 0, sms = 152;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return bytes_for(sizes_for(n, sms));
}

lts_status lts_create(lts_ctx** out, int device, int64_t max_vertices, void* cuda_stream) {
    if (!out || max_vertices < 4 || max_vertices >= (1LL << 31)) return LTS_ERR_ARG;
    *out = nullptr;
    if (cudaSetDevice(device) != cudaSuccess) return LTS_ERR_CUDA;
    lts_ctx* c = new lts_ctx();
    c->device = device;
    c->stream = static_cast<cudaStream_t>(cuda_stream);
    cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, device);
    const Sizes z = sizes_for(max_vertices, c->sms);
    Work& w = c->w;
    w.nmax = (int)max_vertices;
    w.max_tiles = (int)z.tiles;
    w.lanes = (int)z.lanes;
    w.class_cap = (int)z.half;
    w.log_cap = z.log_cap; w.spill_cap = z.spill_cap; w.heap_cap = z.heap_cap; w.lo_cap = z.lo_cap;
    w.nblk = (int)z.nblk;
    w.scan_tmp_cap = (int)z.scan_tiles;
    bool ok = true;
    ok = ok && dev_alloc(c, &w.keyA, z.n) && dev_alloc(c, &w.valA, z.n) && dev_alloc(c, &w.keyB, z.n) &&
         dev_alloc(c, &w.valB, z.n);
    ok = ok && dev_alloc(c, &w.sort_status, (size_t)z.tiles * 256) && dev_alloc(c, &w.sort_hist, 1024) &&
         dev_alloc(c, &w.sort_offsets, 1024) && dev_alloc(c, &w.tile_counter, 4) &&
         dev_alloc(c, &w.bin_cursor, 1024);
    ok = ok && dev_alloc(c, &w.authbits, (z.n + 31) / 32);
    ok = ok && dev_alloc(c, &w.owner, z.n) && dev_alloc(c, &w.loc, z.n) && dev_alloc(c, &w.qmark, z.n);
    ok = ok && dev_alloc(c, &w.U, z.half) && dev_alloc(c, &w.parent, z.half) && dev_alloc(c, &w.wait_v, z.half) &&
         dev_alloc(c, &w.cnt, z.n) && dev_alloc(c, &w.tasks, z.half) &&
         dev_alloc(c, &w.sib_head, z.half) && dev_alloc(c, &w.sib_next, z.half) &&
         dev_alloc(c, &w.spill_base, z.half) && dev_alloc(c, &w.spill_n, z.half);
    ok = ok && dev_alloc(c, &w.spill_pool, z.spill_cap) && dev_alloc(c, &w.heap_pool, z.heap_cap) &&
         dev_alloc(c, &w.vlog, z.log_cap);
    ok = ok && dev_alloc(c, &w.class2reg, z.half) && dev_alloc(c, &w.reg_class, z.half) &&
         dev_alloc(c, &w.reg_saddle, z.half) && dev_alloc(c, &w.reg_size, z.half) &&
         dev_alloc(c, &w.reg_start, z.half + 1) && dev_alloc(c, &w.reg_top, z.half) &&
         dev_alloc(c, &w.reg_sod, z.half) && dev_alloc(c, &w.reg_place, z.half) && dev_alloc(c, &w.reg_head, z.half) &&
         dev_alloc(c, &w.reg_att, z.half) && dev_alloc(c, &w.reg_floods, z.half);
    ok = ok && dev_alloc(c, &w.members, z.n) && dev_alloc(c, &w.lhat, z.n) && dev_alloc(c, &w.tier_list, 2 * z.half) &&
         dev_alloc(c, &w.member_reg, z.n);
    ok = ok && dev_alloc(c, &w.lo_v, z.lo_cap) && dev_alloc(c, &w.lo_L, z.lo_cap) && dev_alloc(c, &w.lo_L2, z.lo_cap) &&
         dev_alloc(c, &w.lo_heap, z.lo_cap) && dev_alloc(c, &w.lo_flag, z.lo_cap);
    ok = ok && dev_alloc(c, &w.rblk, z.nblk) && dev_alloc(c, &w.sad_att, z.half) && dev_alloc(c, &w.cumA, z.half + 1);
    ok = ok && dev_alloc(c, &w.scan_tmp, z.scan_tiles) && dev_alloc(c, &w.ctr, 1) && dev_alloc(c, &w.pstats, 2);
    if (ok && cudaMallocHost((void**)&w.h_ctr, sizeof(DevCounters) + 2 * sizeof(PassStats)) != cudaSuccess) ok = false;
    if (!ok) {
        cudaGetLastError();
        free_all(c);
        delete c;
        return LTS_ERR_OOM;
    }
    for (auto& e : c->ev) cudaEventCreate(&e);
    c->events = true;
    cudaMemsetAsync(w.owner, 0xff, sizeof(int) * (size_t)z.n, c->stream);
    cudaMemsetAsync(w.cnt, 0, sizeof(int) * (size_t)z.n, c->stream);
    cudaMemsetAsync(w.sort_status, 0, (size_t)z.tiles * 256 * sizeof(unsigned long long), c->stream);
    cudaMemsetAsync(w.qmark, 0, sizeof(unsigned long long) * (size_t)z.n, c->stream);
    w.pass_tag = 0;
    cudaMemsetAsync(w.ctr, 0, sizeof(DevCounters), c->stream);
    w.epoch = 0;
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) {
        free_all(c);
        delete c;
        return LTS_ERR_CUDA;
    }
    *out = c;
    return LTS_OK;
}

void lts_destroy(lts_ctx* c) {
    if (!c) return;
    cudaSetDevice(c->device);
    cudaStreamSynchronize(c->stream);
    free_all(c);
    delete c;
}

const char* lts_last_error(const lts_ctx* c) { return c ? c->err.c_str() : "null context"; }

static bool overlap(const void* a, size_t na, const void* b, size_t nb) {
    const char* x = static_cast<const char*>(a);
    const char* y = static_cast<const char*>(b);
    return x < y + nb && y < x + na;
}

lts_status lts_simplify(lts_ctx* c, const lts_grid* gr, const float* d_field, const int32_t* d_authorized,
                        int64_t n_authorized, lts_mode mode, float* d_out_field, int32_t* d_out_order,
                        lts_stats* opt_stats) {
    if (!c) return LTS_ERR_ARG;
    c->err.clear();
    long long n;
    if (!grid_ok(gr, &n)) return fail(c, LTS_ERR_ARG, "invalid grid");
    if (n > c->w.nmax) return fail(c, LTS_ERR_ARG, "grid larger than the context's max_vertices");
    if (mode < LTS_MODE_MIN || mode > LTS_MODE_BOTH) return fail(c, LTS_ERR_ARG, "invalid mode");
    if (!d_field || !d_out_field || !d_out_order) return fail(c, LTS_ERR_ARG, "null data pointer");
    if (n_authorized < 0 || (n_authorized > 0 && !d_authorized)) return fail(c, LTS_ERR_ARG, "invalid authorized list");
    const size_t nb = (size_t)n * 4;
    if (overlap(d_field, nb, d_out_field, nb) || overlap(d_field, nb, d_out_order, nb) ||
        overlap(d_out_field, nb, d_out_order, nb))
        return fail(c, LTS_ERR_ARG, "outputs overlap the input or each other");
    if (cudaSetDevice(c->device) != cudaSuccess) return fail(c, LTS_ERR_CUDA, "cudaSetDevice");
    cudaStream_t s = c->stream;
    Work& w = c->w;
    cudaError_t e;
    if (c->dirty) {
        if ((e = clean_workspace(c)) != cudaSuccess) return cuda_fail(c, e, "clean");
        c->dirty = false;
    }
    Geom g;
    g.ndim = gr->ndim;
    g.nn = gr->ndim == 2 ? 6 : 14;
    g.X = (int)gr->dims[0]; g.Y = (int)gr->dims[1]; g.Z = (int)gr->dims[2];
    g.n = (int)n;
    g.XY = g.X * g.Y;
    g.dX = make_fastdiv((unsigned)g.X);
    g.dXY = make_fastdiv((unsigned)g.XY);
    w.nblk_cur = (int)((n + 31) / 32);
    const int sms = c->sms;
    int* O = d_out_order;
    float* gout = d_out_field;

    cudaMemsetAsync(w.ctr, 0, sizeof(DevCounters), s);
    cudaMemsetAsync(w.pstats, 0, 2 * sizeof(PassStats), s);
    w.launches = 0;
    cudaEventRecord(c->ev[0], s);
    build_authbits(w, g, d_authorized, n_authorized, s);
    order_field(w, g, d_field, gout, O, s);
    cudaEventRecord(c->ev[1], s);
    int evi = 2;
    for (int side = 0; side < 2; ++side) {
        const bool run = side == 0 ? (mode & LTS_MODE_MIN) != 0 : (mode & LTS_MODE_MAX) != 0;
        if (!run) {
            for (int k = 0; k < 5; ++k) cudaEventRecord(c->ev[evi++], s);
            continue;
        }
        pass_reset(w, s);
        if (side == 0) {
            classify<-1>(w, g, O, s);               cudaEventRecord(c->ev[evi++], s);
            propagate<-1>(w, g, O, sms, s);         cudaEventRecord(c->ev[evi++], s);
            extract_regions<-1>(w, g, O, sms, s);   cudaEventRecord(c->ev[evi++], s);
            local_orders<-1>(w, g, O, sms, s);      cudaEventRecord(c->ev[evi++], s);
            reorder_flatten<-1>(w, g, O, gout, sms, s); cudaEventRecord(c->ev[evi++], s);
        } else {
            classify<1>(w, g, O, s);                cudaEventRecord(c->ev[evi++], s);
            propagate<1>(w, g, O, sms, s);          cudaEventRecord(c->ev[evi++], s);
            extract_regions<1>(w, g, O, sms, s);    cudaEventRecord(c->ev[evi++], s);
            local_orders<1>(w, g, O, sms, s);       cudaEventRecord(c->ev[evi++], s);
            reorder_flatten<1>(w, g, O, gout, sms, s); cudaEventRecord(c->ev[evi++], s);
        }
        save_pass_kernel<<<1, 1, 0, s>>>(w.ctr, w.reg_start, w.pstats + side);
        w.launches += 1;
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(c, e, "launch");
    cudaMemcpyAsync(w.h_ctr, w.ctr, sizeof(DevCounters), cudaMemcpyDeviceToHost, s);
    PassStats* hps = reinterpret_cast<PassStats*>(w.h_ctr + 1);
    cudaMemcpyAsync(hps, w.pstats, 2 * sizeof(PassStats), cudaMemcpyDeviceToHost, s);
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return cuda_fail(c, e, "synchronize");
    const int status = w.h_ctr->status;
    if (opt_stats) {
        lts_stats& o = *opt_stats;
        memset(&o, 0, sizeof o);
        o.n_vertices = n;
        for (int k = 0; k < 2; ++k) {
            o.removed[k] = hps[k].removed;
            o.regions[k] = hps[k].regions;
            o.region_vertices[k] = hps[k].region_vertices;
            o.max_region[k] = hps[k].max_region;
            o.max_local_floods[k] = (int32_t)hps[k].max_floods;
            o.total_local_floods[k] = hps[k].total_floods;
            o.heap_spills[k] = hps[k].heap_spills;
        }
        float ms = 0;
        cudaEventElapsedTime(&ms, c->ev[0], c->ev[1]);
        o.stage_us[0] = ms * 1000.f;
        for (int st = 0; st < 5; ++st) {
            float acc = 0;
            for (int side = 0; side < 2; ++side) {
                const int a = 1 + side * 5 + st;
                if (cudaEventElapsedTime(&ms, c->ev[a], c->ev[a + 1]) == cudaSuccess) acc += ms;
            }
            o.stage_us[1 + st] = acc * 1000.f;
        }
        cudaEventElapsedTime(&ms, c->ev[0], c->ev[11]);
        o.stage_us[6] = ms * 1000.f;
        o.kernel_launches = w.launches;
    }
    if (status != 0) {
        c->dirty = true;
        const char* what = status == LTS_ERR_NAN ? "the field holds a NaN"
                         : status == LTS_ERR_NO_AUTHORIZED ? "a pass has unauthorized extrema but no authorized one"
                         : status == LTS_ERR_ARG ? "an authorized id is out of range"
                         : status == LTS_ERR_OOM ? "a workspace pool was exhausted"
                         : status == LTS_ERR_TIMEOUT ? "a bounded device wait expired"
                         : "internal consistency check failed";
        c->err = what;
        return (lts_status)status;
    }
    return LTS_OK;
}

}  // extern "C"
