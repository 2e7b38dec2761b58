// C ABI of the library (include/lts.h): contexts and their workspaces,
// argument checks, and the sequence of stages of one simplification, run
// synchronously (lts_simplify), over a batch of fields spread on several
// workspaces at once (lts_simplify_batch), or as queued requests
// (lts_submit / lts_poll).
#include <algorithm>
#include <climits>
#include <cstdio>
#include <deque>
#include <cstring>
#include <cstdlib>
#include <numeric>
#include <string>
#include <vector>

#include "lts_internal.cuh"

namespace lts {
int propagate_lanes(int sms);
long long propagate_log_slack(int lanes);
long long propagate_spill_slack(int lanes);
long long propagate_heap_slack(int lanes);
int scan_tiles_for(long long max_count);
}  // namespace lts

using namespace lts;

namespace lts {
// Final state of one request, written on the device after its last kernel.
struct ReqResult {
    int status;
    int oom_pool;
    PassStats ps[2];
    unsigned long long ticket;
};
}  // namespace lts

namespace {

constexpr int kMaxLanes = 32;      // the context's own workspace and up to 31 more
constexpr int kMaxServe = 15;      // serving workspaces at most (lts_serve_config)
// Workspaces a batch spreads over (fields with large regions take long on one
// warp per region; running many fields side by side overlaps them: measured
// on the 256-field batch, 4 -> 63, 8 -> 94, 16 -> 158 Mvertices/s).
constexpr int kBatchLanes = 32;
constexpr int kRing = 1024;        // serving requests in flight per context
constexpr int kPoolRetries = 3;    // times a call may enlarge an exhausted flood pool and run again

// A workspace with the stream its work is enqueued on.
struct Lane {
    Work w{};
    long long nmax = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    cudaEvent_t ev[16];
    bool events = false;
    void* allocs[96];
    int nallocs = 0;
    bool dirty = false;            // a CUDA error left the workspace in an unknown state
};

}  // namespace

struct lts_ctx {
    int device = 0;
    int sms = 0;
    Lane lane[kMaxLanes];
    int nlanes = 1;
    std::string err;
    // batches
    ReqResult* batch_dev = nullptr;
    ReqResult* batch_host = nullptr;
    int batch_cap = 0;
    cudaEvent_t fork = nullptr, join[kMaxLanes] = {};
    // serving
    ReqResult* ring_host = nullptr;   // pinned, mapped
    ReqResult* ring_dev = nullptr;
    cudaEvent_t ring_ev[kRing];
    bool ring_ready = false;
    unsigned long long next_ticket = 1;
    int serve_max = kMaxServe;        // serving workspaces (lanes 1..serve_max); 0: the context's own
    long long serve_budget = 120LL << 30;
    std::deque<std::pair<unsigned long long, long long>> inflight[kMaxLanes];   // (ticket, vertices) per lane
    lts_tuning tune{};                // launch tuning (0: default)
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
    z.spill_cap = std::min<long long>(8 * n + propagate_spill_slack((int)z.lanes), (1LL << 31) - 1);
    z.heap_cap = 4 * n + propagate_heap_slack((int)z.lanes);
    z.lo_cap = n + z.half;
    z.nblk = (n + 31) / 32;
    z.scan_tiles = std::max<long long>(scan_tiles_for(z.half + 1), (z.nblk + 4095) / 4096 + 1);
    return z;
}

size_t bytes_for(const Sizes& z) {
    size_t b = 0;
    b += 4 * 4 * (size_t)z.n;                       // sort key/value double buffers
    b += (size_t)z.tiles * 256 * 8 + 8192 * 2 + 32; // look-back words, histograms, digit offsets
    b += 3 * 4 * 8192 + 48;                         // distinct-key table
    b += ((size_t)z.n + 31) / 32 * 4;               // authorized bitmap
    b += 3 * 4 * (size_t)z.n;                       // owner, loc, qmark
    b += 10 * 4 * (size_t)z.half;                   // U and class records
    b += 32 * (size_t)z.half;                       // task records, heap records
    b += 4 * (size_t)z.n;                           // saddle arrival counters
    b += 4 * (size_t)z.spill_cap + 8 * (size_t)z.heap_cap + 4 * (size_t)z.log_cap;
    b += 16 * (size_t)z.log_cap + 4 * (size_t)z.half;   // log classes, per-entry region data, class regions
    b += 11 * 4 * (size_t)z.half;                   // region records
    b += 3 * 4 * (size_t)z.n;                       // members, member regions, lhat
    b += 21 * (size_t)z.lo_cap;                     // local-order scratch
    b += 16 * (size_t)z.n;                          // local adjacency of the largest regions
    b += sizeof(RankBlk) * (size_t)z.nblk + 2 * 4 * (size_t)z.half;
    b += 8 * (size_t)z.scan_tiles + sizeof(DevCounters) + 2 * sizeof(PassStats);
    b += 256 * 8;                                   // test-only look-back words
    b += 64 + (1 << 14) + 6 * 8;                    // link tables, critical point counts
    return b;
}

// tests only: while LTS_TEST_FAIL_ALLOC is set, every device allocation of the
// library fails as if the device had no memory left
bool test_alloc_fails() {
    const char* v = getenv("LTS_TEST_FAIL_ALLOC");
    return v && v[0] && v[0] != '0';
}

template <typename T>
bool dev_alloc(Lane& L, T** p, size_t count) {
    if (L.nallocs >= (int)(sizeof L.allocs / sizeof L.allocs[0])) return false;
    if (test_alloc_fails()) return false;
    void* q = nullptr;
    if (cudaMalloc(&q, std::max<size_t>(count, 1) * sizeof(T)) != cudaSuccess) return false;
    L.allocs[L.nallocs++] = q;
    *p = static_cast<T*>(q);
    return true;
}

void lane_free(Lane& L) {
    for (int i = 0; i < L.nallocs; ++i) cudaFree(L.allocs[i]);
    L.nallocs = 0;
    if (L.w.h_ctr) cudaFreeHost(L.w.h_ctr);
    L.w.h_ctr = nullptr;
    if (L.events)
        for (auto& e : L.ev) cudaEventDestroy(e);
    L.events = false;
    // side streams and their events (null unless created; Work{} zeroes them)
    for (int i = 0; i < 4; ++i)
        if (L.w.aux[i]) cudaStreamDestroy(L.w.aux[i]);
    for (int i = 0; i < 3; ++i)
        if (L.w.join_ev[i]) cudaEventDestroy(L.w.join_ev[i]);
    if (L.w.fork_ev) cudaEventDestroy(L.w.fork_ev);
    if (L.w.pre_fork) cudaEventDestroy(L.w.pre_fork);
    if (L.w.pre_join) cudaEventDestroy(L.w.pre_join);
    if (L.own_stream && L.stream) cudaStreamDestroy(L.stream);
    L.stream = nullptr;
    L.own_stream = false;
    L.w = Work{};
    L.nmax = 0;
}

// Allocates and initializes a workspace for grids of up to nmax vertices.
// On failure the lane is freed again, including `stream` if own_stream.
lts_status lane_alloc(Lane& L, long long nmax, int sms, cudaStream_t stream, bool own_stream, bool side_streams) {
    L.stream = stream;
    L.own_stream = own_stream;
    L.nmax = nmax;
    const Sizes z = sizes_for(nmax, sms);
    Work& w = L.w;
    w.nmax = (int)nmax;
    w.max_tiles = (int)z.tiles;
    w.lanes = (int)z.lanes;
    w.class_cap = (int)z.half;
    w.log_cap = z.log_cap; w.spill_cap = z.spill_cap; w.heap_cap = z.heap_cap; w.lo_cap = z.lo_cap;
    w.nblk = (int)z.nblk;
    w.scan_tmp_cap = (int)z.scan_tiles;
    w.sms = sms;
    w.eng_bpsm = 8;
    w.team_bpsm = 12;
    // tests only: LTS_TEST_MIN_TIER=k (1..5) runs step 2 of small regions in tier k
    // (the results do not depend on the tier)
    w.min_tier = 0;
    if (const char* mt = getenv("LTS_TEST_MIN_TIER")) w.min_tier = std::max(0, std::min(5, atoi(mt)));
    // tests only: look-back words that nothing sets (see LTS_TEST_STALL_SORT in order_field.cu)
    unsigned long long* stall_words = nullptr;
    bool ok = true;
    ok = ok && dev_alloc(L, &w.keyA, z.n) && dev_alloc(L, &w.valA, z.n) && dev_alloc(L, &w.keyB, z.n) &&
         dev_alloc(L, &w.valB, z.n);
    ok = ok && dev_alloc(L, &w.sort_status, (size_t)z.tiles * 256) && dev_alloc(L, &w.sort_hist, 2048) &&
         dev_alloc(L, &w.sort_offsets, 2048) && dev_alloc(L, &w.tile_counter, 8) &&
         dev_alloc(L, &w.dk_keys, 8192) && dev_alloc(L, &w.dk_cnts, 8192) && dev_alloc(L, &w.dk_rank, 8192) &&
         dev_alloc(L, &w.dk_info, 4) &&
         dev_alloc(L, &w.bin_cursor, 1024);
    ok = ok && dev_alloc(L, &w.authbits, (z.n + 31) / 32);
    ok = ok && dev_alloc(L, &w.owner, z.n) && dev_alloc(L, &w.loc, z.n) && dev_alloc(L, &w.qmark, z.n);
    ok = ok && dev_alloc(L, &w.U, z.half) && dev_alloc(L, &w.parent, z.half) && dev_alloc(L, &w.wait_v, z.half) &&
         dev_alloc(L, &w.ctop, z.half) &&
         dev_alloc(L, &w.cnt, z.n) && dev_alloc(L, &w.tasks, z.half) &&
         dev_alloc(L, &w.sib_head, z.half) && dev_alloc(L, &w.sib_next, z.half) &&
         dev_alloc(L, &w.spill_base, z.half) && dev_alloc(L, &w.spill_n, z.half) && dev_alloc(L, &w.heaprec, z.half);
    ok = ok && dev_alloc(L, &w.spill_pool, z.spill_cap) && dev_alloc(L, &w.heap_pool, z.heap_cap) &&
         dev_alloc(L, &w.vlog, z.log_cap) && dev_alloc(L, &w.vlog_cls, z.log_cap) &&
         dev_alloc(L, &w.ent_rid, z.log_cap) && dev_alloc(L, &w.ent_loc, z.log_cap) &&
         dev_alloc(L, &w.ent_od, z.log_cap) && dev_alloc(L, &w.cls2rid, z.half);
    ok = ok && dev_alloc(L, &w.class2reg, z.half) && dev_alloc(L, &w.reg_class, z.half) &&
         dev_alloc(L, &w.reg_saddle, z.half) && dev_alloc(L, &w.reg_size, z.half) &&
         dev_alloc(L, &w.reg_start, z.half + 1) && dev_alloc(L, &w.reg_top, z.half) &&
         dev_alloc(L, &w.reg_sod, z.half) && dev_alloc(L, &w.reg_place, z.half) && dev_alloc(L, &w.reg_head, z.half) &&
         dev_alloc(L, &w.reg_att, z.half) && dev_alloc(L, &w.reg_swallowed, z.half);
    ok = ok && dev_alloc(L, &w.members, z.n) && dev_alloc(L, &w.lhat, z.n) && dev_alloc(L, &w.tier_list, 2 * z.half) &&
         dev_alloc(L, &w.member_reg, z.n);
    ok = ok && dev_alloc(L, &w.lo_v, z.lo_cap) && dev_alloc(L, &w.lo_L, z.lo_cap) && dev_alloc(L, &w.lo_L2, z.lo_cap) &&
         dev_alloc(L, &w.lo_heap, z.lo_cap) && dev_alloc(L, &w.lo_flag, z.lo_cap) && dev_alloc(L, &w.lo_P, z.lo_cap) &&
         dev_alloc(L, &w.lo_adj, 4 * z.n + 4096);
    w.lo_adj_cap = 4 * z.n + 4096;
    ok = ok && dev_alloc(L, &w.rblk, z.nblk) && dev_alloc(L, &w.sad_att, z.half) && dev_alloc(L, &w.cumA, z.half + 1);
    ok = ok && dev_alloc(L, &w.scan_tmp, z.scan_tiles) && dev_alloc(L, &w.ctr, 1) && dev_alloc(L, &w.pstats, 2);
    ok = ok && dev_alloc(L, &stall_words, 256);
    ok = ok && dev_alloc(L, &w.link6, 64) && dev_alloc(L, &w.link14, 1 << 14) && dev_alloc(L, &w.crit_counts, 6);
    w.test_stall = stall_words;
    if (ok && cudaMallocHost((void**)&w.h_ctr, sizeof(DevCounters) + 2 * sizeof(PassStats)) != cudaSuccess) ok = false;
    if (!ok) {
        cudaGetLastError();
        lane_free(L);
        return LTS_ERR_OOM;
    }
    for (auto& e : L.ev) cudaEventCreate(&e);
    L.events = true;
    w.aux_on = false;
    if (side_streams) {
        // a handle whose creation failed is left null, so lane_free skips it
        auto mk_event = [](cudaEvent_t* e) {
            if (cudaEventCreateWithFlags(e, cudaEventDisableTiming) == cudaSuccess) return true;
            *e = nullptr;
            return false;
        };
        auto mk_stream = [](cudaStream_t* st) {
            if (cudaStreamCreateWithFlags(st, cudaStreamNonBlocking) == cudaSuccess) return true;
            *st = nullptr;
            return false;
        };
        bool aux_ok = mk_event(&w.fork_ev) && mk_event(&w.pre_fork) && mk_event(&w.pre_join);
        for (int i = 0; i < 4 && aux_ok; ++i) aux_ok = mk_stream(&w.aux[i]) && (i == 3 || mk_event(&w.join_ev[i]));
        if (!aux_ok) {
            cudaGetLastError();
            lane_free(L);
            return LTS_ERR_CUDA;
        }
        w.aux_on = true;
    }
    cudaStream_t s = L.stream;
    cudaMemsetAsync(w.owner, 0xff, sizeof(int) * (size_t)z.n, s);
    cudaMemsetAsync(w.cnt, 0, sizeof(int) * (size_t)z.n, s);
    cudaMemsetAsync(w.sort_status, 0, (size_t)z.tiles * 256 * sizeof(unsigned long long), s);
    cudaMemsetAsync(w.qmark, 0xff, sizeof(int) * (size_t)z.n, s);
    if (stall_words) cudaMemsetAsync(stall_words, 0, 256 * sizeof(unsigned long long), s);
    build_link_tables(w.link6, w.link14, s);
    cudaMemsetAsync(w.ctr, 0, sizeof(DevCounters), s);
    w.epoch = 0;
    if (cudaStreamSynchronize(s) != cudaSuccess) {
        cudaGetLastError();
        lane_free(L);
        return LTS_ERR_CUDA;
    }
    return LTS_OK;
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

Geom geom_of(const lts_grid* gr, long long n) {
    Geom g;
    g.ndim = gr->ndim;
    g.nn = gr->ndim == 2 ? 6 : 14;
    g.X = (int)gr->dims[0]; g.Y = (int)gr->dims[1]; g.Z = (int)gr->dims[2];
    g.n = (int)n;
    g.XY = g.X * g.Y;
    g.dX = make_fastdiv((unsigned)g.X);
    g.dXY = make_fastdiv((unsigned)g.XY);
    return g;
}

lts_status fail(lts_ctx* c, lts_status s, const std::string& msg) {
    c->err = msg;
    return s;
}

lts_status cuda_fail(lts_ctx* c, Lane& L, cudaError_t e, const char* where) {
    c->err = std::string(where) + ": " + cudaGetErrorString(e);
    L.dirty = true;
    return LTS_ERR_CUDA;
}

std::string status_text(int status, int oom_pool = 0) {
    if (status == LTS_ERR_OOM) {
        const char* pool = oom_pool == 1 ? " (flood overflow heaps)" : oom_pool == 2 ? " (queue spill pool)"
                         : oom_pool == 3 ? " (visited-vertex log)" : "";
        return std::string("a workspace pool was exhausted") + pool;
    }
    return status == LTS_ERR_NAN ? "the field holds a NaN"
         : status == LTS_ERR_NO_AUTHORIZED ? "a pass has unauthorized extrema but no authorized one"
         : status == LTS_ERR_ARG ? "an authorized id is out of range"
         : status == LTS_ERR_TIMEOUT ? "a bounded device wait expired"
         : "internal consistency check failed";
}

// reset the per-vertex state after a CUDA error
cudaError_t clean_workspace(Lane& L) {
    Work& w = L.w;
    cudaMemsetAsync(w.owner, 0xff, sizeof(int) * (size_t)w.nmax, L.stream);
    cudaMemsetAsync(w.cnt, 0, sizeof(int) * (size_t)w.nmax, L.stream);
    cudaMemsetAsync(w.sort_status, 0, (size_t)w.max_tiles * 256 * sizeof(unsigned long long), L.stream);
    w.epoch = 0;
    return cudaGetLastError();
}

bool overlap(const void* a, size_t na, const void* b, size_t nb) {
    const char* x = static_cast<const char*>(a);
    const char* y = static_cast<const char*>(b);
    return x < y + nb && y < x + na;
}

// Checks one field's arguments; n receives its vertex count.
lts_status check_field(lts_ctx* c, const lts_grid* gr, long long nmax, const void* d_field,
                       const int32_t* d_authorized, int64_t n_authorized, lts_mode mode, const void* d_out_field,
                       const int32_t* d_out_order, long long* n, const std::string& what, int vbytes = 4) {
    if (!grid_ok(gr, n)) return fail(c, LTS_ERR_ARG, what + "invalid grid");
    if (*n > nmax) return fail(c, LTS_ERR_ARG, what + "grid larger than the context's max_vertices");
    if ((mode & ~LTS_MODE_RESTORE) < LTS_MODE_MIN || (mode & ~LTS_MODE_RESTORE) > LTS_MODE_BOTH)
        return fail(c, LTS_ERR_ARG, what + "invalid mode");
    if (!d_field || !d_out_field || !d_out_order) return fail(c, LTS_ERR_ARG, what + "null data pointer");
    if (n_authorized < 0 || (n_authorized > 0 && !d_authorized))
        return fail(c, LTS_ERR_ARG, what + "invalid authorized list");
    const size_t nv = (size_t)*n * vbytes, no = (size_t)*n * 4;
    if (overlap(d_field, nv, d_out_field, nv) || overlap(d_field, nv, d_out_order, no) ||
        overlap(d_out_field, nv, d_out_order, no))
        return fail(c, LTS_ERR_ARG, what + "outputs overlap the input or each other");
    return LTS_OK;
}

}  // namespace

namespace lts {
cudaError_t pass_reset(Work& w, cudaStream_t s) {
    // every counter but the status word and the pool it names
    cudaMemsetAsync(reinterpret_cast<char*>(w.ctr) + 2 * sizeof(int), 0, sizeof(DevCounters) - 2 * sizeof(int), s);
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
    ps->fallbacks = ctr->lo_fallbacks;
    ps->restored = ctr->n_restored;
}

// the request's final status and pass statistics
__global__ void capture_kernel(const DevCounters* ctr, const PassStats* ps, ReqResult* out, unsigned long long ticket) {
    out->status = ctr->status;
    out->oom_pool = ctr->oom_pool;
    out->ps[0] = ps[0];
    out->ps[1] = ps[1];
    out->ticket = ticket;
}

// After a failed request (and only then) the claims and arrival counters it
// left behind are cleared, so that the next request on this workspace,
// already enqueued behind it, starts from a clean state.
__global__ void fail_clean_kernel(const DevCounters* ctr, int* owner, int* cnt, int nmax) {
    if (*(volatile const int*)&ctr->status == 0) return;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nmax; i += (long long)gridDim.x * blockDim.x) {
        owner[i] = -1;
        cnt[i] = 0;
    }
}
}  // namespace
}  // namespace lts

namespace {

// How a pass selects the extrema it keeps: the caller's list, or
// persistence above eps measured by the pass itself (Sec. 4.5).
struct Selection {
    const int32_t* ids;
    int64_t n_ids;
    bool by_persistence;
    double eps;
};

// Enqueues one simplification on the lane's stream: stage events ev[0..11],
// the result capture (when res is set) and the clean-up after a failure.
// With a persistence selection each pass first runs the propagations from
// every extremum of its kind (counted in the classification stage), which
// set the authorized bitmap, and then the pass proper.
cudaError_t enqueue_simplify(Lane& L, const Geom& g, const void* d_field, const Selection& sel, lts_mode mode,
                             void* gout, int* O, int sms, ReqResult* res, unsigned long long ticket,
                             bool f64 = false) {
    cudaStream_t s = L.stream;
    Work& w = L.w;
    w.nblk_cur = (g.n + 31) / 32;
    cudaMemsetAsync(w.ctr, 0, sizeof(DevCounters), s);
    cudaMemsetAsync(w.pstats, 0, 2 * sizeof(PassStats), s);
    w.launches = 0;
    cudaEventRecord(L.ev[0], s);
    if (!sel.by_persistence) build_authbits(w, g, sel.ids, sel.n_ids, s);
    if (f64) order_field_f64(w, g, static_cast<const double*>(d_field), static_cast<double*>(gout), O, s);
    else order_field(w, g, static_cast<const float*>(d_field), static_cast<float*>(gout), O, s);
    cudaEventRecord(L.ev[1], s);
    int evi = 2;
    for (int side = 0; side < 2; ++side) {
        const bool run = side == 0 ? (mode & LTS_MODE_MIN) != 0 : (mode & LTS_MODE_MAX) != 0;
        if (!run) {
            for (int k = 0; k < 5; ++k) cudaEventRecord(L.ev[evi++], s);
            continue;
        }
        pass_reset(w, s);
        if (sel.by_persistence) {
            cudaMemsetAsync(w.authbits, 0, sizeof(unsigned) * (((size_t)g.n + 31) / 32), s);
            if (side == 0) {
                classify<-1>(w, g, O, s);
                select_persistent<-1>(w, g, O, static_cast<const float*>(gout), sel.eps, sms, s);
            } else {
                classify<1>(w, g, O, s);
                select_persistent<1>(w, g, O, static_cast<const float*>(gout), sel.eps, sms, s);
            }
            pass_reset(w, s);
        }
        // The reorder's rank prefix needs the regions only: on the context's own
        // workspace it runs on a side stream beside the local orders (its time
        // is then inside the local-order stage).
        auto prefix_fork = [&]() {
            if (w.aux_on) {
                cudaEventRecord(w.pre_fork, s);
                cudaStreamWaitEvent(w.aux[3], w.pre_fork, 0);
                reorder_prefix(w, g, sms, w.aux[3]);
                cudaEventRecord(w.pre_join, w.aux[3]);
            } else {
                reorder_prefix(w, g, sms, s);
            }
        };
        auto prefix_join = [&]() {
            if (w.aux_on) cudaStreamWaitEvent(s, w.pre_join, 0);
        };
        if (side == 0) {
            classify<-1>(w, g, O, s);               cudaEventRecord(L.ev[evi++], s);
            propagate<-1>(w, g, O, sms, s);         cudaEventRecord(L.ev[evi++], s);
            extract_regions<-1>(w, g, O, sms, s);   cudaEventRecord(L.ev[evi++], s);
            prefix_fork();
            local_orders<-1>(w, g, O, sms, s);      prefix_join();
            if (mode & LTS_MODE_RESTORE) restore_swallowed<-1>(w, g, O, sms, s);
            cudaEventRecord(L.ev[evi++], s);
            reorder_flatten<-1>(w, g, O, gout, f64, sms, s); cudaEventRecord(L.ev[evi++], s);
        } else {
            classify<1>(w, g, O, s);                cudaEventRecord(L.ev[evi++], s);
            propagate<1>(w, g, O, sms, s);          cudaEventRecord(L.ev[evi++], s);
            extract_regions<1>(w, g, O, sms, s);    cudaEventRecord(L.ev[evi++], s);
            prefix_fork();
            local_orders<1>(w, g, O, sms, s);       prefix_join();
            if (mode & LTS_MODE_RESTORE) restore_swallowed<1>(w, g, O, sms, s);
            cudaEventRecord(L.ev[evi++], s);
            reorder_flatten<1>(w, g, O, gout, f64, sms, s); cudaEventRecord(L.ev[evi++], s);
        }
        save_pass_kernel<<<1, 1, 0, s>>>(w.ctr, w.reg_start, w.pstats + side);
        w.launches += 1;
    }
    if (res) {
        capture_kernel<<<1, 1, 0, s>>>(w.ctr, w.pstats, res, ticket);
        w.launches += 1;
    }
    fail_clean_kernel<<<sms * 4, 256, 0, s>>>(w.ctr, w.owner, w.cnt, w.nmax);
    w.launches += 1;
    return cudaGetLastError();
}

void fill_stats(lts_stats& o, long long n, const PassStats* ps, long long launches) {
    memset(&o, 0, sizeof o);
    o.n_vertices = n;
    for (int k = 0; k < 2; ++k) {
        o.removed[k] = ps[k].removed;
        o.regions[k] = ps[k].regions;
        o.region_vertices[k] = ps[k].region_vertices;
        o.max_region[k] = ps[k].max_region;
        o.max_local_floods[k] = (int32_t)ps[k].max_floods;
        o.total_local_floods[k] = ps[k].total_floods;
        o.heap_spills[k] = ps[k].heap_spills;
        o.fallback_regions[k] = ps[k].fallbacks;
        o.restored[k] = ps[k].restored;
    }
    o.kernel_launches = launches;
}

void fill_stage_times(lts_stats& o, Lane& L) {
    float ms = 0;
    if (cudaEventElapsedTime(&ms, L.ev[0], L.ev[1]) == cudaSuccess) o.stage_us[0] = ms * 1000.f;
    for (int st = 0; st < 5; ++st) {
        float acc = 0;
        for (int side = 0; side < 2; ++side) {
            const int a = 1 + side * 5 + st;
            if (cudaEventElapsedTime(&ms, L.ev[a], L.ev[a + 1]) == cudaSuccess) acc += ms;
        }
        o.stage_us[1 + st] = acc * 1000.f;
    }
    if (cudaEventElapsedTime(&ms, L.ev[0], L.ev[11]) == cudaSuccess) o.stage_us[6] = ms * 1000.f;
}

lts_status ensure_ring(lts_ctx* c) {
    if (c->ring_ready) return LTS_OK;
    if (cudaHostAlloc((void**)&c->ring_host, kRing * sizeof(ReqResult), cudaHostAllocMapped) != cudaSuccess) {
        cudaGetLastError();
        return fail(c, LTS_ERR_OOM, "cannot allocate the request ring");
    }
    memset(c->ring_host, 0, kRing * sizeof(ReqResult));
    if (cudaHostGetDevicePointer((void**)&c->ring_dev, c->ring_host, 0) != cudaSuccess) {
        cudaGetLastError();
        cudaFreeHost(c->ring_host);
        c->ring_host = nullptr;
        return fail(c, LTS_ERR_CUDA, "cannot map the request ring");
    }
    for (auto& e : c->ring_ev) cudaEventCreateWithFlags(&e, cudaEventDisableTiming);
    c->ring_ready = true;
    return LTS_OK;
}

// Outstanding vertices of a lane's served requests (finished ones retired).
long long lane_backlog(lts_ctx* c, int li) {
    auto& q = c->inflight[li];
    while (!q.empty()) {
        const unsigned long long t = q.front().first;
        // a ticket whose ring slot was reused is finished (submit waited for it)
        if (t + kRing < c->next_ticket || cudaEventQuery(c->ring_ev[t % kRing]) == cudaSuccess) {
            q.pop_front();
            continue;
        }
        cudaGetLastError();
        break;
    }
    long long b = 0;
    for (const auto& r : q) b += r.second;
    return b;
}

// Continuous batching: a request goes to an idle serving workspace, or to a
// new one while the budget and the device's free memory allow, or else to the
// workspace with the fewest outstanding vertices.  Every serving workspace
// fits the context's largest grid and runs on its own stream.  With no
// serving workspace (serve_max == 0, or nothing could be allocated) requests
// run on the context's own workspace and stream, one after another.
int pick_serve_lane(lts_ctx* c, long long n) {
    const long long nmax = c->lane[0].nmax;
    const size_t per_lane = bytes_for(sizes_for(nmax, c->sms));
    int best = -1;
    long long best_load = LLONG_MAX;
    int nalloc = 0, free_slot = -1;
    for (int i = 1; i <= c->serve_max; ++i) {
        Lane& L = c->lane[i];
        if (!L.stream || L.nmax < nmax) {
            // absent, or a smaller workspace left by a batch: usable once re-allocated while idle
            if (free_slot < 0 && (!L.stream || (lane_backlog(c, i) == 0 && cudaStreamQuery(L.stream) == cudaSuccess)))
                free_slot = i;
            continue;
        }
        ++nalloc;
        const long long b = lane_backlog(c, i);
        if (b < best_load) { best_load = b; best = i; }
    }
    (void)n;
    if (best >= 0 && best_load == 0) return best;
    if (free_slot >= 0 && (long long)((nalloc + 1) * per_lane) <= c->serve_budget) {
        size_t fr = 0, tot = 0;
        if (cudaMemGetInfo(&fr, &tot) == cudaSuccess && fr > per_lane + (1ull << 30)) {
            Lane& L = c->lane[free_slot];
            if (L.stream) lane_free(L);
            cudaStream_t s;
            if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) == cudaSuccess) {
                if (lane_alloc(L, nmax, c->sms, s, true, false) == LTS_OK) {
                    c->nlanes = std::max(c->nlanes, free_slot + 1);
                    return free_slot;
                }
                // a failed lane_alloc has already freed the lane and destroyed the stream it owned
            }
        }
        cudaGetLastError();
    }
    return best >= 0 ? best : 0;
}

}  // namespace

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
    cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, device);
    const lts_status st = lane_alloc(c->lane[0], max_vertices, c->sms, static_cast<cudaStream_t>(cuda_stream), false, true);
    if (st != LTS_OK) {
        delete c;
        return st;
    }
    *out = c;
    return LTS_OK;
}

void lts_destroy(lts_ctx* c) {
    if (!c) return;
    cudaSetDevice(c->device);
    cudaStreamSynchronize(c->lane[0].stream);
    for (int i = 1; i < kMaxLanes; ++i)
        if (c->lane[i].stream) cudaStreamSynchronize(c->lane[i].stream);
    for (int i = 0; i < kMaxLanes; ++i) lane_free(c->lane[i]);
    if (c->batch_dev) cudaFree(c->batch_dev);
    if (c->batch_host) cudaFreeHost(c->batch_host);
    if (c->fork) cudaEventDestroy(c->fork);
    for (auto& e : c->join)
        if (e) cudaEventDestroy(e);
    if (c->ring_ready) {
        for (auto& e : c->ring_ev) cudaEventDestroy(e);
        cudaFreeHost(c->ring_host);
    }
    delete c;
}

const char* lts_last_error(const lts_ctx* c) { return c ? c->err.c_str() : "null context"; }

lts_status lts_set_tuning(lts_ctx* c, const lts_tuning* t) {
    if (!c) return LTS_ERR_ARG;
    c->err.clear();
    if (!t) {
        c->tune = lts_tuning{};
        return LTS_OK;
    }
    if (t->engine_blocks_per_sm < 0 || t->engine_blocks_per_sm > 8)
        return fail(c, LTS_ERR_ARG, "engine_blocks_per_sm outside [0, 8]");
    if (t->team_blocks_per_sm < 0 || t->team_blocks_per_sm > 16)
        return fail(c, LTS_ERR_ARG, "team_blocks_per_sm outside [0, 16]");
    if (t->batch_workspaces < 0 || t->batch_workspaces > kBatchLanes)
        return fail(c, LTS_ERR_ARG, "batch_workspaces outside [0, 32]");
    for (int r : t->reserved)
        if (r != 0) return fail(c, LTS_ERR_ARG, "reserved tuning fields must be 0");
    c->tune = *t;
    return LTS_OK;
}

lts_status lts_get_tuning(const lts_ctx* c, lts_tuning* out) {
    if (!c || !out) return LTS_ERR_ARG;
    *out = lts_tuning{};
    out->engine_blocks_per_sm = c->tune.engine_blocks_per_sm > 0 ? c->tune.engine_blocks_per_sm : 8;
    out->team_blocks_per_sm = c->tune.team_blocks_per_sm > 0 ? c->tune.team_blocks_per_sm : 12;
    out->batch_workspaces = c->tune.batch_workspaces > 0 ? c->tune.batch_workspaces : kBatchLanes;
    return LTS_OK;
}

}  // extern "C"

namespace {

// Replaces one tracked allocation of the lane by a larger one (contents are not kept).
template <typename T>
bool regrow(Lane& L, T** p, size_t count) {
    void* q = nullptr;
    if (test_alloc_fails()) return false;
    if (cudaMalloc(&q, count * sizeof(T)) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    for (int i = 0; i < L.nallocs; ++i)
        if (L.allocs[i] == static_cast<void*>(*p)) {
            cudaFree(L.allocs[i]);
            L.allocs[i] = q;
            *p = static_cast<T*>(q);
            return true;
        }
    cudaFree(q);
    return false;
}

// Doubles the flood overflow-heap pool (pool 1) or the queue spill pool
// (pool 2, whose offsets are 32-bit) of a workspace.
bool grow_pool(Lane& L, int pool) {
    Work& w = L.w;
    if (cudaStreamSynchronize(L.stream) != cudaSuccess) return false;
    if (pool == 1) {
        const long long cap = 2 * w.heap_cap;
        if (!regrow(L, &w.heap_pool, (size_t)cap)) return false;
        w.heap_cap = cap;
        return true;
    }
    const long long cap = std::min<long long>(2 * w.spill_cap, (1LL << 31) - 1);
    if (cap <= w.spill_cap || !regrow(L, &w.spill_pool, (size_t)cap)) return false;
    w.spill_cap = cap;
    return true;
}

// The context's launch tuning, copied into a workspace before a call uses it.
void tune_lane(const lts_ctx* c, Lane& L) {
    L.w.eng_bpsm = c->tune.engine_blocks_per_sm > 0 ? c->tune.engine_blocks_per_sm : 8;
    L.w.team_bpsm = c->tune.team_blocks_per_sm > 0 ? c->tune.team_blocks_per_sm : 12;
}

lts_status simplify_one(lts_ctx* c, const lts_grid* gr, const void* d_field, const Selection& sel, lts_mode mode,
                        void* d_out_field, int32_t* d_out_order, lts_stats* opt_stats, bool f64 = false) {
    Lane& L = c->lane[0];
    long long n;
    lts_status st = check_field(c, gr, L.nmax, d_field, sel.ids, sel.n_ids, mode, d_out_field, d_out_order, &n, "",
                                f64 ? 8 : 4);
    if (st != LTS_OK) return st;
    if (cudaSetDevice(c->device) != cudaSuccess) return fail(c, LTS_ERR_CUDA, "cudaSetDevice");
    cudaError_t e;
    if (L.dirty) {
        if ((e = clean_workspace(L)) != cudaSuccess) return cuda_fail(c, L, e, "clean");
        L.dirty = false;
    }
    const Geom g = geom_of(gr, n);
    Work& w = L.w;
    PassStats* hps = reinterpret_cast<PassStats*>(w.h_ctr + 1);
    int status = 0;
    for (int attempt = 0;; ++attempt) {
        tune_lane(c, L);
        if ((e = enqueue_simplify(L, g, d_field, sel, mode, d_out_field, d_out_order, c->sms, nullptr, 0, f64)) !=
            cudaSuccess)
            return cuda_fail(c, L, e, "launch");
        cudaMemcpyAsync(w.h_ctr, w.ctr, sizeof(DevCounters), cudaMemcpyDeviceToHost, L.stream);
        cudaMemcpyAsync(hps, w.pstats, 2 * sizeof(PassStats), cudaMemcpyDeviceToHost, L.stream);
        if ((e = cudaStreamSynchronize(L.stream)) != cudaSuccess) return cuda_fail(c, L, e, "synchronize");
        status = w.h_ctr->status;
        // A flood pool ran out (the propagations' queues outgrew it: regions of a
        // large share of the grid): enlarge that pool and run the call again.  The
        // failed run left the workspace clean (fail_clean_kernel) and did not
        // touch the input.
        const int pool = w.h_ctr->oom_pool;
        if (status == LTS_ERR_OOM && (pool == 1 || pool == 2) && attempt < kPoolRetries) {
            if (!grow_pool(L, pool)) break;
            continue;
        }
        break;
    }
    if (opt_stats) {
        fill_stats(*opt_stats, n, hps, w.launches);
        fill_stage_times(*opt_stats, L);
    }
    if (status != 0) return fail(c, (lts_status)status, status_text(status, w.h_ctr->oom_pool));
    return LTS_OK;
}

}  // namespace

extern "C" {

lts_status lts_simplify(lts_ctx* c, const lts_grid* gr, const float* d_field, const int32_t* d_authorized,
                        int64_t n_authorized, lts_mode mode, float* d_out_field, int32_t* d_out_order,
                        lts_stats* opt_stats) {
    if (!c) return LTS_ERR_ARG;
    c->err.clear();
    const Selection sel{d_authorized, n_authorized, false, 0.0};
    return simplify_one(c, gr, d_field, sel, mode, d_out_field, d_out_order, opt_stats);
}

lts_status lts_simplify_f64(lts_ctx* c, const lts_grid* gr, const double* d_field, const int32_t* d_authorized,
                            int64_t n_authorized, lts_mode mode, double* d_out_field, int32_t* d_out_order,
                            lts_stats* opt_stats) {
    if (!c) return LTS_ERR_ARG;
    c->err.clear();
    const Selection sel{d_authorized, n_authorized, false, 0.0};
    return simplify_one(c, gr, d_field, sel, mode, d_out_field, d_out_order, opt_stats, true);
}

lts_status lts_classify(lts_ctx* c, const lts_grid* gr, const int32_t* d_order, int8_t* d_lower, int8_t* d_upper,
                        int64_t* counts) {
    if (!c) return LTS_ERR_ARG;
    c->err.clear();
    Lane& L = c->lane[0];
    long long n;
    if (!grid_ok(gr, &n)) return fail(c, LTS_ERR_ARG, "invalid grid");
    if (n > L.nmax) return fail(c, LTS_ERR_ARG, "grid larger than the context's max_vertices");
    if (!d_order || !counts) return fail(c, LTS_ERR_ARG, "null pointer");
    if ((d_lower && overlap(d_lower, (size_t)n, d_order, (size_t)n * 4)) ||
        (d_upper && overlap(d_upper, (size_t)n, d_order, (size_t)n * 4)) ||
        (d_lower && d_upper && overlap(d_lower, (size_t)n, d_upper, (size_t)n)))
        return fail(c, LTS_ERR_ARG, "outputs overlap the order field or each other");
    if (cudaSetDevice(c->device) != cudaSuccess) return fail(c, LTS_ERR_CUDA, "cudaSetDevice");
    Work& w = L.w;
    const Geom g = geom_of(gr, n);
    cudaError_t e = critical_points(w, g, d_order, reinterpret_cast<signed char*>(d_lower),
                                    reinterpret_cast<signed char*>(d_upper), w.crit_counts, L.stream);
    unsigned long long h[6] = {0, 0, 0, 0, 0, 0};
    if (e == cudaSuccess) e = cudaMemcpyAsync(h, w.crit_counts, sizeof h, cudaMemcpyDeviceToHost, L.stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(L.stream);
    if (e != cudaSuccess) return cuda_fail(c, L, e, "classify");
    for (int i = 0; i < 6; ++i) counts[i] = (int64_t)h[i];
    return LTS_OK;
}

lts_status lts_simplify_persistence(lts_ctx* c, const lts_grid* gr, const float* d_field, double epsilon,
                                    lts_mode mode, float* d_out_field, int32_t* d_out_order, lts_stats* opt_stats) {
    if (!c) return LTS_ERR_ARG;
    c->err.clear();
    if (!(epsilon >= 0.0)) return fail(c, LTS_ERR_ARG, "epsilon must be a non-negative number");
    const Selection sel{nullptr, 0, true, epsilon};
    return simplify_one(c, gr, d_field, sel, mode, d_out_field, d_out_order, opt_stats);
}

lts_status lts_simplify_batch(lts_ctx* c, int32_t nf, const lts_grid* grids, const float* const* d_fields,
                              const int32_t* const* d_authorized, const int64_t* n_authorized, lts_mode mode,
                              float* const* d_out_fields, int32_t* const* d_out_orders, lts_stats* opt_stats) {
    if (!c) return LTS_ERR_ARG;
    c->err.clear();
    if (nf < 0) return fail(c, LTS_ERR_ARG, "negative field count");
    if (nf == 0) return LTS_OK;
    if (!grids || !d_fields || !d_authorized || !n_authorized || !d_out_fields || !d_out_orders)
        return fail(c, LTS_ERR_ARG, "null array argument");
    std::vector<long long> n(nf);
    long long nbig = 0;
    for (int i = 0; i < nf; ++i) {
        const lts_status st = check_field(c, &grids[i], c->lane[0].nmax, d_fields[i], d_authorized[i],
                                          n_authorized[i], mode, d_out_fields[i], d_out_orders[i], &n[i],
                                          "field " + std::to_string(i) + ": ");
        if (st != LTS_OK) return st;
        nbig = std::max(nbig, n[i]);
    }
    if (cudaSetDevice(c->device) != cudaSuccess) return fail(c, LTS_ERR_CUDA, "cudaSetDevice");
    cudaError_t e;
    // workspaces: the context's own, and up to kBatchLanes - 1 more sized for
    // the largest field, while the device has room for them (a batch runs on
    // as many as it could get; it needs at least one more than the context's
    // own when it has several fields)
    int want = std::min(c->tune.batch_workspaces > 0 ? c->tune.batch_workspaces : kBatchLanes, nf);
    const size_t per_lane = bytes_for(sizes_for(nbig, c->sms));
    for (int i = 1; i < want; ++i) {
        Lane& L = c->lane[i];
        if (L.nmax >= nbig) continue;
        if (L.stream) cudaStreamSynchronize(L.stream);
        lane_free(L);
        size_t fr = 0, tot = 0;
        lts_status st = LTS_ERR_OOM;
        cudaStream_t s;
        if (cudaMemGetInfo(&fr, &tot) == cudaSuccess && fr > per_lane + (1ull << 30)) {
            if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) {
                cudaGetLastError();
                return fail(c, LTS_ERR_CUDA, "cannot create a stream");
            }
            st = lane_alloc(L, nbig, c->sms, s, true, false);   // frees the lane and its stream on failure
        }
        cudaGetLastError();
        if (st != LTS_OK) {
            if (i == 1) return fail(c, LTS_ERR_OOM, "cannot allocate a batch workspace");
            want = i;
            break;
        }
    }
    c->nlanes = std::max(c->nlanes, want);
    if (!c->fork) {
        cudaEventCreateWithFlags(&c->fork, cudaEventDisableTiming);
        for (auto& j : c->join) cudaEventCreateWithFlags(&j, cudaEventDisableTiming);
    }
    if (c->batch_cap < nf) {
        if (c->batch_dev) cudaFree(c->batch_dev);
        if (c->batch_host) cudaFreeHost(c->batch_host);
        c->batch_dev = nullptr;
        c->batch_host = nullptr;
        c->batch_cap = 0;
        if (test_alloc_fails() || cudaMalloc((void**)&c->batch_dev, nf * sizeof(ReqResult)) != cudaSuccess ||
            cudaMallocHost((void**)&c->batch_host, nf * sizeof(ReqResult)) != cudaSuccess) {
            cudaGetLastError();
            return fail(c, LTS_ERR_OOM, "cannot allocate batch results");
        }
        c->batch_cap = nf;
    }
    for (int i = 0; i < want; ++i)
        if (c->lane[i].dirty) {
            if ((e = clean_workspace(c->lane[i])) != cudaSuccess) return cuda_fail(c, c->lane[i], e, "clean");
            c->lane[i].dirty = false;
        }
    // every lane starts after what the context's stream holds
    cudaStream_t s0 = c->lane[0].stream;
    cudaEventRecord(c->fork, s0);
    for (int i = 1; i < want; ++i) cudaStreamWaitEvent(c->lane[i].stream, c->fork, 0);
    // largest fields first, each to the least loaded lane
    std::vector<int> order(nf);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return n[a] > n[b]; });
    std::vector<long long> load(want, 0);
    std::vector<long long> launches(nf, 0);
    for (int i : order) {
        const int l = (int)(std::min_element(load.begin(), load.end()) - load.begin());
        load[l] += n[i];
        Lane& L = c->lane[l];
        const Geom g = geom_of(&grids[i], n[i]);
        const Selection sel{d_authorized[i], n_authorized[i], false, 0.0};
        tune_lane(c, L);
        if ((e = enqueue_simplify(L, g, d_fields[i], sel, mode, d_out_fields[i], d_out_orders[i], c->sms,
                                  c->batch_dev + i, 0)) != cudaSuccess)
            return cuda_fail(c, L, e, "launch");
        launches[i] = L.w.launches;
    }
    for (int i = 1; i < want; ++i) {
        cudaEventRecord(c->join[i], c->lane[i].stream);
        cudaStreamWaitEvent(s0, c->join[i], 0);
    }
    cudaMemcpyAsync(c->batch_host, c->batch_dev, nf * sizeof(ReqResult), cudaMemcpyDeviceToHost, s0);
    if ((e = cudaStreamSynchronize(s0)) != cudaSuccess) return cuda_fail(c, c->lane[0], e, "synchronize");
    int first_bad = -1;
    for (int i = 0; i < nf; ++i) {
        if (opt_stats) fill_stats(opt_stats[i], n[i], c->batch_host[i].ps, launches[i]);
        if (first_bad < 0 && c->batch_host[i].status != 0) first_bad = i;
    }
    if (first_bad >= 0) {
        const int status = c->batch_host[first_bad].status;
        return fail(c, (lts_status)status, "field " + std::to_string(first_bad) + ": " +
                                               status_text(status, c->batch_host[first_bad].oom_pool));
    }
    return LTS_OK;
}

lts_status lts_serve_config(lts_ctx* c, int32_t max_concurrent, int64_t hbm_budget_bytes) {
    if (!c) return LTS_ERR_ARG;
    c->err.clear();
    if (max_concurrent < 0 || max_concurrent > kMaxServe || hbm_budget_bytes < 0)
        return fail(c, LTS_ERR_ARG, "max_concurrent must be in [0, 15] and the budget non-negative");
    c->serve_max = max_concurrent;
    c->serve_budget = hbm_budget_bytes;
    return LTS_OK;
}

lts_status lts_submit(lts_ctx* c, const lts_grid* gr, const float* d_field, const int32_t* d_authorized,
                      int64_t n_authorized, lts_mode mode, float* d_out_field, int32_t* d_out_order,
                      uint64_t* ticket) {
    if (!c) return LTS_ERR_ARG;
    c->err.clear();
    if (!ticket) return fail(c, LTS_ERR_ARG, "null ticket");
    long long n;
    lts_status st = check_field(c, gr, c->lane[0].nmax, d_field, d_authorized, n_authorized, mode, d_out_field,
                                d_out_order, &n, "");
    if (st != LTS_OK) return st;
    if (cudaSetDevice(c->device) != cudaSuccess) return fail(c, LTS_ERR_CUDA, "cudaSetDevice");
    if ((st = ensure_ring(c)) != LTS_OK) return st;
    cudaError_t e;
    const unsigned long long t = c->next_ticket;
    const int li = pick_serve_lane(c, n);
    Lane& L = c->lane[li];
    if (L.dirty) {
        if ((e = clean_workspace(L)) != cudaSuccess) return cuda_fail(c, L, e, "clean");
        L.dirty = false;
    }
    const int slot = (int)(t % kRing);
    // the slot's previous request must be finished before the slot is reused
    if (t > kRing && (e = cudaEventSynchronize(c->ring_ev[slot])) != cudaSuccess) return cuda_fail(c, L, e, "wait");
    c->ring_host[slot].ticket = 0;
    if (li != 0) {
        // a serving workspace starts after what the caller enqueued on the context's stream
        if (!c->fork) {
            cudaEventCreateWithFlags(&c->fork, cudaEventDisableTiming);
            for (auto& j : c->join) cudaEventCreateWithFlags(&j, cudaEventDisableTiming);
        }
        cudaEventRecord(c->fork, c->lane[0].stream);
        cudaStreamWaitEvent(L.stream, c->fork, 0);
    }
    const Geom g = geom_of(gr, n);
    const Selection sel{d_authorized, n_authorized, false, 0.0};
    tune_lane(c, L);
    if ((e = enqueue_simplify(L, g, d_field, sel, mode, d_out_field, d_out_order, c->sms, c->ring_dev + slot, t)) !=
        cudaSuccess)
        return cuda_fail(c, L, e, "launch");
    if ((e = cudaEventRecord(c->ring_ev[slot], L.stream)) != cudaSuccess) return cuda_fail(c, L, e, "record");
    c->inflight[li].emplace_back(t, n);
    c->next_ticket = t + 1;
    *ticket = t;
    return LTS_OK;
}

lts_status lts_poll(lts_ctx* c, uint64_t ticket, int* done) {
    if (!c) return LTS_ERR_ARG;
    c->err.clear();
    if (!done) return fail(c, LTS_ERR_ARG, "null done flag");
    *done = 0;
    if (ticket == 0 || ticket >= c->next_ticket || !c->ring_ready) return fail(c, LTS_ERR_ARG, "unknown ticket");
    if (ticket + kRing < c->next_ticket) return fail(c, LTS_ERR_ARG, "ticket expired (its slot was reused)");
    const int slot = (int)(ticket % kRing);
    if (cudaSetDevice(c->device) != cudaSuccess) return fail(c, LTS_ERR_CUDA, "cudaSetDevice");
    const cudaError_t q = cudaEventQuery(c->ring_ev[slot]);
    if (q == cudaErrorNotReady) return LTS_OK;
    if (q != cudaSuccess) return cuda_fail(c, c->lane[0], q, "query");
    const volatile ReqResult* r = c->ring_host + slot;
    if (r->ticket != ticket) return fail(c, LTS_ERR_INTERNAL, "request result missing");
    *done = 1;
    const int status = r->status;
    if (status != 0) return fail(c, (lts_status)status, status_text(status, r->oom_pool));
    return LTS_OK;
}

}  // extern "C"
