// Internal declarations shared by the CUDA translation units of the library.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "lts.h"

namespace lts {

// ---------------------------------------------------------------------------
// Grid geometry: Freudenthal neighbours are the offsets in {0,1}^d and
// -{0,1}^d.  Offset k < nn/2 is the k+1-th non-zero 0/1 vector (bit b = axis b)
// and offset k + nn/2 its negative.
// ---------------------------------------------------------------------------
// Division by a run-time constant d >= 2 as a multiply-high and shifts
// (the round-up method of Granlund and Montgomery, exact for every 32-bit
// unsigned numerator): l = ceil(log2 d), m = floor(2^32 (2^l - d) / d) + 1,
// q = (t + ((n - t) >> 1)) >> (l - 1) with t = mulhi(m, n).
struct FastDiv {
    unsigned d, m, l;
};

inline FastDiv make_fastdiv(unsigned d) {
    FastDiv f;
    f.d = d;
    unsigned l = 0;
    while ((1ull << l) < d) ++l;
    f.l = l;
    f.m = (unsigned)(((1ull << 32) * ((1ull << l) - d)) / d + 1);
    return f;
}

__device__ __forceinline__ unsigned fdiv(unsigned n, const FastDiv& f) {
    const unsigned t = __umulhi(f.m, n);
    return (t + ((n - t) >> 1)) >> (f.l - 1);
}

struct Geom {
    int ndim;
    int nn;            // 6 or 14
    int X, Y, Z;       // Z = 1 in 2D
    int n;             // X*Y*Z
    int XY;
    FastDiv dX, dXY;
};

// Neighbour k of (x,y,z): returns its id, or -1 outside the grid.
__device__ __forceinline__ int nbr_of(const Geom& g, int x, int y, int z, int k) {
    const int half = g.nn >> 1;
    const int m = (k < half ? k : k - half) + 1;
    const int s = k < half ? 1 : -1;
    const int dx = (m & 1) * s, dy = ((m >> 1) & 1) * s, dz = ((m >> 2) & 1) * s;
    const int a = x + dx, b = y + dy, c = z + dz;
    if ((unsigned)a >= (unsigned)g.X || (unsigned)b >= (unsigned)g.Y || (unsigned)c >= (unsigned)g.Z) return -1;
    return a + g.X * b + g.XY * c;
}

__device__ __forceinline__ void coords_of(const Geom& g, int v, int& x, int& y, int& z) {
    z = (int)fdiv((unsigned)v, g.dXY);
    const int r = v - z * g.XY;
    y = (int)fdiv((unsigned)r, g.dX);
    x = r - y * g.X;
}

// Pass-oriented order: the maxima pass works on O, the minima pass on N-1-O,
// so that every pass treats maxima.
template <int DIR>
__device__ __forceinline__ int od(int o, int n) { return DIR > 0 ? o : n - 1 - o; }

// ---------------------------------------------------------------------------
// Device status word: the first error wins.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void set_status(int* st, int code) { atomicCAS(st, 0, code); }
__device__ __forceinline__ bool failed(const int* st) { return *(volatile const int*)st != 0; }

// Bounded spin budget for every device-side wait on another block.
constexpr long long kSpinLimit = 1LL << 26;
// The budget of the test-only wait that nothing ends (LTS_TEST_STALL_SORT).
constexpr long long kTestSpinLimit = 1LL << 14;

// Scalars produced and consumed on the device, read back once per call.
struct DevCounters {
    int status;
    int oom_pool;          // the pool that ran out: 1 overflow heap, 2 spill, 3 vertex log
    int n_unauth;          // |U| of the current pass
    int n_auth_ext;        // authorized extrema present in the current pass
    int n_regions;
    int n_saddles;         // distinct saddles (head regions)
    int log_cursor;        // visited-vertex log length (chunk reserved)
    int seed_cursor;
    long long spill_cursor; // spill pool (ints)
    long long heap_cursor; // lane heap pool (entries)
    int max_region;
    int max_floods;
    long long region_vertices;
    long long total_floods;
    int heap_spills;
    int n_t16;             // regions for the 16-lane team tier of step 2 (3 <= r <= 16)
    int n_t32;             // regions for the 32-lane team tier of step 2
    int n_med;             // regions for the small dense warp tier of step 2
    int n_large;           // regions for the large dense warp tier of step 2
    int n_huge;            // regions for the 4096-vertex dense warp tier of step 2
    int n_big;             // regions for the HBM tier of step 2
    int n_tasks;           // propagation tasks left after the first step
    long long lo_adj_cursor; // local adjacency pool of the largest local-order tier (ints)
    int lo_fallbacks;      // regions step 2 redid with every boundary vertex as a seed
    int n_rs_regions;      // regions with swallowed authorized extrema (restoration)
    long long n_restored;  // swallowed authorized extrema restored
};

__device__ __forceinline__ void set_oom(DevCounters* ctr, int pool) {
    atomicCAS(&ctr->oom_pool, 0, pool);
    set_status(&ctr->status, LTS_ERR_OOM);
}

// Per-pass statistics accumulated into the host stats.
struct PassStats {
    long long removed, regions, region_vertices, max_region, max_floods, total_floods, heap_spills, fallbacks, restored;
};

// Rank-space block of 32 ranks (16 bytes, one vector load): members and
// saddles present, and the counts of members and saddles before the block.
struct __align__(16) RankBlk {
    unsigned int mmask;
    unsigned int smask;
    unsigned int mpre;
    unsigned int spre;
};
constexpr int kRankShift = 5;

// ---------------------------------------------------------------------------
// Workspace (all device memory, sized for max_vertices).
// ---------------------------------------------------------------------------
struct Work {
    int nmax;
    int max_tiles;
    // order field (radix sort)
    unsigned int* keyA; unsigned int* valA; unsigned int* keyB; unsigned int* valB;
    unsigned long long* sort_status;     // tiles x 256 look-back words
    unsigned int* sort_hist;             // 8 x 256 (digits of a 64-bit key; 4 for float32 fields)
    unsigned int* sort_offsets;          // 8 x 256
    unsigned int* tile_counter;          // 4
    unsigned int* bin_cursor;            // id bins of the last radix pass
    unsigned int* dk_keys; unsigned int* dk_cnts; unsigned int* dk_rank;   // distinct keys (hash table)
    unsigned int* dk_info;               // distinct count, overflow flag, two-pass mode
    unsigned int epoch;
    // authorized bitmap
    unsigned int* authbits;              // ceil(n/32)
    // propagation
    int* owner;                          // per vertex: class, region tag, or -1
    int* qmark;                          // per vertex: the last class that queued it (-1 after a clear)
    int* loc;                            // per vertex: local index within its region
    int* U;                              // unauthorized extrema
    int* parent; int* wait_v;            // per class
    int2* ctop;                          // per class: highest extremum and its Od (persistence-driven selection)
    int* sib_head; int* sib_next;        // per class: regions listed under the claimer of their saddle
    int4* tasks;                         // propagation tasks after the first step
    int* cnt;                            // per vertex: arrival counter of a saddle
    int* spill_base; int* spill_n; int4* heaprec;
    int* spill_pool; long long spill_cap;
    unsigned long long* heap_pool; long long heap_cap;
    int* vlog; long long log_cap;
    int* vlog_cls;                       // per log entry: the class that claimed the vertex
    int* ent_rid; int* ent_loc; int* ent_od;   // per log entry: region, local index, Od (regions stage)
    int* cls2rid;                        // per class: region of its root, -1 if none
    // regions
    int* class2reg; int* reg_class; int* reg_saddle; int* reg_size; int* reg_start;
    int* reg_top; int* reg_sod; int* reg_place; int* reg_head; int* reg_att;
    int* reg_swallowed;                  // per region: swallowed authorized extrema (restoration)
    int* members; int* lhat; int* member_reg;   // CSR members, their local order, their region
    int* tier_list;                      // [0,cap): 16-lane tier; then quarters of cap: 32-lane, dense <=128, dense <=1024, HBM
    // local-order scratch (slots: members + one saddle per region)
    int* lo_v; int* lo_L; int* lo_L2; int* lo_heap; unsigned char* lo_flag; int* lo_P;
    int* lo_adj; long long lo_adj_cap;   // local adjacency of the largest regions (bump pool)
    long long lo_cap;
    // the local-order tiers run side by side: three more streams, forked from
    // and joined back to the workspace's stream with events (the context's own
    // workspace only: batches and served requests overlap whole fields)
    bool aux_on;
    cudaStream_t aux[4];                 // [0..2] local-order tiers, [3] the reorder's rank prefix
    cudaEvent_t fork_ev, join_ev[3], pre_fork, pre_join;
    // reorder
    RankBlk* rblk; int nblk; int nblk_cur;
    int* sad_att; int* cumA;
    // scans
    unsigned long long* scan_tmp; int scan_tmp_cap;
    // counters
    DevCounters* ctr;
    PassStats* pstats;                   // [0] minima pass, [1] maxima pass
    DevCounters* h_ctr;                  // pinned host copy (followed by two PassStats)
    int min_tier;                        // tests only: step-2 regions go to at least this tier (0: by size)
    const unsigned long long* test_stall; // tests only: look-back words nothing sets, or null
    int sms;                             // multiprocessors of the workspace's device
    int eng_bpsm;                        // resident blocks per SM of the propagation engine
    int team_bpsm;                       // blocks per SM of the local-order team kernels
    unsigned char* link6; unsigned char* link14;   // link component tables of interior vertices (2D, 3D)
    unsigned long long* crit_counts;     // critical point counts of lts_classify
    int lanes;                           // propagation lanes (threads)
    int class_cap;                       // capacity of the class and region arrays
    long long launches;                  // kernels launched by the current call
};

// ---- launch helpers (defined in the .cu files) ----
cudaError_t order_field(Work& w, const Geom& g, const float* f, float* gout, int* O, cudaStream_t s);
cudaError_t order_field_f64(Work& w, const Geom& g, const double* f, double* gout, int* O, cudaStream_t s);
cudaError_t build_authbits(Work& w, const Geom& g, const int* ids, long long nids, cudaStream_t s);
template <int DIR>
cudaError_t classify(Work& w, const Geom& g, const int* O, cudaStream_t s);
template <int DIR>
cudaError_t propagate(Work& w, const Geom& g, const int* O, int sms, cudaStream_t s);
template <int DIR>
cudaError_t select_persistent(Work& w, const Geom& g, const int* O, const float* F, double eps, int sms,
                              cudaStream_t s);
template <int DIR>
cudaError_t extract_regions(Work& w, const Geom& g, const int* O, int sms, cudaStream_t s);
template <int DIR>
cudaError_t local_orders(Work& w, const Geom& g, const int* O, int sms, cudaStream_t s);
template <int DIR>
cudaError_t restore_swallowed(Work& w, const Geom& g, const int* O, int sms, cudaStream_t s);
cudaError_t reorder_prefix(Work& w, const Geom& g, int sms, cudaStream_t s);
cudaError_t build_link_tables(unsigned char* t6, unsigned char* t14, cudaStream_t s);
cudaError_t critical_points(Work& w, const Geom& g, const int* O, signed char* lower, signed char* upper,
                            unsigned long long* d_counts, cudaStream_t s);
template <int DIR>
cudaError_t reorder_flatten(Work& w, const Geom& g, int* O, void* gout, bool f64, int sms, cudaStream_t s);
cudaError_t pass_reset(Work& w, cudaStream_t s);
int local_order_tiny_max();
int local_order_med_max();
int local_order_huge_max();

// warp-level reductions before one atomic (all 32 lanes must call)
__device__ __forceinline__ void warp_atomic_max(int* dst, int v) {
    v = __reduce_max_sync(0xffffffffu, v);
    if ((threadIdx.x & 31) == 0 && v > 0) atomicMax(dst, v);
}
__device__ __forceinline__ void warp_atomic_add(int* dst, int v) {
    v = __reduce_add_sync(0xffffffffu, v);
    if ((threadIdx.x & 31) == 0 && v) atomicAdd(dst, v);
}
__device__ __forceinline__ void warp_atomic_add64(long long* dst, long long v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0 && v) atomicAdd((unsigned long long*)dst, (unsigned long long)v);
}

// device-wide exclusive scan of `count` values (count read on the device)
cudaError_t scan_excl_i32(Work& w, const int* in, int* out, const int* d_count, int max_count,
                          cudaStream_t s);

}  // namespace lts
