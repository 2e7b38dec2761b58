// Step 1 with hill chains (Sec. 4.2 step 1, Sec. 4.3, Sec. 4.4): one
// superlevel set propagation per unauthorized maximum, all in one persistent
// kernel.
//
// Each lane runs one propagation (a "class") at a time.  Its priority queue
// is a binary max-heap of (Od, vertex) in the lane's slice of shared memory;
// when it outgrows that slice it moves to a block of an HBM pool and keeps
// growing there.  Popping v:
//   - v already in the class: skip;
//   - claim v (atomicCAS on owner[v]); the vertex log records every claim;
//   - k = higher neighbours of v in the class, h = all higher neighbours;
//     k == h: v is regular for the class, push its lower neighbours;
//   - otherwise v is a saddle for the class (an arrival): the class links
//     itself into v's wait list (headed by the class that claimed v), copies
//     its queue to the spill pool, and adds k to the arrival counter of v.
//     The arrival that brings the counter to h is the last one: it unites
//     every class waiting at v with itself (union-find), melds their spilled
//     queues into its own and continues below v.  Any other arrival stops.
// A class thus only passes a saddle once every higher neighbour belongs to a
// class that has arrived there, so the regions do not depend on the order in
// which lanes run.  Nothing here waits on another lane: a stopped class just
// ends its task, and the kernel ends when every seed has been taken.
#include "lts_internal.cuh"

namespace lts {

namespace {

constexpr int kThreads = 128;
constexpr int kHCap = 32;          // shared-memory queue entries per lane
constexpr int kSeedBatch = 2;
constexpr int kLogChunk = 64;
constexpr int kSpillChunk = 256;

struct PropArgs {
    const int* U;
    int* owner;
    unsigned long long* qmark;   // (pass tag << 32 | class) of the last class that queued the vertex
    unsigned long long tag;      // this pass's tag, in the high 32 bits
    int* parent;
    int* wait_v;
    int* cnt;
    int* listhead;
    int* next_w;
    int* spill_base;
    int* spill_n;
    int* spill_pool;
    long long spill_cap;
    unsigned long long* heap_pool;
    long long heap_cap;
    int* vlog;
    long long log_cap;
    DevCounters* ctr;
};

// A lane's priority queue: in its shared-memory slice (stride = block size)
// until it outgrows it, then in an HBM block that the lane keeps for its
// later propagations and enlarges when needed.
struct Heap {
    unsigned long long* h;
    int n, cap, stride;
    unsigned long long* gblk;    // the lane's HBM block (or null)
    int gcap;
};

__device__ __forceinline__ unsigned long long& at(Heap& H, int i) { return H.h[(long long)i * H.stride]; }

// Union-find root with path halving; parent links only ever point to
// ancestors, so the benign races of halving keep every path valid.
__device__ __forceinline__ int find_root(int* parent, int x) {
    for (;;) {
        int p = __ldcg(parent + x);
        if (p == x) return x;
        int gp = __ldcg(parent + p);
        if (gp == p) return p;
        __stcg(parent + x, gp);
        x = gp;
    }
}

__device__ __forceinline__ bool in_class(int* parent, int ow, int c) {
    return ow >= 0 && (ow == c || find_root(parent, ow) == c);
}

__device__ bool heap_grow(Heap& H, const PropArgs& a) {
    if (H.gblk == nullptr || H.gcap <= H.cap) {
        const int ncap = max(4 * H.cap, 256);
        const long long off = atomicAdd((unsigned long long*)&a.ctr->heap_cursor, (unsigned long long)ncap);
        if (off + ncap > a.heap_cap) { set_status(&a.ctr->status, LTS_ERR_OOM); return false; }
        H.gblk = a.heap_pool + off;
        H.gcap = ncap;
    }
    if (H.stride != 1) atomicAdd(&a.ctr->heap_spills, 1);
    for (int i = 0; i < H.n; ++i) H.gblk[i] = at(H, i);   // forward copy: safe within the same block
    H.h = H.gblk; H.cap = H.gcap; H.stride = 1;
    return true;
}

__device__ __forceinline__ bool heap_push(Heap& H, unsigned long long e, const PropArgs& a) {
    if (H.n == H.cap && !heap_grow(H, a)) return false;
    int i = H.n++;
    while (i > 0) {
        const int p = (i - 1) >> 1;
        const unsigned long long pe = at(H, p);
        if (pe >= e) break;
        at(H, i) = pe;
        i = p;
    }
    at(H, i) = e;
    return true;
}

__device__ __forceinline__ unsigned long long heap_pop(Heap& H) {
    const unsigned long long top = at(H, 0);
    const int n = --H.n;
    if (n == 0) return top;
    const unsigned long long last = at(H, n);
    int i = 0;
    for (;;) {
        const int l = 2 * i + 1;
        if (l >= n) break;
        int c = l;
        unsigned long long ce = at(H, l);
        if (l + 1 < n) {
            const unsigned long long re = at(H, l + 1);
            if (re > ce) { c = l + 1; ce = re; }
        }
        if (ce <= last) break;
        at(H, i) = ce;
        i = c;
    }
    at(H, i) = last;
    return top;
}

// Queue vertex u (order ou) for class c unless c queued it already.
__device__ __forceinline__ bool enqueue(Heap& H, const PropArgs& a, int u, int ou, int c) {
    const unsigned long long mark = a.tag | (unsigned)c;
    if (__ldcg(a.qmark + u) == mark) return true;
    __stcg(a.qmark + u, mark);
    return heap_push(H, ((unsigned long long)ou << 32) | (unsigned)u, a);
}

template <int DIR>
__global__ void __launch_bounds__(kThreads) propagate_kernel(Geom g, const int* __restrict__ O, PropArgs a) {
    extern __shared__ unsigned long long sheap[];
    DevCounters* ctr = a.ctr;
    int* st = &ctr->status;
    if (failed(st)) return;
    const int nU = *(volatile int*)&ctr->n_unauth;
    if (nU > 0 && *(volatile int*)&ctr->n_auth_ext == 0) { set_status(st, LTS_ERR_NO_AUTHORIZED); return; }

    unsigned long long* const myslice = sheap + threadIdx.x;   // interleaved: entry i at [i * kThreads]
    int seed_lo = 0, seed_hi = 0;
    long long log_pos = 0, log_end = 0;
    long long sp_pos = 0, sp_end = 0;
    Heap H{myslice, 0, kHCap, kThreads, nullptr, 0};

    for (;;) {
        if (seed_lo == seed_hi) {
            const int b = atomicAdd(&ctr->seed_cursor, kSeedBatch);
            if (b >= nU) break;
            seed_lo = b;
            seed_hi = min(b + kSeedBatch, nU);
        }
        int c = seed_lo++;
        H.h = myslice; H.n = 0; H.cap = kHCap; H.stride = kThreads;
        {
            const int m = __ldg(a.U + c);
            enqueue(H, a, m, od<DIR>(__ldg(O + m), g.n), c);
        }
        for (;;) {                                   // run class c until it stops at a saddle
            if (H.n == 0) { set_status(st, LTS_ERR_INTERNAL); goto bail; }
            const unsigned long long e = heap_pop(H);
            const int v = (int)(e & 0xffffffffu);
            const int kv = (int)(e >> 32);
            int o = __ldcg(a.owner + v);
            if (in_class(a.parent, o, c)) continue;
            bool claimed = false;
            if (o < 0) {
                const int prev = atomicCAS(a.owner + v, -1, c);
                if (prev == -1) {
                    claimed = true;
                    o = c;
                    if (log_pos == log_end) {
                        log_pos = atomicAdd(&ctr->log_cursor, kLogChunk);
                        log_end = log_pos + kLogChunk;
                        if (log_end > a.log_cap) { log_pos = log_end = 0; set_status(st, LTS_ERR_OOM); goto bail; }
                    }
                    a.vlog[log_pos++] = v;
                } else {
                    o = prev;
                    if (in_class(a.parent, o, c)) continue;
                }
            }
            int x, y, z;
            coords_of(g, v, x, y, z);
            int nbv[14], nbo[14];
            int h = 0, k = 0;
            for (int q = 0; q < g.nn; ++q) {
                const int nb = nbr_of(g, x, y, z, q);
                nbv[q] = nb;
                if (nb < 0) continue;
                const int onb = od<DIR>(__ldg(O + nb), g.n);
                nbo[q] = onb;
                if (onb > kv) {
                    ++h;
                    if (in_class(a.parent, __ldcg(a.owner + nb), c)) ++k;
                }
            }
            if (k == h) {                            // regular for this class
                for (int q = 0; q < g.nn; ++q) {
                    const int nb = nbv[q];
                    if (nb < 0 || nbo[q] > kv) continue;
                    if (in_class(a.parent, __ldcg(a.owner + nb), c)) continue;
                    if (!enqueue(H, a, nb, nbo[q], c)) goto bail;
                }
                continue;
            }
            // ---- arrival at the saddle v ----
            const int head = claimed ? c : o;
            if (!claimed) {
                const int old = atomicExch(a.listhead + head, c);
                __stcg(a.next_w + c, old);
            }
            // the queue must be readable by whoever releases this class
            if (sp_end - sp_pos < H.n) {
                const int want = max(H.n, kSpillChunk);
                sp_pos = atomicAdd(&ctr->spill_cursor, want);
                sp_end = sp_pos + want;
                if (sp_end > a.spill_cap) { set_status(st, LTS_ERR_OOM); goto bail; }
            }
            for (int i = 0; i < H.n; ++i) __stcg(a.spill_pool + sp_pos + i, (int)(at(H, i) & 0xffffffffu));
            __stcg(a.spill_base + c, (int)sp_pos);
            __stcg(a.spill_n + c, H.n);
            sp_pos += H.n;
            __stcg(a.wait_v + c, v);
            __threadfence();
            const int tot = atomicAdd(a.cnt + head, k) + k;
            if (tot < h) break;                      // a higher neighbour is still unvisited: stop
            // ---- last arrival: merge every class stopped at v ----
            __threadfence();
            int cur = head;
            bool first = true;
            while (cur >= 0) {
                if (cur != c) {
                    __stcg(a.parent + cur, c);
                    const int sb = __ldcg(a.spill_base + cur), sn = __ldcg(a.spill_n + cur);
                    for (int i = 0; i < sn; ++i) {
                        const int u = __ldcg(a.spill_pool + sb + i);
                        if (!enqueue(H, a, u, od<DIR>(__ldg(O + u), g.n), c)) goto bail;
                    }
                }
                cur = first ? __ldcg(a.listhead + head) : __ldcg(a.next_w + cur);
                first = false;
            }
            __stcg(a.wait_v + c, -1);
            if (head == c) { __stcg(a.cnt + c, 0); __stcg(a.listhead + c, -1); }
            __threadfence();
            for (int q = 0; q < g.nn; ++q) {         // v now belongs to c: continue below it
                const int nb = nbv[q];
                if (nb < 0 || nbo[q] > kv) continue;
                if (in_class(a.parent, __ldcg(a.owner + nb), c)) continue;
                if (!enqueue(H, a, nb, nbo[q], c)) goto bail;
            }
        }
    }
bail:
    // every reserved log slot must hold a vertex or -1
    while (log_pos < log_end) a.vlog[log_pos++] = -1;
}

}  // namespace

template <int DIR>
cudaError_t propagate(Work& w, const Geom& g, const int* O, int sms, cudaStream_t s) {
    PropArgs a;
    a.U = w.U; a.owner = w.owner; a.qmark = w.qmark; a.tag = (unsigned long long)(++w.pass_tag) << 32;
    a.parent = w.parent; a.wait_v = w.wait_v; a.cnt = w.cnt;
    a.listhead = w.listhead; a.next_w = w.next_w; a.spill_base = w.spill_base; a.spill_n = w.spill_n;
    a.spill_pool = w.spill_pool; a.spill_cap = w.spill_cap; a.heap_pool = w.heap_pool; a.heap_cap = w.heap_cap;
    a.vlog = w.vlog; a.log_cap = w.log_cap; a.ctr = w.ctr;
    const size_t smem = (size_t)kThreads * kHCap * sizeof(unsigned long long);
    const int blocks = w.lanes / kThreads;
    propagate_kernel<DIR><<<blocks, kThreads, smem, s>>>(g, O, a);
    w.launches += 1;
    return cudaGetLastError();
}

int propagate_lanes(int sms) { return sms * 6 * kThreads; }
long long propagate_log_slack(int lanes) { return (long long)lanes * kLogChunk; }
long long propagate_spill_slack(int lanes) { return (long long)lanes * kSpillChunk; }
long long propagate_heap_slack(int lanes) { return (long long)lanes * 512; }

template cudaError_t propagate<1>(Work&, const Geom&, const int*, int, cudaStream_t);
template cudaError_t propagate<-1>(Work&, const Geom&, const int*, int, cudaStream_t);

}  // namespace lts
