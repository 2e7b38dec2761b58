// Step 1 with hill chains (Sec. 4.2 step 1, Sec. 4.3, Sec. 4.4): one
// superlevel set propagation per unauthorized maximum, all in one persistent
// kernel.
//
// Each propagation (a "class") is run by a team of lanes (a whole warp, so
// that no two propagations share an instruction stream): lane q handles neighbour q of the
// popped vertex, so the loads of all neighbours go out in one round trip and
// every branch is uniform within the team.  The priority queue of the class
// is a top-K frontier in the team's registers (E slots per lane), popped with
// a team max-reduction; entries that do not fit go to a per-team binary heap
// in an HBM pool.  Popping v:
//   - v already in the class: skip;
//   - claim v (atomicCAS on owner[v]); the vertex log records every claim;
//   - k = higher neighbours of v in the class, h = all higher neighbours;
//     k == h: v is regular for the class, queue its lower neighbours;
//   - otherwise v is a saddle for the class (an arrival): the class links
//     itself into v's wait list (headed by the class that claimed v), copies
//     its queue to the spill pool, and adds k to the arrival counter of v.
//     The arrival that brings the counter to h is the last one: it unites
//     every class waiting at v with itself (union-find), melds their spilled
//     queues into its own and continues below v.  Any other arrival stops.
// A class thus only passes a saddle once every higher neighbour belongs to a
// class that has arrived there, so the regions do not depend on the order in
// which teams run.  Nothing here waits on another team: a stopped class just
// ends its task, and the kernel ends when every seed has been taken.
// Decisions that read shared mutable state (owner[], parent[]) are taken by
// one lane and broadcast, so a team never diverges.
#include <climits>

#include <cuda/atomic>

#include "lts_internal.cuh"

namespace lts {

namespace {

constexpr int kThreads = 128;
constexpr int kSeedBatch = 16;
constexpr int kLogChunk = 64;
constexpr int kSpillChunk = 4096;

template <int NN> struct TeamCfg;
template <> struct TeamCfg<14> { static constexpr int TS = 32; static constexpr int E = 4; };
template <> struct TeamCfg<6> { static constexpr int TS = 32; static constexpr int E = 4; };

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

// Neighbour q of (x,y,z) for a compile-time neighbour count NN.
template <int NN>
__device__ __forceinline__ int nbr_q(const Geom& g, int x, int y, int z, int q) {
    constexpr int half = NN / 2;
    const int m = (q < half ? q : q - half) + 1;
    const int sgn = q < half ? 1 : -1;
    const int a = x + (m & 1) * sgn, b = y + ((m >> 1) & 1) * sgn, c = z + ((m >> 2) & 1) * sgn;
    if ((unsigned)a >= (unsigned)g.X || (unsigned)b >= (unsigned)g.Y || (unsigned)c >= (unsigned)g.Z) return -1;
    return a + g.X * b + g.XY * c;
}

__device__ __forceinline__ unsigned long long pack(int key, int v) {
    return ((unsigned long long)(unsigned)key << 32) | (unsigned)v;
}

// The overflow heap of a team (binary max-heap in HBM), used by lane 0 only.
struct Overflow {
    unsigned long long* h;
    int n, cap;
};

__device__ bool ov_push(Overflow& H, unsigned long long e, const PropArgs& a) {
    if (H.n == H.cap) {
        const int ncap = max(4 * H.cap, 256);
        const long long off = atomicAdd((unsigned long long*)&a.ctr->heap_cursor, (unsigned long long)ncap);
        if (off + ncap > a.heap_cap) { set_status(&a.ctr->status, LTS_ERR_OOM); return false; }
        unsigned long long* nh = a.heap_pool + off;
        for (int i = 0; i < H.n; ++i) nh[i] = H.h[i];
        if (H.cap == 0) atomicAdd(&a.ctr->heap_spills, 1);
        H.h = nh;
        H.cap = ncap;
    }
    int i = H.n++;
    while (i > 0) {
        const int p = (i - 1) >> 1;
        const unsigned long long pe = H.h[p];
        if (pe >= e) break;
        H.h[i] = pe;
        i = p;
    }
    H.h[i] = e;
    return true;
}

__device__ unsigned long long ov_pop(Overflow& H) {
    const unsigned long long top = H.h[0];
    const int n = --H.n;
    if (n == 0) return top;
    const unsigned long long last = H.h[n];
    int i = 0;
    for (;;) {
        const int l = 2 * i + 1;
        if (l >= n) break;
        int c = l;
        unsigned long long ce = H.h[l];
        if (l + 1 < n && H.h[l + 1] > ce) { c = l + 1; ce = H.h[l + 1]; }
        if (ce <= last) break;
        H.h[i] = ce;
        i = c;
    }
    H.h[i] = last;
    return top;
}

template <int NN>
struct TeamState {
    static constexpr int TS = TeamCfg<NN>::TS;
    static constexpr int E = TeamCfg<NN>::E;
    int sk[E];        // frontier slots: key (Od), -1 = empty
    int sv[E];        //                 vertex
    int rot;          // rotation of the slot assignment (spreads entries over lanes)
    unsigned tmask;
    int tb, lane;
    Overflow ov;      // meaningful in team lane 0
    int ovn;          // uniform copy of ov.n
    int ov_top;       // uniform: key on top of the overflow heap, -1 if empty
};

template <int NN>
__device__ __forceinline__ void ov_sync(TeamState<NN>& T) {
    int n = T.ov.n;
    int top = n > 0 ? (int)(T.ov.h[0] >> 32) : -1;
    T.ovn = __shfl_sync(T.tmask, n, T.tb);
    T.ov_top = __shfl_sync(T.tmask, top, T.tb);
}

// Adds one candidate per lane (has, key, vert) to the team frontier.
// Returns false (uniformly) if the overflow pool is exhausted.
template <int NN>
__device__ bool insert_batch(TeamState<NN>& T, bool has, int key, int vert, const PropArgs& a) {
    constexpr int TS = TeamState<NN>::TS, E = TeamState<NN>::E;
    const int tl = T.lane - T.tb;
    const int src = T.tb + ((tl - T.rot) & (TS - 1));
    const bool hc = __shfl_sync(T.tmask, has, src);
    const int ck = __shfl_sync(T.tmask, key, src);
    const int cv = __shfl_sync(T.tmask, vert, src);
    T.rot = (T.rot + NN) & (TS - 1);
    bool need = false;
    if (hc) {
        bool placed = false;
#pragma unroll
        for (int e = 0; e < E; ++e)
            if (!placed && T.sk[e] < 0) { T.sk[e] = ck; T.sv[e] = cv; placed = true; }
        need = !placed;
    }
    unsigned um = __ballot_sync(T.tmask, need);
    bool ok = true;
    while (um) {
        const int L = __ffs(um) - 1;
        um &= um - 1;
        const int k2 = __shfl_sync(T.tmask, ck, L);
        const int v2 = __shfl_sync(T.tmask, cv, L);
        bool free_here = false;
#pragma unroll
        for (int e = 0; e < E; ++e) free_here |= T.sk[e] < 0;
        const unsigned fm = __ballot_sync(T.tmask, free_here);
        if (fm) {
            if (T.lane == __ffs(fm) - 1) {
                bool placed = false;
#pragma unroll
                for (int e = 0; e < E; ++e)
                    if (!placed && T.sk[e] < 0) { T.sk[e] = k2; T.sv[e] = v2; placed = true; }
            }
            continue;
        }
        // the frontier is full: the smallest of (team minimum, candidate) goes to HBM
        int mk = INT_MAX, ms = 0;
#pragma unroll
        for (int e = 0; e < E; ++e)
            if (T.sk[e] < mk) { mk = T.sk[e]; ms = e; }
        const int MK = __reduce_min_sync(T.tmask, mk);
        unsigned long long out;
        if (k2 < MK) {
            out = pack(k2, v2);
        } else {
            const int M = __ffs(__ballot_sync(T.tmask, mk == MK)) - 1;
            int ev = 0;
#pragma unroll
            for (int e = 0; e < E; ++e)
                if (e == ms) ev = T.sv[e];
            ev = __shfl_sync(T.tmask, ev, M);
            if (T.lane == M) {
#pragma unroll
                for (int e = 0; e < E; ++e)
                    if (e == ms) { T.sk[e] = k2; T.sv[e] = v2; }
            }
            out = pack(MK, ev);
        }
        int r = 1;
        if (T.lane == T.tb) r = ov_push(T.ov, out, a) ? 1 : 0;
        r = __shfl_sync(T.tmask, r, T.tb);
        ov_sync(T);
        if (!r) { ok = false; break; }
    }
    return ok;
}

template <int DIR, int NN>
__global__ void __launch_bounds__(kThreads, 12) propagate_kernel(Geom g, const int* __restrict__ O, PropArgs a) {
    constexpr int TS = TeamCfg<NN>::TS, E = TeamCfg<NN>::E;
    DevCounters* ctr = a.ctr;
    int* st = &ctr->status;
    if (failed(st)) return;
    const int nU = *(volatile int*)&ctr->n_unauth;
    if (nU > 0 && *(volatile int*)&ctr->n_auth_ext == 0) {
        if (threadIdx.x == 0) set_status(st, LTS_ERR_NO_AUTHORIZED);
        return;
    }
    TeamState<NN> T;
    T.lane = threadIdx.x & 31;
    T.tb = T.lane & ~(TS - 1);
    T.tmask = (TS == 32) ? 0xffffffffu : (((1u << TS) - 1u) << T.tb);
    const int tl = T.lane - T.tb;
    const bool leader = tl == 0;
    T.rot = 0;
    T.ov.h = nullptr; T.ov.n = 0; T.ov.cap = 0;
    T.ovn = 0; T.ov_top = -1;
#pragma unroll
    for (int e = 0; e < E; ++e) { T.sk[e] = -1; T.sv[e] = 0; }

    // team-leader state
    int seed_lo = 0, seed_hi = 0;
    long long log_pos = 0, log_end = 0;
    long long sp_pos = 0, sp_end = 0;
    int c = -1;
    bool merged = false;     // c has absorbed other classes: membership needs find_root

    for (;;) {
        if (c < 0) {                                   // take the next seed
            int nc = -1;
            if (leader) {
                if (seed_lo == seed_hi) {
                    // guided batches: large while many seeds remain, single ones at the end
                    const int rem = nU - *(volatile int*)&ctr->seed_cursor;
                    const int nwarps = gridDim.x * (blockDim.x / 32);
                    const int bsz = max(1, min(kSeedBatch, rem / (4 * nwarps)));
                    const int b = atomicAdd(&ctr->seed_cursor, bsz);
                    seed_lo = b;
                    seed_hi = min(b + bsz, nU);
                }
                if (seed_lo < seed_hi && !failed(st)) nc = seed_lo++;
            }
            nc = __shfl_sync(T.tmask, nc, T.tb);
            if (nc < 0) break;
            c = nc;
            merged = false;
#pragma unroll
            for (int e = 0; e < E; ++e) T.sk[e] = -1;
            T.ov.n = 0; T.ovn = 0; T.ov_top = -1;
            // The seed is a maximum: no other class can reach it (classes only queue
            // lower neighbours) and all its neighbours are lower, so it is claimed
            // with a plain store and every neighbour is queued at once.
            const int m = __ldg(a.U + c);
            int okl = 1;
            if (leader) {
                __stcg(a.owner + m, c);
                if (log_pos == log_end) {
                    log_pos = atomicAdd(&ctr->log_cursor, kLogChunk);
                    log_end = log_pos + kLogChunk;
                    if (log_end > a.log_cap) { log_pos = log_end = 0; set_status(st, LTS_ERR_OOM); okl = 0; }
                }
                if (okl) a.vlog[log_pos++] = m;
            }
            if (!__shfl_sync(T.tmask, okl, T.tb)) break;
            int mx, my, mz;
            coords_of(g, m, mx, my, mz);
            const int mnb = tl < NN ? nbr_q<NN>(g, mx, my, mz, tl) : -1;
            const unsigned long long mk = a.tag | (unsigned)c;
            int mo = 0;
            if (mnb >= 0) {
                mo = od<DIR>(__ldg(O + mnb), g.n);
                __stcg(a.qmark + mnb, mk);
            }
            if (!insert_batch(T, mnb >= 0, mo, mnb, a)) break;
        }
        const unsigned long long mark = a.tag | (unsigned)c;
        // ---- pop the highest queued vertex ----
        int bk = -1, bs = 0;
#pragma unroll
        for (int e = 0; e < E; ++e)
            if (T.sk[e] > bk) { bk = T.sk[e]; bs = e; }
        const int K = __reduce_max_sync(T.tmask, bk);
        if (K < 0 && T.ov_top < 0) {                  // cannot happen with an authorized maximum
            if (leader) set_status(st, LTS_ERR_INTERNAL);
            break;
        }
        int v, kv;
        if (T.ov_top > K) {
            unsigned long long e = 0;
            if (leader) e = ov_pop(T.ov);
            e = __shfl_sync(T.tmask, e, T.tb);
            ov_sync(T);
            v = (int)(e & 0xffffffffu);
            kv = (int)(e >> 32);
        } else {
            const int L = __ffs(__ballot_sync(T.tmask, bk == K)) - 1;
            int myv = 0;
#pragma unroll
            for (int e = 0; e < E; ++e)
                if (e == bs) myv = T.sv[e];
            if (T.lane == L) {
#pragma unroll
                for (int e = 0; e < E; ++e)
                    if (e == bs) T.sk[e] = -1;
            }
            v = __shfl_sync(T.tmask, myv, L);
            kv = K;
        }
        // the leader claims v first, so that the atomic overlaps the neighbour loads
        int prev = 0;
        if (leader) prev = atomicCAS(a.owner + v, -1, c);
        // ---- one round of loads: order, owner, mark of every neighbour ----
        int x, y, z;
        coords_of(g, v, x, y, z);
        const int nb = tl < NN ? nbr_q<NN>(g, x, y, z, tl) : -1;
        int on = -1, ow = -1;
        unsigned long long qm = 0;
        if (nb >= 0) {
            on = od<DIR>(__ldg(O + nb), g.n);
            ow = __ldcg(a.owner + nb);
            qm = __ldcg(a.qmark + nb);
        }
        // the leader claims v (or learns its owner) and broadcasts the outcome
        int o = -1, decision = 0;     // decision: 0 skip, 1 claimed, 2 owned by another class
        if (leader) {
            if (prev == -1) {
                decision = 1;
                o = c;
                if (log_pos == log_end) {
                    log_pos = atomicAdd(&ctr->log_cursor, kLogChunk);
                    log_end = log_pos + kLogChunk;
                    if (log_end > a.log_cap) {
                        log_pos = log_end = 0;
                        set_status(st, LTS_ERR_OOM);
                        decision = -1;
                    }
                }
                if (decision == 1) a.vlog[log_pos++] = v;
            } else {
                o = prev;
                decision = (prev == c || (merged && find_root(a.parent, prev) == c)) ? 0 : 2;
            }
        }
        decision = __shfl_sync(T.tmask, decision, T.tb);
        if (decision < 0) break;
        if (decision == 0) continue;
        o = __shfl_sync(T.tmask, o, T.tb);
        const bool claimed = decision == 1;
        const bool higher = nb >= 0 && on > kv;
        bool inC = nb >= 0 && ow >= 0 && (ow == c || (merged && find_root(a.parent, ow) == c));
        const int h = __popc(__ballot_sync(T.tmask, higher));
        const int k = __popc(__ballot_sync(T.tmask, higher && inC));
        if (k != h) {
            // ---- arrival at the saddle v ----
            const int head = claimed ? c : o;
            if (leader && !claimed) {
                const int old = atomicExch(a.listhead + head, c);
                __stcg(a.next_w + c, old);
            }
            // the queue must be readable by whoever releases this class
            int nreg = 0;
#pragma unroll
            for (int e = 0; e < E; ++e) nreg += T.sk[e] >= 0;
            const int total = __reduce_add_sync(T.tmask, nreg) + T.ovn;
            long long base = 0;
            int okr = 1;
            if (leader) {
                if (sp_end - sp_pos < 2 * total) {
                    const int want = max(2 * total, kSpillChunk);
                    sp_pos = atomicAdd(&ctr->spill_cursor, want);
                    sp_end = sp_pos + want;
                    if (sp_end > a.spill_cap) { set_status(st, LTS_ERR_OOM); okr = 0; sp_pos = sp_end = 0; }
                }
                base = sp_pos;
                sp_pos += 2 * total;
            }
            okr = __shfl_sync(T.tmask, okr, T.tb);
            if (!okr) break;
            base = __shfl_sync(T.tmask, base, T.tb);
            long long pos = base;
            const unsigned below = (1u << T.lane) - 1u;
#pragma unroll
            for (int e = 0; e < E; ++e) {
                const bool hs = T.sk[e] >= 0;
                const unsigned m = __ballot_sync(T.tmask, hs);
                if (hs) {
                    const long long at2 = pos + 2 * __popc(m & below);
                    __stcg(a.spill_pool + at2, T.sv[e]);
                    __stcg(a.spill_pool + at2 + 1, T.sk[e]);
                }
                pos += 2 * __popc(m);
            }
            if (T.ovn > 0) {
                const unsigned long long* oh = reinterpret_cast<const unsigned long long*>(
                    __shfl_sync(T.tmask, reinterpret_cast<unsigned long long>(T.ov.h), T.tb));
                for (int i = tl; i < T.ovn; i += TS) {
                    __stcg(a.spill_pool + pos + 2 * i, (int)(oh[i] & 0xffffffffu));
                    __stcg(a.spill_pool + pos + 2 * i + 1, (int)(oh[i] >> 32));
                }
            }
            __syncwarp(T.tmask);                       // orders the team's spill writes before the leader's fence
            int tot = 0;
            if (leader) {
                __stcg(a.spill_base + c, (int)base);
                __stcg(a.spill_n + c, total);
                __stcg(a.wait_v + c, v);
                // release: this class's spill and records; acquire: those of the
                // classes that arrived before
                cuda::atomic_ref<int, cuda::thread_scope_device> counter(a.cnt[head]);
                tot = counter.fetch_add(k, cuda::memory_order_acq_rel) + k;
            }
            tot = __shfl_sync(T.tmask, tot, T.tb);
            if (tot < h) { c = -1; continue; }        // a higher neighbour is still unvisited: stop
            // ---- last arrival: merge every class stopped at v ----
            __syncwarp(T.tmask);
            merged = true;
            int cur = head;
            bool first = true;
            bool okm = true;
            while (cur >= 0 && okm) {
                if (cur != c) {
                    int sb = 0, sn = 0;
                    if (leader) {
                        __stcg(a.parent + cur, c);
                        sb = __ldcg(a.spill_base + cur);
                        sn = __ldcg(a.spill_n + cur);
                    }
                    sb = __shfl_sync(T.tmask, sb, T.tb);
                    sn = __shfl_sync(T.tmask, sn, T.tb);
                    for (int i = 0; i < sn && okm; i += TS) {
                        const int idx = i + tl;
                        bool hs = idx < sn;
                        int u = 0, ou = 0;
                        if (hs) {
                            u = __ldcg(a.spill_pool + sb + 2 * idx);
                            ou = __ldcg(a.spill_pool + sb + 2 * idx + 1);
                            __stcg(a.qmark + u, mark);
                        }
                        okm = insert_batch(T, hs, ou, u, a);
                    }
                }
                int nx = -1;
                if (leader) nx = first ? __ldcg(a.listhead + head) : __ldcg(a.next_w + cur);
                cur = __shfl_sync(T.tmask, nx, T.tb);
                first = false;
            }
            if (!okm) break;
            if (leader) {
                __stcg(a.wait_v + c, -1);
                if (head == c) { __stcg(a.cnt + c, 0); __stcg(a.listhead + c, -1); }
                __threadfence();
            }
            __syncwarp(T.tmask);
            // classes merged into c: recheck which neighbours are in c
            inC = nb >= 0 && in_class(a.parent, ow, c);
        }
        // ---- v belongs to c: queue its lower neighbours ----
        const bool cand = nb >= 0 && on < kv && !inC && qm != mark;
        if (cand) __stcg(a.qmark + nb, mark);
        if (!insert_batch(T, cand, on, nb, a)) break;
    }
    // every reserved log slot must hold a vertex or -1
    if (leader)
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
    const int blocks = w.lanes / kThreads;
    if (g.nn == 14) propagate_kernel<DIR, 14><<<blocks, kThreads, 0, s>>>(g, O, a);
    else propagate_kernel<DIR, 6><<<blocks, kThreads, 0, s>>>(g, O, a);
    w.launches += 1;
    return cudaGetLastError();
}

int propagate_lanes(int sms) { return sms * 12 * kThreads; }
long long propagate_log_slack(int lanes) { return (long long)lanes * kLogChunk; }
long long propagate_spill_slack(int lanes) { return (long long)lanes * kSpillChunk; }
long long propagate_heap_slack(int lanes) { return (long long)lanes * 64; }

template cudaError_t propagate<1>(Work&, const Geom&, const int*, int, cudaStream_t);
template cudaError_t propagate<-1>(Work&, const Geom&, const int*, int, cudaStream_t);

}  // namespace lts
