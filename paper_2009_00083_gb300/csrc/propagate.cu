// Step 1 with hill chains (Sec. 4.2 step 1, Sec. 4.3, Sec. 4.4): one
// superlevel set propagation per unauthorized maximum (a "class").
//
// The first step of every propagation is data parallel and runs as one
// thread-per-class kernel: the seed (a maximum: nothing else can reach it)
// is claimed with a plain store and its highest neighbour u is found; then
// every class pops u.  All its neighbours are lower than the seed, so u is
// the first vertex any schedule pops.  If the seed is the only higher
// neighbour of u, the class claims u and goes on in the engine below.
// Otherwise u is a saddle (an arrival, see below), and most classes stop
// there for good.  The queue of a class stopped at its first pop is the
// seed's neighbourhood minus u, so it is rebuilt when needed instead of
// spilled.  These arrivals cross a kernel boundary before anything reads
// them, so they need no memory fence.  Each class that goes on becomes a
// task record (class, u, Od(u), seed or -1 after a meeting).
//
// The persistent engine then runs the classes that go on.  Each is run by a
// team of lanes (a whole warp, so that no two propagations share an
// instruction stream): lane q handles neighbour q of the popped vertex, so the loads of all
// neighbours go out in one round trip and every branch is uniform within the
// team.  The priority queue of the class is a top-K frontier in the team's
// registers (E slots per lane), popped with a team max-reduction; entries that
// do not fit go to the team's overflow queue in an HBM pool (a radix queue,
// see RQ below; a 32-ary heap in the persistence-driven selection).  Popping v:
//   - v already in the class: skip;
//   - claim v (atomicCAS on owner[v]); the vertex log records every claim;
//   - k = higher neighbours of v in the class, h = all higher neighbours;
//     k == h: v is regular for the class, queue its lower neighbours;
//   - otherwise v is a saddle for the class (an arrival): the class copies
//     its queue to the spill pool and adds k to the arrival counter of v.
//     The arrival that brings the counter to h is the last one.  Every
//     higher neighbour of v then belongs to a class waiting at v, so the
//     waiting classes are the union-find roots of those neighbours' owners,
//     found by the lanes in parallel (no wait list).  The last arrival
//     unites them with itself, melds their queues into its own and
//     continues below v.  Any other arrival stops.
// A class thus only passes a saddle once every higher neighbour belongs to a
// class that has arrived there, so the regions do not depend on the order in
// which teams run.  Nothing here waits on another team: a stopped class just
// ends its task, and the kernel ends when every task has been taken.
// Arrival counters are indexed by the saddle vertex: once a saddle is
// released nothing touches its counter again in the pass, so the releaser
// resets it with a plain store.
// Decisions that read shared mutable state (owner[], parent[]) are taken by
// one lane and broadcast, so a team never diverges.
//
// Persistence-driven selection (Sec. 4.5) runs the same engine from every
// extremum of the pass (PERS = true): a class also keeps its highest
// extremum (the oldest of the classes it absorbed; a stopped class leaves it
// in ctop[]) and, before it takes a popped vertex v, compares the scalar
// difference between that extremum and v with eps in double precision.
// Beyond eps the class ends and its highest extremum is marked persistent
// in the authorized bitmap; a class whose queue runs dry has covered the
// grid and its extremum, the global one, is marked too.  A class that
// waits at a saddle for ever, or that was absorbed, marks nothing.  The
// selection is then the set of extrema whose Elder-rule persistence exceeds
// eps (with the global one): at a saddle where a class stops for good, the
// class on the other side has a higher extremum, and a class that crossed a
// saddle was within eps of its extremum there.
#include <algorithm>
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
    int* qmark;                  // the last class that queued the vertex (cleared to -1 before each launch)
    int* parent;
    int* wait_v;
    int* cnt;
    int* spill_base;
    int* spill_n;
    int4* heaprec;               // a stopped class's overflow queue: (table offset low, high, entries, 0),
                                 // or for the selection's heap (block offset low, high, entries, capacity)
    int* spill_pool;
    long long spill_cap;
    unsigned long long* heap_pool;
    long long heap_cap;
    int* vlog;
    int* vlog_cls;               // the class that claimed each logged vertex (at the time of the claim)
    long long log_cap;
    const int4* tasks;           // (class, u, Od(u), seed; -1 after a meeting at u)
    DevCounters* ctr;
    // persistence-driven selection only
    const float* F;              // the field of the pass
    double eps;
    int2* ctop;                  // per class: (highest extremum, its Od), written when the class stops
    unsigned* authbits;          // persistent extrema are set here
};

// The difference between the class's highest extremum and v exceeds eps
// (maxima pass: f(top) - f(v); minima pass: f(v) - f(top)).
template <int DIR>
__device__ __forceinline__ bool beyond_eps(float ftop, float fv, double eps) {
    const double d = DIR > 0 ? (double)ftop - (double)fv : (double)fv - (double)ftop;
    return d > eps;
}

__device__ __forceinline__ void mark_persistent(unsigned* bits, int v) {
    atomicOr(bits + (v >> 5), 1u << (v & 31));
}

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

// The overflow queue of a team (entries beyond the register frontier): a
// radix queue in HBM.  Pops of a propagation come in decreasing order (a
// vertex is taken only when every higher neighbour is in the class, so what
// it queues is lower than it), and every queued key is at most the key of
// the class's last pop.  So the queue keeps a base key b at least as high as
// every key it holds and files an entry with key k in bucket 0 if k == b,
// else in bucket 32 - clz(b ^ k) (the highest bit where they differ, + 1):
// every key of a lower bucket is higher than every key of a higher one.  A
// push appends to its bucket; a pop takes bucket 0 if it holds anything,
// else refiles the lowest non-empty bucket under a new base, its highest key
// (each entry moves to a lower bucket: a few moves per entry over its
// life).  The team's bucket table (32 blocks of the HBM pool, with their
// lengths and highest entries) lives in shared memory and every operation
// is run by the whole team, so appends and refiling move 32 entries per
// round of coalesced loads.  A class that stops leaves its buckets in the
// pool with a copy of the table; the class that absorbs it refiles the
// smaller queue into the larger one.
struct RQ {
    long long off[32];                 // pool offset of each bucket's block
    int len[32], cap[32];
    unsigned long long mx[32];         // each non-empty bucket's highest entry
    int base;                          // every queued key is at most base
    unsigned nz;                       // non-empty buckets
    int total;                         // queued entries
    long long tpos, tend;              // the team's reserve of pool words for stopped queues' tables
};

// one queue per team of the engine's blocks (shared memory)
__shared__ RQ g_team_rq[kThreads / 32];

__device__ __forceinline__ RQ& team_rq() { return g_team_rq[threadIdx.x >> 5]; }

__device__ __forceinline__ int rq_bucket(int base, int key) {
    return key == base ? 0 : 32 - __clz((unsigned)(base ^ key));
}

__device__ __forceinline__ void rq_reset(RQ& q, int lane) {
    q.len[lane] = 0;
    q.cap[lane] = 0;
    q.off[lane] = 0;
    q.mx[lane] = 0ull;
    if (lane == 0) { q.base = INT_MAX; q.nz = 0u; q.total = 0; }
    __syncwarp();
}

// key of the highest queued entry, -1 if the queue is empty
__device__ __forceinline__ int rq_top(const RQ& q) {
    return q.nz ? (int)(q.mx[__ffs(q.nz) - 1] >> 32) : -1;
}

// Bucket t gets room for `more` entries (a block twice as large from the
// pool, the entries copied by the team).  false (uniform) when the pool is spent.
__device__ bool rq_reserve(RQ& q, int t, int more, int lane, const PropArgs& a) {
    const int len = q.len[t], cap = q.cap[t];
    if (len + more <= cap) return true;
    const int ncap = max(2 * cap, max(64, len + more));
    long long noff = 0;
    if (lane == 0) {
        noff = (long long)atomicAdd((unsigned long long*)&a.ctr->heap_cursor, (unsigned long long)ncap);
        if (noff + ncap > a.heap_cap) { set_oom(a.ctr, 1); noff = -1; }
        else if (cap == 0 && q.total == 0) atomicAdd(&a.ctr->heap_spills, 1);
    }
    noff = __shfl_sync(0xffffffffu, noff, 0);
    if (noff < 0) return false;
    const unsigned long long* src = a.heap_pool + q.off[t];
    unsigned long long* dst = a.heap_pool + noff;
    for (int i = lane; i < len; i += 32) __stcg(dst + i, __ldcg(src + i));
    __syncwarp();
    if (lane == 0) { q.off[t] = noff; q.cap[t] = ncap; }
    __syncwarp();
    return true;
}

// Files the entries e of the lanes with `has` under the queue's base (one
// round: lanes with the same bucket form a group; the buckets that lack room
// grow first, then each group's leader reserves its slots with one
// shared-memory atomic).
__device__ bool rq_file(RQ& q, bool has, unsigned long long e, int lane, const PropArgs& a) {
    const int t = has ? rq_bucket(q.base, (int)(e >> 32)) : -1;
    const unsigned grp = __match_any_sync(0xffffffffu, t);
    const int leader = __ffs(grp) - 1;
    const int cnt = __popc(grp);
    const bool lead = has && lane == leader;
    // buckets without room for their group grow (rare), one at a time
    unsigned short_m = __ballot_sync(0xffffffffu, lead && q.len[t] + cnt > q.cap[t]);
    while (short_m) {
        const int L = __ffs(short_m) - 1;
        short_m &= short_m - 1;
        if (!rq_reserve(q, __shfl_sync(0xffffffffu, t, L), __shfl_sync(0xffffffffu, cnt, L), lane, a))
            return false;
    }
    int base = 0;
    if (lead) {
        base = atomicAdd(&q.len[t], cnt);
        atomicOr(&q.nz, 1u << t);
    }
    base = __shfl_sync(0xffffffffu, base, leader);
    if (has) {
        __stcg(a.heap_pool + q.off[t] + base + __popc(grp & ((1u << lane) - 1u)), e);
        atomicMax(&q.mx[t], e);                  // an empty bucket's highest entry is 0
    }
    const unsigned hm = __ballot_sync(0xffffffffu, has);
    if (lane == 0) atomicAdd(&q.total, __popc(hm));
    __syncwarp();
    return true;
}

// Pushes one entry (the same e in every lane).
__device__ __forceinline__ bool rq_push(RQ& q, unsigned long long e, int lane, const PropArgs& a) {
    const int t = rq_bucket(q.base, (int)(e >> 32));
    if (q.len[t] == q.cap[t] && !rq_reserve(q, t, 1, lane, a)) return false;
    if (lane == 0) {
        const int l = q.len[t];
        __stcg(a.heap_pool + q.off[t] + l, e);
        if (e > q.mx[t]) q.mx[t] = e;
        q.len[t] = l + 1;
        q.nz |= 1u << t;
        ++q.total;
    }
    __syncwarp();
    return true;
}

// Files the `n` entries at pool offset `off` (read in rounds of 32).
__device__ bool rq_file_block(RQ& q, long long off, int n, int lane, const PropArgs& a) {
    for (int i0 = 0; i0 < n; i0 += 32) {
        const bool has = i0 + lane < n;
        const unsigned long long e = has ? __ldcg(a.heap_pool + off + i0 + lane) : 0ull;
        if (!rq_file(q, has, e, lane, a)) return false;
    }
    return true;
}

// Pops the highest entry (the queue is not empty).  false (uniform) when
// refiling ran out of pool.
__device__ bool rq_pop(RQ& q, unsigned long long& out, int lane, const PropArgs& a) {
    int b = __ffs(q.nz) - 1;
    if (b > 0 && q.len[b] == 1) {
        // a bucket of one entry: it is the highest, and taking it leaves every bucket valid
        out = q.mx[b];
        __syncwarp();
        if (lane == 0) {
            q.len[b] = 0;
            q.mx[b] = 0ull;
            q.nz &= ~(1u << b);
            --q.total;
        }
        __syncwarp();
        return true;
    }
    if (b > 0) {
        // refile bucket b under its highest key (its entries go to lower buckets)
        const long long off = q.off[b];
        const int n = q.len[b];
        const unsigned long long top = q.mx[b];
        __syncwarp();
        if (lane == 0) {
            q.len[b] = 0;
            q.mx[b] = 0ull;
            q.nz &= ~(1u << b);
            q.total -= n;
            q.base = (int)(top >> 32);
        }
        __syncwarp();
        if (!rq_file_block(q, off, n, lane, a)) return false;
        b = 0;
    }
    // bucket 0 holds entries of key base: copies of one vertex, all equal to its highest entry
    out = q.mx[0];
    __syncwarp();
    if (lane == 0) {
        if (--q.len[0] == 0) { q.nz &= ~1u; q.mx[0] = 0ull; }
        --q.total;
    }
    __syncwarp();
    return true;
}

// A stopped class's queue: its table (base, non-empty buckets, then per
// bucket: offset, capacity and length, highest entry) written to the pool.  Returns the
// table's pool offset (-1 for an empty queue, -2 when the pool is spent).
__device__ long long rq_store_table(RQ& q, int lane, const PropArgs& a) {
    const int nb = __popc(q.nz);
    const int words = 1 + 3 * nb;
    if (q.tend - q.tpos < words) {             // a new reserve (one global atomic per 1024 words)
        long long r = 0;
        if (lane == 0) {
            r = (long long)atomicAdd((unsigned long long*)&a.ctr->heap_cursor, 1024ull);
            if (r + 1024 > a.heap_cap) { set_oom(a.ctr, 1); r = -2; }
        }
        r = __shfl_sync(0xffffffffu, r, 0);
        if (r < 0) return r;
        __syncwarp();
        if (lane == 0) { q.tpos = r; q.tend = r + 1024; }
        __syncwarp();
    }
    const long long t = q.tpos;
    __syncwarp();
    if (lane == 0) q.tpos = t + words;
    unsigned long long* w = a.heap_pool + t;
    if (lane == 0) __stcg(w, ((unsigned long long)q.nz << 32) | (unsigned)q.base);
    if ((q.nz >> lane) & 1u) {
        const int r = __popc(q.nz & ((1u << lane) - 1u));
        __stcg(w + 1 + 3 * r, (unsigned long long)q.off[lane]);
        __stcg(w + 2 + 3 * r, ((unsigned long long)(unsigned)q.cap[lane] << 32) | (unsigned)q.len[lane]);
        __stcg(w + 3 + 3 * r, q.mx[lane]);
    }
    return t;
}

__device__ __forceinline__ long long rq_store(RQ& q, int lane, const PropArgs& a) {
    return q.total == 0 ? -1 : rq_store_table(q, lane, a);
}

// The team's queue absorbs a stopped class's queue (table at pool offset t,
// `n` entries): the smaller queue is refiled into the larger one.  false
// (uniform) when the pool is spent.
__device__ bool rq_absorb(RQ& q, long long t, int n, int lane, const PropArgs& a) {
    const unsigned long long* w = a.heap_pool + t;
    const unsigned long long h = __ldcg(w);
    const unsigned onz = (unsigned)(h >> 32);
    const int obase = (int)(unsigned)h;
    const int r = __popc(onz & ((1u << lane) - 1u));
    const bool has = (onz >> lane) & 1u;
    long long ooff = 0;
    int olen = 0, ocap = 0;
    unsigned long long omx = 0ull;
    if (has) {
        ooff = (long long)__ldcg(w + 1 + 3 * r);
        const unsigned long long lc = __ldcg(w + 2 + 3 * r);
        olen = (int)(unsigned)lc;
        ocap = (int)(lc >> 32);
        omx = __ldcg(w + 3 + 3 * r);
    }
    if (n > q.total) {
        // adopt the other queue's buckets, then refile this queue's entries into it
        const long long moff = q.off[lane];
        const int mlen = q.len[lane];
        const unsigned mnz = q.nz;
        __syncwarp();
        q.off[lane] = ooff;
        q.len[lane] = olen;
        q.cap[lane] = ocap;
        q.mx[lane] = omx;
        if (lane == 0) { q.base = obase; q.nz = onz; q.total = n; }
        __syncwarp();
        for (int b = 0; b < 32; ++b)
            if (((mnz >> b) & 1u) && !rq_file_block(q, __shfl_sync(0xffffffffu, moff, b),
                                                    __shfl_sync(0xffffffffu, mlen, b), lane, a))
                return false;
        return true;
    }
    for (int b = 0; b < 32; ++b)
        if (((onz >> b) & 1u) && !rq_file_block(q, __shfl_sync(0xffffffffu, ooff, b),
                                                __shfl_sync(0xffffffffu, olen, b), lane, a))
            return false;
    return true;
}

// The persistence-driven selection keeps a 32-ary max-heap in HBM instead
// (a pop sifts down one level per coalesced load of 32 children and a team
// reduction; lane 0 holds the state and pushes): its propagations end at eps
// with most of their queue unpopped, and a heap touches only what it pops,
// where refiling would move entries that are never taken.
struct Overflow {
    unsigned long long* h;
    int n, cap;
};

__device__ bool ov_push(Overflow& H, unsigned long long e, const PropArgs& a) {
    if (H.n == H.cap) {
        const int ncap = max(2 * H.cap, 256);
        const long long off = atomicAdd((unsigned long long*)&a.ctr->heap_cursor, (unsigned long long)ncap);
        if (off + ncap > a.heap_cap) { set_oom(a.ctr, 1); return false; }
        unsigned long long* nh = a.heap_pool + off;
        for (int i = 0; i < H.n; ++i) nh[i] = H.h[i];
        if (H.cap == 0) atomicAdd(&a.ctr->heap_spills, 1);
        H.h = nh;
        H.cap = ncap;
    }
    int i = H.n++;
    while (i > 0) {
        const int p = (i - 1) >> 5;
        const unsigned long long pe = H.h[p];
        if (pe >= e) break;
        H.h[i] = pe;
        i = p;
    }
    H.h[i] = e;
    return true;
}

template <int NN>
struct TeamState {
    static constexpr int TS = TeamCfg<NN>::TS;
    static constexpr int E = TeamCfg<NN>::E;
    static_assert(TS == 32, "the overflow queue is run by whole warps");
    int sk[E];        // frontier slots: key (Od), -1 = empty
    int sv[E];        //                 vertex
    int rot;          // rotation of the slot assignment (spreads entries over lanes)
    unsigned tmask;
    int tb, lane;
    int ov_top;       // uniform: key of the overflow queue's highest entry, -1 if empty
    bool qused;       // uniform: the team's queue holds blocks of the current class
    Overflow ov;      // the selection's heap (meaningful in team lane 0)
};

template <int NN>
__device__ __forceinline__ void ov_sync(TeamState<NN>& T) {
    const int n = T.ov.n;
    const int top = n > 0 ? (int)(T.ov.h[0] >> 32) : -1;
    T.ov_top = __shfl_sync(T.tmask, top, T.tb);
}

// Pops the top of the team's overflow heap (all team lanes call it).
template <int NN>
__device__ unsigned long long ov_pop_team(TeamState<NN>& T) {
    __syncwarp(T.tmask);                       // the leader's pushes before the team's loads
    unsigned long long* h = reinterpret_cast<unsigned long long*>(
        __shfl_sync(T.tmask, reinterpret_cast<unsigned long long>(T.ov.h), T.tb));
    const int n = __shfl_sync(T.tmask, T.ov.n, T.tb) - 1;
    const bool leader = T.lane == T.tb;
    const unsigned long long top = __ldcg(h);
    if (n > 0) {
        const unsigned long long last = __ldcg(h + n);
        int i = 0;
        for (;;) {
            const int c0 = 32 * i + 1;
            if (c0 >= n) break;
            unsigned long long ce = 0ull;
            int ci = -1;
            const int c = c0 + (T.lane - T.tb);
            if (c < n) {
                ce = __ldcg(h + c);
                ci = c;
            }
            const unsigned hi = (unsigned)(ce >> 32), lo = (unsigned)ce;
            const unsigned kh = __reduce_max_sync(T.tmask, hi);
            const unsigned kl = __reduce_max_sync(T.tmask, hi == kh ? lo : 0u);
            const int L = __ffs(__ballot_sync(T.tmask, ci >= 0 && hi == kh && lo == kl)) - 1;
            const unsigned long long mv = ((unsigned long long)kh << 32) | kl;
            if (mv <= last) break;
            if (leader) __stcg(h + i, mv);
            i = __shfl_sync(T.tmask, ci, L);
        }
        if (leader) __stcg(h + i, last);
    }
    if (leader) T.ov.n = n;
    __syncwarp(T.tmask);
    return top;
}

// Adds one candidate per lane (has, key, vert) to the team frontier.
// Returns false (uniformly) if the overflow pool is exhausted.
template <bool PERS, int NN>
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
        bool r;
        if constexpr (PERS) {
            int rr = 1;
            if (T.lane == T.tb) rr = ov_push(T.ov, out, a) ? 1 : 0;
            r = __shfl_sync(T.tmask, rr, T.tb) != 0;
            ov_sync(T);
        } else {
            r = rq_push(team_rq(), out, T.lane, a);
            T.qused = true;
            T.ov_top = rq_top(team_rq());
        }
        if (!r) { ok = false; break; }
    }
    return ok;
}

// The queue of a class that stopped at its first pop u: the neighbours of its
// seed m but u, inserted unless the class `mark` already queued them.
template <int DIR, int NN, bool PERS>
__device__ __forceinline__ bool rebuild_first_queue(TeamState<NN>& T, const Geom& g, const int* __restrict__ O, int m,
                                                    int u, int mark, const PropArgs& a, int tl) {
    int x, y, z;
    coords_of(g, m, x, y, z);
    const int nb = tl < NN ? nbr_q<NN>(g, x, y, z, tl) : -1;
    bool cand = nb >= 0 && nb != u;
    int key = 0;
    if (cand) {
        key = od<DIR>(__ldg(O + nb), g.n);
        if (__ldcg(a.qmark + nb) == mark) cand = false;
        else __stcg(a.qmark + nb, mark);
    }
    return insert_batch<PERS>(T, cand, key, nb, a);
}

// First step (thread per class c): claim the seed m and log it (log slots
// [0, nU) hold the seeds, [nU, 2 nU) the first pops; the engine's log starts
// at 2 nU), find m's highest neighbour u (kept in wait_v[c]) and pop it.  If
// m is u's only higher neighbour, c claims u and becomes an engine task.
// Otherwise c arrives at u with k = 1 (its one vertex, the seed; spill_n[c]
// stays -1: its queue is rebuilt from the seed); the arrival that completes
// u's count makes a task that melds every class waiting at u.  The others
// stop here.  u is not a seed, so its claim never meets a seed's plain store,
// and u's neighbourhood overlaps m's, so most of its loads hit L1.
template <int DIR, int NN, bool PERS>
__global__ void __launch_bounds__(256) first_step_kernel(Geom g, const int* __restrict__ O, PropArgs a, int4* tasks) {
    __shared__ int s_n, s_base;
    DevCounters* ctr = a.ctr;
    if (failed(&ctr->status)) return;
    const int nU = ctr->n_unauth;
    if (!PERS && nU > 0 && ctr->n_auth_ext == 0) {
        if (blockIdx.x == 0 && threadIdx.x == 0) set_status(&ctr->status, LTS_ERR_NO_AUTHORIZED);
        return;
    }
    if (2LL * nU > a.log_cap) {
        if (blockIdx.x == 0 && threadIdx.x == 0) set_oom(ctr, 3);
        return;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) ctr->log_cursor = 2 * nU;
    const int lane = threadIdx.x & 31;
    for (long long b = (long long)blockIdx.x * blockDim.x; b < nU; b += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(b + threadIdx.x);
        int4 task = make_int4(-1, 0, 0, 0);
        int m = -1, u = -1, ku = -1;
        if (c < nU) {
            m = __ldg(a.U + c);
            a.owner[m] = c;
            a.vlog[c] = m;
            a.vlog_cls[c] = c;
            int x, y, z;
            coords_of(g, m, x, y, z);
#pragma unroll
            for (int q = 0; q < NN; ++q) {
                const int nb = nbr_q<NN>(g, x, y, z, q);
                if (nb >= 0) {
                    const int k = od<DIR>(__ldg(O + nb), g.n);
                    if (k > ku) { ku = k; u = nb; }
                }
            }
            if (PERS) {
                a.ctop[c] = make_int2(m, od<DIR>(__ldg(O + m), g.n));
                if (beyond_eps<DIR>(__ldg(a.F + m), __ldg(a.F + u), a.eps)) {   // ends before its first pop
                    mark_persistent(a.authbits, m);
                    a.vlog[nU + c] = -1;
                    u = -1;
                }
            }
        }
        if (u >= 0) {
            a.wait_v[c] = u;
            const int prev = atomicCAS(a.owner + u, -1, c);
            a.vlog[nU + c] = prev == -1 ? u : -1;
            a.vlog_cls[nU + c] = c;
            int x, y, z;
            coords_of(g, u, x, y, z);
            int h = 0;
#pragma unroll
            for (int q = 0; q < NN; ++q) {
                const int nb = nbr_q<NN>(g, x, y, z, q);
                if (nb >= 0 && od<DIR>(__ldg(O + nb), g.n) > ku) ++h;
            }
            if (h == 1) {
                if (prev == -1) task = make_int4(c, u, ku, m);
                else set_status(&ctr->status, LTS_ERR_INTERNAL);   // only the seed's class can reach u
            } else if (atomicAdd(a.cnt + u, 1) + 1 == h) {
                task = make_int4(c, u, ku, -1);
            }
        }
        // task slots: one global atomic per block
        if (threadIdx.x == 0) s_n = 0;
        __syncthreads();
        const unsigned want = __ballot_sync(0xffffffffu, task.x >= 0);
        int wb = 0;
        if (lane == 0 && want) wb = atomicAdd(&s_n, __popc(want));
        wb = __shfl_sync(0xffffffffu, wb, 0);
        __syncthreads();
        if (threadIdx.x == 0) s_base = s_n ? atomicAdd(&ctr->n_tasks, s_n) : 0;
        __syncthreads();
        if (task.x >= 0) tasks[s_base + wb + __popc(want & ((1u << lane) - 1u))] = task;
        __syncthreads();
    }
}

template <int DIR, int NN, bool PERS>
__global__ void __launch_bounds__(kThreads, 8) propagate_kernel(Geom g, const int* __restrict__ O, PropArgs a) {
    constexpr int TS = TeamCfg<NN>::TS, E = TeamCfg<NN>::E;
    DevCounters* ctr = a.ctr;
    int* st = &ctr->status;
    if (failed(st)) return;
    const int nT = *(volatile int*)&ctr->n_tasks;
    TeamState<NN> T;
    T.lane = threadIdx.x & 31;
    T.tb = T.lane & ~(TS - 1);
    T.tmask = (TS == 32) ? 0xffffffffu : (((1u << TS) - 1u) << T.tb);
    const int tl = T.lane - T.tb;
    const bool leader = tl == 0;
    T.rot = 0;
    T.ov.h = nullptr; T.ov.n = 0; T.ov.cap = 0;
    if constexpr (!PERS) {
        if (T.lane == 0) { team_rq().tpos = 0; team_rq().tend = 0; }
        rq_reset(team_rq(), T.lane);
    }
    T.qused = false;
    T.ov_top = -1;
#pragma unroll
    for (int e = 0; e < E; ++e) { T.sk[e] = -1; T.sv[e] = 0; }

    // team-leader state
    int task_lo = 0, task_hi = 0;
    long long log_pos = 0, log_end = 0;
    long long sp_pos = 0, sp_end = 0;
    int c = -1;
    bool merged = false;     // c has absorbed other classes: membership needs find_root
    int top_v = -1, top_k = -1;   // persistence-driven: the class's highest extremum and its Od (uniform)
    float top_f = 0.f;

    for (;;) {
        int v, kv;
        bool resumed = false;    // v is the first pop of a task, already owned by the class
        if (c < 0) {                                   // take the next task
            int4 t = make_int4(-1, 0, 0, 0);
            if (leader) {
                if (task_lo == task_hi) {
                    // guided batches: large while many tasks remain, single ones at the end
                    const int rem = nT - *(volatile int*)&ctr->seed_cursor;
                    const int nteams = gridDim.x * (blockDim.x / TS);
                    const int bsz = max(1, min(kSeedBatch, rem / (4 * nteams)));
                    const int b = atomicAdd(&ctr->seed_cursor, bsz);
                    task_lo = b;
                    task_hi = min(b + bsz, nT);
                }
                if (task_lo < task_hi && !failed(st)) t = __ldcg(a.tasks + task_lo++);
            }
            c = __shfl_sync(T.tmask, t.x, T.tb);
            if (c < 0) break;
            const int u = __shfl_sync(T.tmask, t.y, T.tb);
            kv = __shfl_sync(T.tmask, t.z, T.tb);
            const int seed = __shfl_sync(T.tmask, t.w, T.tb);
#pragma unroll
            for (int e = 0; e < E; ++e) T.sk[e] = -1;
            if constexpr (PERS) {
                T.ov.h = nullptr; T.ov.n = 0; T.ov.cap = 0;
            } else if (T.qused) {
                rq_reset(team_rq(), T.lane);
            }
            T.qused = false;
            T.ov_top = -1;
            const int mk = c;
            bool ok;
            if (seed >= 0) {                           // u has one higher neighbour, the seed of c
                merged = false;
                if (PERS) {
                    top_v = seed;
                    top_k = od<DIR>(__ldg(O + seed), g.n);
                    top_f = __ldg(a.F + seed);
                }
                ok = rebuild_first_queue<DIR, NN, PERS>(T, g, O, seed, u, mk, a, tl);
            } else {
                // a meeting at u: its higher neighbours are the seeds of the classes that met
                merged = true;
                int ux, uy, uz;
                coords_of(g, u, ux, uy, uz);
                const int unb = tl < NN ? nbr_q<NN>(g, ux, uy, uz, tl) : -1;
                bool hi = false;
                int own = -1, ok_u = -1;
                if (unb >= 0) {
                    ok_u = od<DIR>(__ldg(O + unb), g.n);
                    hi = ok_u > kv;
                    own = __ldcg(a.owner + unb);
                }
                unsigned hm = __ballot_sync(T.tmask, hi);
                if (PERS) {                            // the highest of the seeds that met at u
                    top_k = __reduce_max_sync(T.tmask, hi ? ok_u : -1);
                    top_v = __shfl_sync(T.tmask, unb, __ffs(__ballot_sync(T.tmask, hi && ok_u == top_k)) - 1);
                    top_f = __ldg(a.F + top_v);
                }
                ok = true;
                while (hm && ok) {
                    const int L = __ffs(hm) - 1;
                    hm &= hm - 1;
                    const int w = __shfl_sync(T.tmask, unb, L);
                    const int r = __shfl_sync(T.tmask, own, L);
                    if (leader && r != c) __stcg(a.parent + r, c);
                    ok = rebuild_first_queue<DIR, NN, PERS>(T, g, O, w, u, mk, a, tl);
                }
                if (leader) __stcg(a.cnt + u, 0);
            }
            if (!ok) break;
            if (leader) __stcg(a.wait_v + c, -1);
            __syncwarp(T.tmask);
            v = u;
            resumed = true;
        } else {
            // ---- pop the highest queued vertex ----
            int bk = -1, bs = 0;
#pragma unroll
            for (int e = 0; e < E; ++e)
                if (T.sk[e] > bk) { bk = T.sk[e]; bs = e; }
            const int K = __reduce_max_sync(T.tmask, bk);
            if (K < 0 && T.ov_top < 0) {
                if (PERS) {                            // the class covered the grid: the global extremum
                    if (leader) mark_persistent(a.authbits, top_v);
                    c = -1;
                    continue;
                }
                if (leader) set_status(st, LTS_ERR_INTERNAL);   // cannot happen with an authorized maximum
                break;
            }
            if (T.ov_top > K) {
                unsigned long long e;
                if constexpr (PERS) {
                    e = ov_pop_team(T);
                    ov_sync(T);
                } else {
                    if (!rq_pop(team_rq(), e, T.lane, a)) break;
                    T.ov_top = rq_top(team_rq());
                }
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
        }
        const int mark = c;
        // the leader claims v first, so that the atomic overlaps the neighbour loads
        int prev = 0;
        float fv = 0.f;
        if (leader && !resumed) {
            if (PERS) fv = __ldg(a.F + v);
            prev = atomicCAS(a.owner + v, -1, c);
        }
        // ---- one round of loads: order, owner, mark of every neighbour ----
        int x, y, z;
        coords_of(g, v, x, y, z);
        const int nb = tl < NN ? nbr_q<NN>(g, x, y, z, tl) : -1;
        int on = -1, ow = -1;
        int qm = -1;
        if (nb >= 0) {
            on = od<DIR>(__ldg(O + nb), g.n);
            ow = __ldcg(a.owner + nb);
            qm = __ldcg(a.qmark + nb);
        }
        // the leader claims v (or learns its owner) and broadcasts the outcome
        int decision = 0;             // 0 skip, 1 claimed (or resumed), 2 owned by another class, 3 ends (Sec. 4.5)
        if (leader) {
            if (resumed) {
                decision = 1;
            } else if (prev == -1) {
                decision = 1;
                if (log_pos == log_end) {
                    log_pos = atomicAdd(&ctr->log_cursor, kLogChunk);
                    log_end = log_pos + kLogChunk;
                    if (log_end > a.log_cap) {
                        log_pos = log_end = 0;
                        set_oom(ctr, 3);
                        decision = -1;
                    }
                }
                if (decision == 1) {
                    a.vlog_cls[log_pos] = c;
                    a.vlog[log_pos++] = v;
                }
            } else {
                decision = (prev == c || (merged && find_root(a.parent, prev) == c)) ? 0 : 2;
            }
            // persistence-driven: v is more than eps below the class's extremum
            if (PERS && decision > 0 && !resumed && beyond_eps<DIR>(top_f, fv, a.eps)) decision = 3;
        }
        decision = __shfl_sync(T.tmask, decision, T.tb);
        if (decision < 0) break;
        if (decision == 0) continue;
        if (PERS && decision == 3) {                  // the class ends: its extremum is persistent
            if (leader) mark_persistent(a.authbits, top_v);
            c = -1;
            continue;
        }
        const bool higher = nb >= 0 && on > kv;
        bool inC = nb >= 0 && ow >= 0 && (ow == c || (merged && find_root(a.parent, ow) == c));
        const int h = __popc(__ballot_sync(T.tmask, higher));
        const int k = __popc(__ballot_sync(T.tmask, higher && inC));
        if (k != h) {
            if (resumed) {                            // every higher neighbour of a task's u is in the class
                if (leader) set_status(st, LTS_ERR_INTERNAL);
                break;
            }
            // ---- arrival at the saddle v ----
            // The queue must be readable by whoever releases this class: the
            // register part is copied to the spill pool, and the overflow heap
            // stays where it is, its block recorded with the class.
            int nreg = 0;
#pragma unroll
            for (int e = 0; e < E; ++e) nreg += T.sk[e] >= 0;
            const int total = __reduce_add_sync(T.tmask, nreg);
            long long base = 0;
            int okr = 1;
            if (leader) {
                if (sp_end - sp_pos < 2 * total) {
                    const int want = max(2 * total, kSpillChunk);
                    sp_pos = (long long)atomicAdd((unsigned long long*)&ctr->spill_cursor, (unsigned long long)want);
                    sp_end = sp_pos + want;
                    if (sp_end > a.spill_cap) { set_oom(ctr, 2); okr = 0; sp_pos = sp_end = 0; }
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
            // the overflow queue stays in the pool; its table is written there
            long long qrec = -1;
            int qn = 0, qcap = 0;
            if constexpr (PERS) {
                // the heap block stays where it is, recorded with the class
                qrec = T.ov.h ? (long long)(T.ov.h - a.heap_pool) : 0;
                qn = T.ov.n;
                qcap = T.ov.cap;
            } else {
                qrec = T.qused ? rq_store(team_rq(), T.lane, a) : -1;
                if (qrec == -2) break;
                qn = qrec >= 0 ? team_rq().total : 0;
            }
            __syncwarp(T.tmask);                       // orders the team's spill and queue writes before the leader's release
            int tot = 0;
            if (leader) {
                __stcg(a.spill_base + c, (int)base);
                __stcg(a.spill_n + c, total);
                __stcg(a.wait_v + c, v);
                __stcg(a.heaprec + c, make_int4((int)(qrec & 0xffffffffLL), (int)(qrec >> 32), qn, qcap));
                if (PERS) __stcg(a.ctop + c, make_int2(top_v, top_k));
                // release: this class's spill and records; acquire: those of the
                // classes that arrived before
                cuda::atomic_ref<int, cuda::thread_scope_device> counter(a.cnt[v]);
                tot = counter.fetch_add(k, cuda::memory_order_acq_rel) + k;
            }
            tot = __shfl_sync(T.tmask, tot, T.tb);
            if (tot < h) {                             // a higher neighbour is still unvisited: stop
                c = -1;
                if constexpr (PERS) {
                    T.ov.h = nullptr; T.ov.n = 0; T.ov.cap = 0;   // the heap block now belongs to the class
                } else if (T.qused) {
                    rq_reset(team_rq(), T.lane);               // the queue's blocks now belong to the class
                }
                T.qused = false;
                T.ov_top = -1;
                continue;
            }
            // ---- last arrival: merge every class stopped at v ----
            // Every higher neighbour of v now belongs to a class waiting at v:
            // those classes are the roots of the neighbours' owners.
            __syncwarp(T.tmask);
            const int ow2 = nb >= 0 ? __ldcg(a.owner + nb) : -1;
            const int rt = ow2 >= 0 ? find_root(a.parent, ow2) : -1;
            const unsigned hmask = __ballot_sync(T.tmask, higher);
            const unsigned grp = __match_any_sync(T.tmask, rt);
            const bool rep_lane = higher && rt != c && rt >= 0 && (__ffs(grp & hmask) - 1) == T.lane;
            int sb = 0, sn = 0;
            int4 hr = make_int4(0, 0, 0, 0);
            int2 ct = make_int2(-1, -1);
            if (rep_lane) {                            // one lane per class to merge
                sb = __ldcg(a.spill_base + rt);
                sn = __ldcg(a.spill_n + rt);
                if (sn >= 0) hr = __ldcg(a.heaprec + rt);
                if (PERS) ct = __ldcg(a.ctop + rt);
                __stcg(a.parent + rt, c);
            }
            unsigned todo = __ballot_sync(T.tmask, rep_lane);
            if (PERS) {                                // the elder of the merged classes survives
                const int mk2 = __reduce_max_sync(T.tmask, ct.y);
                if (mk2 > top_k) {
                    top_k = mk2;
                    top_v = __shfl_sync(T.tmask, ct.x, __ffs(__ballot_sync(T.tmask, ct.y == mk2)) - 1);
                    top_f = __ldg(a.F + top_v);
                }
            }
            merged = true;
            bool okm = true;
            while (todo && okm) {
                const int L = __ffs(todo) - 1;
                todo &= todo - 1;
                const int rsb = __shfl_sync(T.tmask, sb, L);
                const int rsn = __shfl_sync(T.tmask, sn, L);
                if (rsn < 0) {                         // stopped at its first pop: v, below its seed
                    okm = rebuild_first_queue<DIR, NN, PERS>(T, g, O, __shfl_sync(T.tmask, nb, L), v, mark, a, tl);
                }
                for (int i = 0; i < rsn && okm; i += TS) {
                    const int idx = i + tl;
                    bool hs = idx < rsn;
                    int u = 0, ou = 0;
                    if (hs) {
                        // entries the class already queued are dropped: melded
                        // queues of neighbouring classes share much of their frontier
                        u = __ldcg(a.spill_pool + rsb + 2 * idx);
                        ou = __ldcg(a.spill_pool + rsb + 2 * idx + 1);
                        if (__ldcg(a.qmark + u) == mark) hs = false;
                        else __stcg(a.qmark + u, mark);
                    }
                    okm = insert_batch<PERS>(T, hs, ou, u, a);
                }
                // its overflow queue: the smaller of the two queues is refiled into the larger
                const int rhn = __shfl_sync(T.tmask, hr.z, L);
                if (rhn > 0 && okm) {
                    const int rlo = __shfl_sync(T.tmask, hr.x, L), rhi = __shfl_sync(T.tmask, hr.y, L);
                    const long long roff = ((long long)rhi << 32) | (unsigned)rlo;
                    if constexpr (PERS) {
                        // keep the larger heap, push the smaller one's entries into it
                        const int rcap = __shfl_sync(T.tmask, hr.w, L);
                        int hok = 1;
                        if (leader) {
                            Overflow R{a.heap_pool + roff, rhn, rcap};
                            if (R.n > T.ov.n) { const Overflow t2 = T.ov; T.ov = R; R = t2; }
                            for (int i = 0; i < R.n && hok; ++i) hok = ov_push(T.ov, __ldcg(R.h + i), a) ? 1 : 0;
                        }
                        okm = __shfl_sync(T.tmask, hok, T.tb) != 0;
                        ov_sync(T);
                    } else {
                        okm = rq_absorb(team_rq(), roff, rhn, T.lane, a);
                        T.qused = true;
                        T.ov_top = rq_top(team_rq());
                    }
                }
            }
            if (!okm) break;
            // v is released: nothing reads its counter again in this pass
            if (leader) {
                __stcg(a.wait_v + c, -1);
                __stcg(a.cnt + v, 0);
            }
            __syncwarp(T.tmask);
            // a neighbour is in c if its root is c or the root of a higher neighbour
            inC = nb >= 0 && rt >= 0 && (rt == c || (grp & hmask) != 0);
        }
        // ---- v belongs to c: queue its lower neighbours ----
        const bool cand = nb >= 0 && on < kv && !inC && qm != mark;
        if (cand) __stcg(a.qmark + nb, mark);
        if (!insert_batch<PERS>(T, cand, on, nb, a)) break;
    }
    // every reserved log slot must hold a vertex or -1
    if (leader)
        while (log_pos < log_end) a.vlog[log_pos++] = -1;
}

// Persistence-driven selection leaves claims and arrival counters behind
// (classes that ended or wait for ever): clear them for the pass proper.
__global__ void pers_clear_kernel(const DevCounters* ctr, const int* __restrict__ vlog, const int* __restrict__ wait_v,
                                  int* owner, int* cnt, long long log_cap) {
    if (failed(&ctr->status)) return;
    const long long nlog = min((long long)ctr->log_cursor, log_cap);
    const int nU = ctr->n_unauth;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nlog; i += stride) {
        const int v = vlog[i];
        if (v >= 0) owner[v] = -1;
    }
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < nU; c += stride) {
        const int v = wait_v[c];
        if (v >= 0) cnt[v] = 0;
    }
}

template <int DIR, bool PERS>
cudaError_t launch_propagate(Work& w, const Geom& g, const int* O, const float* F, double eps, int sms,
                             cudaStream_t s) {
    PropArgs a;
    a.U = w.U; a.owner = w.owner; a.qmark = w.qmark;
    // queue marks are class ids of this launch: clear them (-1) first
    cudaMemsetAsync(w.qmark, 0xff, sizeof(int) * (size_t)g.n, s);
    a.parent = w.parent; a.wait_v = w.wait_v; a.cnt = w.cnt;
    a.spill_base = w.spill_base; a.spill_n = w.spill_n; a.heaprec = w.heaprec;
    a.spill_pool = w.spill_pool; a.spill_cap = w.spill_cap; a.heap_pool = w.heap_pool; a.heap_cap = w.heap_cap;
    a.vlog = w.vlog; a.vlog_cls = w.vlog_cls; a.log_cap = w.log_cap; a.tasks = w.tasks; a.ctr = w.ctr;
    a.F = F; a.eps = eps; a.ctop = w.ctop; a.authbits = w.authbits;
    const int pb = sms * 8;
    const int blocks = std::min(w.lanes / kThreads, sms * std::max(1, std::min(w.eng_bpsm, 8)));
    if (g.nn == 14) {
        first_step_kernel<DIR, 14, PERS><<<pb, 256, 0, s>>>(g, O, a, w.tasks);
        propagate_kernel<DIR, 14, PERS><<<blocks, kThreads, 0, s>>>(g, O, a);
    } else {
        first_step_kernel<DIR, 6, PERS><<<pb, 256, 0, s>>>(g, O, a, w.tasks);
        propagate_kernel<DIR, 6, PERS><<<blocks, kThreads, 0, s>>>(g, O, a);
    }
    w.launches += 2;
    if (PERS) {
        pers_clear_kernel<<<sms * 4, 256, 0, s>>>(w.ctr, w.vlog, w.wait_v, w.owner, w.cnt, w.log_cap);
        w.launches += 1;
    }
    return cudaGetLastError();
}

}  // namespace

template <int DIR>
cudaError_t propagate(Work& w, const Geom& g, const int* O, int sms, cudaStream_t s) {
    return launch_propagate<DIR, false>(w, g, O, nullptr, 0.0, sms, s);
}

template <int DIR>
cudaError_t select_persistent(Work& w, const Geom& g, const int* O, const float* F, double eps, int sms,
                              cudaStream_t s) {
    return launch_propagate<DIR, true>(w, g, O, F, eps, sms, s);
}

int propagate_lanes(int sms) { return sms * 8 * kThreads; }
// pool slack: every warp may hold one partly used reservation of each pool
long long propagate_log_slack(int lanes) { return (long long)(lanes / 32) * kLogChunk; }
long long propagate_spill_slack(int lanes) { return (long long)(lanes / 32) * kSpillChunk; }
long long propagate_heap_slack(int lanes) { return (long long)(lanes / 32) * 2048; }

template cudaError_t propagate<1>(Work&, const Geom&, const int*, int, cudaStream_t);
template cudaError_t propagate<-1>(Work&, const Geom&, const int*, int, cudaStream_t);
template cudaError_t select_persistent<1>(Work&, const Geom&, const int*, const float*, double, int, cudaStream_t);
template cudaError_t select_persistent<-1>(Work&, const Geom&, const int*, const float*, double, int, cudaStream_t);

}  // namespace lts
