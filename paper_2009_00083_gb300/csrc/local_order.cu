// Step 2 (Sec. 4.2, Eq. 3-5): a local order for every region R with saddle s.
//
//   l0 = Od on R, l0(s) = +inf, and l0(a) = -inf for one vertex a != s of R
//   that has a neighbour outside R.  a must not be a cut vertex of R (else the
//   first propagation does not end on it and no authorized minimum is left):
//   candidates are tried by increasing Od, and a candidate is kept when the
//   superlevel propagation from s visits it last, which happens exactly when
//   its removal leaves R connected.
//   Then alternate: superlevel propagation from s (largest first; inverse
//   visiting order = new local order) while some minimum lacks an outside
//   neighbour, and sublevel propagation from the current authorized minima,
//   the minima of the local order with an outside neighbour (smallest first;
//   visiting order = new local order) while some vertex other than s is a
//   maximum.
//   That alternation can cycle for ever.  A region whose alternation has not
//   ended after 2|R|+2 propagations (or has no authorized minimum to start
//   from) is redone from the first propagation's order with every vertex of
//   R\{s} that has an outside neighbour as a seed of each sublevel
//   propagation.  An order that repeats after a superlevel propagation proves
//   a cycle and ends the first attempt early (Brent's method: one saved
//   order, compared after every superlevel propagation and replaced after 1,
//   2, 4, ... of them); that only saves work, the result is the cap's.
// Propagations only use edges inside R.
//
// Tiers by region size r = |R|:
//   r <= 16 and r <= 32: one region per team of 16 / 32 lanes, one vertex per
//     lane in registers (adjacency as a bit mask over the team's lanes); a
//     propagation step is one team max/min reduction over the frontier and
//     one broadcast of the popped vertex's adjacency;
//   r <= 128, r <= 1024 and r <= 4096: one region per warp, arrays in shared
//     memory; a propagation runs in key space (the members' priorities are
//     ranks 0..r-1, the queue a bitmap over them with summary levels), so a
//     step is a few shared-memory loads and the neighbours' pushes;
//   larger: one region per warp, the same key-space queue in shared memory
//     with the key-indexed adjacency in HBM scratch (a 32-ary heap in shared
//     memory when the scratch pool is spent, and one region per lane with
//     binary heaps in HBM scratch when that heap overflows).
#include <algorithm>
#include <climits>

#include "lts_internal.cuh"

namespace lts {

namespace {

constexpr unsigned char kBnd = 1, kVis = 2, kTried = 4, kSeed = 16;
constexpr int kMedR = 1024;
constexpr int kHugeR = 4096;
constexpr int kNoNbr = 0xffff;

// ---------------------------------------------------------------------------
// storage policies: V (vertex), L / L2 (local orders), Hp (heap of local
// indices), F (flags), nbr(i, q) (local index of neighbour q, or -1)
// ---------------------------------------------------------------------------

// HBM scratch; neighbours recomputed from the grid and the region tags
template <int NN>
struct BigStore {
    int* v; int* l; int* l2; int* hp; unsigned char* f; int* p;
    Geom g; const int* owner; const int* loc; int tag; int s; int m;
    const int* O; int dir;
    // l0 without the minus-infinity vertex: Od on the members, s on top
    __device__ int L0(int i) const {
        if (i == m) return INT_MAX;
        const int o = __ldg(O + v[i]);
        return dir > 0 ? o : g.n - 1 - o;
    }
    __device__ int& V(int i) const { return v[i]; }
    __device__ int& L(int i) const { return l[i]; }
    __device__ int& L2(int i) const { return l2[i]; }
    __device__ int& P(int i) const { return p[i]; }
    __device__ int hp_get(int i) const { return hp[i]; }
    __device__ void hp_set(int i, int x) const { hp[i] = x; }
    __device__ unsigned char& F(int i) const { return f[i]; }
    __device__ int nbr(int i, int q) const {
        int x, y, z;
        coords_of(g, v[i], x, y, z);
        const int nb = nbr_of(g, x, y, z, q);
        if (nb < 0) return -1;
        if (nb == s) return m;
        if (__ldg(owner + nb) != tag) return -1;
        return __ldg(loc + nb);
    }
};

// ---------------------------------------------------------------------------
// the algorithm (one thread)
// ---------------------------------------------------------------------------

template <bool MAXF, class S>
__device__ __forceinline__ bool better(const S& T, int a, int b) {
    return MAXF ? T.L(a) > T.L(b) : T.L(a) < T.L(b);
}

template <bool MAXF, class S>
__device__ void hpush(const S& T, int& n, int i) {
    int p = n++;
    while (p > 0) {
        const int q = (p - 1) >> 1;
        const int hq = T.hp_get(q);
        if (!better<MAXF>(T, i, hq)) break;
        T.hp_set(p, hq);
        p = q;
    }
    T.hp_set(p, i);
}

template <bool MAXF, class S>
__device__ int hpop(const S& T, int& n) {
    const int top = T.hp_get(0);
    const int last = T.hp_get(--n);
    if (n == 0) return top;
    int p = 0;
    for (;;) {
        int l = 2 * p + 1;
        if (l >= n) break;
        if (l + 1 < n && better<MAXF>(T, T.hp_get(l + 1), T.hp_get(l))) ++l;
        const int hl = T.hp_get(l);
        if (!better<MAXF>(T, hl, last)) break;
        T.hp_set(p, hl);
        p = l;
    }
    T.hp_set(p, last);
    return top;
}

// superlevel propagation from s (local index m); L2 = inverse visiting
// order; returns the last vertex visited (-2 if R was not covered)
template <int NN, class S>
__device__ int max_flood(const S& T, int m, int r) {
    for (int i = 0; i < r; ++i) T.F(i) &= (unsigned char)~kVis;
    int n = 0, cnt = 0, last = -1;
    T.F(m) |= kVis;
    hpush<true>(T, n, m);
    while (n > 0) {
        const int i = hpop<true>(T, n);
        T.L2(i) = r - 1 - cnt++;
        last = i;
#pragma unroll
        for (int q = 0; q < NN; ++q) {
            const int j = T.nbr(i, q);
            if (j < 0 || (T.F(j) & kVis)) continue;
            T.F(j) |= kVis;
            hpush<true>(T, n, j);
        }
    }
    return cnt == r ? last : -2;
}

// sublevel propagation from the vertices flagged kSeed
template <int NN, class S>
__device__ bool min_flood(const S& T, int m, int r) {
    for (int i = 0; i < r; ++i) T.F(i) &= (unsigned char)~kVis;
    int n = 0, cnt = 0;
    for (int i = 0; i < m; ++i)
        if (T.F(i) & kSeed) { T.F(i) |= kVis; hpush<false>(T, n, i); }
    while (n > 0) {
        const int i = hpop<false>(T, n);
        T.L2(i) = cnt++;
#pragma unroll
        for (int q = 0; q < NN; ++q) {
            const int j = T.nbr(i, q);
            if (j < 0 || (T.F(j) & kVis)) continue;
            T.F(j) |= kVis;
            hpush<false>(T, n, j);
        }
    }
    return cnt == r;
}

template <int NN, class S>
__device__ bool has_unauth_min(const S& T, int r) {
    for (int i = 0; i < r; ++i) {
        if (T.F(i) & kBnd) continue;
        bool ismin = true;
#pragma unroll
        for (int q = 0; q < NN; ++q) {
            const int j = T.nbr(i, q);
            if (j >= 0 && T.L(j) < T.L(i)) ismin = false;
        }
        if (ismin) return true;
    }
    return false;
}

// flags the seeds of a sublevel propagation: the vertices of R\{s} with an
// outside neighbour that are minima of L (literal) or all of them; returns
// whether there is one
template <int NN, class S>
__device__ bool mark_seeds(const S& T, int m, bool literal) {
    bool any = false;
    for (int i = 0; i < m; ++i) {
        bool sd = (T.F(i) & kBnd) != 0;
        if (sd && literal) {
#pragma unroll
            for (int q = 0; q < NN; ++q) {
                const int j = T.nbr(i, q);
                if (j >= 0 && T.L(j) < T.L(i)) sd = false;
            }
        }
        T.F(i) = (unsigned char)(sd ? (T.F(i) | kSeed) : (T.F(i) & ~kSeed));
        any |= sd;
    }
    return any;
}

template <int NN, class S>
__device__ bool has_unauth_max(const S& T, int m) {
    for (int i = 0; i < m; ++i) {
        bool ismax = true;
#pragma unroll
        for (int q = 0; q < NN; ++q) {
            const int j = T.nbr(i, q);
            if (j >= 0 && T.L(j) > T.L(i)) ismax = false;
        }
        if (ismax) return true;
    }
    return false;
}

// Propagation count of a region that was redone with every boundary vertex
// as a seed (or-ed into the count returned by local_order_run).
constexpr int kFellBack = 1 << 30;

// Runs step 2 on a region whose V, L (= L0) and F (kBnd) are set.  On success
// L holds the local order; returns the number of propagations of the run
// whose result is kept (| kFellBack if the region was redone), or -1.
template <int NN, class S>
__device__ int local_order_run(const S& T, int m) {
    const int r = m + 1;
    bool ok = false;
    int a = -1;
    for (;;) {
        a = -1;
        for (int i = 0; i < m; ++i)
            if ((T.F(i) & (kBnd | kTried)) == kBnd && (a < 0 || T.L(i) < T.L(a))) a = i;
        if (a < 0) break;
        const int keep = T.L(a);
        T.L(a) = INT_MIN;
        const int last = max_flood<NN>(T, m, r);
        if (last == -2) break;
        if (last == a) { ok = true; break; }
        T.L(a) = keep;
        T.F(a) |= kTried;
    }
    if (!ok) return -1;
    const int cap = 2 * r + 2;
    for (int pass = 0; pass < 2; ++pass) {
        const bool literal = pass == 0;
        if (!literal) {                     // rebuild l1 in L2
            for (int i = 0; i < r; ++i) T.L(i) = T.L0(i);
            T.L(a) = INT_MIN;
            if (max_flood<NN>(T, m, r) != a) return -1;
        }
        for (int i = 0; i < r; ++i) { T.L(i) = T.L2(i); T.P(i) = T.L2(i); }
        int nfl = 1, res = 0;               // res: 1 done, -1 does not end, -2 error
        long long power = 1, lam = 0;
        for (;;) {
            if (!has_unauth_min<NN>(T, r)) { res = 1; break; }
            if (!mark_seeds<NN>(T, m, literal)) { res = -1; break; }
            if (++nfl > cap) { res = -1; break; }
            if (!min_flood<NN>(T, m, r)) { res = -2; break; }
            for (int i = 0; i < r; ++i) T.L(i) = T.L2(i);
            if (!has_unauth_max<NN>(T, m)) { res = 1; break; }
            if (++nfl > cap) { res = -1; break; }
            if (max_flood<NN>(T, m, r) < 0) { res = -2; break; }
            for (int i = 0; i < r; ++i) T.L(i) = T.L2(i);
            if (literal) {
                bool same = true;
                for (int i = 0; i < r && same; ++i) same = T.P(i) == T.L(i);
                if (same) { res = -1; break; }
                if (++lam == power) {
                    for (int i = 0; i < r; ++i) T.P(i) = T.L(i);
                    power *= 2;
                    lam = 0;
                }
            }
        }
        if (res == 1) return literal ? nfl : (nfl | kFellBack);
        if (res == -2 || !literal) return -1;
    }
    return -1;
}

struct LOArgs {
    const int* O; const int* owner; const int* loc; const int* members; const int* reg_start;
    const int* reg_size; const int* reg_saddle; int* lhat;
    int* lo_v; int* lo_L; int* lo_L2; int* lo_heap; unsigned char* lo_flag; int* lo_P;
    const int* tier_list; DevCounters* ctr;
    int* lo_adj; long long lo_adj_cap;
};

// ---- tiers 1-2: one region per team of TS lanes (r <= TS), registers ----

template <int TS>
struct TeamLO {
    unsigned tm;   // team mask
    int tb, tl, lane;
};

// superlevel propagation from the lane holding s; returns the team lane of
// the last visited vertex, -2 if R was not covered; l2 = inverse visit order
template <int TS>
__device__ __forceinline__ int team_max_flood(const TeamLO<TS>& T, bool act, int L, unsigned adj, int m, int r,
                                              int& l2) {
    bool inq = T.tl == m, vis = false;
    int last = -2;
    for (int step = 0; step < r; ++step) {
        const int key = (act && inq && !vis) ? L : INT_MIN;
        const int K = __reduce_max_sync(T.tm, key);
        if (K == INT_MIN) return -2;
        const int p = __ffs(__ballot_sync(T.tm, act && inq && !vis && key == K)) - 1;
        if (T.lane == p) { vis = true; l2 = r - 1 - step; }
        const unsigned ap = __shfl_sync(T.tm, adj, p);
        if ((ap >> T.tl) & 1u) inq = true;
        last = p - T.tb;
    }
    return last;
}

// sublevel propagation from every lane with an outside neighbour but s
template <int TS>
__device__ __forceinline__ bool team_min_flood(const TeamLO<TS>& T, bool act, int L, unsigned adj, bool seed,
                                               int r, int& l2) {
    bool inq = act && seed, vis = false;
    for (int step = 0; step < r; ++step) {
        const int key = (act && inq && !vis) ? L : INT_MAX;
        const int K = __reduce_min_sync(T.tm, key);
        if (K == INT_MAX) return false;
        const int p = __ffs(__ballot_sync(T.tm, act && inq && !vis && key == K)) - 1;
        if (T.lane == p) { vis = true; l2 = step; }
        const unsigned ap = __shfl_sync(T.tm, adj, p);
        if ((ap >> T.tl) & 1u) inq = true;
    }
    return true;
}

// is this lane's vertex a strict extremum of L among its neighbours in R
template <int TS>
__device__ __forceinline__ void team_extremum(const TeamLO<TS>& T, int L, unsigned adj, bool& is_min,
                                              bool& is_max) {
    is_min = true;
    is_max = true;
#pragma unroll
    for (int q = 0; q < TS; ++q) {
        const int lq = __shfl_sync(T.tm, L, T.tb + q);
        if ((adj >> q) & 1u) {
            if (lq < L) is_min = false;
            if (lq > L) is_max = false;
        }
    }
}

template <int DIR, int NN, int TS>
__global__ void __launch_bounds__(128, 12) lo_team_kernel(Geom g, LOArgs a, const int* list, const int* d_count) {
    if (failed(&a.ctr->status)) return;
    TeamLO<TS> T;
    T.lane = threadIdx.x & 31;
    T.tb = T.lane & ~(TS - 1);
    T.tl = T.lane - T.tb;
    T.tm = TS == 32 ? 0xffffffffu : (((1u << TS) - 1u) << T.tb);
    const int team = (blockIdx.x * blockDim.x + threadIdx.x) / TS;
    const int nteams = gridDim.x * blockDim.x / TS;
    const int cnt = list ? *d_count : a.ctr->n_regions;
    int mx = 0, nfb = 0;
    long long tot = 0;
    for (int k = team; k < cnt; k += nteams) {
        const int rid = list ? list[k] : k;
        const int m = a.reg_size[rid];
        const int r = m + 1;
        if (r > TS) continue;
        const int s = a.reg_saddle[rid];
        const int tag = -2 - rid;
        const int st0 = a.reg_start[rid];
        const bool act = T.tl < r;
        const bool mem = T.tl < m;
        int vtx = -1;
        if (act) vtx = mem ? a.members[st0 + T.tl] : s;
        unsigned adj = 0;
        bool bnd = false;
        int L = INT_MIN;
        if (act) {
            int x, y, z;
            coords_of(g, vtx, x, y, z);
            int nbv[NN], ow[NN];
#pragma unroll
            for (int q = 0; q < NN; ++q) {
                nbv[q] = nbr_of(g, x, y, z, q);
                ow[q] = (nbv[q] >= 0 && nbv[q] != s) ? __ldg(a.owner + nbv[q]) : 0;
            }
#pragma unroll
            for (int q = 0; q < NN; ++q) {
                const int nb = nbv[q];
                if (nb < 0) continue;
                if (nb == s) adj |= 1u << m;
                else if (ow[q] == tag) adj |= 1u << __ldg(a.loc + nb);
                else bnd = true;
            }
            L = mem ? od<DIR>(__ldg(a.O + vtx), g.n) : INT_MAX;
        }
        // the minus-infinity vertex: lowest boundary-adjacent non-cut member
        bool tried = false, ok = false;
        int l2 = 0;
        const int keepL = L;
        for (;;) {
            const int ck = (mem && bnd && !tried) ? L : INT_MAX;
            const int cmin = __reduce_min_sync(T.tm, ck);
            if (cmin == INT_MAX) break;
            const int ap = __ffs(__ballot_sync(T.tm, ck == cmin && mem && bnd && !tried)) - 1;
            if (T.lane == ap) L = -1;               // -infinity: every Od is >= 0
            const int last = team_max_flood(T, act, L, adj, m, r, l2);
            if (last == -2) break;
            if (last == ap - T.tb) { ok = true; break; }
            if (T.lane == ap) { L = keepL; tried = true; }
        }
        int nfl = -1;
        bool fell_back = false;
        if (ok) {
            const int l1 = l2;
            const int cap = 2 * r + 2;
            for (int pass = 0; pass < 2 && nfl < 0; ++pass) {
                const bool literal = pass == 0;
                L = l1;
                int saved = l1, fl = 1, res = 0;   // res: 1 done, -1 does not end, -2 error
                int power = 1, lam = 0;
                for (;;) {
                    bool mn, mxx;
                    team_extremum(T, L, adj, mn, mxx);
                    if (!__any_sync(T.tm, act && !bnd && mn)) { res = 1; break; }
                    const bool sd = mem && bnd && (!literal || mn);
                    if (!__any_sync(T.tm, sd)) { res = -1; break; }
                    if (++fl > cap) { res = -1; break; }
                    if (!team_min_flood(T, act, L, adj, sd, r, l2)) { res = -2; break; }
                    L = l2;
                    team_extremum(T, L, adj, mn, mxx);
                    if (!__any_sync(T.tm, mem && mxx)) { res = 1; break; }
                    if (++fl > cap) { res = -1; break; }
                    if (team_max_flood(T, act, L, adj, m, r, l2) < 0) { res = -2; break; }
                    L = l2;
                    if (literal) {
                        if (__all_sync(T.tm, !act || L == saved)) { res = -1; break; }
                        if (++lam == power) { saved = L; power *= 2; lam = 0; }
                    }
                }
                if (res == 1) { nfl = fl; fell_back = !literal; }
                else if (res == -2) break;
            }
        }
        if (nfl < 0) {
            if (T.tl == 0) set_status(&a.ctr->status, LTS_ERR_INTERNAL);
            continue;
        }
        if (mem) a.lhat[st0 + T.tl] = L;
        mx = max(mx, nfl);
        tot += nfl;
        nfb += fell_back;
    }
    // one count per region: only the team's first lane reports
    if (T.tl != 0) { mx = 0; tot = 0; nfb = 0; }
    __syncwarp();
    warp_atomic_max(&a.ctr->max_floods, mx);
    warp_atomic_add64(&a.ctr->total_floods, tot);
    warp_atomic_add(&a.ctr->lo_fallbacks, nfb);
}

// ---- tiers 3-5: one warp per region of at most 128, 1024 or 4096 vertices ----

template <int NN>
struct Dense {
    int* v; int* L; int* L2; int* P; unsigned short* adj; unsigned char* f;   // f: kBnd | kVis | kTried | kInq | kSeed
    unsigned short* rk;      // rank of each member's Od among the members (key-space propagations)
    unsigned short* kidx;    // key -> local index
    // queue bitmaps over the keys: bit k of b1; bit w of b2: b1 word w is not 0;
    // bit u of b3: b2 word u is not 0 (b2 has one word below 1025 keys, b3 is then unused)
    unsigned* b1; unsigned* b2; unsigned* b3;
};
constexpr unsigned char kInq = 8;

template <int NN>
__device__ __forceinline__ void dense_checks(const Dense<NN>& D, int r, int m, int lane, bool& umin, bool& umax) {
    bool a_min = false, a_max = false;
    for (int i = lane; i < r; i += 32) {
        const int l = D.L[i];
        bool is_min = true, is_max = true;
#pragma unroll
        for (int q = 0; q < NN; ++q) {
            const unsigned short j = D.adj[i * NN + q];
            if (j == kNoNbr) continue;
            const int lj = D.L[j];
            if (lj < l) is_min = false;
            if (lj > l) is_max = false;
        }
        if (is_min && !(D.f[i] & kBnd)) a_min = true;
        if (is_max && i < m) a_max = true;
    }
    umin = __any_sync(0xffffffffu, a_min);
    umax = __any_sync(0xffffffffu, a_max);
}

// Superlevel (MAXF) or sublevel propagation over the region in key space:
// the priority of local index i is a key in 0..r-1 in the order of L, so the
// queue is a bitmap over the keys with one or two summary levels: a pop takes
// the highest (lowest) set bit in two or three shared-memory loads, a push sets
// as many bits, and the visiting order is that of any priority queue on the
// same keys.  Keys: with tryc >= 0 (a candidate try of the first propagation)
// the candidate has key 0, s key r-1 and the other members their Od rank
// (shifted up by one below the candidate's); otherwise L itself, a
// permutation of 0..r-1 after the first propagation.
template <bool MAXF, int NN, int RMAX>
__device__ __forceinline__ int dense_flood_keys(const Dense<NN>& D, int r, int lane, int tryc) {
    constexpr bool kL3 = RMAX > 1024;
    const int rtry = tryc >= 0 ? D.rk[tryc] : 0;
    auto key = [&](int i) -> int {
        if (tryc < 0) return D.L[i];
        if (i == tryc) return 0;
        if (i == r - 1) return r - 1;
        const int k = D.rk[i];
        return k < rtry ? k + 1 : k;
    };
    auto push = [&](int kk) {
        atomicOr(&D.b1[kk >> 5], 1u << (kk & 31));
        atomicOr(&D.b2[kk >> 10], 1u << ((kk >> 5) & 31));
        if (kL3) atomicOr(&D.b3[0], 1u << (kk >> 10));
    };
    const int w1n = (r + 31) >> 5;
    for (int w = lane; w < w1n; w += 32) D.b1[w] = 0u;
    if (lane < 4) D.b2[lane] = 0u;
    if (kL3 && lane == 0) D.b3[0] = 0u;
    for (int i = lane; i < r; i += 32) D.kidx[key(i)] = (unsigned short)i;
    __syncwarp();
    for (int i = lane; i < r; i += 32)
        if (D.f[i] & kInq) push(key(i));
    __syncwarp();
    int last = -2;
    for (int step = 0; step < r; ++step) {
        int i2 = 0;
        unsigned w3 = 0u;
        if (kL3) {
            w3 = D.b3[0];
            if (!w3) return -2;
            i2 = MAXF ? 31 - __clz(w3) : __ffs(w3) - 1;
        }
        const unsigned w2 = D.b2[i2];
        if (!w2) return -2;
        const int i1 = i2 * 32 + (MAXF ? 31 - __clz(w2) : __ffs(w2) - 1);
        const unsigned w1 = D.b1[i1];
        if (!w1) return -2;                               // inconsistent levels: reported as an error
        const int b = MAXF ? 31 - __clz(w1) : __ffs(w1) - 1;
        const int p = D.kidx[i1 * 32 + b];
        __syncwarp();
        if (lane == 0) {
            const unsigned n1 = w1 & ~(1u << b);
            D.b1[i1] = n1;
            if (!n1) {
                const unsigned n2 = w2 & ~(1u << (i1 & 31));
                D.b2[i2] = n2;
                if (kL3 && !n2) D.b3[0] = w3 & ~(1u << i2);
            }
            D.f[p] |= kVis;
            D.L2[p] = MAXF ? r - 1 - step : step;
        }
        __syncwarp();
        if (lane < NN) {
            const unsigned short j = D.adj[p * NN + lane];
            if (j != kNoNbr) {
                const unsigned char fj = D.f[j];
                if (!(fj & kInq)) {                       // enters the queue once (the neighbours of p are distinct)
                    D.f[j] = fj | kInq;
                    push(key(j));
                }
            }
        }
        __syncwarp();
        last = p;
    }
    return last;
}

// rk[i] = rank of L[i] among L[0..m-1] (distinct values): a bitonic sort of
// the values in P (padded with INT_MAX to a power of two), then a binary
// search per member
template <int NN>
__device__ __forceinline__ void dense_ranks(const Dense<NN>& D, int m, int lane) {
    int n2 = 1;
    while (n2 < m) n2 <<= 1;
    for (int i = lane; i < n2; i += 32) D.P[i] = i < m ? D.L[i] : INT_MAX;
    __syncwarp();
    for (int k = 2; k <= n2; k <<= 1)
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int t = lane; t < (n2 >> 1); t += 32) {
                const int i = ((t & ~(j - 1)) << 1) | (t & (j - 1));   // bit j of i is clear
                const int a = D.P[i], b = D.P[i + j];
                if ((a > b) == ((i & k) == 0)) { D.P[i] = b; D.P[i + j] = a; }
            }
            __syncwarp();
        }
    for (int i = lane; i < m; i += 32) {
        const int li = D.L[i];
        int lo = 0, hi = m;
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (D.P[mid] < li) lo = mid + 1;
            else hi = mid;
        }
        D.rk[i] = (unsigned short)lo;
    }
    __syncwarp();
}

// flags the seeds of a sublevel propagation (see mark_seeds); returns whether there is one
template <int NN>
__device__ __forceinline__ bool dense_mark_seeds(const Dense<NN>& D, int m, int lane, bool literal) {
    bool any = false;
    for (int i = lane; i < m; i += 32) {
        bool sd = (D.f[i] & kBnd) != 0;
        if (sd && literal) {
            const int l = D.L[i];
#pragma unroll
            for (int q = 0; q < NN; ++q) {
                const unsigned short j = D.adj[i * NN + q];
                if (j != kNoNbr && D.L[j] < l) sd = false;
            }
        }
        D.f[i] = (unsigned char)(sd ? (D.f[i] | kSeed) : (D.f[i] & ~kSeed));
        any |= sd;
    }
    return __any_sync(0xffffffffu, any);
}

// The bounded cut search of the warp tier (wr_cuts below) on a dense tier's
// shared-memory adjacency: before candidate a's first propagation, a search
// from each neighbour of a in R (but s, local index m) over R \ {a} that ends
// within 64 vertices without reaching s or a vertex an earlier search for a
// reached has found a piece that a cuts off, so the propagation would not end
// on a.  mark[] (P) holds a * 16 + t for the vertices the t-th search for a
// reached; q (L2, free before the propagation) holds the search queue and, in
// q[64], its length.
template <int NN>
__device__ bool dense_cuts(const Dense<NN>& D, int ai, int m, int lane) {
    constexpr int kBudget = 64;
    int* mark = D.P;
    int* q = D.L2;
    const int nb = lane < NN ? (int)D.adj[ai * NN + lane] : (int)kNoNbr;
    unsigned todo = __ballot_sync(0xffffffffu, nb != kNoNbr && nb != m);
    const int base = ai * 16;
    int t = 0;
    while (todo) {
        const int src = __ffs(todo) - 1;
        todo &= todo - 1;
        const int b0 = __shfl_sync(0xffffffffu, nb, src);
        const int mb = mark[b0];
        if (mb >= base && mb < base + 16) continue;   // reached by an earlier search for a
        const int stamp = base + t++;
        __syncwarp();
        if (lane == 0) {
            mark[b0] = stamp;
            q[0] = b0;
            q[kBudget] = 1;
        }
        __syncwarp();
        int head = 0;
        bool reach = false, over = false;
        for (;;) {
            const int tail = q[kBudget];
            if (head >= tail) break;
            const int i = head + lane < tail ? q[head + lane] : -1;
            head = min(tail, head + 32);
            bool rs = false;
            if (i >= 0) {
#pragma unroll
                for (int k = 0; k < NN; ++k) {
                    const int j = (int)D.adj[i * NN + k];
                    if (j == (int)kNoNbr || j == ai) continue;
                    if (j == m) { rs = true; continue; }
                    const int old = atomicExch(mark + j, stamp);
                    if (old == stamp) continue;
                    if (old >= base && old < base + 16) { rs = true; continue; }   // joins an earlier search's piece
                    const int slot = atomicAdd(q + kBudget, 1);
                    if (slot < kBudget) q[slot] = j;
                }
            }
            __syncwarp();
            reach = __any_sync(0xffffffffu, rs);
            over = q[kBudget] > kBudget;
            if (reach || over) break;
        }
        if (!reach && !over) return true;
    }
    return false;
}

// per warp: v, L, L2, P (ints), adj (NN ushorts), rk and kidx (ushorts) per
// vertex; the key bitmaps (b1: RMAX bits, b2: 4 words, b3: 1 word, 16-byte
// slots); the flags (a byte per vertex)
template <int NN, int RMAX>
__host__ __device__ constexpr size_t dense_smem_per_warp() {
    return (size_t)RMAX * (4 * 4 + 2 * NN + 4 + 1) + (size_t)RMAX / 8 + 48;
}

// one region per warp, WPB warps per block, regions of at most RMAX vertices
template <int DIR, int NN, int RMAX, int WPB>
__global__ void __launch_bounds__(32 * WPB) lo_dense_kernel(Geom g, LOArgs a, const int* list, const int* d_count) {
    extern __shared__ unsigned char smem[];
    if (failed(&a.ctr->status)) return;
    const int wib = threadIdx.x >> 5;
    unsigned char* mine = smem + (size_t)wib * dense_smem_per_warp<NN, RMAX>();
    Dense<NN> D;
    D.v = reinterpret_cast<int*>(mine);
    D.L = D.v + RMAX;
    D.L2 = D.L + RMAX;
    D.P = D.L2 + RMAX;
    D.adj = reinterpret_cast<unsigned short*>(D.P + RMAX);
    static_assert(RMAX % 64 == 0 && RMAX <= 4096, "key bitmaps of the dense tiers");
    D.rk = D.adj + RMAX * NN;
    D.kidx = D.rk + RMAX;
    D.b1 = reinterpret_cast<unsigned*>(D.kidx + RMAX);
    D.b2 = D.b1 + RMAX / 32;
    D.b3 = D.b2 + 4;
    D.f = reinterpret_cast<unsigned char*>(D.b3 + 4);
    const int lane = threadIdx.x & 31;
    const int cnt = *d_count;
    const int gw = blockIdx.x * WPB + wib, nw = gridDim.x * WPB;
    for (int k = gw; k < cnt; k += nw) {
        const int rid = list[k];
        const int m = a.reg_size[rid];
        const int r = m + 1;
        const int s = a.reg_saddle[rid];
        const int tag = -2 - rid;
        const int st0 = a.reg_start[rid];
        for (int i = lane; i < r; i += 32) {
            const int vtx = i < m ? a.members[st0 + i] : s;
            D.v[i] = vtx;
            int x, y, z;
            coords_of(g, vtx, x, y, z);
            unsigned char fl = 0;
#pragma unroll
            for (int q = 0; q < NN; ++q) {
                const int nb = nbr_of(g, x, y, z, q);
                unsigned short li = kNoNbr;
                if (nb >= 0) {
                    if (nb == s) li = (unsigned short)m;
                    else if (__ldg(a.owner + nb) == tag) li = (unsigned short)__ldg(a.loc + nb);
                    else fl = kBnd;
                }
                D.adj[i * NN + q] = li;
            }
            D.f[i] = fl;
            D.L[i] = i < m ? od<DIR>(__ldg(a.O + vtx), g.n) : INT_MAX;
        }
        __syncwarp();
        dense_ranks(D, m, lane);                          // Od rank of every member
        for (int i = lane; i < r; i += 32) D.P[i] = -1;  // the cut searches' marks
        __syncwarp();
        // the minus-infinity vertex
        bool ok = false;
        int ai = -1;
        for (;;) {
            int best = INT_MAX, bi = -1;
            for (int i = lane; i < m; i += 32)
                if ((D.f[i] & (kBnd | kTried)) == kBnd && D.L[i] < best) { best = D.L[i]; bi = i; }
            const int K = __reduce_min_sync(0xffffffffu, best);
            if (K == INT_MAX) break;
            const int src = __ffs(__ballot_sync(0xffffffffu, bi >= 0 && best == K)) - 1;
            ai = __shfl_sync(0xffffffffu, bi, src);
            if (dense_cuts(D, ai, m, lane)) {            // ai cuts off a small piece of R
                if (lane == 0) D.f[ai] |= kTried;
                __syncwarp();
                continue;
            }
            const int keep = D.L[ai];
            __syncwarp();
            if (lane == 0) D.L[ai] = -1;
            for (int i = lane; i < r; i += 32) D.f[i] = (unsigned char)((D.f[i] & ~(kVis | kInq)) | (i == m ? kInq : 0));
            __syncwarp();
            const int last = dense_flood_keys<true, NN, RMAX>(D, r, lane, ai);
            if (last == -2) break;
            if (last == ai) { ok = true; break; }
            if (lane == 0) { D.L[ai] = keep; D.f[ai] |= kTried; }
            __syncwarp();
        }
        int nfl = -1;
        bool fell_back = false;
        if (ok) {
            const int cap = 2 * r + 2;
            for (int pass = 0; pass < 2 && nfl < 0; ++pass) {
                const bool literal = pass == 0;
                if (!literal) {
                    // redo from l1: rebuild it in L2 with the accepted candidate at -infinity
                    for (int i = lane; i < r; i += 32) {
                        D.L[i] = i == ai ? -1 : (i < m ? od<DIR>(__ldg(a.O + D.v[i]), g.n) : INT_MAX);
                        D.f[i] = (unsigned char)((D.f[i] & ~(kVis | kInq)) | (i == m ? kInq : 0));
                    }
                    __syncwarp();
                    if (dense_flood_keys<true, NN, RMAX>(D, r, lane, ai) != ai)
                        break;
                }
                for (int i = lane; i < r; i += 32) { D.L[i] = D.L2[i]; D.P[i] = D.L2[i]; }
                __syncwarp();
                int fl = 1, res = 0;          // res: 1 done, -1 does not end, -2 error
                int power = 1, lam = 0;
                for (;;) {
                    bool umin, umax;
                    dense_checks(D, r, m, lane, umin, umax);
                    if (!umin) { res = 1; break; }
                    if (!dense_mark_seeds(D, m, lane, literal)) { res = -1; break; }
                    if (++fl > cap) { res = -1; break; }
                    for (int i = lane; i < r; i += 32)
                        D.f[i] = (unsigned char)((D.f[i] & ~(kVis | kInq)) | ((i < m && (D.f[i] & kSeed)) ? kInq : 0));
                    __syncwarp();
                    if (dense_flood_keys<false, NN, RMAX>(D, r, lane, -1) == -2) {
                        res = -2;
                        break;
                    }
                    for (int i = lane; i < r; i += 32) D.L[i] = D.L2[i];
                    __syncwarp();
                    dense_checks(D, r, m, lane, umin, umax);
                    if (!umax) { res = 1; break; }
                    if (++fl > cap) { res = -1; break; }
                    for (int i = lane; i < r; i += 32)
                        D.f[i] = (unsigned char)((D.f[i] & ~(kVis | kInq)) | (i == m ? kInq : 0));
                    __syncwarp();
                    if (dense_flood_keys<true, NN, RMAX>(D, r, lane, -1) == -2) {
                        res = -2;
                        break;
                    }
                    for (int i = lane; i < r; i += 32) D.L[i] = D.L2[i];
                    __syncwarp();
                    if (literal) {
                        bool same = true;
                        for (int i = lane; i < r; i += 32) same &= D.P[i] == D.L[i];
                        if (__all_sync(0xffffffffu, same)) { res = -1; break; }
                        if (++lam == power) {
                            for (int i = lane; i < r; i += 32) D.P[i] = D.L[i];
                            __syncwarp();
                            power *= 2;
                            lam = 0;
                        }
                    }
                }
                if (res == 1) { nfl = fl; fell_back = !literal; }
                else if (res == -2) break;
            }
        }
        __syncwarp();
        if (nfl < 0) {
            if (lane == 0) set_status(&a.ctr->status, LTS_ERR_INTERNAL);
            continue;
        }
        for (int i = lane; i < m; i += 32) a.lhat[st0 + i] = D.L[i];
        if (lane == 0) {
            atomicMax(&a.ctr->max_floods, nfl);
            atomicAdd((unsigned long long*)&a.ctr->total_floods, (unsigned long long)nfl);
            if (fell_back) atomicAdd(&a.ctr->lo_fallbacks, 1);
        }
        __syncwarp();
    }
}

// ---- tier 6: one warp per region above kHugeR vertices ----
// The same algorithm as local_order_run, run by a warp: the frontier is a
// 32-ary max-heap of (biased key << 32 | local index) in shared memory, so a
// pop sifts down one level per warp-wide load and max-reduction; the keys are
// unique, so the pops come in the same order as with any other heap.  V, L,
// L2 and the flags live in the region's HBM scratch; neighbours are
// recomputed from the grid and the region tags.  A region whose frontier
// outgrows the heap is redone by lane 0 on the single-thread path.
constexpr int kWarpHeapCap = 28672;

struct WarpRegion {
    int* V; int* L; int* L2; unsigned char* F;
    Geom g; const int* owner; const int* loc; int tag; int s; int m; int r;
    int* adj;          // local index of neighbour q of local vertex i at [i * NN + q], or null
};

__device__ __forceinline__ int wr_nbr(const WarpRegion& R, int vtx, int q) {
    int x, y, z;
    coords_of(R.g, vtx, x, y, z);
    const int nb = nbr_of(R.g, x, y, z, q);
    if (nb < 0) return -1;
    if (nb == R.s) return R.m;
    if (__ldg(R.owner + nb) != R.tag) return -1;
    return __ldg(R.loc + nb);
}

// neighbour q of local vertex i (local index, -1 outside R)
template <int NN>
__device__ __forceinline__ int wr_nbr_of(const WarpRegion& R, int i, int q) {
    return R.adj ? R.adj[(long long)i * NN + q] : wr_nbr(R, R.V[i], q);
}

// biased key: unsigned order of the (max-first) or reversed (min-first) key
template <bool MAXF>
__device__ __forceinline__ unsigned long long wr_entry(int key, int i) {
    unsigned k = (unsigned)key ^ 0x80000000u;
    if (!MAXF) k = ~k;
    return ((unsigned long long)k << 32) | (unsigned)i;
}

// lane 0 pushes e; hn is the warp-uniform heap size
__device__ __forceinline__ void wh_push(unsigned long long* H, int& hn, unsigned long long e, int lane) {
    if (lane == 0) {
        int p = hn;
        while (p > 0) {
            const int par = (p - 1) >> 5;
            const unsigned long long hp = H[par];
            if (hp >= e) break;
            H[p] = hp;
            p = par;
        }
        H[p] = e;
    }
    ++hn;
    __syncwarp();
}

__device__ __forceinline__ unsigned long long wh_pop(unsigned long long* H, int& hn, int lane) {
    const unsigned long long top = H[0];
    --hn;
    if (hn == 0) { __syncwarp(); return top; }
    const unsigned long long last = H[hn];
    int p = 0;
    for (;;) {
        const int c0 = p * 32 + 1;
        if (c0 >= hn) break;
        const int c = c0 + lane;
        const unsigned long long hv = c < hn ? H[c] : 0ull;
        const unsigned hi = c < hn ? (unsigned)(hv >> 32) : 0u;
        const unsigned K = __reduce_max_sync(0xffffffffu, hi);
        const int lm = __ffs(__ballot_sync(0xffffffffu, c < hn && hi == K)) - 1;
        const unsigned long long mv = __shfl_sync(0xffffffffu, hv, lm);
        if (mv <= last) break;
        __syncwarp();
        if (lane == 0) H[p] = mv;
        p = c0 + lm;
    }
    __syncwarp();
    if (lane == 0) H[p] = last;
    __syncwarp();
    return top;
}

// superlevel (MAXF) or sublevel propagation; returns the last vertex (max),
// -2 if R was not covered, -3 if the heap overflowed
template <bool MAXF, int NN>
__device__ int wr_flood(const WarpRegion& R, unsigned long long* H, int lane) {
    for (int i = lane; i < R.r; i += 32) R.F[i] &= (unsigned char)~kVis;
    __syncwarp();
    int hn = 0;
    if (MAXF) {
        if (lane == 0) R.F[R.m] |= kVis;
        wh_push(H, hn, wr_entry<true>(R.L[R.m], R.m), lane);
    } else {
        for (int b = 0; b < R.m; b += 32) {
            const int i = b + lane;
            const bool sd = i < R.m && (R.F[i] & kSeed);
            if (sd) R.F[i] |= kVis;
            const int key = sd ? R.L[i] : 0;
            unsigned mk = __ballot_sync(0xffffffffu, sd);
            while (mk) {
                const int l = __ffs(mk) - 1;
                mk &= mk - 1;
                const int ki = __shfl_sync(0xffffffffu, key, l);
                if (hn >= kWarpHeapCap) return -3;
                wh_push(H, hn, wr_entry<false>(ki, b + l), lane);
            }
        }
    }
    int cnt = 0, last = -1;
    while (hn > 0) {
        const unsigned long long top = wh_pop(H, hn, lane);
        const int i = (int)(top & 0xffffffffu);
        if (lane == 0) R.L2[i] = MAXF ? R.r - 1 - cnt : cnt;
        ++cnt;
        last = i;
        int j = -1, key = 0;
        if (lane < NN) {
            j = wr_nbr_of<NN>(R, i, lane);
            if (j >= 0 && !(R.F[j] & kVis)) {
                R.F[j] |= kVis;
                key = R.L[j];
            } else {
                j = -1;
            }
        }
        unsigned mk = __ballot_sync(0xffffffffu, j >= 0);
        while (mk) {
            const int l = __ffs(mk) - 1;
            mk &= mk - 1;
            const int jj = __shfl_sync(0xffffffffu, j, l);
            const int kk = __shfl_sync(0xffffffffu, key, l);
            if (hn >= kWarpHeapCap) return -3;
            wh_push(H, hn, wr_entry<MAXF>(kk, jj), lane);
        }
    }
    if (!MAXF) return cnt == R.r ? 0 : -2;
    return cnt == R.r ? last : -2;
}

// ---- floods in key space (after the first flood L is a permutation of 0..r-1) ----
// NK[k * NN + q] holds the key of neighbour q of the vertex with key k (-1 if
// none); the frontier is a three-level bitmap over the keys in shared memory
// (the summary levels give the highest or lowest set bit in three loads,
// pushes are lane-parallel atomicOr, no capacity limit) and the visited set a
// bitmap.
//
// A propagation pops several keys per round.  The round takes the next keys
// of the queue c_0, c_1, ... (up to 32: every set bit of the 32 bitmap words
// from the top one on, in pop order), one per lane, and loads their NK rows
// together.  Popping them one by one pops c_j right after c_{j-1} exactly
// when no key queued by c_0..c_{j-1} comes before c_j; a queued key is a
// neighbour key not yet visited, so a prefix scan over the lanes of the best
// such key finds the longest prefix c_0..c_{V-1} (V >= 1) that the one-by-one
// propagation pops in that order.  The round pops that prefix (visiting
// order, queue bits cleared) and queues its new neighbours; the rest of the
// candidates stay queued.  The visiting order is the one-by-one order.
struct KeyQueue {
    unsigned* q1; unsigned* q2; unsigned* q3; unsigned* vis;
    int n1, n2, n3;                        // words per level (n3 <= 32)
    int* candk;                            // the round's candidate keys (32 slots)
};

__device__ __forceinline__ void kq_push(const KeyQueue& Q, int k) {
    atomicOr(Q.q1 + (k >> 5), 1u << (k & 31));
    atomicOr(Q.q2 + (k >> 10), 1u << ((k >> 5) & 31));
    atomicOr(Q.q3 + (k >> 15), 1u << ((k >> 10) & 31));
}

// index of the level-1 word that holds the highest (lowest) queued key, -1 if
// the queue is empty
template <bool MAXF>
__device__ __forceinline__ int kq_top_word(const KeyQueue& Q, int lane) {
    const unsigned w3l = lane < Q.n3 ? Q.q3[lane] : 0u;
    const unsigned m3 = __ballot_sync(0xffffffffu, w3l != 0u);
    if (!m3) return -1;
    const int l3 = MAXF ? 31 - __clz(m3) : __ffs(m3) - 1;
    const unsigned w3 = __shfl_sync(0xffffffffu, w3l, l3);
    const int i2 = l3 * 32 + (MAXF ? 31 - __clz(w3) : __ffs(w3) - 1);
    if (i2 >= Q.n2) return -1;                 // inconsistent levels: reported as empty (an error)
    const unsigned w2 = Q.q2[i2];
    if (w2 == 0u) return -1;
    const int i1 = i2 * 32 + (MAXF ? 31 - __clz(w2) : __ffs(w2) - 1);
    return i1 < Q.n1 ? i1 : -1;
}

// removes key k from the queue (lanes may remove keys of one word at once:
// the lane whose removal empties a word clears its summary bit)
__device__ __forceinline__ void kq_remove(const KeyQueue& Q, int k) {
    const unsigned b1 = 1u << (k & 31);
    if ((atomicAnd(Q.q1 + (k >> 5), ~b1) & ~b1) != 0u) return;
    const unsigned b2 = 1u << ((k >> 5) & 31);
    if ((atomicAnd(Q.q2 + (k >> 10), ~b2) & ~b2) != 0u) return;
    atomicAnd(Q.q3 + (k >> 15), ~(1u << ((k >> 10) & 31)));
}

// One propagation in key space over the keys Lk (a permutation of 0..r-1; Lk
// may be L2 itself); L2 gets the visiting order.  Returns the last key popped
// (the maxima flood) or 0, or -2 if R was not covered.
template <bool MAXF, int NN>
__device__ int wr_flood_keys(const WarpRegion& R, const int* Lk, int* NK, int* ordk, const KeyQueue& Q, int lane) {
    const int r = R.r;
    // NK from the local adjacency, four vertices per lane in flight
    constexpr int U = 4;
    for (int i0 = lane; i0 < r; i0 += 32 * U) {
        int k[U];
        int j[U][NN];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int i = i0 + 32 * u;
            k[u] = i < r ? Lk[i] : -1;
#pragma unroll
            for (int q = 0; q < NN; ++q) j[u][q] = i < r ? R.adj[(long long)i * NN + q] : -1;
        }
#pragma unroll
        for (int u = 0; u < U; ++u)
#pragma unroll
            for (int q = 0; q < NN; ++q) j[u][q] = j[u][q] >= 0 ? Lk[j[u][q]] : -1;
#pragma unroll
        for (int u = 0; u < U; ++u)
            if (k[u] >= 0) {
#pragma unroll
                for (int q = 0; q < NN; ++q) NK[(long long)k[u] * NN + q] = j[u][q];
            }
    }
    for (int w = lane; w < Q.n1; w += 32) { Q.q1[w] = 0u; Q.vis[w] = 0u; }
    for (int w = lane; w < Q.n2; w += 32) Q.q2[w] = 0u;
    if (lane < Q.n3) Q.q3[lane] = 0u;
    __syncwarp();
    if (MAXF) {
        if (lane == 0) {
            const int k = Lk[R.m];
            atomicOr(Q.vis + (k >> 5), 1u << (k & 31));
            kq_push(Q, k);
        }
    } else {
        for (int i = lane; i < R.m; i += 32)
            if (R.F[i] & kSeed) {
                const int k = Lk[i];
                atomicOr(Q.vis + (k >> 5), 1u << (k & 31));
                kq_push(Q, k);
            }
    }
    __syncwarp();
    int cnt = 0, last = -1;
    // Rounds pay off where the queue is wide; on a thin region (a path-like
    // propagation) most rounds pop one key, and single pops are cheaper: after
    // 32 rounds that popped fewer than 48 keys the propagation pops one key at
    // a time for the next 512 pops, then tries rounds again.
    int rounds = 0, round_pops = 0, singles = 0;
    while (cnt < r) {
        const int w0 = kq_top_word<MAXF>(Q, lane);
        if (w0 < 0) break;
        if (singles > 0) {
            --singles;
            const unsigned w1 = Q.q1[w0];
            if (!w1) break;                         // inconsistent levels: reported as an error
            const int k = (w0 << 5) + (MAXF ? 31 - __clz(w1) : __ffs(w1) - 1);
            __syncwarp();
            if (lane == 0) {
                ordk[k] = MAXF ? r - 1 - cnt : cnt;
                kq_remove(Q, k);
            }
            ++cnt;
            last = k;
            __syncwarp();
            if (lane < NN) {
                const int kk = NK[(long long)k * NN + lane];
                if (kk >= 0) {
                    const unsigned bit = 1u << (kk & 31);
                    if (!(atomicOr(Q.vis + (kk >> 5), bit) & bit)) kq_push(Q, kk);
                }
            }
            __syncwarp();
            continue;
        }
        // candidates: the set bits of the 32 words from w0 on, in pop order
        const int wi = MAXF ? w0 - lane : w0 + lane;
        unsigned w = (wi >= 0 && wi < Q.n1) ? Q.q1[wi] : 0u;
        const int nb = __popc(w);
        int x = nb;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, x, d);
            if (lane >= d) x += y;
        }
        int slot = x - nb;
        while (w && slot < 32) {
            const int bt = MAXF ? 31 - __clz(w) : __ffs(w) - 1;
            Q.candk[slot++] = (wi << 5) + bt;
            w &= ~(1u << bt);
        }
        const int nc = min(32, __shfl_sync(0xffffffffu, x, 31));
        __syncwarp();
        const int c = lane < nc ? Q.candk[lane] : -1;
        int nk[NN];
#pragma unroll
        for (int q = 0; q < NN; ++q) nk[q] = c >= 0 ? NK[(long long)c * NN + q] : -1;
        // the best key that popping c would queue (not visited yet)
        int best = MAXF ? -1 : INT_MAX;
#pragma unroll
        for (int q = 0; q < NN; ++q) {
            const int kk = nk[q];
            if (kk >= 0 && !(Q.vis[kk >> 5] & (1u << (kk & 31)))) best = MAXF ? max(best, kk) : min(best, kk);
        }
        // the best key queued by the candidates before this lane's
        int pre = best;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, pre, d);
            if (lane >= d) pre = MAXF ? max(pre, y) : min(pre, y);
        }
        pre = __shfl_up_sync(0xffffffffu, pre, 1);
        if (lane == 0) pre = MAXF ? -1 : INT_MAX;
        const unsigned okm = __ballot_sync(0xffffffffu, c >= 0 && (MAXF ? pre < c : pre > c));
        const int V = min(okm == 0xffffffffu ? 32 : __ffs(~okm) - 1, r - cnt);
        if (V <= 0) break;                          // cannot happen: the top key is always popped
        if (lane < V) {
            ordk[c] = MAXF ? r - 1 - (cnt + lane) : cnt + lane;
            kq_remove(Q, c);
        }
        __syncwarp();
        if (lane < V) {
#pragma unroll
            for (int q = 0; q < NN; ++q) {
                const int kk = nk[q];
                if (kk >= 0) {
                    const unsigned bit = 1u << (kk & 31);
                    if (!(atomicOr(Q.vis + (kk >> 5), bit) & bit)) kq_push(Q, kk);
                }
            }
        }
        __syncwarp();
        last = __shfl_sync(0xffffffffu, c, V - 1);
        cnt += V;
        round_pops += V;
        if (++rounds == 32) {
            if (round_pops < 48) singles = 512;
            rounds = round_pops = 0;
        }
    }
#pragma unroll 4
    for (int i = lane; i < r; i += 32) R.L2[i] = ordk[Lk[i]];
    __syncwarp();
    return cnt == r ? (MAXF ? last : 0) : -2;
}

// The scans below run one lane per vertex with kScanU vertices per lane in
// flight (all their adjacency entries, then all their neighbours' orders), so
// that the warp of a large region waits for one round of loads per 32 * kScanU
// vertices instead of one per neighbour.
constexpr int kScanU = 4;

// Whether vertex i is a strict local minimum and maximum of L among its
// neighbours in R, for the kScanU vertices b + lane + 32 u (u < kScanU) below
// lim; li gets their L.
template <int NN>
__device__ __forceinline__ void wr_scan_ext(const WarpRegion& R, int b, int lim, int lane, int (&li)[kScanU],
                                            bool (&is_min)[kScanU], bool (&is_max)[kScanU]) {
    int lj[kScanU][NN];
#pragma unroll
    for (int u = 0; u < kScanU; ++u) {
        const int i = b + lane + 32 * u;
        li[u] = i < lim ? R.L[i] : 0;
#pragma unroll
        for (int q = 0; q < NN; ++q) lj[u][q] = i < lim ? R.adj[(long long)i * NN + q] : -1;
    }
#pragma unroll
    for (int u = 0; u < kScanU; ++u)
#pragma unroll
        for (int q = 0; q < NN; ++q) lj[u][q] = lj[u][q] >= 0 ? R.L[lj[u][q]] : -1;
#pragma unroll
    for (int u = 0; u < kScanU; ++u) {
        bool mn = true, mx = true;
#pragma unroll
        for (int q = 0; q < NN; ++q) {
            const int l = lj[u][q];      // -1: no neighbour in R (L is never negative here)
            if (l >= 0 && l < li[u]) mn = false;
            if (l > li[u]) mx = false;
        }
        is_min[u] = mn;
        is_max[u] = mx;
    }
}

// some vertex (not s, for minima: without an outside neighbour) is a strict
// local minimum (MINF) or maximum of L
template <bool MINF, int NN>
__device__ bool wr_has_extremum(const WarpRegion& R, int lane) {
    const int lim = MINF ? R.r : R.m;
    if (R.adj) {
        for (int b = 0; b < lim; b += 32 * kScanU) {
            int li[kScanU];
            bool mn[kScanU], mx[kScanU];
            wr_scan_ext<NN>(R, b, lim, lane, li, mn, mx);
            bool found = false;
#pragma unroll
            for (int u = 0; u < kScanU; ++u) {
                const int i = b + lane + 32 * u;
                if (i < lim && (MINF ? (mn[u] && !(R.F[i] & kBnd)) : mx[u])) found = true;
            }
            if (__any_sync(0xffffffffu, found)) return true;
        }
        return false;
    }
    bool found = false;
    for (int i = lane; i < lim && !found; i += 32) {
        if (MINF && (R.F[i] & kBnd)) continue;
        const int li = R.L[i];
        bool ext = true;
        for (int q = 0; q < NN && ext; ++q) {
            const int j = wr_nbr_of<NN>(R, i, q);
            if (j >= 0 && (MINF ? R.L[j] < li : R.L[j] > li)) ext = false;
        }
        found = ext;
    }
    return __any_sync(0xffffffffu, found);
}

// flags the seeds of a sublevel propagation (see mark_seeds); returns whether there is one
template <int NN>
__device__ bool wr_mark_seeds(const WarpRegion& R, int lane, bool literal) {
    bool any = false;
    if (R.adj) {
        for (int b = 0; b < R.m; b += 32 * kScanU) {
            int li[kScanU];
            bool mn[kScanU], mx[kScanU];
            if (literal) wr_scan_ext<NN>(R, b, R.m, lane, li, mn, mx);
#pragma unroll
            for (int u = 0; u < kScanU; ++u) {
                const int i = b + lane + 32 * u;
                if (i < R.m) {
                    const unsigned char f = R.F[i];
                    const bool sd = (f & kBnd) && (!literal || mn[u]);
                    R.F[i] = (unsigned char)(sd ? (f | kSeed) : (f & ~kSeed));
                    any |= sd;
                }
            }
        }
        __syncwarp();
        return __any_sync(0xffffffffu, any);
    }
    for (int i = lane; i < R.m; i += 32) {
        bool sd = (R.F[i] & kBnd) != 0;
        if (sd && literal) {
            const int li = R.L[i];
            for (int q = 0; q < NN && sd; ++q) {
                const int j = wr_nbr_of<NN>(R, i, q);
                if (j >= 0 && R.L[j] < li) sd = false;
            }
        }
        R.F[i] = (unsigned char)(sd ? (R.F[i] | kSeed) : (R.F[i] & ~kSeed));
        any |= sd;
    }
    __syncwarp();
    return __any_sync(0xffffffffu, any);
}

// The first propagation with candidate a at minus infinity ends on a exactly
// when R \ {a} is connected.  Candidates that cut off a few vertices are
// common on thin regions, so before propagating, a bounded search from each
// neighbour of a in R (but s) over R \ {a} looks for such a piece: a search
// that ends within kCutBudget vertices without reaching s, or a vertex that
// an earlier search for a reached, has found one, and a is then not the
// minus-infinity vertex.  mark[] holds a * 16 + t for the vertices reached by
// the t-th search for a (other values otherwise); q is kCutBudget + 1 ints of
// shared memory.  false: no such piece within the budget (the propagation
// decides).
constexpr int kCutBudget = 64;

template <int NN>
__device__ bool wr_cuts(const WarpRegion& R, int ai, int* mark, int* q, int lane) {
    const int nb = lane < NN ? R.adj[(long long)ai * NN + lane] : -1;
    unsigned todo = __ballot_sync(0xffffffffu, nb >= 0 && nb != R.m);
    const int base = ai * 16;
    int t = 0;
    while (todo) {
        const int src = __ffs(todo) - 1;
        todo &= todo - 1;
        const int b0 = __shfl_sync(0xffffffffu, nb, src);
        const int mb = __ldcg(mark + b0);
        if (mb >= base && mb < base + 16) continue;   // reached by an earlier search for a
        const int stamp = base + t++;
        __syncwarp();
        if (lane == 0) {
            __stcg(mark + b0, stamp);
            q[0] = b0;
            q[kCutBudget] = 1;
        }
        __syncwarp();
        int head = 0;
        bool reach = false, over = false;
        for (;;) {
            const int tail = q[kCutBudget];
            if (head >= tail) break;
            const int i = head + lane < tail ? q[head + lane] : -1;
            head = min(tail, head + 32);
            bool rs = false;
            if (i >= 0) {
#pragma unroll
                for (int k = 0; k < NN; ++k) {
                    const int j = R.adj[(long long)i * NN + k];
                    if (j < 0 || j == ai) continue;
                    if (j == R.m) { rs = true; continue; }
                    const int old = atomicExch(mark + j, stamp);
                    if (old == stamp) continue;
                    if (old >= base && old < base + 16) { rs = true; continue; }   // joins an earlier search's piece
                    const int slot = atomicAdd(q + kCutBudget, 1);
                    if (slot < kCutBudget) q[slot] = j;
                }
            }
            __syncwarp();
            reach = __any_sync(0xffffffffu, rs);
            over = q[kCutBudget] > kCutBudget;
            if (reach || over) break;
        }
        if (!reach && !over) return true;
    }
    return false;
}

template <int DIR, int NN>
__global__ void __launch_bounds__(32) lo_warp_kernel(Geom g, LOArgs a, const int* list, const int* d_count) {
    extern __shared__ unsigned long long H[];
    if (failed(&a.ctr->status)) return;
    const int lane = threadIdx.x;
    const int cnt = *d_count;
    int mx = 0, nfb = 0;
    long long tot = 0;
    for (int k = blockIdx.x; k < cnt; k += gridDim.x) {
        const int rid = list[k];
        const int m = a.reg_size[rid];
        const int s = a.reg_saddle[rid];
        const int st0 = a.reg_start[rid];
        const long long off = (long long)st0 + rid;
        int* P = a.lo_P + off;                      // the order Brent's check compares with
        WarpRegion R{a.lo_v + off, a.lo_L + off, a.lo_L2 + off, a.lo_flag + off, g, a.owner, a.loc, -2 - rid, s, m,
                     m + 1, nullptr};
        // the local adjacency, from a bump pool (recomputed per pop when the pool is spent)
        long long abase = 0;
        if (lane == 0) abase = (long long)atomicAdd((unsigned long long*)&a.ctr->lo_adj_cursor,
                                                    (unsigned long long)NN * (m + 1));
        abase = __shfl_sync(0xffffffffu, abase, 0);
        int* adj = abase + (long long)NN * (m + 1) <= a.lo_adj_cap ? a.lo_adj + abase : nullptr;
        // the key-space table of the later floods, from the same pool, and the bitmaps in shared memory
        long long nbase = 0;
        if (lane == 0 && adj) nbase = (long long)atomicAdd((unsigned long long*)&a.ctr->lo_adj_cursor,
                                                           (unsigned long long)NN * (m + 1));
        nbase = __shfl_sync(0xffffffffu, nbase, 0);
        KeyQueue Q;
        Q.n1 = (m + 1 + 31) >> 5;                   // keys 0..m
        Q.n2 = (Q.n1 + 31) >> 5;
        Q.n3 = (Q.n2 + 31) >> 5;
        unsigned* sm = reinterpret_cast<unsigned*>(H);
        Q.q1 = sm; Q.vis = sm + Q.n1; Q.q2 = sm + 2 * Q.n1; Q.q3 = sm + 2 * Q.n1 + Q.n2;
        Q.candk = reinterpret_cast<int*>(Q.q3 + 32);
        const bool keyspace = adj && nbase + (long long)NN * (m + 1) <= a.lo_adj_cap && Q.n3 <= 32 &&
                              2LL * Q.n1 + Q.n2 + 64 + kCutBudget + 1 <= 2LL * kWarpHeapCap;
        int* NK = keyspace ? a.lo_adj + nbase : nullptr;
        int* ordk = a.lo_heap + off;
        // members, flags, l0 and the local adjacency, kScanU vertices per lane in flight
        for (int b = 0; b <= m; b += 32 * kScanU) {
            int vtx[kScanU], ov[kScanU];
            int nb[kScanU][NN], j[kScanU][NN];
#pragma unroll
            for (int u = 0; u < kScanU; ++u) {
                const int i = b + lane + 32 * u;
                vtx[u] = i < m ? a.members[st0 + i] : (i == m ? s : -1);
            }
#pragma unroll
            for (int u = 0; u < kScanU; ++u) {
                int x = 0, y = 0, z = 0;
                if (vtx[u] >= 0) coords_of(g, vtx[u], x, y, z);
#pragma unroll
                for (int q = 0; q < NN; ++q) nb[u][q] = vtx[u] >= 0 ? nbr_of(g, x, y, z, q) : -1;
                ov[u] = vtx[u] >= 0 && vtx[u] != s ? __ldg(a.O + vtx[u]) : 0;
            }
#pragma unroll
            for (int u = 0; u < kScanU; ++u)
#pragma unroll
                for (int q = 0; q < NN; ++q)
                    j[u][q] = nb[u][q] >= 0 && nb[u][q] != s ? __ldg(a.owner + nb[u][q]) : 0;
#pragma unroll
            for (int u = 0; u < kScanU; ++u) {
                const int i = b + lane + 32 * u;
                if (vtx[u] < 0) continue;
                R.V[i] = vtx[u];
                unsigned char fl = 0;
#pragma unroll
                for (int q = 0; q < NN; ++q) {
                    int jj = -1;
                    if (nb[u][q] == s) jj = m;
                    else if (nb[u][q] >= 0) {
                        if (j[u][q] != R.tag) fl = kBnd;
                        else jj = __ldg(a.loc + nb[u][q]);
                    }
                    if (adj) adj[(long long)i * NN + q] = jj;
                }
                R.F[i] = fl;
                R.L[i] = i < m ? od<DIR>(ov[u], g.n) : INT_MAX;
            }
        }
        R.adj = adj;
        __syncwarp();
        int nfl = -1;
        bool overflow = false;
        // Dense ranks of Od for the candidate tries in key space: a bitmap over
        // the members' Od range and its prefix popcounts.  V then holds the
        // ranks 0..m-1 of the members (nothing reads the vertex ids again); a
        // try with candidate a uses the keys a: 0, members below a: rank + 1,
        // members above a: rank, s: m, a permutation of 0..m.
        bool dense = false;
        if (keyspace) {
            int mn = INT_MAX, mx = INT_MIN;
            #pragma unroll 4
            for (int i = lane; i < m; i += 32) { mn = min(mn, R.L[i]); mx = max(mx, R.L[i]); }
            mn = __reduce_min_sync(0xffffffffu, mn);
            mx = __reduce_max_sync(0xffffffffu, mx);
            const long long words = ((long long)mx - mn + 1 + 31) >> 5;
            long long bbase = 0;
            if (lane == 0) bbase = (long long)atomicAdd((unsigned long long*)&a.ctr->lo_adj_cursor,
                                                        (unsigned long long)(2 * words));
            bbase = __shfl_sync(0xffffffffu, bbase, 0);
            if (bbase + 2 * words <= a.lo_adj_cap) {
                unsigned* bm = reinterpret_cast<unsigned*>(a.lo_adj + bbase);
                int* pre = a.lo_adj + bbase + words;
                for (long long w = lane; w < words; w += 32) bm[w] = 0u;
                __syncwarp();
                for (int i = lane; i < m; i += 32) {
                    const int o = R.L[i] - mn;
                    atomicOr(bm + (o >> 5), 1u << (o & 31));
                }
                __syncwarp();
                int run = 0;
                for (long long b = 0; b < words; b += 32) {
                    const long long w = b + lane;
                    const int c = w < words ? __popc(bm[w]) : 0;
                    int x = c;
#pragma unroll
                    for (int d = 1; d < 32; d <<= 1) {
                        const int y = __shfl_up_sync(0xffffffffu, x, d);
                        if (lane >= d) x += y;
                    }
                    if (w < words) pre[w] = run + x - c;
                    run += __shfl_sync(0xffffffffu, x, 31);
                }
                __syncwarp();
                for (int i = lane; i < m; i += 32) {
                    const int o = R.L[i] - mn;
                    R.V[i] = pre[o >> 5] + __popc(bm[o >> 5] & ((1u << (o & 31)) - 1u));
                }
                __syncwarp();
                dense = true;
            }
        }
        // the minus-infinity vertex: lowest boundary-adjacent member whose removal keeps R connected
        bool ok = false;
        int ai = -1;
        // the first propagation with candidate ai at -infinity (L2 gets its order);
        // returns the last vertex (key 0 in key space), -2 / -3 on failure / heap overflow
        auto first_flood = [&](int ai) -> int {
            if (dense) {
                // key space: the candidate takes key 0, below every other
                const int ra = R.V[ai];
                for (int i = lane; i <= m; i += 32) {
                    const int ri = i < m ? R.V[i] : m;
                    R.L2[i] = i == ai ? 0 : (i < m && ri < ra ? ri + 1 : ri);
                }
                __syncwarp();
                const int lk = wr_flood_keys<true, NN>(R, R.L2, NK, ordk, Q, lane);
                return lk == 0 ? ai : (lk == -2 ? -2 : -1);
            }
            if (lane == 0) R.L[ai] = INT_MIN;
            __syncwarp();
            return wr_flood<true, NN>(R, H, lane);
        };
        // the bounded searches of wr_cuts: marks in P (free until the alternation), queue at the end of H
        int* cutq = reinterpret_cast<int*>(H + kWarpHeapCap) - (kCutBudget + 1);
        if (R.adj) {
#pragma unroll 4
            for (int i = lane; i <= m; i += 32) P[i] = -1;
            __syncwarp();
        }
        for (;;) {
            int best = INT_MAX, bi = -1;
#pragma unroll 4
            for (int i = lane; i < m; i += 32) {
                const unsigned char f = R.F[i];
                const int l = R.L[i];
                if ((f & (kBnd | kTried)) == kBnd && l < best) { best = l; bi = i; }
            }
            const int K = __reduce_min_sync(0xffffffffu, best);
            if (K == INT_MAX) break;
            ai = __shfl_sync(0xffffffffu, bi, __ffs(__ballot_sync(0xffffffffu, bi >= 0 && best == K)) - 1);
            __syncwarp();
            if (R.adj && m < (1 << 26) && wr_cuts<NN>(R, ai, P, cutq, lane)) {   // marks ai * 16 + t fit an int
                if (lane == 0) R.F[ai] |= kTried;
                __syncwarp();
                continue;
            }
            const int last = first_flood(ai);
            if (last == -3) { overflow = true; break; }
            if (last == -2) break;
            if (last == ai) { ok = true; break; }
            if (lane == 0) { if (!dense) R.L[ai] = K; R.F[ai] |= kTried; }
            __syncwarp();
        }
        bool fell_back = false;
        if (ok) {
            const int cap = 2 * R.r + 2;
            for (int pass = 0; pass < 2 && nfl < 0 && !overflow; ++pass) {
                const bool literal = pass == 0;
                if (!literal) {
                    // redo from l1: rebuild it in L2 (V holds vertex ids unless dense)
                    if (!dense) {
                        for (int i = lane; i <= m; i += 32) R.L[i] = i < m ? od<DIR>(__ldg(a.O + R.V[i]), g.n) : INT_MAX;
                        __syncwarp();
                    }
                    const int last = first_flood(ai);
                    if (last == -3) { overflow = true; break; }
                    if (last != ai) break;
                }
                #pragma unroll 4
                for (int i = lane; i < R.r; i += 32) { R.L[i] = R.L2[i]; P[i] = R.L2[i]; }
                __syncwarp();
                int fl = 1, res = 0;            // res: 1 done, -1 does not end, -2 error, -3 overflow
                int power = 1, lam = 0;
                for (;;) {
                    if (!wr_has_extremum<true, NN>(R, lane)) { res = 1; break; }
                    if (!wr_mark_seeds<NN>(R, lane, literal)) { res = -1; break; }
                    if (++fl > cap) { res = -1; break; }
                    const int rmin = keyspace ? wr_flood_keys<false, NN>(R, R.L, NK, ordk, Q, lane)
                                              : wr_flood<false, NN>(R, H, lane);
                    if (rmin == -3) { res = -3; break; }
                    if (rmin < 0) { res = -2; break; }
                    #pragma unroll 4
                    for (int i = lane; i < R.r; i += 32) R.L[i] = R.L2[i];
                    __syncwarp();
                    if (!wr_has_extremum<false, NN>(R, lane)) { res = 1; break; }
                    if (++fl > cap) { res = -1; break; }
                    const int rmax = keyspace ? wr_flood_keys<true, NN>(R, R.L, NK, ordk, Q, lane)
                                              : wr_flood<true, NN>(R, H, lane);
                    if (rmax == -3) { res = -3; break; }
                    if (rmax < 0) { res = -2; break; }
                    #pragma unroll 4
                    for (int i = lane; i < R.r; i += 32) R.L[i] = R.L2[i];
                    __syncwarp();
                    if (literal) {
                        bool same = true;
                        #pragma unroll 4
                        for (int i = lane; i < R.r; i += 32) same &= P[i] == R.L[i];
                        if (__all_sync(0xffffffffu, same)) { res = -1; break; }
                        if (++lam == power) {
                            #pragma unroll 4
                            for (int i = lane; i < R.r; i += 32) P[i] = R.L[i];
                            __syncwarp();
                            power *= 2;
                            lam = 0;
                        }
                    }
                }
                if (res == 1) { nfl = fl; fell_back = !literal; }
                else if (res == -3) overflow = true;
                else if (res == -2) break;
            }
        }
        __syncwarp();
        if (overflow) {
            // the frontier outgrew the heap: lane 0 redoes the region on the single-thread path
            nfl = -1;
            if (lane == 0) {
                BigStore<NN> T{a.lo_v + off, a.lo_L + off, a.lo_L2 + off, a.lo_heap + off, a.lo_flag + off, P,
                               g, a.owner, a.loc, -2 - rid, s, m, a.O, DIR};
                // V holds vertex ids again (the dense ranks are recomputed from scratch)
                for (int i = 0; i <= m; ++i) T.V(i) = i < m ? a.members[st0 + i] : s;
                for (int i = 0; i <= m; ++i) {
                    T.F(i) &= kBnd;
                    T.L(i) = T.L0(i);
                }
                nfl = local_order_run<NN>(T, m);
                fell_back = nfl >= 0 && (nfl & kFellBack);
                if (nfl >= 0) nfl &= ~kFellBack;
            }
            nfl = __shfl_sync(0xffffffffu, nfl, 0);
            fell_back = __shfl_sync(0xffffffffu, fell_back, 0);
        }
        if (nfl < 0) {
            if (lane == 0) set_status(&a.ctr->status, LTS_ERR_INTERNAL);
            continue;
        }
        #pragma unroll 4
        for (int i = lane; i < m; i += 32) a.lhat[st0 + i] = R.L[i];
        mx = max(mx, nfl);
        tot += nfl;
        nfb += fell_back;
        __syncwarp();
    }
    if (lane != 0) { mx = 0; tot = 0; nfb = 0; }
    warp_atomic_max(&a.ctr->max_floods, mx);
    warp_atomic_add64(&a.ctr->total_floods, tot);
    warp_atomic_add(&a.ctr->lo_fallbacks, nfb);
}

template <int DIR, int NN>
void launch_tiers(Work& w, const Geom& g, const LOArgs& a, int sms, cudaStream_t s) {
    const int q = w.class_cap / 4;
    constexpr size_t small = 4 * dense_smem_per_warp<NN, 128>();
    constexpr size_t large = dense_smem_per_warp<NN, kMedR>();
    constexpr size_t huge = dense_smem_per_warp<NN, kHugeR>();
    static_assert(huge <= 227 * 1024, "shared memory of the 4096-vertex tier");
    cudaFuncSetAttribute(lo_dense_kernel<DIR, NN, 128, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)small);
    cudaFuncSetAttribute(lo_dense_kernel<DIR, NN, kMedR, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)large);
    cudaFuncSetAttribute(lo_dense_kernel<DIR, NN, kHugeR, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)huge);
    const int* tl = w.tier_list + w.class_cap;
    // The tiers hold disjoint regions (each writes only its regions' local
    // orders and scratch slots, and reads the order of their members), so
    // they run side by side: each is latency-bound with a long tail.
    cudaStream_t s0 = s, s1 = s, s2 = s;
    if (w.aux_on) {
        cudaEventRecord(w.fork_ev, s);
        for (int i = 0; i < 3; ++i) cudaStreamWaitEvent(w.aux[i], w.fork_ev, 0);
        s0 = w.aux[0]; s1 = w.aux[1]; s2 = w.aux[2];
    }
    const int tb = sms * std::max(1, std::min(w.team_bpsm, 16));
    lo_team_kernel<DIR, NN, 16><<<tb, 128, 0, s>>>(g, a, w.tier_list, &w.ctr->n_t16);
    lo_team_kernel<DIR, NN, 32><<<tb, 128, 0, s2>>>(g, a, tl, &w.ctr->n_t32);
    lo_dense_kernel<DIR, NN, 128, 4><<<sms * 10, 128, small, s1>>>(g, a, tl + q, &w.ctr->n_med);
    lo_dense_kernel<DIR, NN, kMedR, 1><<<sms * 5, 32, large, s0>>>(g, a, tl + 2 * q, &w.ctr->n_large);
    lo_dense_kernel<DIR, NN, kHugeR, 1><<<sms, 32, huge, s0>>>(g, a, tl + 3 * q, &w.ctr->n_huge);
    constexpr size_t heap_bytes = kWarpHeapCap * sizeof(unsigned long long);
    cudaFuncSetAttribute(lo_warp_kernel<DIR, NN>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)heap_bytes);
    lo_warp_kernel<DIR, NN><<<sms, 32, heap_bytes, s0>>>(g, a, tl + 3 * q + q / 2, &w.ctr->n_big);
    if (w.aux_on) {
        for (int i = 0; i < 3; ++i) {
            cudaEventRecord(w.join_ev[i], w.aux[i]);
            cudaStreamWaitEvent(s, w.join_ev[i], 0);
        }
    }
}

}  // namespace

template <int DIR>
cudaError_t local_orders(Work& w, const Geom& g, const int* O, int sms, cudaStream_t s) {
    LOArgs a{O, w.owner, w.loc, w.members, w.reg_start, w.reg_size, w.reg_saddle, w.lhat,
             w.lo_v, w.lo_L, w.lo_L2, w.lo_heap, w.lo_flag, w.lo_P, w.tier_list, w.ctr, w.lo_adj, w.lo_adj_cap};
    if (g.nn == 14) launch_tiers<DIR, 14>(w, g, a, sms, s);
    else launch_tiers<DIR, 6>(w, g, a, sms, s);
    w.launches += 6;
    return cudaGetLastError();
}

template cudaError_t local_orders<1>(Work&, const Geom&, const int*, int, cudaStream_t);
template cudaError_t local_orders<-1>(Work&, const Geom&, const int*, int, cudaStream_t);

int local_order_tiny_max() { return 16; }
int local_order_med_max() { return kMedR; }
int local_order_huge_max() { return kHugeR; }

}  // namespace lts
