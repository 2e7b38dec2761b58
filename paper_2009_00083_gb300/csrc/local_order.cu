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
//   neighbour, and sublevel propagation from every vertex of R\{s} with an
//   outside neighbour (smallest first; visiting order = new local order)
//   while some vertex other than s is a maximum.
// Propagations only use edges inside R.  Each lane handles one region; the
// per-region arrays live in a scratch area indexed by the region's slots.
#include <climits>

#include "lts_internal.cuh"

namespace lts {

namespace {

constexpr unsigned char kBnd = 1, kVis = 2, kTried = 4;

struct Ctx {
    Geom g;
    const int* owner;
    const int* loc;
    int tag;       // region tag in owner[]
    int s;         // saddle vertex
    int m;         // members; local index of s
    int r;         // m + 1
    const int* V;
    int* L;
    int* L2;
    int* Hp;
    unsigned char* F;
};

// local index of neighbour q of local vertex i, or -1 if outside R / the grid
__device__ __forceinline__ int lnbr(const Ctx& C, int x, int y, int z, int q) {
    const int nb = nbr_of(C.g, x, y, z, q);
    if (nb < 0) return -1;
    if (nb == C.s) return C.m;
    if (__ldg(C.owner + nb) != C.tag) return -1;
    return __ldg(C.loc + nb);
}

// heap of local indices; MAXF: largest L first, else smallest first
template <bool MAXF>
__device__ __forceinline__ bool better(const int* L, int a, int b) { return MAXF ? L[a] > L[b] : L[a] < L[b]; }

template <bool MAXF>
__device__ void hpush(const Ctx& C, int& n, int i) {
    int p = n++;
    while (p > 0) {
        const int q = (p - 1) >> 1;
        if (!better<MAXF>(C.L, i, C.Hp[q])) break;
        C.Hp[p] = C.Hp[q];
        p = q;
    }
    C.Hp[p] = i;
}

template <bool MAXF>
__device__ int hpop(const Ctx& C, int& n) {
    const int top = C.Hp[0];
    const int last = C.Hp[--n];
    if (n == 0) return top;
    int p = 0;
    for (;;) {
        int l = 2 * p + 1;
        if (l >= n) break;
        if (l + 1 < n && better<MAXF>(C.L, C.Hp[l + 1], C.Hp[l])) ++l;
        if (!better<MAXF>(C.L, C.Hp[l], last)) break;
        C.Hp[p] = C.Hp[l];
        p = l;
    }
    C.Hp[p] = last;
    return top;
}

// Superlevel propagation from s; L2 = inverse visiting order.  Returns the
// last vertex visited.
__device__ int max_flood(const Ctx& C) {
    for (int i = 0; i < C.r; ++i) C.F[i] &= (unsigned char)~kVis;
    int n = 0, cnt = 0, last = -1;
    C.F[C.m] |= kVis;
    hpush<true>(C, n, C.m);
    while (n > 0) {
        const int i = hpop<true>(C, n);
        C.L2[i] = C.r - 1 - cnt++;
        last = i;
        int x, y, z;
        coords_of(C.g, C.V[i], x, y, z);
        for (int q = 0; q < C.g.nn; ++q) {
            const int j = lnbr(C, x, y, z, q);
            if (j < 0 || (C.F[j] & kVis)) continue;
            C.F[j] |= kVis;
            hpush<true>(C, n, j);
        }
    }
    return cnt == C.r ? last : -2;
}

// Sublevel propagation from every vertex of R\{s} with an outside neighbour;
// L2 = visiting order.
__device__ bool min_flood(const Ctx& C) {
    for (int i = 0; i < C.r; ++i) C.F[i] &= (unsigned char)~kVis;
    int n = 0, cnt = 0;
    for (int i = 0; i < C.m; ++i)
        if (C.F[i] & kBnd) { C.F[i] |= kVis; hpush<false>(C, n, i); }
    while (n > 0) {
        const int i = hpop<false>(C, n);
        C.L2[i] = cnt++;
        int x, y, z;
        coords_of(C.g, C.V[i], x, y, z);
        for (int q = 0; q < C.g.nn; ++q) {
            const int j = lnbr(C, x, y, z, q);
            if (j < 0 || (C.F[j] & kVis)) continue;
            C.F[j] |= kVis;
            hpush<false>(C, n, j);
        }
    }
    return cnt == C.r;
}

// some vertex without an outside neighbour is a minimum of L on R
__device__ bool has_unauth_min(const Ctx& C) {
    for (int i = 0; i < C.r; ++i) {
        if (C.F[i] & kBnd) continue;
        int x, y, z;
        coords_of(C.g, C.V[i], x, y, z);
        bool ismin = true;
        for (int q = 0; q < C.g.nn && ismin; ++q) {
            const int j = lnbr(C, x, y, z, q);
            if (j >= 0 && C.L[j] < C.L[i]) ismin = false;
        }
        if (ismin) return true;
    }
    return false;
}

// some vertex other than s is a maximum of L on R
__device__ bool has_unauth_max(const Ctx& C) {
    for (int i = 0; i < C.m; ++i) {
        int x, y, z;
        coords_of(C.g, C.V[i], x, y, z);
        bool ismax = true;
        for (int q = 0; q < C.g.nn && ismax; ++q) {
            const int j = lnbr(C, x, y, z, q);
            if (j >= 0 && C.L[j] > C.L[i]) ismax = false;
        }
        if (ismax) return true;
    }
    return false;
}

__device__ __forceinline__ void copy_l2(const Ctx& C) {
    for (int i = 0; i < C.r; ++i) C.L[i] = C.L2[i];
}

template <int DIR>
__global__ void __launch_bounds__(128) local_order_kernel(Geom g, const int* __restrict__ O,
                                                          const int* __restrict__ owner, const int* __restrict__ loc,
                                                          const int* __restrict__ members,
                                                          const int* __restrict__ reg_start,
                                                          const int* __restrict__ reg_size,
                                                          const int* __restrict__ reg_saddle, int* lhat, int* lo_v,
                                                          int* lo_L, int* lo_L2, int* lo_heap, unsigned char* lo_flag,
                                                          DevCounters* ctr) {
    if (failed(&ctr->status)) return;
    const int nreg = ctr->n_regions;
    for (int rid = blockIdx.x * blockDim.x + threadIdx.x; rid < nreg; rid += gridDim.x * blockDim.x) {
        Ctx C;
        C.g = g; C.owner = owner; C.loc = loc;
        C.tag = -2 - rid;
        C.s = reg_saddle[rid];
        C.m = reg_size[rid];
        C.r = C.m + 1;
        const int st0 = reg_start[rid];
        const long long off = (long long)st0 + rid;
        int* V = lo_v + off;
        C.V = V; C.L = lo_L + off; C.L2 = lo_L2 + off; C.Hp = lo_heap + off; C.F = lo_flag + off;
        for (int i = 0; i < C.m; ++i) V[i] = members[st0 + i];
        V[C.m] = C.s;
        for (int i = 0; i < C.r; ++i) {
            const int v = V[i];
            int x, y, z;
            coords_of(g, v, x, y, z);
            unsigned char fl = 0;
            for (int q = 0; q < g.nn; ++q) {
                const int nb = nbr_of(g, x, y, z, q);
                if (nb < 0) continue;
                if (nb != C.s && __ldg(owner + nb) != C.tag) { fl = kBnd; break; }
            }
            C.F[i] = fl;
            C.L[i] = od<DIR>(__ldg(O + v), g.n);
        }
        C.L[C.m] = INT_MAX;
        // the minus-infinity vertex: lowest boundary-adjacent non-cut vertex
        int floods = 0;
        bool ok = false;
        for (;;) {
            int a = -1;
            for (int i = 0; i < C.m; ++i)
                if ((C.F[i] & (kBnd | kTried)) == kBnd && (a < 0 || C.L[i] < C.L[a])) a = i;
            if (a < 0) break;
            const int keep = C.L[a];
            C.L[a] = INT_MIN;
            const int last = max_flood(C);
            ++floods;
            if (last == -2) break;
            if (last == a) { ok = true; break; }
            C.L[a] = keep;
            C.F[a] |= kTried;
        }
        if (!ok) { set_status(&ctr->status, LTS_ERR_INTERNAL); continue; }
        copy_l2(C);
        const int cap = 2 * C.r + 2;
        int nfl = 1;   // propagations of the alternation (the accepted first one included)
        for (;;) {
            if (!has_unauth_min(C)) break;
            if (!min_flood(C)) { ok = false; break; }
            copy_l2(C);
            ++nfl;
            if (!has_unauth_max(C)) break;
            if (max_flood(C) < 0) { ok = false; break; }
            copy_l2(C);
            ++nfl;
            if (nfl > cap) { ok = false; break; }
        }
        if (!ok) { set_status(&ctr->status, LTS_ERR_INTERNAL); continue; }
        for (int i = 0; i < C.m; ++i) lhat[st0 + i] = C.L[i];
        atomicMax(&ctr->max_floods, nfl);
        atomicAdd((unsigned long long*)&ctr->total_floods, (unsigned long long)nfl);
        (void)floods;
    }
}

}  // namespace

template <int DIR>
cudaError_t local_orders(Work& w, const Geom& g, const int* O, int sms, cudaStream_t s) {
    local_order_kernel<DIR><<<sms * 16, 128, 0, s>>>(g, O, w.owner, w.loc, w.members, w.reg_start, w.reg_size,
                                                     w.reg_saddle, w.lhat, w.lo_v, w.lo_L, w.lo_L2, w.lo_heap,
                                                     w.lo_flag, w.ctr);
    w.launches += 1;
    return cudaGetLastError();
}

template cudaError_t local_orders<1>(Work&, const Geom&, const int*, int, cudaStream_t);
template cudaError_t local_orders<-1>(Work&, const Geom&, const int*, int, cudaStream_t);

}  // namespace lts
