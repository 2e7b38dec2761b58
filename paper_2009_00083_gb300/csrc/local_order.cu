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
// Propagations only use edges inside R.
//
// The algorithm is written once over a storage policy and run in three
// tiers by region size: regions of at most 16 vertices (nearly all of them)
// one per lane with every array in shared memory; up to 1024 vertices one
// per warp, the adjacency built by the whole warp and the propagations run
// by one lane in shared memory; larger ones one per lane in HBM scratch.
#include <climits>

#include "lts_internal.cuh"

namespace lts {

namespace {

constexpr unsigned char kBnd = 1, kVis = 2, kTried = 4;
constexpr int kTinyR = 16;
constexpr int kTinyThreads = 128;
constexpr int kMedR = 1024;
constexpr int kNoNbr = 0xffff;

// ---------------------------------------------------------------------------
// storage policies: V (vertex), L / L2 (local orders), Hp (heap of local
// indices), F (flags), nbr(i, q) (local index of neighbour q, or -1)
// ---------------------------------------------------------------------------

// one lane, shared memory, slot i of lane t at [i * stride + t]
template <int NN>
struct TinyStore {
    int* v; int* l; int* l2; unsigned char* hp; unsigned char* f; unsigned char* adj;
    int stride;
    __device__ int& V(int i) const { return v[i * stride]; }
    __device__ int& L(int i) const { return l[i * stride]; }
    __device__ int& L2(int i) const { return l2[i * stride]; }
    __device__ int hp_get(int i) const { return hp[i * stride]; }
    __device__ void hp_set(int i, int x) const { hp[i * stride] = (unsigned char)x; }
    __device__ unsigned char& F(int i) const { return f[i * stride]; }
    __device__ int nbr(int i, int q) const {
        const unsigned char x = adj[(i * NN + q) * stride];
        return x == 0xff ? -1 : x;
    }
};

// one warp per region, shared memory (unit stride)
template <int NN>
struct MedStore {
    int* v; int* l; int* l2; unsigned short* hp; unsigned char* f; unsigned short* adj;
    __device__ int& V(int i) const { return v[i]; }
    __device__ int& L(int i) const { return l[i]; }
    __device__ int& L2(int i) const { return l2[i]; }
    __device__ int hp_get(int i) const { return hp[i]; }
    __device__ void hp_set(int i, int x) const { hp[i] = (unsigned short)x; }
    __device__ unsigned char& F(int i) const { return f[i]; }
    __device__ int nbr(int i, int q) const {
        const unsigned short x = adj[i * NN + q];
        return x == kNoNbr ? -1 : x;
    }
};

// HBM scratch; neighbours recomputed from the grid and the region tags
template <int NN>
struct BigStore {
    int* v; int* l; int* l2; int* hp; unsigned char* f;
    Geom g; const int* owner; const int* loc; int tag; int s; int m;
    __device__ int& V(int i) const { return v[i]; }
    __device__ int& L(int i) const { return l[i]; }
    __device__ int& L2(int i) const { return l2[i]; }
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

// sublevel propagation from every vertex of R\{s} with an outside neighbour
template <int NN, class S>
__device__ bool min_flood(const S& T, int m, int r) {
    for (int i = 0; i < r; ++i) T.F(i) &= (unsigned char)~kVis;
    int n = 0, cnt = 0;
    for (int i = 0; i < m; ++i)
        if (T.F(i) & kBnd) { T.F(i) |= kVis; hpush<false>(T, n, i); }
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

// Runs step 2 on a region whose V, L (Od; L(m) = INT_MAX) and F (kBnd)
// are set.  On success L holds the local order; returns the number of
// propagations of the alternation, or -1 on failure.
template <int NN, class S>
__device__ int local_order_run(const S& T, int m) {
    const int r = m + 1;
    bool ok = false;
    for (;;) {
        int a = -1;
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
    for (int i = 0; i < r; ++i) T.L(i) = T.L2(i);
    const int cap = 2 * r + 2;
    int nfl = 1;
    for (;;) {
        if (!has_unauth_min<NN>(T, r)) break;
        if (!min_flood<NN>(T, m, r)) return -1;
        for (int i = 0; i < r; ++i) T.L(i) = T.L2(i);
        ++nfl;
        if (!has_unauth_max<NN>(T, m)) break;
        if (max_flood<NN>(T, m, r) < 0) return -1;
        for (int i = 0; i < r; ++i) T.L(i) = T.L2(i);
        ++nfl;
        if (nfl > cap) return -1;
    }
    return nfl;
}

struct LOArgs {
    const int* O; const int* owner; const int* loc; const int* members; const int* reg_start;
    const int* reg_size; const int* reg_saddle; int* lhat;
    int* lo_v; int* lo_L; int* lo_L2; int* lo_heap; unsigned char* lo_flag;
    const int* tier_list; DevCounters* ctr;
};

struct FloodStat {
    int mx = 0;
    long long tot = 0;
    __device__ void add(DevCounters* ctr, int nfl) {
        if (nfl < 0) { set_status(&ctr->status, LTS_ERR_INTERNAL); return; }
        mx = max(mx, nfl);
        tot += nfl;
    }
    __device__ void flush(DevCounters* ctr) {   // all 32 lanes
        warp_atomic_max(&ctr->max_floods, mx);
        warp_atomic_add64(&ctr->total_floods, tot);
    }
};

// ---- tier 1: one lane per region of at most kTinyR vertices ----
template <int DIR, int NN>
__global__ void __launch_bounds__(kTinyThreads) lo_tiny_kernel(Geom g, LOArgs a) {
    extern __shared__ unsigned char smem[];
    if (failed(&a.ctr->status)) return;
    const int t = threadIdx.x;
    const int B = kTinyThreads;
    int* sv = reinterpret_cast<int*>(smem);
    int* sl = sv + kTinyR * B;
    int* sl2 = sl + kTinyR * B;
    unsigned char* shp = reinterpret_cast<unsigned char*>(sl2 + kTinyR * B);
    unsigned char* sf = shp + kTinyR * B;
    unsigned char* sadj = sf + kTinyR * B;
    TinyStore<NN> T{sv + t, sl + t, sl2 + t, shp + t, sf + t, sadj + t, B};
    FloodStat fs;
    const int nreg = a.ctr->n_regions;
    for (int rid = blockIdx.x * B + t; rid < nreg; rid += gridDim.x * B) {
        const int m = a.reg_size[rid];
        if (m + 1 > kTinyR) continue;
        const int s = a.reg_saddle[rid];
        const int tag = -2 - rid;
        const int st0 = a.reg_start[rid];
        for (int i = 0; i < m; ++i) T.V(i) = a.members[st0 + i];
        T.V(m) = s;
        for (int i = 0; i <= m; ++i) {
            const int vtx = T.V(i);
            int x, y, z;
            coords_of(g, vtx, x, y, z);
            unsigned char fl = 0;
#pragma unroll
            for (int q = 0; q < NN; ++q) {
                const int nb = nbr_of(g, x, y, z, q);
                unsigned char li = 0xff;
                if (nb >= 0) {
                    if (nb == s) li = (unsigned char)m;
                    else if (__ldg(a.owner + nb) == tag) li = (unsigned char)__ldg(a.loc + nb);
                    else fl = kBnd;
                }
                sadj[((i * NN + q) * B) + t] = li;
            }
            T.F(i) = fl;
            T.L(i) = od<DIR>(__ldg(a.O + vtx), g.n);
        }
        T.L(m) = INT_MAX;
        const int nfl = local_order_run<NN>(T, m);
        fs.add(a.ctr, nfl);
        if (nfl < 0) continue;
        for (int i = 0; i < m; ++i) a.lhat[st0 + i] = T.L(i);
    }
    __syncwarp();
    fs.flush(a.ctr);
}

// ---- tier 2: one warp per region of at most kMedR vertices ----
template <int DIR, int NN>
__global__ void __launch_bounds__(32) lo_med_kernel(Geom g, LOArgs a, const int* list, const int* d_count) {
    extern __shared__ unsigned char smem[];
    if (failed(&a.ctr->status)) return;
    int* sv = reinterpret_cast<int*>(smem);
    int* sl = sv + kMedR;
    int* sl2 = sl + kMedR;
    unsigned short* shp = reinterpret_cast<unsigned short*>(sl2 + kMedR);
    unsigned short* sadj = shp + kMedR;
    unsigned char* sf = reinterpret_cast<unsigned char*>(sadj + kMedR * NN);
    MedStore<NN> T{sv, sl, sl2, shp, sf, sadj};
    const int lane = threadIdx.x;
    const int cnt = *d_count;
    for (int k = blockIdx.x; k < cnt; k += gridDim.x) {
        const int rid = list[k];
        const int m = a.reg_size[rid];
        const int s = a.reg_saddle[rid];
        const int tag = -2 - rid;
        const int st0 = a.reg_start[rid];
        for (int i = lane; i <= m; i += 32) sv[i] = i < m ? a.members[st0 + i] : s;
        __syncwarp();
        for (int i = lane; i <= m; i += 32) {
            const int vtx = sv[i];
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
                sadj[i * NN + q] = li;
            }
            sf[i] = fl;
            sl[i] = i < m ? od<DIR>(__ldg(a.O + vtx), g.n) : INT_MAX;
        }
        __syncwarp();
        int nfl = 0;
        if (lane == 0) {
            nfl = local_order_run<NN>(T, m);
            FloodStat fs;
            fs.add(a.ctr, nfl);
            if (nfl >= 0) {
                atomicMax(&a.ctr->max_floods, nfl);
                atomicAdd((unsigned long long*)&a.ctr->total_floods, (unsigned long long)nfl);
            }
        }
        nfl = __shfl_sync(0xffffffffu, nfl, 0);
        __syncwarp();
        if (nfl >= 0)
            for (int i = lane; i < m; i += 32) a.lhat[st0 + i] = sl[i];
        __syncwarp();
    }
}

// ---- tier 3: one lane per region above kMedR vertices, HBM scratch ----
template <int DIR, int NN>
__global__ void __launch_bounds__(128) lo_big_kernel(Geom g, LOArgs a, const int* list, const int* d_count) {
    if (failed(&a.ctr->status)) return;
    const int cnt = *d_count;
    FloodStat fs;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < cnt; k += gridDim.x * blockDim.x) {
        const int rid = list[k];
        const int m = a.reg_size[rid];
        const int s = a.reg_saddle[rid];
        const int st0 = a.reg_start[rid];
        const long long off = (long long)st0 + rid;
        BigStore<NN> T{a.lo_v + off, a.lo_L + off, a.lo_L2 + off, a.lo_heap + off, a.lo_flag + off,
                       g, a.owner, a.loc, -2 - rid, s, m};
        for (int i = 0; i < m; ++i) T.V(i) = a.members[st0 + i];
        T.V(m) = s;
        for (int i = 0; i <= m; ++i) {
            const int vtx = T.V(i);
            int x, y, z;
            coords_of(g, vtx, x, y, z);
            unsigned char fl = 0;
            for (int q = 0; q < NN; ++q) {
                const int nb = nbr_of(g, x, y, z, q);
                if (nb >= 0 && nb != s && __ldg(a.owner + nb) != T.tag) fl = kBnd;
            }
            T.F(i) = fl;
            T.L(i) = od<DIR>(__ldg(a.O + vtx), g.n);
        }
        T.L(m) = INT_MAX;
        const int nfl = local_order_run<NN>(T, m);
        fs.add(a.ctr, nfl);
        if (nfl < 0) continue;
        for (int i = 0; i < m; ++i) a.lhat[st0 + i] = T.L(i);
    }
    __syncwarp();
    fs.flush(a.ctr);
}

template <int NN>
constexpr size_t tiny_smem() { return (size_t)kTinyR * kTinyThreads * (3 * 4 + 2 + NN); }
template <int NN>
constexpr size_t med_smem() { return (size_t)kMedR * (3 * 4 + 2 + 2 * NN + 1); }

template <int DIR, int NN>
void launch_tiers(Work& w, const Geom& g, const LOArgs& a, int sms, cudaStream_t s) {
    cudaFuncSetAttribute(lo_tiny_kernel<DIR, NN>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tiny_smem<NN>());
    cudaFuncSetAttribute(lo_med_kernel<DIR, NN>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)med_smem<NN>());
    lo_tiny_kernel<DIR, NN><<<sms * 4, kTinyThreads, tiny_smem<NN>(), s>>>(g, a);
    lo_med_kernel<DIR, NN><<<sms * 4, 32, med_smem<NN>(), s>>>(g, a, w.tier_list, &w.ctr->n_med);
    lo_big_kernel<DIR, NN><<<sms, 128, 0, s>>>(g, a, w.tier_list + w.class_cap / 2, &w.ctr->n_big);
}

}  // namespace

template <int DIR>
cudaError_t local_orders(Work& w, const Geom& g, const int* O, int sms, cudaStream_t s) {
    LOArgs a{O, w.owner, w.loc, w.members, w.reg_start, w.reg_size, w.reg_saddle, w.lhat,
             w.lo_v, w.lo_L, w.lo_L2, w.lo_heap, w.lo_flag, w.tier_list, w.ctr};
    if (g.nn == 14) launch_tiers<DIR, 14>(w, g, a, sms, s);
    else launch_tiers<DIR, 6>(w, g, a, sms, s);
    w.launches += 3;
    return cudaGetLastError();
}

template cudaError_t local_orders<1>(Work&, const Geom&, const int*, int, cudaStream_t);
template cudaError_t local_orders<-1>(Work&, const Geom&, const int*, int, cudaStream_t);

int local_order_tiny_max() { return kTinyR; }
int local_order_med_max() { return kMedR; }

}  // namespace lts
