// Extremum classification for one pass (Sec. 3.1, Eq. 1).
//
// A vertex is a maximum of the pass-oriented order Od when none of its
// Freudenthal neighbours is higher.  Authorized maxima are counted; the
// unauthorized ones form the list U of propagation seeds, appended with one
// atomic per warp, and each gets a fresh class record for step 1.
#include "lts_internal.cuh"

namespace lts {

namespace {

constexpr int kRun = 16;              // consecutive vertices per thread
constexpr int kCT = 256;              // threads per block; a tile is kCT * kRun vertices

// Every thread classifies a run of kRun consecutive vertices; the block
// scans the per-thread counts and appends the whole tile's unauthorized
// extrema with a single atomic (per-warp atomics on one counter serialise).
template <int DIR>
__global__ void __launch_bounds__(kCT) classify_kernel(Geom g, const int* __restrict__ O,
                                                       const unsigned* __restrict__ authbits, int* __restrict__ U,
                                                       int* __restrict__ parent, int* __restrict__ wait_v,
                                                       int* __restrict__ cnt, int* __restrict__ listhead,
                                                       int* __restrict__ next_w, int* __restrict__ spill_n,
                                                       int cap, DevCounters* ctr) {
    __shared__ int s_warp[kCT / 32];
    __shared__ int s_base;
    if (failed(&ctr->status)) return;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int my_auth = 0;
    for (long long tile = blockIdx.x;; tile += gridDim.x) {
        const long long base = tile * (long long)(kCT * kRun);
        if (base >= g.n) break;
        const long long v0 = base + (long long)threadIdx.x * kRun;
        unsigned mu = 0;
#pragma unroll 4
        for (int i = 0; i < kRun; ++i) {
            const long long vv = v0 + i;
            if (vv >= g.n) break;
            const int v = (int)vv;
            const int ov = od<DIR>(__ldg(O + v), g.n);
            int x, y, z;
            coords_of(g, v, x, y, z);
            bool ext = true;
            for (int k = 0; k < g.nn; ++k) {
                const int nb = nbr_of(g, x, y, z, k);
                if (nb >= 0 && od<DIR>(__ldg(O + nb), g.n) > ov) { ext = false; break; }
            }
            if (!ext) continue;
            if ((__ldg(authbits + (v >> 5)) >> (v & 31)) & 1u) ++my_auth;
            else mu |= 1u << i;
        }
        // block-wide exclusive scan of the per-thread counts
        const int c = __popc(mu);
        int x = c;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) s_warp[warp] = x;
        __syncthreads();
        if (threadIdx.x == 0) {
            int run = 0;
            for (int w = 0; w < kCT / 32; ++w) { const int t = s_warp[w]; s_warp[w] = run; run += t; }
            s_base = run ? atomicAdd(&ctr->n_unauth, run) : 0;
        }
        __syncthreads();
        int pos = s_base + s_warp[warp] + x - c;
        while (mu) {
            const int i = __ffs(mu) - 1;
            mu &= mu - 1;
            const int cl = pos++;
            if (cl >= cap) { set_status(&ctr->status, LTS_ERR_INTERNAL); continue; }
            U[cl] = (int)(v0 + i);
            parent[cl] = cl;
            wait_v[cl] = -1;
            cnt[cl] = 0;
            listhead[cl] = -1;
            next_w[cl] = -1;
            spill_n[cl] = 0;
        }
        __syncthreads();
    }
    warp_atomic_add(&ctr->n_auth_ext, my_auth);
}

}  // namespace

template <int DIR>
cudaError_t classify(Work& w, const Geom& g, const int* O, cudaStream_t s) {
    const long long tiles = ((long long)g.n + kCT * kRun - 1) / (kCT * kRun);
    const long long blocks = std::min<long long>(tiles, 152LL * 8);
    classify_kernel<DIR><<<(int)blocks, kCT, 0, s>>>(g, O, w.authbits, w.U, w.parent, w.wait_v, w.cnt,
                                                         w.listhead, w.next_w, w.spill_n, w.class_cap, w.ctr);
    w.launches += 1;
    return cudaGetLastError();
}

template cudaError_t classify<1>(Work&, const Geom&, const int*, cudaStream_t);
template cudaError_t classify<-1>(Work&, const Geom&, const int*, cudaStream_t);

}  // namespace lts
