// Extremum classification for one pass (Sec. 3.1, Eq. 1).
//
// A vertex is a maximum of the pass-oriented order Od when none of its
// Freudenthal neighbours is higher.  Authorized maxima are counted; the
// unauthorized ones form the list U of propagation seeds, appended with one
// atomic per warp, and each gets a fresh class record for step 1.
#include "lts_internal.cuh"

namespace lts {

namespace {

template <int DIR>
__global__ void __launch_bounds__(256) classify_kernel(Geom g, const int* __restrict__ O,
                                                       const unsigned* __restrict__ authbits, int* __restrict__ U,
                                                       int* __restrict__ parent, int* __restrict__ wait_v,
                                                       int* __restrict__ cnt, int* __restrict__ listhead,
                                                       int* __restrict__ next_w, int* __restrict__ spill_n,
                                                       int cap, DevCounters* ctr) {
    if (failed(&ctr->status)) return;
    const int lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long b = (long long)blockIdx.x * blockDim.x; b < g.n; b += stride) {
        const long long vv = b + threadIdx.x;
        bool ext = false;
        int v = (int)vv;
        if (vv < g.n) {
            const int ov = od<DIR>(__ldg(O + v), g.n);
            int x, y, z;
            coords_of(g, v, x, y, z);
            ext = true;
            for (int k = 0; k < g.nn; ++k) {
                const int nb = nbr_of(g, x, y, z, k);
                if (nb >= 0 && od<DIR>(__ldg(O + nb), g.n) > ov) { ext = false; break; }
            }
        }
        const bool auth = ext && ((__ldg(authbits + (v >> 5)) >> (v & 31)) & 1u);
        const bool un = ext && !auth;
        const unsigned ma = __ballot_sync(0xffffffffu, auth);
        const unsigned mu = __ballot_sync(0xffffffffu, un);
        int basepos = 0;
        if (lane == 0) {
            if (ma) atomicAdd(&ctr->n_auth_ext, __popc(ma));
            if (mu) basepos = atomicAdd(&ctr->n_unauth, __popc(mu));
        }
        basepos = __shfl_sync(0xffffffffu, basepos, 0);
        if (un) {
            const int c = basepos + __popc(mu & lt);
            if (c >= cap) { set_status(&ctr->status, LTS_ERR_INTERNAL); continue; }
            U[c] = v;
            parent[c] = c;
            wait_v[c] = -1;
            cnt[c] = 0;
            listhead[c] = -1;
            next_w[c] = -1;
            spill_n[c] = 0;
        }
    }
}

}  // namespace

template <int DIR>
cudaError_t classify(Work& w, const Geom& g, const int* O, cudaStream_t s) {
    const int threads = 256;
    const long long blocks = std::min<long long>(((long long)g.n + threads - 1) / threads, 152LL * 16);
    classify_kernel<DIR><<<(int)blocks, threads, 0, s>>>(g, O, w.authbits, w.U, w.parent, w.wait_v, w.cnt,
                                                         w.listhead, w.next_w, w.spill_n, w.class_cap, w.ctr);
    w.launches += 1;
    return cudaGetLastError();
}

template cudaError_t classify<1>(Work&, const Geom&, const int*, cudaStream_t);
template cudaError_t classify<-1>(Work&, const Geom&, const int*, cudaStream_t);

}  // namespace lts
