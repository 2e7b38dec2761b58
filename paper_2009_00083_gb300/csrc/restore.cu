// Optional post-process of step 3 (Sec. 4.2): restoring authorized extrema of
// the other kind that a region swallowed (mode flag LTS_MODE_RESTORE).
//
// In the maxima pass (the minima pass mirrors it on Od = N-1-O) a region R
// can contain authorized minima of the pass's input order.  Every neighbour
// of such a minimum lies in R (it is higher, so above the saddle s and
// connected to it), and the local order of step 2 makes none of them a
// minimum.  The paper restores one by making it smaller than all its
// neighbours.  Here each region's swallowed authorized minima are taken in
// increasing Od; one moves below every vertex of the region's block (below
// the ones already restored, which are never its neighbours) unless one of
// its neighbours u would be left without a higher neighbour: u would become a
// maximum, an unauthorized extremum.  Vertices outside R next to a vertex of
// R other than s sit below the block of R, so only s and members of R can be
// higher.  The block's local order is then renumbered: the restored vertices
// first, in the order they were restored, then the others in their order.
//
// rs_mark_kernel: one thread per member finds the swallowed candidates and
// lists their regions; rs_apply_kernel: one thread per listed region (rare:
// only arbitrary authorized sets put authorized extrema inside regions).
#include <climits>

#include "lts_internal.cuh"

namespace lts {

namespace {

__device__ __forceinline__ bool auth_bit(const unsigned* bits, int v) { return (__ldg(bits + (v >> 5)) >> (v & 31)) & 1u; }

// v is a minimum of Od: every neighbour is higher
template <int DIR>
__device__ bool is_min_od(const Geom& g, const int* __restrict__ O, int v) {
    int x, y, z;
    coords_of(g, v, x, y, z);
    const int ov = od<DIR>(__ldg(O + v), g.n);
    for (int q = 0; q < g.nn; ++q) {
        const int nb = nbr_of(g, x, y, z, q);
        if (nb >= 0 && od<DIR>(__ldg(O + nb), g.n) < ov) return false;
    }
    return true;
}

template <int DIR>
__global__ void rs_mark_kernel(Geom g, const int* __restrict__ O, const unsigned* __restrict__ authbits,
                               const int* __restrict__ members, const int* __restrict__ member_reg,
                               const int* __restrict__ reg_start, int* reg_cnt, int* rs_list, DevCounters* ctr) {
    if (failed(&ctr->status)) return;
    const int nreg = ctr->n_regions;
    const int total = nreg > 0 ? reg_start[nreg] : 0;
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < total; p += gridDim.x * blockDim.x) {
        const int w = members[p];
        if (!auth_bit(authbits, w) || !is_min_od<DIR>(g, O, w)) continue;
        const int r = member_reg[p];
        if (atomicAdd(reg_cnt + r, 1) == 0) rs_list[atomicAdd(&ctr->n_rs_regions, 1)] = r;
    }
}

// K: the current key of every local index of a region (members 0..m-1);
// restored vertices have keys below every other.
template <int DIR>
__global__ void rs_apply_kernel(Geom g, const int* __restrict__ O, const unsigned* __restrict__ authbits,
                                const int* __restrict__ members, const int* __restrict__ reg_start,
                                const int* __restrict__ reg_size, const int* __restrict__ reg_saddle,
                                const int* __restrict__ owner, const int* __restrict__ loc, int* lhat,
                                const int* __restrict__ rs_list, int* lo_K, int* lo_orig, DevCounters* ctr) {
    if (failed(&ctr->status)) return;
    const int nl = ctr->n_rs_regions;
    long long restored = 0;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < nl; k += gridDim.x * blockDim.x) {
        const int r = rs_list[k];
        const int st0 = reg_start[r], m = reg_size[r], s = reg_saddle[r];
        const int tag = -2 - r;
        int* K = lo_K + st0 + r;                        // the region's local-order scratch slots
        int* orig = lo_orig + st0 + r;
        for (int i = 0; i < m; ++i) K[i] = lhat[st0 + i];
        int done = 0, last = -1;
        for (;;) {
            // the next swallowed authorized minimum in increasing Od
            int w = -1, ow = INT_MAX;
            for (int i = 0; i < m; ++i) {
                const int v = members[st0 + i];
                const int o = od<DIR>(__ldg(O + v), g.n);
                if (o <= last || o >= ow || !auth_bit(authbits, v) || !is_min_od<DIR>(g, O, v)) continue;
                w = v;
                ow = o;
            }
            if (w < 0) break;
            last = ow;
            // every neighbour u of w must keep a higher neighbour other than w
            bool ok = true;
            int x, y, z;
            coords_of(g, w, x, y, z);
            for (int q = 0; q < g.nn && ok; ++q) {
                const int u = nbr_of(g, x, y, z, q);
                if (u < 0) continue;
                if (__ldg(owner + u) != tag) {            // cannot happen: a region is a superlevel component
                    set_status(&ctr->status, LTS_ERR_INTERNAL);
                    ok = false;
                    break;
                }
                const int ku = K[__ldg(loc + u)];
                int ux, uy, uz;
                coords_of(g, u, ux, uy, uz);
                bool higher = false;
                for (int q2 = 0; q2 < g.nn && !higher; ++q2) {
                    const int xx = nbr_of(g, ux, uy, uz, q2);
                    if (xx < 0 || xx == w) continue;
                    if (xx == s) higher = true;
                    else if (__ldg(owner + xx) == tag && K[__ldg(loc + xx)] > ku) higher = true;
                }
                ok = higher;
            }
            if (!ok) continue;
            const int iw = __ldg(loc + w);
            orig[done] = K[iw];
            K[iw] = INT_MIN + done;
            ++done;
        }
        if (done == 0) continue;
        for (int i = 0; i < m; ++i) {
            int nv;
            if (K[i] < 0) {
                nv = K[i] - INT_MIN;
            } else {
                int below = 0;
                for (int j = 0; j < done; ++j) below += orig[j] < K[i];
                nv = done + K[i] - below;
            }
            lhat[st0 + i] = nv;
        }
        restored += done;
    }
    if (restored) atomicAdd((unsigned long long*)&ctr->n_restored, (unsigned long long)restored);
}

}  // namespace

template <int DIR>
cudaError_t restore_swallowed(Work& w, const Geom& g, const int* O, int sms, cudaStream_t s) {
    cudaMemsetAsync(w.reg_swallowed, 0, sizeof(int) * (size_t)w.class_cap, s);
    rs_mark_kernel<DIR><<<sms * 8, 256, 0, s>>>(g, O, w.authbits, w.members, w.member_reg, w.reg_start,
                                                w.reg_swallowed, w.tier_list, w.ctr);
    rs_apply_kernel<DIR><<<sms, 128, 0, s>>>(g, O, w.authbits, w.members, w.reg_start, w.reg_size, w.reg_saddle,
                                             w.owner, w.loc, w.lhat, w.tier_list, w.lo_L, w.lo_L2, w.ctr);
    w.launches += 2;
    return cudaGetLastError();
}

template cudaError_t restore_swallowed<1>(Work&, const Geom&, const int*, int, cudaStream_t);
template cudaError_t restore_swallowed<-1>(Work&, const Geom&, const int*, int, cudaStream_t);

}  // namespace lts
