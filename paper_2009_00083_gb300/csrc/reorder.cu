// Steps 3 and 4 (Sec. 4.2, Eq. 6; numerical perturbation with zeta = 0).
//
// In pass-oriented ranks j = Od(v), every region forms a contiguous block
// right below its saddle and all other vertices keep their relative order.
// So a non-member at rank j moves to
//     j - M(j) + A(j)
// with M(j) the members ranked below j and A(j) the members whose saddle is
// ranked at or below j.  Both are read from a rank-space bitmap of 32-rank
// blocks holding the member and saddle bits and their prefix counts (16
// bytes per block, one vector load, 0.5 byte per vertex, so it stays in L2),
// plus the prefix sums of the block sizes per saddle.  A member w of region R at saddle s goes to
//     newrank(s) - attached(s) + offset(R) + lhat(w)
// and takes g(s) bit for bit.  No global sort is needed.
#include "lts_internal.cuh"

namespace lts {

namespace {

constexpr int kT = 256;
constexpr int kPer = 16;

// ---- exclusive scan of the rank blocks' (member, saddle) popcounts ----
__global__ void blk_sums_kernel(const RankBlk* __restrict__ b, int nb, unsigned long long* tsum) {
    __shared__ unsigned long long s[kT];
    const int base = blockIdx.x * kT * kPer;
    unsigned long long acc = 0;
    for (int i = 0; i < kPer; ++i) {
        const int k = base + threadIdx.x * kPer + i;
        if (k < nb) acc += (unsigned long long)__popc(b[k].mmask) | ((unsigned long long)__popc(b[k].smask) << 32);
    }
    s[threadIdx.x] = acc;
    __syncthreads();
    for (int o = kT / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) s[threadIdx.x] += s[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) tsum[blockIdx.x] = s[0];
}

__global__ void tile_scan_kernel(unsigned long long* tsum, int nt) {
    // single block of 1024 threads: exclusive scan in place
    __shared__ unsigned long long s[1024];
    const int per = (nt + 1023) / 1024;
    const int b = threadIdx.x * per;
    unsigned long long acc = 0;
    for (int i = 0; i < per; ++i) if (b + i < nt) acc += tsum[b + i];
    s[threadIdx.x] = acc;
    __syncthreads();
    for (int o = 1; o < 1024; o <<= 1) {
        unsigned long long v = threadIdx.x >= o ? s[threadIdx.x - o] : 0;
        __syncthreads();
        s[threadIdx.x] += v;
        __syncthreads();
    }
    unsigned long long run = s[threadIdx.x] - acc;
    for (int i = 0; i < per; ++i)
        if (b + i < nt) { unsigned long long t = tsum[b + i]; tsum[b + i] = run; run += t; }
}

__global__ void blk_apply_kernel(RankBlk* b, int nb, const unsigned long long* __restrict__ tsum) {
    __shared__ unsigned long long s[kT];
    const int base = blockIdx.x * kT * kPer;
    unsigned long long acc = 0;
    for (int i = 0; i < kPer; ++i) {
        const int k = base + threadIdx.x * kPer + i;
        if (k < nb) acc += (unsigned long long)__popc(b[k].mmask) | ((unsigned long long)__popc(b[k].smask) << 32);
    }
    s[threadIdx.x] = acc;
    __syncthreads();
    for (int o = 1; o < kT; o <<= 1) {
        unsigned long long v = threadIdx.x >= o ? s[threadIdx.x - o] : 0;
        __syncthreads();
        s[threadIdx.x] += v;
        __syncthreads();
    }
    unsigned long long run = tsum[blockIdx.x] + s[threadIdx.x] - acc;
    for (int i = 0; i < kPer; ++i) {
        const int k = base + threadIdx.x * kPer + i;
        if (k < nb) {
            b[k].mpre = (unsigned)run;
            b[k].spre = (unsigned)(run >> 32);
            run += (unsigned long long)__popc(b[k].mmask) | ((unsigned long long)__popc(b[k].smask) << 32);
        }
    }
}

// saddle number k (by rank) -> block total attached below it
__global__ void saddle_index_kernel(const RankBlk* __restrict__ rb, const int* __restrict__ reg_head,
                                    const int* __restrict__ reg_sod, const int* __restrict__ reg_att, int* sad_att,
                                    const DevCounters* ctr) {
    if (failed(&ctr->status)) return;
    const int nreg = ctr->n_regions;
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < nreg; r += gridDim.x * blockDim.x) {
        if (!reg_head[r]) continue;
        const int j = reg_sod[r];
        const RankBlk b = rb[j >> kRankShift];
        const int k = (int)b.spre + __popc(b.smask & ((1u << (j & 31)) - 1u));
        sad_att[k] = reg_att[r];
    }
}

__device__ __forceinline__ int new_rank(const RankBlk* __restrict__ rb, const int* __restrict__ cumA, int j) {
    const uint4 b = __ldg(reinterpret_cast<const uint4*>(rb) + (j >> kRankShift));   // mmask, smask, mpre, spre
    const int bit = j & 31;
    const unsigned lt = (1u << bit) - 1u;
    const unsigned le = lt | (1u << bit);
    const int M = (int)b.z + __popc(b.x & lt);
    const int A = __ldg(cumA + (int)b.w + __popc(b.y & le));
    return j - M + A;
}

template <int DIR>
__global__ void __launch_bounds__(kT) stream_kernel(int n, int* O, const RankBlk* __restrict__ rb,
                                                    const int* __restrict__ cumA, const DevCounters* ctr) {
    if (failed(&ctr->status)) return;
    if (ctr->n_regions == 0) return;
    const long long stride = (long long)gridDim.x * blockDim.x;
    const long long n4 = (reinterpret_cast<unsigned long long>(O) & 15ull) == 0 ? (n >> 2) : 0;
    int4* O4 = reinterpret_cast<int4*>(O);
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n4; i += stride) {
        int4 o = O4[i];
        o.x = od<DIR>(new_rank(rb, cumA, od<DIR>(o.x, n)), n);
        o.y = od<DIR>(new_rank(rb, cumA, od<DIR>(o.y, n)), n);
        o.z = od<DIR>(new_rank(rb, cumA, od<DIR>(o.z, n)), n);
        o.w = od<DIR>(new_rank(rb, cumA, od<DIR>(o.w, n)), n);
        O4[i] = o;
    }
    for (long long i = 4 * n4 + blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += stride)
        O[i] = od<DIR>(new_rank(rb, cumA, od<DIR>(O[i], n)), n);
}

// one thread per member (CSR position); the first threads also reset the
// saddles' claims
template <int DIR, typename T>
__global__ void members_place_kernel(int n, int* O, T* gout, int* owner, const int* __restrict__ members,
                                     const int* __restrict__ member_reg, const int* __restrict__ lhat,
                                     const int* __restrict__ reg_saddle, const int* __restrict__ reg_sod,
                                     const int* __restrict__ reg_place, const int* __restrict__ reg_start,
                                     const RankBlk* __restrict__ rb, const int* __restrict__ cumA,
                                     const DevCounters* ctr) {
    if (failed(&ctr->status)) return;
    const int nreg = ctr->n_regions;
    const int total = nreg > 0 ? reg_start[nreg] : 0;
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < total; p += gridDim.x * blockDim.x) {
        const int r = member_reg[p];
        const int w = members[p];
        const int s = reg_saddle[r];
        O[w] = od<DIR>(new_rank(rb, cumA, reg_sod[r]) + reg_place[r] + lhat[p], n);
        gout[w] = gout[s];
        owner[w] = -1;
    }
}

// the final saddles: release their claims and clear their arrival counters
__global__ void saddles_reset_kernel(int* owner, int* cnt, const int* __restrict__ reg_saddle, const DevCounters* ctr) {
    const int nreg = ctr->n_regions;
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < nreg; r += gridDim.x * blockDim.x) {
        const int sv = reg_saddle[r];
        owner[sv] = -1;
        cnt[sv] = 0;
    }
}

}  // namespace

// The rank prefix of step 3: member and saddle counts before every 32-rank
// block, and the members attached to each saddle, summed over the saddles.
// It needs the regions only, not their local orders.
cudaError_t reorder_prefix(Work& w, const Geom& g, int sms, cudaStream_t s) {
    const int nb = w.nblk_cur;
    const int per_tile = kT * kPer;
    const int nt = (nb + per_tile - 1) / per_tile;
    blk_sums_kernel<<<nt, kT, 0, s>>>(w.rblk, nb, w.scan_tmp);
    tile_scan_kernel<<<1, 1024, 0, s>>>(w.scan_tmp, nt);
    blk_apply_kernel<<<nt, kT, 0, s>>>(w.rblk, nb, w.scan_tmp);
    saddle_index_kernel<<<sms * 8, 256, 0, s>>>(w.rblk, w.reg_head, w.reg_sod, w.reg_att, w.sad_att, w.ctr);
    scan_excl_i32(w, w.sad_att, w.cumA, &w.ctr->n_saddles, g.n / 2 + 1, s);
    w.launches += 4;
    return cudaGetLastError();
}

template <int DIR>
cudaError_t reorder_flatten(Work& w, const Geom& g, int* O, void* gout, bool f64, int sms, cudaStream_t s) {
    stream_kernel<DIR><<<sms * 8, kT, 0, s>>>(g.n, O, w.rblk, w.cumA, w.ctr);
    if (f64)
        members_place_kernel<DIR, double><<<sms * 8, 256, 0, s>>>(g.n, O, static_cast<double*>(gout), w.owner,
                                                                  w.members, w.member_reg, w.lhat, w.reg_saddle,
                                                                  w.reg_sod, w.reg_place, w.reg_start, w.rblk,
                                                                  w.cumA, w.ctr);
    else
        members_place_kernel<DIR, float><<<sms * 8, 256, 0, s>>>(g.n, O, static_cast<float*>(gout), w.owner,
                                                                 w.members, w.member_reg, w.lhat, w.reg_saddle,
                                                                 w.reg_sod, w.reg_place, w.reg_start, w.rblk,
                                                                 w.cumA, w.ctr);
    saddles_reset_kernel<<<sms * 4, 256, 0, s>>>(w.owner, w.cnt, w.reg_saddle, w.ctr);
    w.launches += 3;
    return cudaGetLastError();
}

template cudaError_t reorder_flatten<1>(Work&, const Geom&, int*, void*, bool, int, cudaStream_t);
template cudaError_t reorder_flatten<-1>(Work&, const Geom&, int*, void*, bool, int, cudaStream_t);

}  // namespace lts
