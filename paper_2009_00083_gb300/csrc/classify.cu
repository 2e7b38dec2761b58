// Extremum classification for one pass (Sec. 3.1, Eq. 1).
//
// A vertex is a maximum of the pass-oriented order Od when none of its
// Freudenthal neighbours is higher.  Authorized maxima are counted; the
// unauthorized ones form the list U of propagation seeds, and each gets a
// fresh class record for step 1.
#include "lts_internal.cuh"

namespace lts {

namespace {

// The Freudenthal neighbourhood of v is the union of two unit cubes: the one
// with v as its lowest corner and the one with v as its highest corner
// (offsets {0,1}^d and -{0,1}^d).  The order is injective, so v is a maximum
// exactly when it is the maximum of both cubes.  Each cube is two 2x2
// squares of consecutive z planes: with A_z(x,y) the maximum of the square
// {x,x+1} x {y,y+1} of plane z and B_z(x,y) that of {x-1,x} x {y-1,y},
//     v is a maximum  <=>  v == max(A_z, A_z+1)  and  v == max(B_z, B_z-1).
// A warp owns 30 consecutive x of one row y (its lanes span x-1 .. x+30, so
// the two end lanes only provide neighbours) and marches kZC planes along z.
// Per plane a lane loads its vertex in rows y-1, y, y+1 (the neighbouring
// warps of the block read the same lines, so most of these hit L1), takes
// x-1 and x+1 from its neighbour lanes and keeps the squares of its column in
// registers.  The minima pass compares with min instead of max on O itself
// (outside the grid: -1 for maxima, N for minima), so no value is
// transformed.  A 2D grid is the case Z = 1.  Unauthorized extrema are
// gathered per warp in shared memory and appended to U with one atomic per
// flush.
constexpr int kWarps = 8;                    // rows per block
constexpr int kCT = 32 * kWarps;
constexpr int kOut = 30;                     // outputs per warp row
constexpr int kZC = 64;                      // planes per warp
constexpr int kWL = 256;                     // gathered extrema per warp before a flush

template <int DIR>
__device__ __forceinline__ int top2(int a, int b) { return DIR > 0 ? max(a, b) : min(a, b); }

template <int DIR>
__global__ void __launch_bounds__(kCT) classify_kernel(Geom g, const int* __restrict__ O,
                                                       const unsigned* __restrict__ authbits, int* __restrict__ U,
                                                       int* __restrict__ parent, int* __restrict__ wait_v,
                                                       int* __restrict__ spill_n, int* __restrict__ sib_head,
                                                       int cap, DevCounters* ctr) {
    __shared__ int s_list[kWarps][kWL];
    if (failed(&ctr->status)) return;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int outside = DIR > 0 ? -1 : g.n;
    const int ntx = (g.X + kOut - 1) / kOut, nty = (g.Y + kWarps - 1) / kWarps, nzc = (g.Z + kZC - 1) / kZC;
    const int ntxy = ntx * nty;
    const int nblk = ntxy * nzc;
    int* L = s_list[warp];
    int cnt = 0;                             // gathered in L (warp-uniform)
    int my_auth = 0;

    auto flush = [&]() {
        if (cnt == 0) return;
        int base = 0;
        if (lane == 0) base = atomicAdd(&ctr->n_unauth, cnt);
        base = __shfl_sync(0xffffffffu, base, 0);
        for (int i = lane; i < cnt; i += 32) {
            const int cl = base + i;
            if (cl >= cap) { set_status(&ctr->status, LTS_ERR_INTERNAL); continue; }
            U[cl] = L[i];
            parent[cl] = cl;
            wait_v[cl] = -1;
            spill_n[cl] = -1;                // never spilled: a queue rebuilt from the seed
            sib_head[cl] = -1;
        }
        __syncwarp();
        cnt = 0;
    };

    for (int b = blockIdx.x; b < nblk; b += gridDim.x) {
        const int zc = b / ntxy, t = b - zc * ntxy;
        const int ty = t / ntx, tx = t - ty * ntx;
        const int y = ty * kWarps + warp;
        if (y >= g.Y) continue;                          // warp-uniform: no output row
        const int x = tx * kOut - 1 + lane;
        const bool xin = (unsigned)x < (unsigned)g.X;
        const bool out_lane = lane >= 1 && lane <= kOut && x < g.X;
        const int zs = zc * kZC, ze = min(zs + kZC, g.Z);
        const bool r0 = y >= 1 && xin, r1 = xin, r2 = y + 1 < g.Y && xin;
        // rows y-1, y, y+1 of plane zs-1 at x (pointer arithmetic only where valid)
        const int* p = O + ((long long)g.XY * (zs - 1) + (long long)g.X * y + (xin ? x : 0));
        const long long XY = g.XY;
        const int X = g.X;
        auto load = [&](int pz, const int* q, int& a0, int& a1, int& a2) {
            const bool pin = (unsigned)pz < (unsigned)g.Z;
            a0 = (pin && r0) ? __ldg(q - X) : outside;
            a1 = (pin && r1) ? __ldg(q) : outside;
            a2 = (pin && r2) ? __ldg(q + X) : outside;
        };
        // squares of the lane's column in one plane
        auto squares = [&](int a0, int a1, int a2, int& A, int& B) {
            const int n1 = __shfl_down_sync(0xffffffffu, a1, 1), n2 = __shfl_down_sync(0xffffffffu, a2, 1);
            const int p0 = __shfl_up_sync(0xffffffffu, a0, 1), p1 = __shfl_up_sync(0xffffffffu, a1, 1);
            A = top2<DIR>(top2<DIR>(a1, n1), top2<DIR>(a2, n2));
            B = top2<DIR>(top2<DIR>(a1, p1), top2<DIR>(a0, p0));
        };
        int c0, c1, c2, d0, d1, d2;
        load(zs - 1, p, c0, c1, c2);
        load(zs, p + XY, d0, d1, d2);
        int Am, Bm, A0, B0;
        squares(c0, c1, c2, Am, Bm);                    // plane zs-1: only B is used
        squares(d0, d1, d2, A0, B0);                    // plane zs
        int v0 = d1;
        p += 2 * XY;                                    // plane zs+1
        int e0, e1, e2;
        load(zs + 1, p, e0, e1, e2);
        for (int z = zs; z < ze; ++z) {
            const int w0 = e0, w1 = e1, w2 = e2;        // plane z+1
            p += XY;
            if (z + 2 <= ze) load(z + 2, p, e0, e1, e2); // one plane ahead
            int A1, B1;
            squares(w0, w1, w2, A1, B1);
            const bool is_ext = out_lane && v0 == top2<DIR>(A0, A1) && v0 == top2<DIR>(B0, Bm);
            bool unauth = false;
            int v = 0;
            if (is_ext) {
                v = x + X * y + g.XY * z;
                if ((__ldg(authbits + (v >> 5)) >> (v & 31)) & 1u) ++my_auth;
                else unauth = true;
            }
            const unsigned m = __ballot_sync(0xffffffffu, unauth);
            if (m) {
                if (unauth) L[cnt + __popc(m & ((1u << lane) - 1u))] = v;
                cnt += __popc(m);
                __syncwarp();
                if (cnt > kWL - 32) flush();
            }
            Bm = B0;
            A0 = A1; B0 = B1; v0 = w1;
        }
    }
    flush();
    warp_atomic_add(&ctr->n_auth_ext, my_auth);
}

}  // namespace

template <int DIR>
cudaError_t classify(Work& w, const Geom& g, const int* O, cudaStream_t s) {
    const long long nblk = (long long)((g.X + kOut - 1) / kOut) * ((g.Y + kWarps - 1) / kWarps) * ((g.Z + kZC - 1) / kZC);
    const int blocks = (int)std::min<long long>(nblk, (long long)w.sms * 8 * 4);
    classify_kernel<DIR><<<blocks, kCT, 0, s>>>(g, O, w.authbits, w.U, w.parent, w.wait_v, w.spill_n, w.sib_head,
                                                w.class_cap, w.ctr);
    w.launches += 1;
    return cudaGetLastError();
}

template cudaError_t classify<1>(Work&, const Geom&, const int*, cudaStream_t);
template cudaError_t classify<-1>(Work&, const Geom&, const int*, cudaStream_t);

}  // namespace lts
