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
// exactly when it is the maximum of both cubes.  A block loads a tile of the
// pass-oriented order with a one-vertex halo into shared memory (outside the
// grid: -1, below every rank), computes the maxima of all 2x2x2 cubes
// separably, and compares.  The tile's unauthorized extrema are appended
// with one atomic.
constexpr int TX = 32, TY = 8, TZ = 8;       // outputs per tile (3D); 2D uses TZ = 1
constexpr int kCT = 256;

template <int DIR, int TZT>
__global__ void __launch_bounds__(kCT) classify_kernel(Geom g, const int* __restrict__ O,
                                                       const unsigned* __restrict__ authbits, int* __restrict__ U,
                                                       int* __restrict__ parent, int* __restrict__ wait_v,
                                                       int* __restrict__ spill_n, int* __restrict__ sib_head,
                                                       int cap, DevCounters* ctr) {
    constexpr int SX = TX + 2, SY = TY + 2, SZ = TZT + 2;
    __shared__ int S[SZ][SY][SX];            // order with halo
    __shared__ int s_warp[kCT / 32];
    __shared__ int s_base;
    if (failed(&ctr->status)) return;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int ntx = (g.X + TX - 1) / TX, nty = (g.Y + TY - 1) / TY, ntz = (g.Z + TZT - 1) / TZT;
    const long long ntiles = (long long)ntx * nty * ntz;
    int my_auth = 0;
    for (long long t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const int tx = (int)(t % ntx), ty = (int)((t / ntx) % nty), tz = (int)(t / ((long long)ntx * nty));
        const int x0 = tx * TX - 1, y0 = ty * TY - 1, z0 = tz * TZT - 1;
        // rows of SX values (one per (y, z) of the halo tile), one row per warp
        // step; every lane issues its loads before storing any of them
        constexpr int ROWS = SY * SZ;
        constexpr int RPW = (ROWS + kCT / 32 - 1) / (kCT / 32);   // rows per warp
        int vals[RPW][2];
#pragma unroll
        for (int k = 0; k < RPW; ++k) {
            const int rr = warp + k * (kCT / 32);
            const int ly = rr % SY, lz = rr / SY;
            const int y = y0 + ly, z = z0 + lz;
            const bool rowok = rr < ROWS && (unsigned)y < (unsigned)g.Y && (unsigned)z < (unsigned)g.Z;
            const int* rowp = O + (long long)g.XY * z + (long long)g.X * y;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int lx = lane + 32 * h;
                const int x = x0 + lx;
                vals[k][h] = (rowok && lx < SX && (unsigned)x < (unsigned)g.X) ? od<DIR>(__ldg(rowp + x), g.n) : -1;
            }
        }
#pragma unroll
        for (int k = 0; k < RPW; ++k) {
            const int rr = warp + k * (kCT / 32);
            if (rr >= ROWS) break;
            const int ly = rr % SY, lz = rr / SY;
            S[lz][ly][lane] = vals[k][0];
            if (lane + 32 < SX) S[lz][ly][lane + 32] = vals[k][1];
        }
        __syncthreads();
        // each thread: PER consecutive outputs along x of one (y, z) row; the two
        // cubes of an output use 7 rows of S: (dy,dz) in {0,1}^2 and -{0,1}^2
        unsigned mu = 0;
        constexpr int PER = TX * TY * TZT / kCT;
        constexpr int GROUPS = TX / PER;   // threads along x per row
        const int gx = threadIdx.x % GROUPS, row = threadIdx.x / GROUPS;
        const int oy = row % TY, oz = row / TY;
        const int z = z0 + 1 + oz, y = y0 + 1 + oy;
        const int vfirst = (x0 + 1 + gx * PER) + g.X * y + g.XY * z;
        if (oz < TZT && z < g.Z && y < g.Y) {
            const int bx = gx * PER;           // S column of x - 1 for the first output
            constexpr int DY[7] = {0, 1, 0, 1, -1, 0, -1};
            constexpr int DZ[7] = {0, 0, 1, 1, 0, -1, -1};
            int pm[7][PER + 1];                // pairwise x maxima of each row
#pragma unroll
            for (int r = 0; r < 7; ++r) {
                int prevv = S[oz + 1 + DZ[r]][oy + 1 + DY[r]][bx];
#pragma unroll
                for (int i = 0; i <= PER; ++i) {
                    const int cur = S[oz + 1 + DZ[r]][oy + 1 + DY[r]][bx + 1 + i];
                    pm[r][i] = max(prevv, cur);
                    prevv = cur;
                }
            }
#pragma unroll
            for (int i = 0; i < PER; ++i) {
                const int x = x0 + 1 + bx + i;
                if (x >= g.X) break;
                const int ov = S[oz + 1][oy + 1][bx + 1 + i];
                const int cpos = max(max(pm[0][i + 1], pm[1][i + 1]), max(pm[2][i + 1], pm[3][i + 1]));
                const int cneg = max(max(pm[0][i], pm[4][i]), max(pm[5][i], pm[6][i]));
                if (ov == cpos && ov == cneg) {
                    const int v = vfirst + i;
                    if ((__ldg(authbits + (v >> 5)) >> (v & 31)) & 1u) ++my_auth;
                    else mu |= 1u << i;
                }
            }
        }
        // block-wide exclusive scan of the per-thread counts, one atomic per tile
        const int c = __popc(mu);
        int x = c;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int yv = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += yv;
        }
        if (lane == 31) s_warp[warp] = x;
        __syncthreads();
        if (threadIdx.x == 0) {
            int run = 0;
            for (int w = 0; w < kCT / 32; ++w) { const int tt = s_warp[w]; s_warp[w] = run; run += tt; }
            s_base = run ? atomicAdd(&ctr->n_unauth, run) : 0;
        }
        __syncthreads();
        int pos = s_base + s_warp[warp] + x - c;
        while (mu) {
            const int i = __ffs(mu) - 1;
            mu &= mu - 1;
            const int cl = pos++;
            if (cl >= cap) { set_status(&ctr->status, LTS_ERR_INTERNAL); continue; }
            U[cl] = vfirst + i;
            parent[cl] = cl;
            wait_v[cl] = -1;
            spill_n[cl] = -1;            // never spilled: a queue rebuilt from the seed
            sib_head[cl] = -1;
        }
        __syncthreads();
    }
    warp_atomic_add(&ctr->n_auth_ext, my_auth);
}

}  // namespace

template <int DIR>
cudaError_t classify(Work& w, const Geom& g, const int* O, cudaStream_t s) {
    const long long tiles = (long long)((g.X + TX - 1) / TX) * ((g.Y + TY - 1) / TY) *
                            (g.ndim == 3 ? (g.Z + TZ - 1) / TZ : 1);
    const int blocks = (int)std::min<long long>(tiles, 152LL * 8);
    if (g.ndim == 3)
        classify_kernel<DIR, TZ><<<blocks, kCT, 0, s>>>(g, O, w.authbits, w.U, w.parent, w.wait_v,
                                                        w.spill_n, w.sib_head, w.class_cap, w.ctr);
    else
        classify_kernel<DIR, 1><<<blocks, kCT, 0, s>>>(g, O, w.authbits, w.U, w.parent, w.wait_v,
                                                       w.spill_n, w.sib_head, w.class_cap, w.ctr);
    w.launches += 1;
    return cudaGetLastError();
}

template cudaError_t classify<1>(Work&, const Geom&, const int*, cudaStream_t);
template cudaError_t classify<-1>(Work&, const Geom&, const int*, cudaStream_t);

}  // namespace lts
