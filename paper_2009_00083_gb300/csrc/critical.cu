// Critical points of an order field (Sec. 3.1): for every vertex, the number
// of connected components of its lower link and of its upper link.  Minimum:
// empty lower link; maximum: empty upper link; regular: both connected and
// non-empty; otherwise a saddle (in 3D: lower link split = join saddle, upper
// link split = split saddle).
//
// The link of a vertex in the Freudenthal (Kuhn) triangulation is the graph
// on its neighbour offsets in which offsets a and b are adjacent when
// {0, a, b} is a simplex: both non-negative with strictly nested supports,
// both non-positive with strictly nested supports, or one non-negative and
// the other non-positive with disjoint supports (a hexagon in 2D; 36 edges
// on 14 offsets in 3D).  An interior vertex has every neighbour, so its
// (lower, upper) component counts depend only on which neighbours are lower:
// a table of 2^nn entries, built once per workspace, answers them with one
// load.  A vertex on the grid boundary has missing neighbours, and its
// counts come from a union-find over the present ones instead.
#include "lts_internal.cuh"

namespace lts {

namespace {

// Offset k < nn/2 is the (k+1)-th non-zero 0/1 vector (bit b = axis b),
// offset k + nn/2 its negative.
__device__ __forceinline__ bool link_adjacent(int a, int b, int half) {
    const bool pa = a < half, pb = b < half;
    const int ma = (pa ? a : a - half) + 1, mb = (pb ? b : b - half) + 1;
    if (pa == pb) return ma != mb && ((ma & mb) == ma || (ma & mb) == mb);   // nested supports
    return (ma & mb) == 0;                                                    // disjoint supports
}

// Components of the link restricted to the offsets in `mask` (bit k: offset k).
__device__ int link_components(unsigned mask, int nn) {
    int parent[14];
    const int half = nn >> 1;
    for (int k = 0; k < nn; ++k) parent[k] = k;
    int comps = 0;
    for (int a = 0; a < nn; ++a) {
        if (!((mask >> a) & 1u)) continue;
        ++comps;
        for (int b = 0; b < a; ++b) {
            if (!((mask >> b) & 1u) || !link_adjacent(a, b, half)) continue;
            int ra = a, rb = b;
            while (parent[ra] != ra) ra = parent[ra];
            while (parent[rb] != rb) rb = parent[rb];
            if (ra != rb) {
                parent[ra] = rb;
                --comps;
            }
        }
    }
    return comps;
}

// table[mask] = lower components | upper components << 4, for a vertex with
// every neighbour present and the neighbours in `mask` lower
__global__ void link_table_kernel(unsigned char* table, int nn) {
    const unsigned full = (1u << nn) - 1u;
    for (unsigned m = blockIdx.x * blockDim.x + threadIdx.x; m <= full; m += gridDim.x * blockDim.x)
        table[m] = (unsigned char)(link_components(m, nn) | (link_components(full & ~m, nn) << 4));
}

__global__ void critical_kernel(Geom g, const int* __restrict__ O, const unsigned char* __restrict__ table,
                                signed char* lower_out, signed char* upper_out, unsigned long long* counts) {
    unsigned long long c_min = 0, c_max = 0, c_reg = 0, c_sad = 0, c_lo = 0, c_up = 0;
    for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < g.n;
         v += (long long)gridDim.x * blockDim.x) {
        int x, y, z;
        coords_of(g, (int)v, x, y, z);
        const int ov = __ldg(O + v);
        unsigned lower = 0, present = 0;
        for (int q = 0; q < g.nn; ++q) {
            const int nb = nbr_of(g, x, y, z, q);
            if (nb < 0) continue;
            present |= 1u << q;
            if (__ldg(O + nb) < ov) lower |= 1u << q;
        }
        int nl, nu;
        if (present == (1u << g.nn) - 1u) {
            const unsigned char t = __ldg(table + lower);
            nl = t & 15;
            nu = t >> 4;
        } else {
            nl = link_components(lower, g.nn);
            nu = link_components(present & ~lower, g.nn);
        }
        if (lower_out) lower_out[v] = (signed char)nl;
        if (upper_out) upper_out[v] = (signed char)nu;
        if (nl == 0) ++c_min;
        else if (nu == 0) ++c_max;
        else if (nl == 1 && nu == 1) ++c_reg;
        else ++c_sad;
        if (nl > 1) c_lo += nl - 1;
        if (nu > 1) c_up += nu - 1;
    }
    unsigned long long vals[6] = {c_min, c_max, c_reg, c_sad, c_lo, c_up};
#pragma unroll
    for (int i = 0; i < 6; ++i) {
        unsigned long long t = vals[i];
        for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
        if ((threadIdx.x & 31) == 0 && t) atomicAdd(counts + i, t);
    }
}

}  // namespace

cudaError_t build_link_tables(unsigned char* t6, unsigned char* t14, cudaStream_t s) {
    link_table_kernel<<<1, 64, 0, s>>>(t6, 6);
    link_table_kernel<<<64, 256, 0, s>>>(t14, 14);
    return cudaGetLastError();
}

cudaError_t critical_points(Work& w, const Geom& g, const int* O, signed char* lower, signed char* upper,
                            unsigned long long* d_counts, cudaStream_t s) {
    cudaMemsetAsync(d_counts, 0, 6 * sizeof(unsigned long long), s);
    critical_kernel<<<w.sms * 8, 256, 0, s>>>(g, O, g.nn == 14 ? w.link14 : w.link6, lower, upper, d_counts);
    w.launches += 1;
    return cudaGetLastError();
}

}  // namespace lts
