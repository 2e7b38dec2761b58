// Device-wide exclusive scan of int32 values whose count lives on the
// device: out[i] = sum(in[0..i)), out[count] = total.  Three phases (tile
// sums, one-block scan of the tile sums, tile-local scan plus offset); tiles
// beyond the device count do nothing.
#include "lts_internal.cuh"

namespace lts {

namespace {

constexpr int kT = 256;
constexpr int kPer = 16;
constexpr int kTile = kT * kPer;

__global__ void sums_kernel(const int* __restrict__ in, const int* __restrict__ d_count,
                            unsigned long long* tsum) {
    __shared__ unsigned long long s[kT];
    const int cnt = *d_count;
    const long long base = (long long)blockIdx.x * kTile;
    unsigned long long acc = 0;
    if (base < cnt) {
        for (int i = 0; i < kPer; ++i) {
            const long long k = base + threadIdx.x * kPer + i;
            if (k < cnt) acc += (unsigned)in[k];
        }
    }
    s[threadIdx.x] = acc;
    __syncthreads();
    for (int o = kT / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) s[threadIdx.x] += s[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) tsum[blockIdx.x] = s[0];
}

__global__ void top_kernel(unsigned long long* tsum, int nt) {
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

__global__ void apply_kernel(const int* __restrict__ in, int* __restrict__ out, const int* __restrict__ d_count,
                             const unsigned long long* __restrict__ tsum) {
    __shared__ unsigned long long s[kT];
    const int cnt = *d_count;
    const long long base = (long long)blockIdx.x * kTile;
    if (base > cnt) return;
    unsigned long long acc = 0;
    for (int i = 0; i < kPer; ++i) {
        const long long k = base + threadIdx.x * kPer + i;
        if (k < cnt) acc += (unsigned)in[k];
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
        const long long k = base + threadIdx.x * kPer + i;
        if (k < cnt) { out[k] = (int)run; run += (unsigned)in[k]; }
        else if (k == cnt) out[k] = (int)run;
    }
}

}  // namespace

cudaError_t scan_excl_i32(Work& w, const int* in, int* out, const int* d_count, int max_count, cudaStream_t s) {
    const int nt = (max_count + 1 + kTile - 1) / kTile;
    if (nt > w.scan_tmp_cap) return cudaErrorInvalidValue;
    sums_kernel<<<nt, kT, 0, s>>>(in, d_count, w.scan_tmp);
    top_kernel<<<1, 1024, 0, s>>>(w.scan_tmp, nt);
    apply_kernel<<<nt, kT, 0, s>>>(in, out, d_count, w.scan_tmp);
    w.launches += 3;
    return cudaGetLastError();
}

int scan_tiles_for(long long max_count) { return (int)((max_count + 1 + kTile - 1) / kTile); }

}  // namespace lts
