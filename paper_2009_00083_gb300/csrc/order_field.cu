// Order field (Sec. 4.1): vertices sorted by (f, vertex id); O(v) = rank.
//
// Onesweep LSD radix sort of 32-bit order-preserving keys with the vertex id
// as value: one histogram pass over f (which also copies f into the output
// field g), then four 8-bit digit passes.  Each pass takes tiles in launch
// order from an atomic counter, ranks its keys with warp match-any groups,
// finds its global digit offsets by decoupled look-back over the tiles before
// it (bounded spins), and scatters through shared memory so that every digit
// run is written contiguously.  The last pass does not scatter O[id] = rank
// over the whole array (random 4-byte writes cost a read-modify-write of a
// DRAM sector each): it appends the (id, rank) pairs to bins of 2^22 ids,
// and an inverse pass then writes O bin by bin, so that the random writes of
// one bin stay inside a 16 MB window of O that L2 merges into full sectors.
#include <cstdio>
#include <mutex>

#include "lts_internal.cuh"

namespace lts {

namespace {

constexpr int kThreads = 256;
constexpr int kItems = 16;
constexpr int kTile = kThreads * kItems;   // 4096 keys
constexpr int kWarps = kThreads / 32;
constexpr int kBinShift = 22;
constexpr int kMaxBins = 1 << (31 - kBinShift);

// IEEE order as unsigned order; -0.0 is folded onto +0.0.
__device__ __forceinline__ unsigned order_key(float x, int* st) {
    unsigned u = __float_as_uint(x);
    if ((u & 0x7fffffffu) > 0x7f800000u) set_status(st, LTS_ERR_NAN);
    if (u == 0x80000000u) u = 0u;
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

// Histograms of the four digits; each thread walks 16 consecutive keys and
// flushes a digit count only when the digit changes (runs of equal high
// digits are common in smooth fields, so this avoids contended atomics).
__global__ void __launch_bounds__(kThreads) hist_copy_kernel(const float* __restrict__ f, float* __restrict__ gout,
                                                             int n, unsigned* __restrict__ hist, int* st) {
    __shared__ unsigned sh[4][256];
    for (int i = threadIdx.x; i < 1024; i += blockDim.x) (&sh[0][0])[i] = 0;
    __syncthreads();
    const long long chunk = 16;
    const long long nchunks = (n + chunk - 1) / chunk;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < nchunks;
         c += (long long)gridDim.x * blockDim.x) {
        const long long b = c * chunk;
        unsigned cur[4] = {0xffffffffu, 0xffffffffu, 0xffffffffu, 0xffffffffu};
        unsigned cc[4] = {0, 0, 0, 0};
        const bool vec = ((reinterpret_cast<unsigned long long>(f) | reinterpret_cast<unsigned long long>(gout)) & 15ull) == 0;
        if (vec && b + chunk <= n) {
            const float4* p = reinterpret_cast<const float4*>(f + b);
            float4* q = reinterpret_cast<float4*>(gout + b);
            float v[16];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                float4 t = __ldcs(p + j);
                __stcs(q + j, t);
                v[4 * j] = t.x; v[4 * j + 1] = t.y; v[4 * j + 2] = t.z; v[4 * j + 3] = t.w;
            }
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                unsigned k = order_key(v[j], st);
#pragma unroll
                for (int d = 0; d < 4; ++d) {
                    unsigned dg = (k >> (8 * d)) & 255u;
                    if (dg != cur[d]) {
                        if (cc[d]) atomicAdd(&sh[d][cur[d]], cc[d]);
                        cur[d] = dg; cc[d] = 0;
                    }
                    ++cc[d];
                }
            }
        } else {
            for (long long i = b; i < n; ++i) {
                float x = f[i];
                gout[i] = x;
                unsigned k = order_key(x, st);
                for (int d = 0; d < 4; ++d) {
                    unsigned dg = (k >> (8 * d)) & 255u;
                    if (dg != cur[d]) {
                        if (cc[d]) atomicAdd(&sh[d][cur[d]], cc[d]);
                        cur[d] = dg; cc[d] = 0;
                    }
                    ++cc[d];
                }
            }
        }
#pragma unroll
        for (int d = 0; d < 4; ++d)
            if (cc[d]) atomicAdd(&sh[d][cur[d]], cc[d]);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < 1024; i += blockDim.x) {
        unsigned v = (&sh[0][0])[i];
        if (v) atomicAdd(&hist[i], v);
    }
}

// Exclusive prefix of each digit's histogram: global start of every bucket.
__global__ void digit_offsets_kernel(const unsigned* __restrict__ hist, unsigned* __restrict__ off) {
    const int d = blockIdx.x;          // 4 blocks of 256 threads
    const int t = threadIdx.x;
    __shared__ unsigned s[256];
    s[t] = hist[d * 256 + t];
    __syncthreads();
    for (int o = 1; o < 256; o <<= 1) {
        unsigned v = t >= o ? s[t - o] : 0;
        __syncthreads();
        s[t] += v;
        __syncthreads();
    }
    off[d * 256 + t] = s[t] - hist[d * 256 + t];
}

__device__ __forceinline__ unsigned long long pack_status(unsigned epoch, unsigned flag, unsigned val) {
    return ((unsigned long long)epoch << 34) | ((unsigned long long)flag << 32) | val;
}

// One digit pass.  FIRST: keys come from f and values are the indices.
// LAST: instead of writing the sorted pairs, write O[value] = rank.
template <bool FIRST, bool LAST>
__global__ void __launch_bounds__(kThreads, 4) onesweep_kernel(
    const float* __restrict__ f, const unsigned* __restrict__ kin, const unsigned* __restrict__ vin,
    unsigned* __restrict__ kout, unsigned* __restrict__ vout, unsigned* bin_cursor, int n, int shift,
    const unsigned* __restrict__ goff, unsigned long long* status, unsigned* tile_ctr, unsigned epoch, int* st) {
    __shared__ unsigned s_tile;
    __shared__ unsigned wh[kWarps][256];
    __shared__ unsigned s_gstart[256];
    __shared__ unsigned s_lstart[256];
    __shared__ unsigned s_wsum[kWarps];
    __shared__ unsigned skey[kTile];
    __shared__ unsigned sval[kTile];
    __shared__ unsigned s_bcnt[LAST ? kMaxBins : 1];
    __shared__ unsigned s_bstart[LAST ? kMaxBins : 1];

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) s_tile = atomicAdd(tile_ctr, 1u);
    for (int i = tid; i < kWarps * 256; i += kThreads) (&wh[0][0])[i] = 0;
    __syncthreads();
    const unsigned tile = s_tile;
    const long long base = (long long)tile * kTile + warp * (32 * kItems);

    unsigned key[kItems], val[kItems], rank[kItems];
#pragma unroll
    for (int i = 0; i < kItems; ++i) {
        const long long idx = base + i * 32 + lane;
        if (idx < n) {
            if (FIRST) { key[i] = order_key(__ldg(f + idx), st); val[i] = (unsigned)idx; }
            else { key[i] = __ldcs(kin + idx); val[i] = __ldcs(vin + idx); }
        } else {
            key[i] = 0xffffffffu; val[i] = 0xffffffffu;   // sorts last within the tile, never written
        }
    }
    const unsigned lt = (1u << lane) - 1u;
#pragma unroll
    for (int i = 0; i < kItems; ++i) {
        const unsigned d = (key[i] >> shift) & 255u;
        const unsigned peers = __match_any_sync(0xffffffffu, d);
        const int leader = __ffs(peers) - 1;
        unsigned b = 0;
        if (lane == leader) b = atomicAdd(&wh[warp][d], (unsigned)__popc(peers));
        b = __shfl_sync(0xffffffffu, b, leader);
        rank[i] = b + __popc(peers & lt);
    }
    __syncthreads();
    // per digit: exclusive offsets of the warps, tile count
    const int d = tid;
    unsigned run = 0;
#pragma unroll
    for (int w = 0; w < kWarps; ++w) { unsigned t = wh[w][d]; wh[w][d] = run; run += t; }
    const unsigned cnt = run;
    // publish the aggregate (tile 0 publishes its inclusive prefix right away)
    volatile unsigned long long* vs = status;
    if (tile == 0) vs[d] = pack_status(epoch, 2u, cnt);
    else vs[(long long)tile * 256 + d] = pack_status(epoch, 1u, cnt);
    unsigned excl = 0;
    if (tile > 0) {
        long long t = (long long)tile - 1;
        long long spins = 0;
        while (t >= 0) {
            unsigned long long w = vs[t * 256 + d];
            const unsigned e = (unsigned)(w >> 34), fl = (unsigned)(w >> 32) & 3u;
            if (e != epoch || fl == 0u) {
                if (++spins > kSpinLimit) { set_status(st, LTS_ERR_TIMEOUT); break; }
                continue;
            }
            excl += (unsigned)w;
            if (fl == 2u) break;
            --t;
        }
        __threadfence();
        vs[(long long)tile * 256 + d] = pack_status(epoch, 2u, excl + cnt);
    }
    s_gstart[d] = goff[d] + excl;
    // tile-local start of every digit (block-wide exclusive scan of cnt)
    unsigned x = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        unsigned y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) s_wsum[warp] = x;
    __syncthreads();
    unsigned wpre = 0;
    for (int w = 0; w < warp; ++w) wpre += s_wsum[w];
    s_lstart[d] = wpre + x - cnt;
    __syncthreads();

    if (LAST) {
        // group the tile's (id, rank) pairs by id bin in shared memory
        const int nbins = (int)(((unsigned)n + (1u << kBinShift) - 1) >> kBinShift);
        for (int b = tid; b < nbins; b += kThreads) s_bcnt[b] = 0;
        __syncthreads();
        unsigned lidx[kItems];
#pragma unroll
        for (int i = 0; i < kItems; ++i) {
            // few bins: aggregate per warp before the shared atomic
            const long long idx = base + i * 32 + lane;
            const unsigned bin = idx < n ? (val[i] >> kBinShift) : 0xffffffffu;
            const unsigned peers = __match_any_sync(0xffffffffu, bin);
            const int leader = __ffs(peers) - 1;
            unsigned b = 0;
            if (lane == leader && bin != 0xffffffffu) b = atomicAdd(&s_bcnt[bin], (unsigned)__popc(peers));
            b = __shfl_sync(0xffffffffu, b, leader);
            lidx[i] = b + __popc(peers & lt);
        }
        __syncthreads();
        if (tid == 0) {
            unsigned run = 0;
            for (int b = 0; b < nbins; ++b) { const unsigned c = s_bcnt[b]; s_bstart[b] = run; run += c; }
        }
        __syncthreads();
#pragma unroll
        for (int i = 0; i < kItems; ++i) {
            const long long idx = base + i * 32 + lane;
            if (idx < n) {
                const unsigned dg = (key[i] >> shift) & 255u;
                const unsigned gp = s_gstart[dg] + wh[warp][dg] + rank[i];
                const unsigned lp = s_bstart[val[i] >> kBinShift] + lidx[i];
                sval[lp] = val[i];
                skey[lp] = gp;
            }
        }
        __syncthreads();
        // one atomic per non-empty bin reserves the tile's run in that bin
        for (int b = tid; b < nbins; b += kThreads) {
            const unsigned c = s_bcnt[b];
            s_bcnt[b] = c ? atomicAdd(&bin_cursor[b], c) - s_bstart[b] : 0u;   // global start minus local start
        }
        __syncthreads();
        const long long tb = (long long)tile * kTile;
        const int valid = (int)min((long long)kTile, (long long)n - tb);
        for (int j = tid; j < valid; j += kThreads) {
            const unsigned id = sval[j];
            const unsigned gpos = s_bcnt[id >> kBinShift] + (unsigned)j;
            if (gpos >= (unsigned)n || skey[j] >= (unsigned)n) continue;   // only after a look-back timeout
            __stcs(kout + gpos, id);
            __stcs(vout + gpos, skey[j]);
        }
    } else {
#pragma unroll
        for (int i = 0; i < kItems; ++i) {
            const unsigned dg = (key[i] >> shift) & 255u;
            const unsigned lp = s_lstart[dg] + wh[warp][dg] + rank[i];
            skey[lp] = key[i];
            sval[lp] = val[i];
        }
        __syncthreads();
        const long long tb = (long long)tile * kTile;
        const int valid = (int)min((long long)kTile, (long long)n - tb);
        for (int j = tid; j < valid; j += kThreads) {
            const unsigned k = skey[j];
            const unsigned dg = (k >> shift) & 255u;
            const unsigned gp = s_gstart[dg] + (unsigned)j - s_lstart[dg];
            if (gp >= (unsigned)n) continue;                   // only after a look-back timeout
            __stcs(kout + gp, k);
            __stcs(vout + gp, sval[j]);
        }
    }
}

// bins of 2^kBinShift ids: bin b is filled from position b << kBinShift
__global__ void bin_init_kernel(unsigned* bin_cursor, int nbins) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b < nbins) bin_cursor[b] = (unsigned)b << kBinShift;
}

// O[id] = rank for the binned pairs, walked in bin order
__global__ void __launch_bounds__(256) inverse_kernel(const unsigned* __restrict__ ids, const unsigned* __restrict__ ranks,
                                                      int* __restrict__ O, int n) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += stride) {
        const unsigned id = __ldcs(ids + i);
        if (id < (unsigned)n) O[id] = (int)__ldcs(ranks + i);
    }
}

__global__ void authbits_kernel(const int* __restrict__ ids, long long nids, int n, unsigned* bits, int* st) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nids; i += (long long)gridDim.x * blockDim.x) {
        const int v = ids[i];
        if (v < 0 || v >= n) { set_status(st, LTS_ERR_ARG); continue; }
        atomicOr(&bits[v >> 5], 1u << (v & 31));
    }
}

}  // namespace

cudaError_t order_field(Work& w, const Geom& g, const float* f, float* gout, int* O, cudaStream_t s) {
    const int n = g.n;
    const int tiles = (n + kTile - 1) / kTile;
    int* st = &w.ctr->status;
    cudaMemsetAsync(w.sort_hist, 0, 1024 * sizeof(unsigned), s);
    cudaMemsetAsync(w.tile_counter, 0, 4 * sizeof(unsigned), s);
    {
        long long nch = (n + 15) / 16;
        int blocks = (int)std::min<long long>((nch + kThreads - 1) / kThreads, 152LL * 8);
        hist_copy_kernel<<<blocks, kThreads, 0, s>>>(f, gout, n, w.sort_hist, st);
    }
    digit_offsets_kernel<<<4, 256, 0, s>>>(w.sort_hist, w.sort_offsets);
    const int nbins = (int)(((unsigned)n + (1u << kBinShift) - 1) >> kBinShift);
    bin_init_kernel<<<(nbins + 255) / 256, 256, 0, s>>>(w.bin_cursor, nbins);
    w.launches += 8;
    for (int p = 0; p < 4; ++p) {
        unsigned epoch = ++w.epoch;
        if (w.epoch >= (1u << 30) - 8) {   // epoch wrap: clear the look-back words
            cudaMemsetAsync(w.sort_status, 0, (size_t)w.max_tiles * 256 * sizeof(unsigned long long), s);
            w.epoch = 1;
            epoch = 1;
        }
        const unsigned* goff = w.sort_offsets + 256 * p;
        unsigned* tc = w.tile_counter + p;
        if (p == 0)
            onesweep_kernel<true, false><<<tiles, kThreads, 0, s>>>(f, nullptr, nullptr, w.keyA, w.valA, nullptr, n, 0,
                                                                    goff, w.sort_status, tc, epoch, st);
        else if (p == 1)
            onesweep_kernel<false, false><<<tiles, kThreads, 0, s>>>(nullptr, w.keyA, w.valA, w.keyB, w.valB, nullptr, n,
                                                                     8, goff, w.sort_status, tc, epoch, st);
        else if (p == 2)
            onesweep_kernel<false, false><<<tiles, kThreads, 0, s>>>(nullptr, w.keyB, w.valB, w.keyA, w.valA, nullptr, n,
                                                                     16, goff, w.sort_status, tc, epoch, st);
        else
            onesweep_kernel<false, true><<<tiles, kThreads, 0, s>>>(nullptr, w.keyA, w.valA, w.keyB, w.valB,
                                                                    w.bin_cursor, n, 24, goff, w.sort_status, tc,
                                                                    epoch, st);
    }
    inverse_kernel<<<152 * 8, 256, 0, s>>>(w.keyB, w.valB, O, n);
    return cudaGetLastError();
}

cudaError_t build_authbits(Work& w, const Geom& g, const int* ids, long long nids, cudaStream_t s) {
    const size_t words = ((size_t)g.n + 31) / 32;
    cudaMemsetAsync(w.authbits, 0, words * sizeof(unsigned), s);
    if (nids > 0) {
        int blocks = (int)std::min<long long>((nids + 255) / 256, 1024);
        authbits_kernel<<<blocks, 256, 0, s>>>(ids, nids, g.n, w.authbits, &w.ctr->status);
        w.launches += 1;
    }
    return cudaGetLastError();
}

}  // namespace lts

// ---------------------------------------------------------------------------
// lts_order_field_static: the order field (the kernels above) on a scratch
// buffer that is a static device array of this file, for callers that cannot
// allocate device memory when they call (see include/lts.h).  Nothing here is
// used by lts_simplify.
// ---------------------------------------------------------------------------
namespace {

using lts::kTile;
constexpr long long kStMax = LTS_ORDER_STATIC_MAX_VERTICES;
constexpr int kStTiles = (int)((kStMax + kTile - 1) / kTile);
constexpr size_t kStAlign(size_t b) { return (b + 255) & ~(size_t)255; }
// Scratch layout (byte offsets).  The first kStZero bytes must start at zero
// on every call: the look-back words (epoch 0 = "not yet published"), the
// digit histograms (accumulated by atomics), the tile tickets of the four
// passes and the error word.  Everything after them is fully written before
// it is read.
constexpr size_t kStLook = 0;                                           // u64[tiles * 256]
constexpr size_t kStHist = kStLook + (size_t)kStTiles * 256 * 8;         // u32[4 * 256]
constexpr size_t kStTicket = kStHist + 1024 * 4;                        // u32[4]
constexpr size_t kStErr = kStTicket + 16;                               // int32
constexpr size_t kStZero = kStAlign(kStErr + 4);
constexpr size_t kStOff = kStZero;                                      // u32[4 * 256] digit starts
constexpr size_t kStBin = kStAlign(kStOff + 1024 * 4);                  // u32 bin cursors
constexpr size_t kStKeyA = kStAlign(kStBin + 4 * (((size_t)kStMax >> lts::kBinShift) + 1));
constexpr size_t kStValA = kStKeyA + 4 * (size_t)kStMax;
constexpr size_t kStKeyB = kStValA + 4 * (size_t)kStMax;                // also takes the copy of f
constexpr size_t kStValB = kStKeyB + 4 * (size_t)kStMax;
constexpr size_t kStBytes = kStValB + 4 * (size_t)kStMax;
static_assert(kStMax <= (1LL << lts::kBinShift) * 256, "bin cursors");

constexpr int kStMaxDevices = 256;
std::mutex st_setup_mu;
void* st_base[kStMaxDevices] = {};

lts_status st_fail(char* err, size_t len, lts_status s, const char* msg) {
    if (err && len) std::snprintf(err, len, "%s", msg);
    return s;
}

}  // namespace

// 16.5 MiB at LTS_ORDER_STATIC_MAX_VERTICES = 2^20.  CUDA allocates it once
// per device, when this library's module loads there.
static __device__ __align__(256) unsigned long long lts_order_static_scratch[kStBytes / 8];

extern "C" lts_status lts_order_field_static(int device, const lts_grid* gr, const float* d_field,
                                             int32_t* d_order, void* cuda_stream, char* err, size_t err_len) {
    using namespace lts;
    if (err && err_len) err[0] = '\0';
    if (!gr || (gr->ndim != 2 && gr->ndim != 3) || gr->dims[0] < 2 || gr->dims[1] < 2 ||
        (gr->ndim == 3 && gr->dims[2] < 2) || (gr->ndim == 2 && gr->dims[2] != 1) ||
        gr->dims[0] >= (1LL << 31) || gr->dims[1] >= (1LL << 31) || gr->dims[2] >= (1LL << 31))
        return st_fail(err, err_len, LTS_ERR_ARG, "invalid grid");
    const long long n = gr->dims[0] * gr->dims[1] * gr->dims[2];
    if (n > kStMax) {
        char msg[160];
        std::snprintf(msg, sizeof msg, "grid has %lld vertices; lts_order_field_static takes at most %lld "
                      "(LTS_ORDER_STATIC_MAX_VERTICES): use lts_simplify", n, kStMax);
        return st_fail(err, err_len, LTS_ERR_ARG, msg);
    }
    if (!d_field || !d_order) return st_fail(err, err_len, LTS_ERR_ARG, "null data pointer");
    {
        const char* a = reinterpret_cast<const char*>(d_field);
        const char* b = reinterpret_cast<const char*>(d_order);
        if (a < b + 4 * n && b < a + 4 * n) return st_fail(err, err_len, LTS_ERR_ARG, "d_order overlaps d_field");
    }
    if (device < 0 || device >= kStMaxDevices) return st_fail(err, err_len, LTS_ERR_ARG, "invalid device");
    int prev = -1;
    if (cudaGetDevice(&prev) != cudaSuccess) return st_fail(err, err_len, LTS_ERR_CUDA, "cudaGetDevice failed");
    if (cudaSetDevice(device) != cudaSuccess) return st_fail(err, err_len, LTS_ERR_CUDA, "cudaSetDevice failed");
    struct Restore {
        int d;
        ~Restore() { cudaSetDevice(d); }
    } restore{prev};

    // Set-up, once per device, with that device current: the scratch's
    // device address.  The first call on a device does it.
    char* base;
    {
        std::lock_guard<std::mutex> lock(st_setup_mu);
        if (!st_base[device]) {
            void* p = nullptr;
            const cudaError_t e = cudaGetSymbolAddress(&p, lts_order_static_scratch);
            if (e != cudaSuccess || !p) {
                char msg[160];
                std::snprintf(msg, sizeof msg, "cudaGetSymbolAddress of the static scratch failed: %s",
                              cudaGetErrorString(e));
                return st_fail(err, err_len, LTS_ERR_CUDA, msg);
            }
            st_base[device] = p;
        }
        base = static_cast<char*>(st_base[device]);
    }

    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    unsigned long long* look = reinterpret_cast<unsigned long long*>(base + kStLook);
    unsigned* hist = reinterpret_cast<unsigned*>(base + kStHist);
    unsigned* ticket = reinterpret_cast<unsigned*>(base + kStTicket);
    int* st = reinterpret_cast<int*>(base + kStErr);
    unsigned* goff = reinterpret_cast<unsigned*>(base + kStOff);
    unsigned* bins = reinterpret_cast<unsigned*>(base + kStBin);
    unsigned* keyA = reinterpret_cast<unsigned*>(base + kStKeyA);
    unsigned* valA = reinterpret_cast<unsigned*>(base + kStValA);
    unsigned* keyB = reinterpret_cast<unsigned*>(base + kStKeyB);
    unsigned* valB = reinterpret_cast<unsigned*>(base + kStValB);
    const int ni = (int)n;
    const int tiles = (int)((n + kTile - 1) / kTile);

    cudaMemsetAsync(base, 0, kStZero, s);
    {
        const long long nch = (n + 15) / 16;
        const int blocks = (int)std::min<long long>((nch + kThreads - 1) / kThreads, 152LL * 8);
        hist_copy_kernel<<<blocks, kThreads, 0, s>>>(d_field, reinterpret_cast<float*>(keyB), ni, hist, st);
    }
    digit_offsets_kernel<<<4, 256, 0, s>>>(hist, goff);
    const int nbins = (int)(((unsigned)ni + (1u << kBinShift) - 1) >> kBinShift);
    bin_init_kernel<<<(nbins + 255) / 256, 256, 0, s>>>(bins, nbins);
    // the look-back words were zeroed above, so the passes take epochs 1..4
    onesweep_kernel<true, false><<<tiles, kThreads, 0, s>>>(d_field, nullptr, nullptr, keyA, valA, nullptr, ni, 0,
                                                            goff, look, ticket, 1u, st);
    onesweep_kernel<false, false><<<tiles, kThreads, 0, s>>>(nullptr, keyA, valA, keyB, valB, nullptr, ni, 8,
                                                             goff + 256, look, ticket + 1, 2u, st);
    onesweep_kernel<false, false><<<tiles, kThreads, 0, s>>>(nullptr, keyB, valB, keyA, valA, nullptr, ni, 16,
                                                             goff + 512, look, ticket + 2, 3u, st);
    onesweep_kernel<false, true><<<tiles, kThreads, 0, s>>>(nullptr, keyA, valA, keyB, valB, bins, ni, 24,
                                                            goff + 768, look, ticket + 3, 4u, st);
    inverse_kernel<<<152 * 8, 256, 0, s>>>(keyB, valB, d_order, ni);
    cudaError_t e = cudaGetLastError();
    int h_status = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h_status, st, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        char msg[160];
        std::snprintf(msg, sizeof msg, "CUDA error: %s", cudaGetErrorString(e));
        return st_fail(err, err_len, LTS_ERR_CUDA, msg);
    }
    if (h_status == LTS_ERR_NAN) return st_fail(err, err_len, LTS_ERR_NAN, "the field holds a NaN");
    if (h_status == LTS_ERR_TIMEOUT) return st_fail(err, err_len, LTS_ERR_TIMEOUT, "a sort look-back wait expired");
    if (h_status != 0) return st_fail(err, err_len, LTS_ERR_INTERNAL, "unexpected device status");
    return LTS_OK;
}
