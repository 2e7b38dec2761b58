// Order field (Sec. 4.1): vertices sorted by (f, vertex id); O(v) = rank.
//
// Onesweep LSD radix sort of 32-bit order-preserving keys with the vertex id
// as value: one histogram pass over f (which also copies f into the output
// field g), then four 8-bit digit passes (two on compressed keys, below).
// Each pass takes tiles in launch order from an atomic counter, ranks its keys
// with warp match-any groups (ballots in the first pass),
// finds its global digit offsets by decoupled look-back over the tiles before
// it (bounded spins), and scatters through shared memory so that every digit
// run is written contiguously.  The last pass does not scatter O[id] = rank
// over the whole array (random 4-byte writes cost a read-modify-write of a
// DRAM sector each): it appends the (id, rank) pairs to bins of 2^22 ids,
// and an inverse pass then writes O bin by bin, so that the random writes of
// one bin stay inside a 16 MB window of O that L2 merges into full sectors.
//
// Few distinct values (quantized fields; heavy ties): the histogram pass also
// collects the distinct keys with their counts in a hash table (per block in
// shared memory, then globally).  If there are at most kDkMax of them, one
// small kernel replaces every key by its rank among the distinct keys (an
// order-preserving compression to 12 bits) and derives the two digit
// histograms of the compressed keys from the counts; the sort then takes two
// digit passes instead of four (the first pass looks the compressed key up,
// the second is the last).  Ties keep their id order: the passes are stable
// whatever the keys.  The choice is made on the device: the passes of the
// other path are launched too and return at once.
#include <cstdio>
#include <mutex>
#include <utility>

#include <cstdlib>

#include "lts_internal.cuh"

namespace lts {

namespace {

constexpr int kThreads = 256;
constexpr int kItems = 16;
constexpr int kTile = kThreads * kItems;   // 4096 keys
constexpr int kWarps = kThreads / 32;
constexpr int kBinShift = 22;
constexpr int kMaxBins = 1 << (31 - kBinShift);
constexpr int kDkMax = 4096;             // distinct keys for the two-pass sort (12-bit compressed keys)
constexpr int kDkSlots = 2 * kDkMax;     // global hash table slots
constexpr int kDkLocal = 1024;           // per-block hash table slots
constexpr int kDkProbe = 8;              // local probes before a key goes to the global table
constexpr unsigned kDkEmpty = 0xffffffffu;   // no order key has this value (it is a NaN pattern)

// dk_info words
constexpr int kDkCount = 0;              // distinct keys inserted in the global table
constexpr int kDkOverflow = 1;           // more than kDkMax distinct keys (or a probe limit hit)
constexpr int kDkMode = 2;               // 1: the compressed two-pass sort runs

__device__ __forceinline__ unsigned dk_hash(unsigned k) { return (k * 0x9E3779B1u) >> 19; }   // 13 bits

// Adds cnt occurrences of key to the global table (bounded probing).
// Returns false once there are too many distinct keys: collecting stops.
__device__ bool dk_insert_global(unsigned* keys, unsigned* cnts, unsigned* info, unsigned key, unsigned cnt) {
    unsigned h = dk_hash(key) & (kDkSlots - 1);
    for (int p = 0; p < kDkSlots; ++p) {
        if (*(volatile unsigned*)(info + kDkOverflow)) return false;
        unsigned cur = *(volatile unsigned*)(keys + h);
        if (cur == kDkEmpty) {
            if (*(volatile unsigned*)(info + kDkCount) >= (unsigned)kDkMax) {
                atomicExch(info + kDkOverflow, 1u);
                return false;
            }
            cur = atomicCAS(keys + h, kDkEmpty, key);
            if (cur == kDkEmpty) {
                atomicAdd(cnts + h, cnt);
                if (atomicAdd(info + kDkCount, 1u) + 1u > (unsigned)kDkMax) {
                    atomicExch(info + kDkOverflow, 1u);
                    return false;
                }
                return true;
            }
        }
        if (cur == key) {
            atomicAdd(cnts + h, cnt);
            return true;
        }
        h = (h + 1) & (kDkSlots - 1);
    }
    atomicExch(info + kDkOverflow, 1u);
    return false;
}

// Adds cnt occurrences of key to the block's table; false if it did not fit
// in kDkProbe probes.  At three quarters full the table takes no new keys
// (*full), so that a block with many distinct keys does not probe a full one.
__device__ bool dk_insert_local(unsigned* lk, unsigned* lc, int* count, int* full, unsigned key, unsigned cnt) {
    if (*(volatile int*)full) {
        // only keys already present
        unsigned h = dk_hash(key) & (kDkLocal - 1);
        for (int p = 0; p < kDkProbe; ++p) {
            const unsigned cur = *(volatile unsigned*)(lk + h);
            if (cur == key) { atomicAdd(lc + h, cnt); return true; }
            if (cur == kDkEmpty) return false;
            h = (h + 1) & (kDkLocal - 1);
        }
        return false;
    }
    unsigned h = dk_hash(key) & (kDkLocal - 1);
    for (int p = 0; p < kDkProbe; ++p) {
        unsigned cur = *(volatile unsigned*)(lk + h);
        bool mine = false;
        if (cur == kDkEmpty) {
            cur = atomicCAS(lk + h, kDkEmpty, key);
            mine = cur == kDkEmpty;
        }
        if (mine || cur == key) {
            atomicAdd(lc + h, cnt);
            if (mine && atomicAdd(count, 1) + 1 >= kDkLocal * 3 / 4) *(volatile int*)full = 1;
            return true;
        }
        h = (h + 1) & (kDkLocal - 1);
    }
    return false;
}

// The compressed key of an order key present in the global table.
__device__ __forceinline__ unsigned dk_lookup(const unsigned* __restrict__ keys, const unsigned* __restrict__ rank,
                                              unsigned key, int* st) {
    unsigned h = dk_hash(key) & (kDkSlots - 1);
    for (int p = 0; p < kDkSlots; ++p) {
        const unsigned cur = __ldg(keys + h);
        if (cur == key) return __ldg(rank + h);
        if (cur == kDkEmpty) break;
        h = (h + 1) & (kDkSlots - 1);
    }
    set_status(st, LTS_ERR_INTERNAL);
    return 0;
}

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
// With dk_keys set, also collects the distinct keys and their counts: runs
// of equal keys within a thread's 16 are counted once, the block's table takes
// them, and the table is added to the global one at the end.
__global__ void __launch_bounds__(kThreads) hist_copy_kernel(const float* __restrict__ f, float* __restrict__ gout,
                                                             int n, unsigned* __restrict__ hist, int* st,
                                                             unsigned* dk_keys, unsigned* dk_cnts, unsigned* dk_info) {
    __shared__ unsigned sh[4][256];
    __shared__ unsigned lk[kDkLocal], lc[kDkLocal];
    __shared__ int s_lcount, s_lfull;
    for (int i = threadIdx.x; i < 1024; i += blockDim.x) (&sh[0][0])[i] = 0;
    for (int i = threadIdx.x; i < kDkLocal; i += blockDim.x) { lk[i] = kDkEmpty; lc[i] = 0; }
    if (threadIdx.x == 0) { s_lcount = 0; s_lfull = 0; }
    __syncthreads();
    unsigned run_key = kDkEmpty, run_cnt = 0;
    bool dk_on = dk_keys != nullptr;       // this thread still collects
    auto dk_flush = [&]() {
        if (run_cnt && !dk_insert_local(lk, lc, &s_lcount, &s_lfull, run_key, run_cnt) &&
            !dk_insert_global(dk_keys, dk_cnts, dk_info, run_key, run_cnt))
            dk_on = false;
        run_cnt = 0;
    };
    auto dk_add = [&](unsigned k) {
        if (k == run_key) { ++run_cnt; return; }
        dk_flush();
        run_key = k;
        run_cnt = 1;
    };
    const long long chunk = 16;
    const long long nchunks = (n + chunk - 1) / chunk;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < nchunks;
         c += (long long)gridDim.x * blockDim.x) {
        const long long b = c * chunk;
        unsigned cur[4] = {0xffffffffu, 0xffffffffu, 0xffffffffu, 0xffffffffu};
        unsigned cc[4] = {0, 0, 0, 0};
        const bool vec = ((reinterpret_cast<unsigned long long>(f) | reinterpret_cast<unsigned long long>(gout)) & 15ull) == 0;
        if (dk_on && *(volatile unsigned*)(dk_info + kDkOverflow)) dk_on = false;
        const bool dk = dk_on;
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
                if (dk) dk_add(k);
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
            const long long e = b + chunk < n ? b + chunk : (long long)n;
            for (long long i = b; i < e; ++i) {
                float x = f[i];
                gout[i] = x;
                unsigned k = order_key(x, st);
                if (dk) dk_add(k);
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
    if (dk_on) dk_flush();
    __syncthreads();
    for (int i = threadIdx.x; i < 1024; i += blockDim.x) {
        unsigned v = (&sh[0][0])[i];
        if (v) atomicAdd(&hist[i], v);
    }
    if (dk_keys && !*(volatile unsigned*)(dk_info + kDkOverflow))
        for (int i = threadIdx.x; i < kDkLocal; i += blockDim.x)
            if (lk[i] != kDkEmpty && !dk_insert_global(dk_keys, dk_cnts, dk_info, lk[i], lc[i])) break;
}

// Ranks the distinct keys (if there are at most kDkMax) and replaces the
// histograms of digits 0 and 1 by those of the compressed keys.  One block.
__global__ void __launch_bounds__(1024) dense_keys_kernel(const unsigned* __restrict__ dk_keys,
                                                          const unsigned* __restrict__ dk_cnts, unsigned* dk_rank,
                                                          unsigned* dk_info, unsigned* hist, const int* st) {
    __shared__ unsigned s_key[kDkMax];
    __shared__ unsigned short s_slot[kDkMax];
    __shared__ unsigned s_h[2][256];
    __shared__ int s_n;
    if (dk_info[kDkOverflow] || failed(st)) {
        if (threadIdx.x == 0) dk_info[kDkMode] = 0;
        return;
    }
    if (threadIdx.x == 0) s_n = 0;
    for (int i = threadIdx.x; i < 512; i += blockDim.x) (&s_h[0][0])[i] = 0;
    __syncthreads();
    for (int i = threadIdx.x; i < kDkSlots; i += blockDim.x) {
        const unsigned k = dk_keys[i];
        if (k == kDkEmpty) continue;
        const int at = atomicAdd(&s_n, 1);
        if (at < kDkMax) { s_key[at] = k; s_slot[at] = (unsigned short)i; }
    }
    __syncthreads();
    const int D = s_n;
    if (D > kDkMax) {                                // cannot happen without the overflow flag
        if (threadIdx.x == 0) dk_info[kDkMode] = 0;
        return;
    }
    for (int i = threadIdx.x; i < D; i += blockDim.x) {
        const unsigned k = s_key[i];
        unsigned r = 0;
        for (int j = 0; j < D; ++j) r += s_key[j] < k;
        dk_rank[s_slot[i]] = r;
        const unsigned c = dk_cnts[s_slot[i]];
        atomicAdd(&s_h[0][r & 255u], c);
        atomicAdd(&s_h[1][r >> 8], c);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < 512; i += blockDim.x) hist[i] = (&s_h[0][0])[i];
    if (threadIdx.x == 0) dk_info[kDkMode] = 1;
}

// float64 fields: IEEE order as unsigned 64-bit order; -0.0 is folded onto +0.0.
__device__ __forceinline__ unsigned long long order_key64(double x, int* st) {
    unsigned long long u = (unsigned long long)__double_as_longlong(x);
    if ((u & 0x7fffffffffffffffull) > 0x7ff0000000000000ull) set_status(st, LTS_ERR_NAN);
    if (u == 0x8000000000000000ull) u = 0ull;
    return (u & 0x8000000000000000ull) ? ~u : (u | 0x8000000000000000ull);
}

// float64 fields: copies f to g, writes (low word of the key, id) as the
// first sort's pairs and the high word of the key by id, and counts the
// eight byte digits of the key (low word: digits 0-3, high word: 4-7).
__global__ void __launch_bounds__(kThreads) hist64_kernel(const double* __restrict__ f, double* __restrict__ gout,
                                                          int n, unsigned* __restrict__ keys, unsigned* __restrict__ vals,
                                                          unsigned* __restrict__ hi, unsigned* __restrict__ hist,
                                                          int* st) {
    __shared__ unsigned sh[8][256];
    for (int i = threadIdx.x; i < 2048; i += blockDim.x) (&sh[0][0])[i] = 0;
    __syncthreads();
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const double x = __ldcs(f + i);
        __stcs(gout + i, x);
        const unsigned long long k = order_key64(x, st);
        const unsigned lo = (unsigned)k, h = (unsigned)(k >> 32);
        __stcs(keys + i, lo);
        __stcs(vals + i, (unsigned)i);
        __stcs(hi + i, h);
#pragma unroll
        for (int d = 0; d < 4; ++d) {
            atomicAdd(&sh[d][(lo >> (8 * d)) & 255u], 1u);
            atomicAdd(&sh[4 + d][(h >> (8 * d)) & 255u], 1u);
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < 2048; i += blockDim.x) {
        const unsigned v = (&sh[0][0])[i];
        if (v) atomicAdd(&hist[i], v);
    }
}

// keys[i] = hi[vals[i]]: the high words in the order of the sort by low words.
__global__ void gather_hi_kernel(const unsigned* __restrict__ vals, const unsigned* __restrict__ hi,
                                 unsigned* __restrict__ keys, int n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        keys[i] = __ldg(hi + __ldcs(vals + i));
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

// Which sort a pass belongs to (read from dk_info on the device).
constexpr int kRoleAlways = 0, kRoleFourPass = 1, kRoleTwoPass = 2;

// One digit pass.  FIRST: keys come from f (compressed when the two-pass
// sort runs) and values are the indices.  LAST: instead of writing the sorted
// pairs, write (id, rank) pairs binned by id for the inverse pass.  A pass
// of the sort that does not run returns at once.
template <bool FIRST, bool LAST>
__global__ void __launch_bounds__(kThreads, 4) onesweep_kernel(
    const float* __restrict__ f, const unsigned* __restrict__ kin, const unsigned* __restrict__ vin,
    unsigned* __restrict__ kout, unsigned* __restrict__ vout, unsigned* bin_cursor, int n, int shift,
    const unsigned* __restrict__ goff, unsigned long long* status, unsigned* tile_ctr, unsigned epoch, int* st,
    const unsigned* __restrict__ dk_keys, const unsigned* __restrict__ dk_rank, const unsigned* dk_info, int role,
    const unsigned long long* stall = nullptr) {
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
    const bool two_pass = dk_info != nullptr && dk_info[kDkMode] == 1u;
    if ((role == kRoleFourPass && two_pass) || (role == kRoleTwoPass && !two_pass)) return;
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
            if (FIRST) {
                key[i] = order_key(__ldg(f + idx), st);
                if (two_pass) key[i] = dk_lookup(dk_keys, dk_rank, key[i], st);
                val[i] = (unsigned)idx;
            }
            else { key[i] = __ldcs(kin + idx); val[i] = __ldcs(vin + idx); }
        } else {
            key[i] = 0xffffffffu; val[i] = 0xffffffffu;   // sorts last within the tile, never written
        }
    }
    const unsigned lt = (1u << lane) - 1u;
#pragma unroll
    for (int i = 0; i < kItems; ++i) {
        const unsigned d = (key[i] >> shift) & 255u;
        // lanes with the same digit: in the first pass the keys come in vertex
        // order, where a smooth field gives long runs of equal digits, and
        // eight ballots beat the match instruction there (measured); later
        // passes use the match instruction
        unsigned peers;
        if (FIRST) {
            peers = 0xffffffffu;
#pragma unroll
            for (int bt = 0; bt < 8; ++bt) {
                const bool on = (d >> bt) & 1u;
                const unsigned bb = __ballot_sync(0xffffffffu, on);
                peers &= on ? bb : ~bb;
            }
        } else {
            peers = __match_any_sync(0xffffffffu, d);
        }
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
        // tests only: with `stall`, tile 1 waits on words that nothing sets, with a short limit
        const bool stalled = stall != nullptr && tile == 1;
        const long long limit = stalled ? kTestSpinLimit : kSpinLimit;
        while (t >= 0) {
            unsigned long long w = stalled ? *(volatile const unsigned long long*)(stall + d) : vs[t * 256 + d];
            const unsigned e = (unsigned)(w >> 34), fl = (unsigned)(w >> 32) & 3u;
            if (e != epoch || fl == 0u) {
                if (++spins > limit) { set_status(st, LTS_ERR_TIMEOUT); break; }
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
    cudaMemsetAsync(w.tile_counter, 0, 8 * sizeof(unsigned), s);
    cudaMemsetAsync(w.dk_keys, 0xff, kDkSlots * sizeof(unsigned), s);
    cudaMemsetAsync(w.dk_cnts, 0, kDkSlots * sizeof(unsigned), s);
    cudaMemsetAsync(w.dk_info, 0, 4 * sizeof(unsigned), s);
    {
        long long nch = (n + 15) / 16;
        int blocks = (int)std::min<long long>((nch + kThreads - 1) / kThreads, (long long)w.sms * 8);
        hist_copy_kernel<<<blocks, kThreads, 0, s>>>(f, gout, n, w.sort_hist, st, w.dk_keys, w.dk_cnts, w.dk_info);
    }
    dense_keys_kernel<<<1, 1024, 0, s>>>(w.dk_keys, w.dk_cnts, w.dk_rank, w.dk_info, w.sort_hist, st);
    digit_offsets_kernel<<<4, 256, 0, s>>>(w.sort_hist, w.sort_offsets);
    const int nbins = (int)(((unsigned)n + (1u << kBinShift) - 1) >> kBinShift);
    bin_init_kernel<<<(nbins + 255) / 256, 256, 0, s>>>(w.bin_cursor, nbins);
    w.launches += 10;
    unsigned ep[4];
    for (int p = 0; p < 4; ++p) {
        ep[p] = ++w.epoch;
        if (w.epoch >= (1u << 30) - 8) {   // epoch wrap: clear the look-back words
            cudaMemsetAsync(w.sort_status, 0, (size_t)w.max_tiles * 256 * sizeof(unsigned long long), s);
            w.epoch = 1;
            ep[p] = 1;
        }
    }
    const unsigned* dkk = w.dk_keys;
    const unsigned* dkr = w.dk_rank;
    const unsigned* dki = w.dk_info;
    // tests only: while LTS_TEST_STALL_SORT is set, tile 1 of the first digit
    // pass waits on look-back words that nothing sets, so that its bounded wait
    // expires (LTS_ERR_TIMEOUT) without any fault
    const char* stall_env = getenv("LTS_TEST_STALL_SORT");
    const unsigned long long* stall =
        (stall_env && stall_env[0] && stall_env[0] != '0') ? w.test_stall : nullptr;
    // digit 0 (both sorts); digit 1: middle pass of the four-pass sort, last
    // pass of the two-pass sort (both write the binned pairs to B); digits 2, 3
    onesweep_kernel<true, false><<<tiles, kThreads, 0, s>>>(f, nullptr, nullptr, w.keyA, w.valA, nullptr, n, 0,
                                                            w.sort_offsets, w.sort_status, w.tile_counter + 0, ep[0],
                                                            st, dkk, dkr, dki, kRoleAlways, stall);
    onesweep_kernel<false, false><<<tiles, kThreads, 0, s>>>(nullptr, w.keyA, w.valA, w.keyB, w.valB, nullptr, n, 8,
                                                             w.sort_offsets + 256, w.sort_status, w.tile_counter + 1,
                                                             ep[1], st, dkk, dkr, dki, kRoleFourPass);
    onesweep_kernel<false, true><<<tiles, kThreads, 0, s>>>(nullptr, w.keyA, w.valA, w.keyB, w.valB, w.bin_cursor, n,
                                                            8, w.sort_offsets + 256, w.sort_status,
                                                            w.tile_counter + 4, ep[1], st, dkk, dkr, dki,
                                                            kRoleTwoPass);
    onesweep_kernel<false, false><<<tiles, kThreads, 0, s>>>(nullptr, w.keyB, w.valB, w.keyA, w.valA, nullptr, n, 16,
                                                             w.sort_offsets + 512, w.sort_status, w.tile_counter + 2,
                                                             ep[2], st, dkk, dkr, dki, kRoleFourPass);
    onesweep_kernel<false, true><<<tiles, kThreads, 0, s>>>(nullptr, w.keyA, w.valA, w.keyB, w.valB, w.bin_cursor, n,
                                                            24, w.sort_offsets + 768, w.sort_status,
                                                            w.tile_counter + 3, ep[3], st, dkk, dkr, dki,
                                                            kRoleFourPass);
    inverse_kernel<<<w.sms * 8, 256, 0, s>>>(w.keyB, w.valB, O, n);
    return cudaGetLastError();
}

// The order field of a float64 field: an LSD radix sort of the 64-bit order
// keys with the vertex ids, as two stable 32-bit sorts (four 8-bit digit
// passes each): first by the low words, then, after the high words are
// gathered in that order, by the high words; ties keep the id order.  The
// last pass bins (id, rank) pairs like the float32 sort.  The high words are
// kept in the member-region array, unused until the passes.
cudaError_t order_field_f64(Work& w, const Geom& g, const double* f, double* gout, int* O, cudaStream_t s) {
    const int n = g.n;
    const int tiles = (n + kTile - 1) / kTile;
    int* st = &w.ctr->status;
    unsigned* hi = reinterpret_cast<unsigned*>(w.member_reg);
    cudaMemsetAsync(w.sort_hist, 0, 2048 * sizeof(unsigned), s);
    cudaMemsetAsync(w.tile_counter, 0, 8 * sizeof(unsigned), s);
    {
        const int blocks = (int)std::min<long long>(((long long)n + kThreads - 1) / kThreads, (long long)w.sms * 8);
        hist64_kernel<<<blocks, kThreads, 0, s>>>(f, gout, n, w.keyA, w.valA, hi, w.sort_hist, st);
    }
    digit_offsets_kernel<<<8, 256, 0, s>>>(w.sort_hist, w.sort_offsets);
    const int nbins = (int)(((unsigned)n + (1u << kBinShift) - 1) >> kBinShift);
    bin_init_kernel<<<(nbins + 255) / 256, 256, 0, s>>>(w.bin_cursor, nbins);
    w.launches += 3;
    unsigned ep[8];
    for (int p = 0; p < 8; ++p) {
        ep[p] = ++w.epoch;
        if (w.epoch >= (1u << 30) - 8) {   // epoch wrap: clear the look-back words
            cudaMemsetAsync(w.sort_status, 0, (size_t)w.max_tiles * 256 * sizeof(unsigned long long), s);
            w.epoch = 1;
            ep[p] = 1;
        }
    }
    unsigned* ka = w.keyA; unsigned* va = w.valA; unsigned* kb = w.keyB; unsigned* vb = w.valB;
    for (int p = 0; p < 8; ++p) {
        if (p == 4) {
            // the low words are sorted (pairs in A): sort on the high words next
            gather_hi_kernel<<<w.sms * 8, 256, 0, s>>>(va, hi, ka, n);
            w.launches += 1;
        }
        const int shift = 8 * (p & 3);
        if (p < 7)
            onesweep_kernel<false, false><<<tiles, kThreads, 0, s>>>(nullptr, ka, va, kb, vb, nullptr, n, shift,
                                                                     w.sort_offsets + 256 * p, w.sort_status,
                                                                     w.tile_counter + p, ep[p], st, nullptr, nullptr,
                                                                     nullptr, kRoleAlways);
        else
            onesweep_kernel<false, true><<<tiles, kThreads, 0, s>>>(nullptr, ka, va, kb, vb, w.bin_cursor, n, shift,
                                                                    w.sort_offsets + 256 * p, w.sort_status,
                                                                    w.tile_counter + p, ep[p], st, nullptr, nullptr,
                                                                    nullptr, kRoleAlways);
        std::swap(ka, kb);
        std::swap(va, vb);
    }
    w.launches += 8;
    // after eight passes the binned (id, rank) pairs are in A again (ka, va)
    inverse_kernel<<<w.sms * 8, 256, 0, s>>>(ka, va, O, n);
    w.launches += 1;
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

    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess || sms <= 0)
        return st_fail(err, err_len, LTS_ERR_CUDA, "cannot read the device's multiprocessor count");
    cudaMemsetAsync(base, 0, kStZero, s);
    {
        const long long nch = (n + 15) / 16;
        const int blocks = (int)std::min<long long>((nch + kThreads - 1) / kThreads, (long long)sms * 8);
        hist_copy_kernel<<<blocks, kThreads, 0, s>>>(d_field, reinterpret_cast<float*>(keyB), ni, hist, st, nullptr,
                                                     nullptr, nullptr);
    }
    digit_offsets_kernel<<<4, 256, 0, s>>>(hist, goff);
    const int nbins = (int)(((unsigned)ni + (1u << kBinShift) - 1) >> kBinShift);
    bin_init_kernel<<<(nbins + 255) / 256, 256, 0, s>>>(bins, nbins);
    // the look-back words were zeroed above, so the passes take epochs 1..4
    onesweep_kernel<true, false><<<tiles, kThreads, 0, s>>>(d_field, nullptr, nullptr, keyA, valA, nullptr, ni, 0,
                                                            goff, look, ticket, 1u, st, nullptr, nullptr, nullptr,
                                                            kRoleAlways);
    onesweep_kernel<false, false><<<tiles, kThreads, 0, s>>>(nullptr, keyA, valA, keyB, valB, nullptr, ni, 8,
                                                             goff + 256, look, ticket + 1, 2u, st, nullptr, nullptr,
                                                             nullptr, kRoleAlways);
    onesweep_kernel<false, false><<<tiles, kThreads, 0, s>>>(nullptr, keyB, valB, keyA, valA, nullptr, ni, 16,
                                                             goff + 512, look, ticket + 2, 3u, st, nullptr, nullptr,
                                                             nullptr, kRoleAlways);
    onesweep_kernel<false, true><<<tiles, kThreads, 0, s>>>(nullptr, keyA, valA, keyB, valB, bins, ni, 24,
                                                            goff + 768, look, ticket + 3, 4u, st, nullptr, nullptr,
                                                            nullptr, kRoleAlways);
    inverse_kernel<<<sms * 8, 256, 0, s>>>(keyB, valB, d_order, ni);
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
