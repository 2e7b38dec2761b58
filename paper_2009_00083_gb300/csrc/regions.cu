// Regions after step 1 (Sec. 4.3: one region per hill chain).
//
// Every class still waiting when the propagation kernel ends is a region:
// its saddle is where it waits and its members are the vertices it (or the
// classes it absorbed) claimed, apart from final saddles.  Regions get dense
// ids, member lists (CSR), their highest member's order (to order regions
// that share a saddle, the reading that makes Eq. 6 a total order), and, per
// saddle, the offset of each sibling block and the block total.
#include "lts_internal.cuh"

namespace lts {

namespace {

__device__ __forceinline__ int warp_reserve(int* counter, bool want) {
    const int lane = threadIdx.x & 31;
    const unsigned m = __ballot_sync(0xffffffffu, want);
    int b = 0;
    if (lane == 0 && m) b = atomicAdd(counter, __popc(m));
    b = __shfl_sync(0xffffffffu, b, 0);
    return b + __popc(m & ((1u << lane) - 1u));
}

// flatten the class forest: parent[c] = root
__global__ void flatten_kernel(int* parent, const DevCounters* ctr) {
    if (failed(&ctr->status)) return;
    const int nU = ctr->n_unauth;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < nU; c += gridDim.x * blockDim.x) {
        int r = c;
        while (parent[r] != r) r = parent[r];
        parent[c] = r;
    }
}

// Every root class is a region waiting at its saddle.  The siblings at a
// saddle are listed under the class that claimed it (sib_head, sib_next).
template <int DIR>
__global__ void roots_kernel(Geom g, const int* __restrict__ O, const int* __restrict__ parent,
                             const int* __restrict__ wait_v, const int* __restrict__ owner, int* sib_head,
                             int* sib_next, int* class2reg,
                             int* reg_class, int* reg_saddle, int* reg_size, int* reg_top, int* reg_sod, int* reg_head,
                             DevCounters* ctr) {
    if (failed(&ctr->status)) return;
    const int nU = ctr->n_unauth;
    for (long long b = (long long)blockIdx.x * blockDim.x; b < nU; b += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(b + threadIdx.x);
        const bool root = c < nU && parent[c] == c;
        const int rid = warp_reserve(&ctr->n_regions, root);
        if (c >= nU) continue;
        if (!root) { class2reg[c] = -1; continue; }
        const int sv = wait_v[c];
        if (sv < 0) { set_status(&ctr->status, LTS_ERR_INTERNAL); class2reg[c] = -1; continue; }
        class2reg[c] = rid;
        reg_class[rid] = c;
        reg_saddle[rid] = sv;
        reg_size[rid] = 0;
        reg_top[rid] = -1;
        reg_sod[rid] = od<DIR>(O[sv], g.n);
        const int hc = owner[sv];                     // the class that claimed the saddle waits there too
        reg_head[rid] = hc == c;
        if (hc < 0) set_status(&ctr->status, LTS_ERR_INTERNAL);
        else if (hc != c) sib_next[c] = atomicExch(sib_head + hc, c);
    }
}

// every class: the region of its root (the forest is flat), -1 if none
__global__ void cls_rid_kernel(const int* __restrict__ parent, const int* __restrict__ class2reg, int* cls2rid,
                               const DevCounters* ctr) {
    if (failed(&ctr->status)) return;
    const int nU = ctr->n_unauth;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < nU; c += gridDim.x * blockDim.x)
        cls2rid[c] = class2reg[parent[c]];
}

// One thread per log entry (a claimed vertex u with the class that claimed
// it): the region of u, its local index (counted), the region's highest
// member, and u's region tag and local index.  The entry's region, local
// index and Od are kept for members_fill_kernel, which then reads nothing at
// random.  A region's final saddle is not a member (entry region -1).
template <int DIR>
__global__ void members_count_kernel(Geom g, const int* __restrict__ O, const int* __restrict__ vlog,
                                     const int* __restrict__ vlog_cls, const int* __restrict__ cls2rid, int* owner,
                                     int* loc, const int* __restrict__ reg_saddle, int* reg_size, int* reg_top,
                                     int* ent_rid, int* ent_loc, int* ent_od, DevCounters* ctr) {
    if (failed(&ctr->status)) return;
    const int nlog = ctr->log_cursor;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nlog; i += gridDim.x * blockDim.x) {
        const int u = vlog[i];
        int rid = -1;
        if (u >= 0) {
            rid = __ldg(cls2rid + vlog_cls[i]);
            if (rid < 0) set_status(&ctr->status, LTS_ERR_INTERNAL);
            else if (__ldg(reg_saddle + rid) == u) rid = -1;    // a final saddle, not a member
        }
        ent_rid[i] = rid;
        if (rid < 0) continue;
        const int l = atomicAdd(reg_size + rid, 1);
        const int o = od<DIR>(__ldg(O + u), g.n);
        atomicMax(reg_top + rid, o);
        loc[u] = l;
        owner[u] = -2 - rid;                                    // region tag
        ent_loc[i] = l;
        ent_od[i] = o;
    }
}

__global__ void members_fill_kernel(const int* __restrict__ vlog, const int* __restrict__ ent_rid,
                                    const int* __restrict__ ent_loc, const int* __restrict__ ent_od,
                                    const int* __restrict__ reg_start, int* members, int* member_reg, RankBlk* rblk,
                                    DevCounters* ctr) {
    if (failed(&ctr->status)) return;
    const int nlog = ctr->log_cursor;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nlog; i += gridDim.x * blockDim.x) {
        const int rid = ent_rid[i];
        if (rid < 0) continue;
        const int p = __ldg(reg_start + rid) + ent_loc[i];
        members[p] = vlog[i];
        member_reg[p] = rid;
        const int j = ent_od[i];
        atomicOr(&rblk[j >> kRankShift].mmask, 1u << (j & 31));
    }
}

// Step-2 tier lists by region size r = members + 1.  A region with a single
// member m needs no work: m is the only candidate for the minus-infinity
// vertex (it has neighbours outside R), the propagation from s visits it
// last, and no vertex lacks an outside neighbour, so lhat(m) = 0 after one
// propagation.
// min_tier > 0 (tests only) moves regions up to tier min_tier (0: 16 lanes,
// 1: 32 lanes, 2: dense <= 128, 3: dense <= med_max, 4: dense <= huge_max,
// 5: HBM) while its list has room, so that every tier runs on small regions.
__global__ void tiers_kernel(const int* __restrict__ reg_size, const int* __restrict__ reg_start, int* lhat,
                             int* tier_list, int cap, int q, int med_max, int huge_max, int min_tier, int nverts,
                             DevCounters* ctr) {
    if (failed(&ctr->status)) return;
    const int nreg = ctr->n_regions;
    int trivial = 0;
    for (long long b = (long long)blockIdx.x * blockDim.x; b < nreg; b += (long long)gridDim.x * blockDim.x) {
        const int r = (int)(b + threadIdx.x);
        const int sz = r < nreg ? reg_size[r] + 1 : 0;
        if (sz == 2) { lhat[reg_start[r]] = 0; ++trivial; }
        int tier = sz <= 2 ? -1 : sz <= 16 ? 0 : sz <= 32 ? 1 : sz <= 128 ? 2 : sz <= med_max ? 3 : sz <= huge_max ? 4 : 5;
        if (tier >= 0 && tier < min_tier) {
            // room in the forced tier's list (quarters of cap; the last one split in halves)
            int* cnt = min_tier == 1 ? &ctr->n_t32 : min_tier == 2 ? &ctr->n_med : min_tier == 3 ? &ctr->n_large
                     : min_tier == 4 ? &ctr->n_huge : &ctr->n_big;
            // leave room for the regions that belong there by size (at most nverts / their least size)
            const int least = min_tier == 1 ? 16 : min_tier == 2 ? 32 : min_tier == 3 ? 128
                            : min_tier == 4 ? med_max : huge_max;
            const int room = (min_tier >= 4 ? q / 2 : q) - nverts / least;
            if (*(volatile int*)cnt < room) {
                const int pos = atomicAdd(cnt, 1);
                if (pos < room) {
                    int* rest = tier_list + cap;
                    const int base = min_tier == 1 ? 0 : min_tier == 2 ? q : min_tier == 3 ? 2 * q
                                   : min_tier == 4 ? 3 * q : 3 * q + q / 2;
                    rest[base + pos] = r;
                    tier = -2;                        // placed
                } else {
                    atomicSub(cnt, 1);
                }
            }
        }
        const bool t16 = tier == 0;
        const int p16 = warp_reserve(&ctr->n_t16, t16);
        if (t16) tier_list[p16] = r;
        int* rest = tier_list + cap;
        const bool t32 = tier == 1;
        const bool med = tier == 2;
        const bool lrg = tier == 3;
        const bool huge = tier == 4;
        const bool big = tier == 5;
        const int p32 = warp_reserve(&ctr->n_t32, t32);
        const int pm = warp_reserve(&ctr->n_med, med);
        const int pl = warp_reserve(&ctr->n_large, lrg);
        const int ph = warp_reserve(&ctr->n_huge, huge);
        const int pb = warp_reserve(&ctr->n_big, big);
        if (t32) rest[p32] = r;
        if (med) rest[q + pm] = r;
        if (lrg) rest[2 * q + pl] = r;
        if (huge) rest[3 * q + ph] = r;
        if (big) rest[3 * q + q / 2 + pb] = r;
    }
    if (trivial) atomicMax(&ctr->max_floods, 1);
    warp_atomic_add64(&ctr->total_floods, trivial);
}

// Per saddle (run by its head region): order the sibling regions by their
// highest member and give each the offset of its block below the saddle.
__global__ void siblings_kernel(const int* __restrict__ reg_class, const int* __restrict__ reg_head,
                                const int* __restrict__ reg_sod, const int* __restrict__ reg_size,
                                const int* __restrict__ reg_top, const int* __restrict__ sib_head,
                                const int* __restrict__ sib_next, const int* __restrict__ class2reg, int* reg_place,
                                int* reg_att, RankBlk* rblk, DevCounters* ctr) {
    if (failed(&ctr->status)) return;
    const int nreg = ctr->n_regions;
    int my_max = 0, my_sad = 0;
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < nreg; r += gridDim.x * blockDim.x) {
        const int sz = reg_size[r];
        my_max = max(my_max, sz);
        if (!reg_head[r]) continue;
        const int hc = reg_class[r];
        const int first = sib_head[hc];
        if (first < 0) {                               // the common case: one region at the saddle
            reg_place[r] = -sz;
            reg_att[r] = sz;
        } else {
            // siblings: the head class and the classes listed under it
            int total = sz;
            for (int cur = first; cur >= 0; cur = sib_next[cur]) total += reg_size[class2reg[cur]];
            int cur = hc;
            while (cur >= 0) {
                const int rr = class2reg[cur];
                const int t = reg_top[rr];
                int below = reg_top[r] < t ? sz : 0;   // sizes of siblings with a lower top
                for (int c2 = first; c2 >= 0; c2 = sib_next[c2]) {
                    const int r2 = class2reg[c2];
                    if (reg_top[r2] < t) below += reg_size[r2];
                }
                reg_place[rr] = below - total;
                cur = cur == hc ? first : sib_next[cur];
            }
            reg_att[r] = total;
        }
        const int j = reg_sod[r];
        atomicOr(&rblk[j >> kRankShift].smask, 1u << (j & 31));
        ++my_sad;
    }
    warp_atomic_max(&ctr->max_region, my_max);
    warp_atomic_add(&ctr->n_saddles, my_sad);
}

}  // namespace

template <int DIR>
cudaError_t extract_regions(Work& w, const Geom& g, const int* O, int sms, cudaStream_t s) {
    const int T = 256;
    const int B = sms * 8;
    flatten_kernel<<<B, T, 0, s>>>(w.parent, w.ctr);
    roots_kernel<DIR><<<B, T, 0, s>>>(g, O, w.parent, w.wait_v, w.owner, w.sib_head, w.sib_next, w.class2reg, w.reg_class, w.reg_saddle,
                                      w.reg_size, w.reg_top, w.reg_sod, w.reg_head, w.ctr);
    cls_rid_kernel<<<B, T, 0, s>>>(w.parent, w.class2reg, w.cls2rid, w.ctr);
    members_count_kernel<DIR><<<B, T, 0, s>>>(g, O, w.vlog, w.vlog_cls, w.cls2rid, w.owner, w.loc, w.reg_saddle,
                                              w.reg_size, w.reg_top, w.ent_rid, w.ent_loc, w.ent_od, w.ctr);
    scan_excl_i32(w, w.reg_size, w.reg_start, &w.ctr->n_regions, g.n / 2 + 1, s);
    members_fill_kernel<<<B, T, 0, s>>>(w.vlog, w.ent_rid, w.ent_loc, w.ent_od, w.reg_start, w.members,
                                        w.member_reg, w.rblk, w.ctr);
    siblings_kernel<<<B, T, 0, s>>>(w.reg_class, w.reg_head, w.reg_sod, w.reg_size, w.reg_top, w.sib_head, w.sib_next,
                                    w.class2reg, w.reg_place, w.reg_att, w.rblk, w.ctr);
    tiers_kernel<<<B, T, 0, s>>>(w.reg_size, w.reg_start, w.lhat, w.tier_list, w.class_cap, w.class_cap / 4,
                                 local_order_med_max(), local_order_huge_max(), w.min_tier, g.n, w.ctr);
    w.launches += 7;
    return cudaGetLastError();
}

template cudaError_t extract_regions<1>(Work&, const Geom&, const int*, int, cudaStream_t);
template cudaError_t extract_regions<-1>(Work&, const Geom&, const int*, int, cudaStream_t);

}  // namespace lts
