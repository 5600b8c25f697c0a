// Sampled-splitter partition of 64-bit keys with equality buckets.
//
// Used by the local sort (reference-split keys of strings).  Every segment of
// positions [start, start+size) is split into B range buckets (s_{b-1} < k <
// s_b) and B-1 equality buckets (k == s_b) by B-1 splitters taken from an
// evenly spaced, sorted sample of the segment's keys.  Equal keys always share a
// bucket, so a key that occurs very often ends in its own equality bucket
// instead of overflowing a range bucket.  The scatter is stable (warp-level
// ranking in position order), so equal keys keep their relative order.
//
// A round is planned on the device (k_lg_plan, one CTA): it reads the list of
// segments pushed by the previous round, orders them (partitioned segments
// first, whole-segment sorts after), and writes every segment's tiles, bucket
// count and offsets plus the round's totals (LsPlan).  Every kernel of the round
// runs on a fixed grid and loops over the counts in LsPlan, so a round needs no
// host round trip and the whole loop can be captured in a CUDA graph.
#pragma once

#include <algorithm>
#include <vector>

#include "sss_device.cuh"
#include "sss_internal.cuh"

namespace {

constexpr int LG_TILE = 1024, LG_T = 256;  // tile of positions per CTA / threads
constexpr int LG_OVS = 16;                 // samples per range bucket
constexpr int LG_BMAX = 256;               // max range buckets per segment
constexpr int LG_NBMAX = 2 * LG_BMAX - 1;  // range + equality buckets

struct LgSegInfo {
    Seg seg;            // start, size, depth
    uint32_t tiles;     // number of tiles
    uint32_t tile0;     // first tile index
    uint32_t nb;        // range buckets B (splitters B-1, buckets 2B-1); 0 for whole-segment sorts
    uint32_t hist_base; // offset into hist (bucket-major: b*tiles + t)
    uint32_t bst_base;  // offset into bucket starts (2B entries)
    uint32_t bk_base;   // index of this segment's first bucket in the flat bucket list
    uint32_t pad[2];
};

struct LgTile {
    uint32_t s;      // segment index
    uint32_t begin;  // absolute first position
    uint32_t end;    // absolute end position
    uint32_t t;      // tile index within segment
};

// Totals of one round: segments [0, npart) are partitioned, [npart, ns) sorted
// whole; tiles [0, ptiles) belong to partitioned segments.
struct LsPlan {
    uint32_t ns, npart, ntiles, ptiles, pbuckets, hist;
    uint32_t pad[2];
};

// Plan a round from the segment list `list` (count cnt[2]); resets the five list
// counters for the pushes of this round and the eight dynamic work counters.
// One CTA of 1024 threads.
__global__ void __launch_bounds__(1024) k_lg_plan(const Seg* __restrict__ list, uint32_t* __restrict__ cnt,
                                                  uint32_t* __restrict__ work, uint32_t direct_max, uint32_t target, uint32_t cap_segs,
                                                  uint32_t cap_tiles, uint32_t cap_hist,
                                                  LgSegInfo* __restrict__ info, LsPlan* __restrict__ plan,
                                                  unsigned* err) {
    __shared__ uint32_t sh_warp[32];
    __shared__ uint32_t s_ns;
    const uint32_t tid = threadIdx.x;
    if (tid == 0) {
        uint32_t c = cnt[2];
        if (c > cap_segs) {
            atomicOr(err, ERRBIT_OVERFLOW);
            c = 0;
        }
        s_ns = c;
    }
    __syncthreads();
    const uint32_t ns = s_ns;
    // partitioned segments first, in list order, then the whole-segment sorts
    uint32_t local = 0;
    for (uint32_t s = tid; s < ns; s += 1024) local += list[s].size > direct_max ? 1u : 0u;
    uint32_t npart;
    BlockScan<1024>::exclusive_sum(local, sh_warp, &npart);
    uint32_t cp = 0, cd = 0;
    for (uint32_t b0 = 0; b0 < ns; b0 += 1024) {
        const uint32_t s = b0 + tid;
        const bool valid = s < ns;
        Seg sg{};
        if (valid) sg = list[s];
        const bool part = valid && sg.size > direct_max;
        uint32_t tp, td;
        uint32_t ep = BlockScan<1024>::exclusive_sum(part ? 1u : 0u, sh_warp, &tp);
        uint32_t ed = BlockScan<1024>::exclusive_sum(valid && !part ? 1u : 0u, sh_warp, &td);
        if (valid) info[part ? cp + ep : npart + cd + ed].seg = sg;
        cp += tp;
        cd += td;
    }
    __syncthreads();
    // tiles, buckets and offsets in the new order
    uint32_t ct = 0, ch = 0, cb = 0, cpt = 0;
    for (uint32_t b0 = 0; b0 < ns; b0 += 1024) {
        const uint32_t s = b0 + tid;
        const bool valid = s < ns;
        Seg sg{};
        if (valid) sg = info[s].seg;
        const bool part = valid && s < npart;
        const uint32_t tiles = valid ? (sg.size + LG_TILE - 1) / LG_TILE : 0u;
        uint32_t nb = 0;
        if (part) {
            nb = (sg.size + target - 1) / target;
            nb = nb < 2u ? 2u : (nb > (uint32_t)LG_BMAX ? (uint32_t)LG_BMAX : nb);
        }
        const uint32_t nbk = part ? 2 * nb - 1 : 0u;
        uint32_t tt, th, tb, tpt;
        uint32_t et = BlockScan<1024>::exclusive_sum(tiles, sh_warp, &tt);
        uint32_t eh = BlockScan<1024>::exclusive_sum(nbk * tiles, sh_warp, &th);
        uint32_t eb = BlockScan<1024>::exclusive_sum(nbk, sh_warp, &tb);
        BlockScan<1024>::exclusive_sum(part ? tiles : 0u, sh_warp, &tpt);
        if (valid) {
            LgSegInfo si{};
            si.seg = sg;
            si.tiles = tiles;
            si.tile0 = ct + et;
            si.nb = nb;
            si.hist_base = ch + eh;
            si.bst_base = s * (LG_NBMAX + 1);
            si.bk_base = cb + eb;
            info[s] = si;
        }
        ct += tt;
        ch += th;
        cb += tb;
        cpt += tpt;
    }
    if (tid == 0) {
        LsPlan pl{ns, npart, ct, cpt, cb, ch, {0, 0}};
        if (ct > cap_tiles || ch > cap_hist) {
            atomicOr(err, ERRBIT_OVERFLOW);
            pl = LsPlan{0, 0, 0, 0, 0, 0, {0, 0}};
        }
        *plan = pl;
        cnt[0] = cnt[1] = cnt[2] = cnt[3] = cnt[4] = cnt[5] = 0;
        for (int k = 0; k < 8; ++k) work[k] = 0;
    }
}

// segment of flat index g among n segments with nondecreasing field f: last
// segment with f <= g
__device__ __forceinline__ uint32_t segment_of_tile(const LgSegInfo* info, uint32_t ns, uint32_t g) {
    uint32_t a = 0, c = ns;
    while (a + 1 < c) {
        uint32_t mid = (a + c) >> 1;
        if (info[mid].tile0 <= g) a = mid; else c = mid;
    }
    return a;
}

__device__ __forceinline__ uint32_t segment_of_bucket(const LgSegInfo* info, uint32_t ns, uint32_t g) {
    uint32_t a = 0, c = ns;
    while (a + 1 < c) {
        uint32_t mid = (a + c) >> 1;
        if (info[mid].bk_base <= g) a = mid; else c = mid;
    }
    return a;
}

__global__ void k_lg_tiles(const LsPlan* __restrict__ plan, const LgSegInfo* __restrict__ info,
                           LgTile* __restrict__ tiles) {
    const uint32_t nt = plan->ntiles, ns = plan->ns;
    for (uint32_t g = blockIdx.x * blockDim.x + threadIdx.x; g < nt; g += gridDim.x * blockDim.x) {
        const uint32_t s = segment_of_tile(info, ns, g);
        const LgSegInfo si = info[s];
        const uint32_t t = g - si.tile0;
        const uint32_t b0 = si.seg.start + t * LG_TILE;
        const uint32_t e = si.seg.start + si.seg.size;
        tiles[g] = LgTile{s, b0, b0 + (uint32_t)LG_TILE < e ? b0 + (uint32_t)LG_TILE : e, t};
    }
}

// Per partitioned segment: evenly spaced samples, sorted; splitter b = sample (b+1)*OVS-1.
__global__ void __launch_bounds__(512) k_lg_samples(const LsPlan* __restrict__ plan,
                                                    const LgSegInfo* __restrict__ info, const uint64_t* __restrict__ K,
                                                    uint64_t* __restrict__ spl) {
    __shared__ uint64_t sh[LG_BMAX * LG_OVS];
    const uint32_t npart = plan->npart;
    for (uint32_t s = blockIdx.x; s < npart; s += gridDim.x) {
        __syncthreads();
        LgSegInfo si = info[s];
        uint32_t S = si.nb * LG_OVS;
        for (uint32_t i = threadIdx.x; i < S; i += 512) {
            uint64_t q = si.seg.start + ((2 * (uint64_t)i + 1) * si.seg.size) / (2 * (uint64_t)S);
            sh[i] = K[q];
        }
        __syncthreads();
        bitonic_sort64<512>(sh, S);
        for (uint32_t b = threadIdx.x; b + 1 < si.nb; b += 512)
            spl[(size_t)s * (LG_BMAX - 1) + b] = sh[(b + 1) * LG_OVS - 1];
    }
}

// first splitter >= k (lower bound) among nsp sorted splitters
__device__ __forceinline__ uint32_t lower_bound64(const uint64_t* s, uint32_t nsp, uint64_t k) {
    uint32_t lo = 0, hi = nsp;
    while (lo < hi) {
        uint32_t mid = (lo + hi) >> 1;
        if (s[mid] < k) lo = mid + 1; else hi = mid;
    }
    return lo;
}

__global__ void __launch_bounds__(LG_T) k_lg_classify(const LsPlan* __restrict__ plan,
                                                      const LgTile* __restrict__ tiles,
                                                      const LgSegInfo* __restrict__ info,
                                                      const uint64_t* __restrict__ K, const uint64_t* __restrict__ spl,
                                                      uint32_t* __restrict__ hist, uint32_t* __restrict__ rankinfo) {
    constexpr int W = LG_T / 32;
    constexpr int PER_WARP = LG_TILE / W;  // contiguous positions per warp
    __shared__ uint64_t ssp[LG_BMAX];
    __shared__ uint32_t cnt[W][LG_NBMAX];
    const uint32_t ptiles = plan->ptiles;
    for (uint32_t g = blockIdx.x; g < ptiles; g += gridDim.x) {
        __syncthreads();
        LgTile tl = tiles[g];
        LgSegInfo si = info[tl.s];
        uint32_t nsp = si.nb - 1, nbk = 2 * si.nb - 1;
        for (uint32_t i = threadIdx.x; i < nsp; i += LG_T) ssp[i] = spl[(size_t)tl.s * (LG_BMAX - 1) + i];
        for (uint32_t i = threadIdx.x; i < (uint32_t)(W * LG_NBMAX); i += LG_T) (&cnt[0][0])[i] = 0;
        __syncthreads();
        int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
        uint32_t lt = (1u << lane) - 1u;
        uint32_t myb[PER_WARP / 32], myr[PER_WARP / 32];
#pragma unroll
        for (int it = 0; it < PER_WARP / 32; ++it) {
            uint32_t q = tl.begin + w * PER_WARP + it * 32 + lane;
            bool valid = q < tl.end;
            uint32_t b = 0xFFFFu;
            if (valid) {
                uint64_t k = K[q];
                uint32_t lb = lower_bound64(ssp, nsp, k);
                b = 2 * lb + ((lb < nsp && ssp[lb] == k) ? 1u : 0u);
            }
            uint32_t peers = __match_any_sync(SSS_FULL, b);
            uint32_t leader = __ffs(peers) - 1;
            uint32_t base = 0;
            if (valid && lane == (int)leader) {
                base = cnt[w][b];
                cnt[w][b] = base + __popc(peers);
            }
            base = __shfl_sync(SSS_FULL, base, leader);
            myb[it] = b;
            myr[it] = base + __popc(peers & lt);
        }
        __syncthreads();
        // exclusive prefix over warps for every bucket; tile total into hist
        for (uint32_t b = threadIdx.x; b < nbk; b += LG_T) {
            uint32_t run = 0;
#pragma unroll
            for (int ww = 0; ww < W; ++ww) {
                uint32_t t = cnt[ww][b];
                cnt[ww][b] = run;
                run += t;
            }
            hist[si.hist_base + b * si.tiles + tl.t] = run;
        }
        __syncthreads();
#pragma unroll
        for (int it = 0; it < PER_WARP / 32; ++it) {
            uint32_t q = tl.begin + w * PER_WARP + it * 32 + lane;
            if (q < tl.end) rankinfo[q] = (myb[it] << 16) | (cnt[w][myb[it]] + myr[it]);
        }
    }
}

// Exclusive prefix of every bucket's row of tile counts (one warp per row, the
// row contiguous, so loads coalesce); the row total goes to the bucket's start
// slot, turned into the start by k_lg_offsets.
__global__ void __launch_bounds__(256) k_lg_rowscan(const LsPlan* __restrict__ plan,
                                                    const LgSegInfo* __restrict__ info, uint32_t* __restrict__ hist,
                                                    uint32_t* __restrict__ bst) {
    const uint32_t nrows = plan->pbuckets, npart = plan->npart;
    const uint32_t lane = threadIdx.x & 31;
    const uint32_t warps = gridDim.x * (blockDim.x >> 5);
    for (uint32_t r = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); r < nrows; r += warps) {
        const uint32_t s = segment_of_bucket(info, npart, r);
        const LgSegInfo si = info[s];
        const uint32_t b = r - si.bk_base;
        uint32_t* h = hist + si.hist_base + b * si.tiles;
        uint32_t carry = 0;
        for (uint32_t t0 = 0; t0 < si.tiles; t0 += 32) {
            const uint32_t t = t0 + lane;
            const uint32_t v = t < si.tiles ? h[t] : 0u;
            uint32_t x = v;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                uint32_t y = __shfl_up_sync(SSS_FULL, x, o);
                if (lane >= (uint32_t)o) x += y;
            }
            if (t < si.tiles) h[t] = carry + x - v;
            carry += __shfl_sync(SSS_FULL, x, 31);
        }
        if (lane == 0) bst[si.bst_base + b] = carry;
    }
}

// Per partitioned segment: bucket starts from the row totals.
__global__ void __launch_bounds__(512) k_lg_offsets(const LsPlan* __restrict__ plan,
                                                    const LgSegInfo* __restrict__ info, uint32_t* __restrict__ bst) {
    __shared__ uint32_t sh_warp[32];
    const uint32_t npart = plan->npart;
    for (uint32_t s = blockIdx.x; s < npart; s += gridDim.x) {
        LgSegInfo si = info[s];
        uint32_t nbk = 2 * si.nb - 1;
        uint32_t b = threadIdx.x;
        uint32_t tot = b < nbk ? bst[si.bst_base + b] : 0u;
        uint32_t total;
        uint32_t ex = BlockScan<512>::exclusive_sum(tot, sh_warp, &total);
        if (b < nbk) bst[si.bst_base + b] = si.seg.start + ex;
        if (b == 0) bst[si.bst_base + nbk] = si.seg.start + si.seg.size;
    }
}

// The scatter of a tile goes through shared memory: its keys are first placed
// in bucket order (the tile's bucket counts, scanned, plus each key's rank within
// its bucket), so that consecutive threads then write consecutive positions of
// one bucket's range.  Written directly, the keys of a warp land in as many
// buckets as they have, and every 8-byte key or 4-byte index costs a whole
// sector of DRAM writes.
__global__ void __launch_bounds__(LG_T) k_lg_scatter(const LsPlan* __restrict__ plan,
                                                     const LgTile* __restrict__ tiles, const LgSegInfo* __restrict__ info,
                                                     const uint32_t* __restrict__ hist, const uint32_t* __restrict__ bst,
                                                     const uint32_t* __restrict__ rankinfo,
                                                     const uint64_t* __restrict__ K, const uint32_t* __restrict__ perm,
                                                     uint64_t* __restrict__ tK, uint32_t* __restrict__ tV,
                                                     unsigned* err) {
    constexpr int PER = LG_TILE / LG_T;
    static_assert(2 * LG_T >= LG_NBMAX, "two buckets per thread in the scan");
    __shared__ uint32_t cnt[2 * LG_T];
    __shared__ uint32_t sh_warp[32];
    __shared__ uint64_t sK[LG_TILE];
    __shared__ uint32_t sV[LG_TILE], sD[LG_TILE];
    const uint32_t tid = threadIdx.x;
    const uint32_t ptiles = plan->ptiles;
    for (uint32_t g = blockIdx.x; g < ptiles; g += gridDim.x) {
        const LgTile tl = tiles[g];
        const LgSegInfo si = info[tl.s];
        const uint32_t nbk = 2 * si.nb - 1;
        __syncthreads();  // the previous tile's keys have left shared memory
        for (uint32_t i = tid; i < 2u * LG_T; i += LG_T) cnt[i] = 0;
        __syncthreads();
        uint32_t ri[PER];
#pragma unroll
        for (int u = 0; u < PER; ++u) {
            const uint32_t q = tl.begin + tid + u * LG_T;
            ri[u] = q < tl.end ? rankinfo[q] : 0xFFFFFFFFu;
            if (q < tl.end) atomicAdd(&cnt[min(ri[u] >> 16, 2u * LG_T - 1u)], 1u);  // b < nbk <= 511
        }
        __syncthreads();
        // the tile's bucket offsets: exclusive scan of the counts
        const uint32_t c0 = cnt[2 * tid], c1 = cnt[2 * tid + 1];
        const uint32_t ex = BlockScan<LG_T>::exclusive_sum(c0 + c1, sh_warp, nullptr);
        cnt[2 * tid] = ex;
        cnt[2 * tid + 1] = ex + c0;
        __syncthreads();
#pragma unroll
        for (int u = 0; u < PER; ++u) {
            const uint32_t q = tl.begin + tid + u * LG_T;
            if (q >= tl.end) continue;
            const uint32_t b = ri[u] >> 16, r = ri[u] & 0xFFFFu;
            const uint32_t slot = cnt[min(b, 2u * LG_T - 1u)] + r;
            uint32_t dst = bst[si.bst_base + b] + hist[si.hist_base + b * si.tiles + tl.t] + r;
            if (b >= nbk || dst < si.seg.start || dst >= si.seg.start + si.seg.size || slot >= LG_TILE) {
                atomicOr(err, ERRBIT_OVERFLOW);
                if (slot >= LG_TILE) continue;
                dst = 0xFFFFFFFFu;
            }
            sK[slot] = K[q];
            sV[slot] = perm[q];
            sD[slot] = dst;
        }
        __syncthreads();
        const uint32_t m = tl.end - tl.begin;
        for (uint32_t i = tid; i < m; i += LG_T) {
            const uint32_t dst = sD[i];
            if (dst == 0xFFFFFFFFu) continue;
            tK[dst] = sK[i];
            tV[dst] = sV[i];
        }
    }
}

// Work memory of the partition for up to `cap_segs` segments covering <= n positions.
struct SpBufs {
    uint64_t* spl;
    uint32_t* hist;
    uint32_t* bst;
    uint32_t* rankinfo;
    LgSegInfo* info;
    LgTile* tiles;
    LsPlan* plan;
    uint32_t cap_segs, cap_tiles, cap_hist;
};

inline void carve_sp(Arena& ar, uint32_t n, uint32_t cap_segs, SpBufs& b) {
    b.cap_segs = cap_segs;
    b.cap_tiles = n / LG_TILE + cap_segs + 2;
    b.cap_hist = LG_NBMAX * b.cap_tiles;
    b.spl = ar.take<uint64_t>((size_t)cap_segs * (LG_BMAX - 1));
    b.hist = ar.take<uint32_t>(b.cap_hist);
    b.bst = ar.take<uint32_t>((size_t)cap_segs * (LG_NBMAX + 1));
    b.rankinfo = ar.take<uint32_t>(n);
    b.info = ar.take<LgSegInfo>(cap_segs);
    b.tiles = ar.take<LgTile>(b.cap_tiles);
    b.plan = ar.take<LsPlan>(1);
}

// The partition of the planned round's partitioned segments (fixed grids).
inline sss_status launch_sp(sss_ctx* ctx, const SpBufs& B, const uint64_t* K, const uint32_t* V, uint64_t* tK,
                            uint32_t* tV, const char* tag_samples, const char* tag_classify, const char* tag_offsets,
                            const char* tag_scatter) {
    const uint32_t sm = (uint32_t)std::max(1, ctx->sm_count);
    SSS_TRY(sss_launch(ctx, tag_samples, k_lg_samples, dim3(sm * 2), dim3(512), 0, (const LsPlan*)B.plan,
                       (const LgSegInfo*)B.info, K, B.spl));
    SSS_TRY(sss_launch(ctx, tag_classify, k_lg_classify, dim3(sm * 6), dim3(LG_T), 0, (const LsPlan*)B.plan,
                       (const LgTile*)B.tiles, (const LgSegInfo*)B.info, K, (const uint64_t*)B.spl, B.hist,
                       B.rankinfo));
    SSS_TRY(sss_launch(ctx, tag_offsets, k_lg_rowscan, dim3(sm * 4), dim3(256), 0, (const LsPlan*)B.plan,
                       (const LgSegInfo*)B.info, B.hist, B.bst));
    SSS_TRY(sss_launch(ctx, tag_offsets, k_lg_offsets, dim3(sm * 2), dim3(512), 0, (const LsPlan*)B.plan,
                       (const LgSegInfo*)B.info, B.bst));
    SSS_TRY(sss_launch(ctx, tag_scatter, k_lg_scatter, dim3(sm * 8), dim3(LG_T), 0, (const LsPlan*)B.plan,
                       (const LgTile*)B.tiles, (const LgSegInfo*)B.info, (const uint32_t*)B.hist,
                       (const uint32_t*)B.bst, (const uint32_t*)B.rankinfo, K, V, tK, tV, ctx->d_err));
    return SSS_OK;
}

}  // namespace
