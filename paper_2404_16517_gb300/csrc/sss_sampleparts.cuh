// Sampled-splitter partition of 64-bit keys with equality buckets.
//
// Used by the local sort (words of strings) and by duplicate detection (prefix
// hashes).  Every segment of positions [start, start+size) is split into B range
// buckets (s_{b-1} < k < s_b) and B-1 equality buckets (k == s_b) by B-1
// splitters taken from an evenly spaced, sorted sample of the segment's keys.
// Equal keys always share a bucket, so a key that occurs very often ends in its
// own equality bucket instead of overflowing a range bucket.  The scatter is
// stable (warp-level ranking in position order), so equal keys keep their
// relative order.
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
    uint32_t nb;        // range buckets B (splitters B-1, buckets 2B-1)
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

// One CTA per segment: evenly spaced samples, sorted; splitter b = sample (b+1)*OVS-1.
__global__ void __launch_bounds__(512) k_lg_samples(const LgSegInfo* __restrict__ info, const uint64_t* __restrict__ K,
                                                    uint64_t* __restrict__ spl) {
    __shared__ uint64_t sh[LG_BMAX * LG_OVS];
    LgSegInfo si = info[blockIdx.x];
    uint32_t S = si.nb * LG_OVS;
    for (uint32_t i = threadIdx.x; i < S; i += 512) {
        uint64_t q = si.seg.start + ((2 * (uint64_t)i + 1) * si.seg.size) / (2 * (uint64_t)S);
        sh[i] = K[q];
    }
    __syncthreads();
    bitonic_sort64<512>(sh, S);
    for (uint32_t b = threadIdx.x; b + 1 < si.nb; b += 512)
        spl[(size_t)blockIdx.x * (LG_BMAX - 1) + b] = sh[(b + 1) * LG_OVS - 1];
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

__global__ void __launch_bounds__(LG_T) k_lg_classify(const LgTile* __restrict__ tiles,
                                                      const LgSegInfo* __restrict__ info,
                                                      const uint64_t* __restrict__ K, const uint64_t* __restrict__ spl,
                                                      uint32_t* __restrict__ hist, uint32_t* __restrict__ rankinfo) {
    constexpr int W = LG_T / 32;
    constexpr int PER_WARP = LG_TILE / W;  // contiguous positions per warp
    __shared__ uint64_t ssp[LG_BMAX];
    __shared__ uint32_t cnt[W][LG_NBMAX];
    LgTile tl = tiles[blockIdx.x];
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

// Per segment: prefix of every bucket over the tiles, then bucket starts.
__global__ void __launch_bounds__(512) k_lg_offsets(const LgSegInfo* __restrict__ info, uint32_t* __restrict__ hist,
                                                    uint32_t* __restrict__ bst) {
    __shared__ uint32_t sh_warp[32];
    LgSegInfo si = info[blockIdx.x];
    uint32_t nbk = 2 * si.nb - 1;
    uint32_t b = threadIdx.x;
    uint32_t tot = 0;
    if (b < nbk) {
        uint32_t* h = hist + si.hist_base + b * si.tiles;
        for (uint32_t t = 0; t < si.tiles; ++t) {
            uint32_t v = h[t];
            h[t] = tot;
            tot += v;
        }
    }
    uint32_t total;
    uint32_t ex = BlockScan<512>::exclusive_sum(tot, sh_warp, &total);
    if (b < nbk) bst[si.bst_base + b] = si.seg.start + ex;
    if (b == 0) bst[si.bst_base + nbk] = si.seg.start + si.seg.size;
}

__global__ void __launch_bounds__(LG_T) k_lg_scatter(const LgTile* __restrict__ tiles, const LgSegInfo* __restrict__ info,
                                                     const uint32_t* __restrict__ hist, const uint32_t* __restrict__ bst,
                                                     const uint32_t* __restrict__ rankinfo,
                                                     const uint64_t* __restrict__ K, const uint32_t* __restrict__ perm,
                                                     uint64_t* __restrict__ tK, uint32_t* __restrict__ tV,
                                                     unsigned* err) {
    LgTile tl = tiles[blockIdx.x];
    LgSegInfo si = info[tl.s];
    for (uint32_t q = tl.begin + threadIdx.x; q < tl.end; q += LG_T) {
        uint32_t ri = rankinfo[q];
        uint32_t b = ri >> 16;
        uint32_t dst = bst[si.bst_base + b] + hist[si.hist_base + b * si.tiles + tl.t] + (ri & 0xFFFFu);
        if (dst < si.seg.start || dst >= si.seg.start + si.seg.size) {
            atomicOr(err, ERRBIT_OVERFLOW);
            continue;
        }
        tK[dst] = K[q];
        tV[dst] = perm[q];
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
}

// Host plan for a list of segments: bucket counts, tiles and offsets, written to
// pinned staging (h_info, h_tiles).  Range buckets target `target` keys each.
// Returns false when a capacity would be exceeded.
inline bool plan_sp(const std::vector<Seg>& segs, uint32_t target, const SpBufs& B, LgSegInfo* h_info,
                    LgTile* h_tiles, uint32_t* out_ntiles, uint32_t* out_nbuckets = nullptr) {
    uint32_t ns = (uint32_t)segs.size();
    if (ns > B.cap_segs) return false;
    uint32_t ntiles = 0, hist_off = 0, nbk = 0;
    for (uint32_t s = 0; s < ns; ++s) {
        const Seg& sg = segs[s];
        uint32_t tiles = (sg.size + LG_TILE - 1) / LG_TILE;
        uint32_t nb = (sg.size + target - 1) / target;
        nb = std::max(2u, std::min((uint32_t)LG_BMAX, nb));
        LgSegInfo si{};
        si.seg = sg;
        si.tiles = tiles;
        si.tile0 = ntiles;
        si.nb = nb;
        si.hist_base = hist_off;
        si.bst_base = s * (LG_NBMAX + 1);
        si.bk_base = nbk;
        nbk += 2 * nb - 1;
        h_info[s] = si;
        if (ntiles + tiles > B.cap_tiles) return false;
        for (uint32_t t = 0; t < tiles; ++t) {
            uint32_t b0 = sg.start + t * LG_TILE;
            h_tiles[ntiles + t] = LgTile{s, b0, std::min(b0 + (uint32_t)LG_TILE, sg.start + sg.size), t};
        }
        ntiles += tiles;
        hist_off += (2 * nb - 1) * tiles;
        if (hist_off > B.cap_hist) return false;
    }
    *out_ntiles = ntiles;
    if (out_nbuckets) *out_nbuckets = nbk;
    return true;
}

// Enqueue samples, classification, offsets and the stable scatter of (K, V) into
// (tK, tV); bucket b of segment s then spans bst[s*(LG_NBMAX+1) + b .. + b+1).
inline sss_status launch_sp(sss_ctx* ctx, const SpBufs& B, uint32_t ns, uint32_t ntiles, const uint64_t* K,
                            const uint32_t* V, uint64_t* tK, uint32_t* tV, const char* tag_samples,
                            const char* tag_classify, const char* tag_offsets, const char* tag_scatter) {
    SSS_TRY(sss_launch(ctx, tag_samples, k_lg_samples, dim3(ns), dim3(512), 0, (const LgSegInfo*)B.info, K, B.spl));
    SSS_TRY(sss_launch(ctx, tag_classify, k_lg_classify, dim3(ntiles), dim3(LG_T), 0, (const LgTile*)B.tiles,
                       (const LgSegInfo*)B.info, K, (const uint64_t*)B.spl, B.hist, B.rankinfo));
    SSS_TRY(sss_launch(ctx, tag_offsets, k_lg_offsets, dim3(ns), dim3(512), 0, (const LgSegInfo*)B.info, B.hist,
                       B.bst));
    SSS_TRY(sss_launch(ctx, tag_scatter, k_lg_scatter, dim3(ntiles), dim3(LG_T), 0, (const LgTile*)B.tiles,
                       (const LgSegInfo*)B.info, (const uint32_t*)B.hist, (const uint32_t*)B.bst,
                       (const uint32_t*)B.rankinfo, K, V, tK, tV, ctx->d_err));
    return SSS_OK;
}

// segment of flat bucket g: last segment with bk_base <= g
__device__ __forceinline__ uint32_t segment_of_bucket(const LgSegInfo* info, uint32_t ns, uint32_t g) {
    uint32_t a = 0, c = ns;
    while (a + 1 < c) {
        uint32_t mid = (a + c) >> 1;
        if (info[mid].bk_base <= g) a = mid; else c = mid;
    }
    return a;
}

}  // namespace
