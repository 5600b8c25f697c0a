// Stage A: local string sort of every partition with LCP-array output
// (Section 3, "Initialization": each PE sorts its local strings; the LCP array
// is a by-product of sorting).  A6: exact distinguishing prefixes (Section 2).
//
// Design (GB300): MSD radix sort with reference-split keys.
//  * A segment is a run of positions whose strings share their first `depth`
//    characters.  Every member is compared with the segment's first member (the
//    reference) from `depth` on: its full LCP v with the reference, its next
//    characters and which side of the reference it falls on make a 64-bit key
//    (ref_key in sss_device.cuh) whose order is string order on the first
//    depth + v + C characters (C = 4..6, by the reference's length).  Each member thus skips its own shared prefix
//    with the reference; a plain common-prefix skip would only advance the whole
//    segment by the smallest v.
//  * Segments of <= 2048 strings are finished inside one CTA: keys are gathered,
//    sorted in shared memory as (group, key, index) and split, until every group
//    is a single string or a run of equal strings.
//  * Larger segments take a multi-CTA round: compute the keys, sample splitters,
//    classify into range and equality buckets (equal keys always share a
//    bucket), stable scatter, sort each range bucket in shared memory, and emit
//    the groups of equal keys as new segments.
//  * LCP values fall out at every split (key_lcp); equal strings get lcp = their
//    length.
#include <algorithm>
#include <cstdio>
#include <vector>

#include "sss_device.cuh"
#include "sss_internal.cuh"
#include "sss_sampleparts.cuh"

namespace {

constexpr uint32_t DONE = 0xFFFFFFFFu;

// size classes
constexpr int WF_WARPS = 8;                     // group finishers: warps per CTA
constexpr int QUAD_W = 4;                       // segments of <= 4 strings: 4 lanes each, 8 per warp
constexpr int TINY_T = 64, TINY_CAP = 64;       // segments of warp_cap+1 .. 64 strings
constexpr int SM_T = 128, SM_CAP = 512;         // segments of 65 .. 512 strings
constexpr int MED_T = 512, MED_CAP = 2048;      // segments of 513 .. cta_cap (<= 2048) strings, 2 CTAs per SM
constexpr int BK_T = 512, BK_CAP = 4096;        // bucket sort CTA (bucket targets above BKS_CAP / 2)
constexpr int BKS_T = 256, BKS_CAP = 2048;      // bucket sort CTA for targets <= BKS_CAP / 2 (4 CTAs per SM)
constexpr int DIRECT_T = 1024, DIRECT_CAP = 8192;  // whole-segment sort CTA (segments <= direct_cap)

struct SegLists {
    Seg* tiny;
    Seg* med;
    Seg* large;
    uint32_t* cnt;  // [0] tiny, [1] med, [2] large, [3] warp, [4] small, [5] quad
    uint32_t cap_tiny, cap_med, cap_large;
    Seg* warp;
    uint32_t cap_warp;
    Seg* small;
    uint32_t cap_small;
    uint32_t warp_max, med_max;  // classes: warp <= warp_max < tiny <= TINY_CAP < small <= SM_CAP < med <= med_max < large
};

__device__ __forceinline__ void push_seg(const SegLists& L, uint32_t start, uint32_t size, uint32_t depth,
                                         unsigned* err) {
    Seg s{start, size, depth, 0};
    if (size <= L.warp_max) {
        // one array for both short classes: segments of <= QUAD_W strings from
        // the bottom (count cnt[5]), the others from the top (count cnt[3]); the
        // two never meet, as the segments of a round are disjoint and hold >= 2
        // strings each (the finishers check it)
        if (size <= (uint32_t)QUAD_W) {
            uint32_t i = atomicAdd(&L.cnt[5], 1u);
            if (i < L.cap_warp) L.warp[i] = s; else atomicOr(err, ERRBIT_OVERFLOW);
        } else {
            uint32_t i = atomicAdd(&L.cnt[3], 1u);
            if (i < L.cap_warp) L.warp[L.cap_warp - 1u - i] = s; else atomicOr(err, ERRBIT_OVERFLOW);
        }
    } else if (size <= (uint32_t)TINY_CAP) {
        uint32_t i = atomicAdd(&L.cnt[0], 1u);
        if (i < L.cap_tiny) L.tiny[i] = s; else atomicOr(err, ERRBIT_OVERFLOW);
    } else if (size <= (uint32_t)SM_CAP && size <= L.med_max) {
        uint32_t i = atomicAdd(&L.cnt[4], 1u);
        if (i < L.cap_small) L.small[i] = s; else atomicOr(err, ERRBIT_OVERFLOW);
    } else if (size <= L.med_max) {
        uint32_t i = atomicAdd(&L.cnt[1], 1u);
        if (i < L.cap_med) L.med[i] = s; else atomicOr(err, ERRBIT_OVERFLOW);
    } else {
        uint32_t i = atomicAdd(&L.cnt[2], 1u);
        if (i < L.cap_large) L.large[i] = s; else atomicOr(err, ERRBIT_OVERFLOW);
    }
}

// push_seg for a whole warp: every lane calls it (converged) and the lanes
// with `want` push their segment.  Lanes pushing to the same list share one
// atomic on its counter: a round can emit millions of short segments, and one
// atomic per segment on the few list counters serialises in L2.
__device__ __forceinline__ void push_seg_warp(const SegLists& L, bool want, uint32_t start, uint32_t size,
                                              uint32_t depth, unsigned* err) {
    if (__ballot_sync(SSS_FULL, want) == 0) return;
    // list of the segment: 0 quad, 1 warp, 2 tiny, 3 small, 4 med, 5 large; 6 none
    uint32_t cls = 6u;
    if (want) {
        if (size <= L.warp_max) cls = size <= (uint32_t)QUAD_W ? 0u : 1u;
        else if (size <= (uint32_t)TINY_CAP) cls = 2u;
        else if (size <= (uint32_t)SM_CAP && size <= L.med_max) cls = 3u;
        else if (size <= L.med_max) cls = 4u;
        else cls = 5u;
    }
    const unsigned peers = __match_any_sync(SSS_FULL, cls);
    if (!want) return;
    const uint32_t lane = threadIdx.x & 31;
    const uint32_t leader = (uint32_t)__ffs(peers) - 1u;
    const uint32_t rank = (uint32_t)__popc(peers & ((1u << lane) - 1u));
    const uint32_t cidx = (0x214035u >> (4u * cls)) & 0xFu;  // counter of the list: 5 3 0 4 1 2
    uint32_t base = 0;
    if (lane == leader) base = atomicAdd(&L.cnt[cidx], (uint32_t)__popc(peers));
    base = __shfl_sync(peers, base, leader);
    const uint32_t i = base + rank;
    const Seg sg{start, size, depth, 0};
    bool ok;
    switch (cls) {
        case 0: ok = i < L.cap_warp; if (ok) L.warp[i] = sg; break;
        case 1: ok = i < L.cap_warp; if (ok) L.warp[L.cap_warp - 1u - i] = sg; break;
        case 2: ok = i < L.cap_tiny; if (ok) L.tiny[i] = sg; break;
        case 3: ok = i < L.cap_small; if (ok) L.small[i] = sg; break;
        case 4: ok = i < L.cap_med; if (ok) L.med[i] = sg; break;
        default: ok = i < L.cap_large; if (ok) L.large[i] = sg; break;
    }
    if (!ok) atomicOr(err, ERRBIT_OVERFLOW);
}

// Dynamic work distribution: the next unit for the whole CTA (units vary a lot
// in cost, so a static block-to-unit map leaves a long tail).
__device__ __forceinline__ uint32_t cta_next_unit(uint32_t* counter) {
    __shared__ uint32_t s_unit;
    __syncthreads();
    if (threadIdx.x == 0) s_unit = atomicAdd(counter, 1u);
    __syncthreads();
    return s_unit;
}

// Candidates for the reference member of a group of `cnt` strings starting at
// `start` with depth `depth`: fixed pseudo-random members, the t-th from
// ref_pick(.., t) (results do not depend on the choice).  The finishers and
// the large path take the longest of several candidates: a member's LCP with
// the reference is capped by the reference's length, so a short reference keeps
// every longer member that shares its whole remainder in one group.  Always
// taking the first member would let an input whose order follows the strings'
// lengths or shared prefixes peel off a few strings per round.
__device__ __forceinline__ uint32_t ref_mix(uint32_t start, uint32_t cnt, uint32_t depth, uint32_t t) {
    uint32_t x = start * 0x9E3779B9u ^ (depth + 0x7F4A7C15u) * 0x85EBCA6Bu ^ cnt * 0xC2B2AE35u ^ t * 0x27D4EB2Fu;
    x ^= x >> 16;
    x *= 0x7FEB352Du;
    x ^= x >> 15;
    x *= 0x846CA68Bu;
    x ^= x >> 16;
    return x;
}
__device__ __forceinline__ uint32_t ref_pick(uint32_t start, uint32_t cnt, uint32_t depth, uint32_t t = 0) {
    return cnt > 1 ? ref_mix(start, cnt, depth, t) % cnt : 0u;
}

// identity order and LCP 0 over positions q0 .. q0 + n (perm and lcp point at q0)
__global__ void k_init_perm(uint32_t* perm, uint32_t* lcp, uint32_t n, uint32_t q0) {
    uint32_t q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q < n) {
        perm[q] = q0 + q;
        lcp[q] = 0;
    }
}

// ---------------------------------------------------------------------------
// CTA finisher: completely sorts one segment of <= CAP strings.
template <int THREADS, int CAP>
__device__ __forceinline__ void finish_segment(const Seg sg, const uint8_t* __restrict__ chars,
                                               const uint64_t* __restrict__ offs, const uint32_t* __restrict__ lens,
                                               uint32_t* __restrict__ perm, uint32_t* __restrict__ lcp, unsigned* err) {
    constexpr int ITEMS = CAP / THREADS;
    extern __shared__ __align__(16) unsigned char smem[];
    uint64_t* sHi = reinterpret_cast<uint64_t*>(smem);  // sort keys (group:16 | word>>16)
    uint64_t* sLo = sHi + CAP;                           // (word<<48 | string index)
    uint32_t* sV = reinterpret_cast<uint32_t*>(sLo + CAP);  // string index at local position
    uint32_t* sG = sV + CAP;                             // group start of element, DONE when final
    uint32_t* sGD = sG + CAP;                            // depth of group (at its start)
    uint32_t* sGM = sGD + CAP;                           // member count (at group start)
    uint32_t* sGF = sGM + CAP;                           // key format of the group (at its start)
    uint32_t* sA = sGF + CAP;                            // scan buffer
    uint32_t* sC = sA + CAP;                             // compacted active positions
    __shared__ uint32_t sh_warp[32];
    constexpr uint32_t FIN_NREF = 68;  // 64 reference words plus a 4-word block of slack
    __shared__ uint64_t refw[FIN_NREF];

    const uint32_t m = sg.size;
    const int tid = threadIdx.x;
    for (uint32_t i = tid; i < m; i += THREADS) {
        sV[i] = perm[sg.start + i];
        sG[i] = 0;
    }
    if (tid == 0) {
        sGD[0] = sg.depth;
        sGM[0] = m;
    }
    __syncthreads();

    // every iteration splits a group or finishes it, so a segment of m strings
    // needs at most about 2m iterations; the bound only guards against bugs
    for (uint32_t iter = 0;; ++iter) {
        if (iter > 4u * (uint32_t)CAP + 64u) {
            if (tid == 0) atomicOr(err, ERRBIT_OVERFLOW);
            break;
        }
        // 1. compact the positions of unfinished elements
        for (uint32_t i = tid; i < (uint32_t)CAP; i += THREADS) sA[i] = (i < m && sG[i] != DONE) ? 1u : 0u;
        __syncthreads();
        uint32_t nact = block_exclusive_sum_inplace<THREADS, ITEMS>(sA, CAP, sh_warp);
        if (nact == 0) break;
        for (uint32_t i = tid; i < m; i += THREADS)
            if (sG[i] != DONE) sC[sA[i]] = i;
        __syncthreads();

        // 2a. every group's reference: its longest member among up to
        //     REF_CAND candidates (all members of a smaller group, scanned from
        //     a pseudo-random one on, else pseudo-random ones; the earliest
        //     candidate on ties), kept at the group start in the scan buffer,
        //     which is free until step 5
        for (uint32_t j = tid; j < nact; j += THREADS) {
            const uint32_t pos = sC[j];
            if (sG[pos] != pos) continue;
            constexpr uint32_t REF_CAND = 8;
            const uint32_t c = sGM[pos], d = sGD[pos];
            uint32_t best = pos, blen = 0;
            if (c <= REF_CAND) {
                const uint32_t t0 = ref_pick(pos, c, d);
                for (uint32_t t = 0; t < c; ++t) {
                    const uint32_t q = pos + (t0 + t < c ? t0 + t : t0 + t - c);
                    const uint32_t l = lens[sV[q]];
                    if (t == 0 || l > blen) { blen = l; best = q; }
                }
            } else {
#pragma unroll
                for (uint32_t t = 0; t < REF_CAND; ++t) {
                    const uint32_t q = pos + ref_pick(pos, c, d, t);
                    const uint32_t l = lens[sV[q]];
                    if (t == 0 || l > blen) { blen = l; best = q; }
                }
            }
            sA[pos] = best;
        }
        __syncthreads();
        // the first iteration has one group, the whole segment: its reference's
        // first 512 characters from the depth on go to shared memory, so that
        // every member reads only its own string (with 16-byte loads)
        if (iter == 0) {
            const uint32_t r0 = sV[sA[0]], rl0 = lens[r0];
            for (uint32_t i = tid; i < FIN_NREF; i += THREADS) refw[i] = load_word_be(chars + offs[r0], rl0, sGD[0] + 8 * i);
            __syncthreads();
        }

        // 2b. reference-split key of every member against its group's
        //     reference; pack (group, key, index)
        for (uint32_t j = tid; j < nact; j += THREADS) {
            uint32_t pos = sC[j];
            uint32_t g = sG[pos];
            uint32_t d = sGD[g];
            const uint32_t refpos = sA[g];
            uint32_t e = sV[pos], r = sV[refpos];
            const uint8_t* rs = chars + offs[r];
            uint32_t rl = lens[r];
            uint64_t w;
            uint32_t v;
            const uint32_t f = key_fmt(rl, d);
            if (pos == g) sGF[g] = f;
            if (pos == refpos) {
                v = rl > d ? rl - d : 0u;
                v = v < VCAP ? v : VCAP;
                w = load_word_be(rs, rl, d + v);
            } else {
                const uint32_t le = lens[e];
                const uint32_t mlen = le < rl ? le : rl;
                v = (iter == 0 && mlen <= d + 8 * (FIN_NREF - 4)) ? lcp_full_w_ref(chars + offs[e], le, rl, refw, d, &w)
                                                                  : lcp_full_w(chars + offs[e], le, rs, rl, d, &w);
            }
            const uint32_t rho = (iter == 0 && (v >> 3) < FIN_NREF)
                                     ? (uint32_t)(refw[v >> 3] >> (56 - 8 * (v & 7))) & 0xFFu
                                     : (uint32_t)(load_word_be(rs, rl, d + v) >> 56);
            uint64_t k = ref_key(v, w, rho, f);
            sHi[j] = ((uint64_t)g << 48) | (k >> 16);
            sLo[j] = (k << 48) | (uint64_t)e;
        }
        __syncthreads();

        // 3. sort (group, key, index)
        block_merge_sort128_fit<THREADS, ITEMS>(sHi, sLo, nact);

        // 5. write back, find new group boundaries, LCP at new boundaries
        for (uint32_t j = tid; j < nact; j += THREADS) {
            uint32_t pos = sC[j];
            uint64_t hi = sHi[j], lo = sLo[j];
            uint32_t g = (uint32_t)(hi >> 48);
            uint64_t k = (hi << 16) | (lo >> 48);
            sV[pos] = (uint32_t)lo;
            bool bnd = true;
            if (j > 0) {
                uint64_t hp = sHi[j - 1], lp = sLo[j - 1];
                uint32_t gp = (uint32_t)(hp >> 48);
                uint64_t kp = (hp << 16) | (lp >> 48);
                if (gp == g) {
                    bnd = (kp != k);
                    if (bnd) lcp[sg.start + pos] = sGD[g] + key_lcp(kp, k, sGF[g]);
                }
            }
            sA[j] = bnd ? pos : 0u;
        }
        __syncthreads();
        block_inclusive_max_inplace<THREADS, ITEMS>(sA, nact, sh_warp);

        // 6. member count of every new group
        for (uint32_t j = tid; j < nact; j += THREADS)
            if (sA[j] == sC[j]) sGM[sC[j]] = 0;
        __syncthreads();
        for (uint32_t j = tid; j < nact; j += THREADS) atomicAdd(&sGM[sA[j]], 1u);
        __syncthreads();

        // 7. classify: single strings and runs of equal strings are final
        uint32_t dnew[ITEMS], fnew[ITEMS];
#pragma unroll
        for (int t = 0; t < ITEMS; ++t) {
            uint32_t j = tid + t * THREADS;
            if (j < nact) {
                dnew[t] = sGD[(uint32_t)(sHi[j] >> 48)];
                fnew[t] = sGF[(uint32_t)(sHi[j] >> 48)];
            }
        }
        __syncthreads();
#pragma unroll
        for (int t = 0; t < ITEMS; ++t) {
            uint32_t j = tid + t * THREADS;
            if (j >= nact) continue;
            uint32_t pos = sC[j];
            uint32_t ng = sA[j];
            uint64_t k = (sHi[j] << 16) | (sLo[j] >> 48);
            uint32_t cnt = sGM[ng];
            if (cnt == 1) {
                sG[pos] = DONE;
            } else if (key_ended(k, fnew[t])) {
                sG[pos] = DONE;
                if (pos != ng) lcp[sg.start + pos] = lens[(uint32_t)sLo[j]];
            } else {
                sG[pos] = ng;
                if (pos == ng) sGD[ng] = dnew[t] + key_v(k, fnew[t]) + fmt_chars(fnew[t]);
            }
        }
        __syncthreads();
    }
    for (uint32_t i = tid; i < m; i += THREADS) perm[sg.start + i] = sV[i];
}

// Segments segs[0 .. count) (count from the device when d_count is given,
// clamped to count), one CTA at a time.
template <int THREADS, int CAP>
__global__ void __launch_bounds__(THREADS) k_finish(const Seg* __restrict__ segs, const uint32_t* __restrict__ d_count,
                                                    uint32_t count, uint32_t* work, const uint8_t* __restrict__ chars,
                                                    const uint64_t* __restrict__ offs,
                                                    const uint32_t* __restrict__ lens, uint32_t* __restrict__ perm,
                                                    uint32_t* __restrict__ lcp, unsigned* err) {
    const uint32_t nseg = d_count ? min(*d_count, count) : count;
    for (uint32_t i = cta_next_unit(work); i < nseg; i = cta_next_unit(work))
        finish_segment<THREADS, CAP>(segs[i], chars, offs, lens, perm, lcp, err);
}

// k_finish held to two CTAs per SM (the 512-thread class: 63 registers)
template <int THREADS, int CAP>
__global__ void __launch_bounds__(THREADS, 2) k_finish2(const Seg* __restrict__ segs, const uint32_t* __restrict__ d_count,
                                                    uint32_t count, uint32_t* work, const uint8_t* __restrict__ chars,
                                                    const uint64_t* __restrict__ offs,
                                                    const uint32_t* __restrict__ lens, uint32_t* __restrict__ perm,
                                                    uint32_t* __restrict__ lcp, unsigned* err) {
    const uint32_t nseg = d_count ? min(*d_count, count) : count;
    for (uint32_t i = cta_next_unit(work); i < nseg; i = cta_next_unit(work))
        finish_segment<THREADS, CAP>(segs[i], chars, offs, lens, perm, lcp, err);
}

// Group finisher: W consecutive lanes of a warp (W = 32, or QUAD_W for the
// shortest segments, 32 / W segments per warp) completely sort one segment of
// <= W strings, lane i of the group holding position i.  Same rounds as the CTA
// finisher (reference-split key of every unfinished member against its group's
// reference, sort by (group, key, index), split), with the sort a bitonic
// network in registers.  Every lane of the warp runs every round (the loop
// ends when no lane of the warp is left unfinished); a group whose segment is
// finished, or that has none (`has` false), carries its lanes along unchanged.
__device__ __forceinline__ void warp_cas128(uint64_t& hi, uint64_t& lo, uint32_t gl, uint32_t j, bool up) {
    uint64_t ohi = __shfl_xor_sync(SSS_FULL, hi, j), olo = __shfl_xor_sync(SSS_FULL, lo, j);
    bool keep_min = (((gl & j) == 0) == up);
    bool other_less = key128_less(ohi, olo, hi, lo);
    if (keep_min ? other_less : key128_less(hi, lo, ohi, olo)) {
        hi = ohi;
        lo = olo;
    }
}

template <int W>
__device__ __forceinline__ void finish_group_segment(const Seg sg, bool has, const uint8_t* __restrict__ chars,
                                                     const uint64_t* __restrict__ offs,
                                                     const uint32_t* __restrict__ lens, uint32_t* __restrict__ perm,
                                                     uint32_t* __restrict__ lcp, unsigned* err) {
    static_assert(W >= 2 && W <= 32 && (W & (W - 1)) == 0, "group width is a power of two <= 32");
    constexpr uint64_t DONE_BIT = 1ull << 47;  // in the low word, above the 32-bit index
    constexpr unsigned WMASK = W == 32 ? ~0u : ((1u << W) - 1u);
    const uint32_t lane = threadIdx.x & 31;
    const uint32_t gl = lane & (W - 1);  // lane within the group
    const uint32_t gb = lane - gl;       // the group's first lane
    const uint32_t m = has ? (sg.size <= (uint32_t)W ? sg.size : (uint32_t)W) : 0u;
    const bool live = gl < m;
    // bitonic span, uniform over the warp: the group width, or for a whole-warp
    // group the next power of two >= m (lanes past it hold padding and sit out)
    const uint32_t span = W < 32 ? (uint32_t)W : (m <= 2u ? 2u : (1u << (32 - __clz((int)(m - 1)))));
    uint32_t e = live ? perm[sg.start + gl] : 0u;
    uint32_t len = live ? lens[e] : 0u;
    uint32_t g = 0, gd = sg.depth, gc = m;  // group start (within the segment), depth, member count
    bool done = !live;
    for (uint32_t iter = 0;; ++iter) {
        if (__ballot_sync(SSS_FULL, !done) == 0) break;
        if (iter > 4u * W + 8u) {
            if (!done) atomicOr(err, ERRBIT_OVERFLOW);
            break;
        }
        // the reference of the lane's group: its longest member, ties broken by
        // a pseudo-random rank (segmented max-scan over the group's lanes; the
        // group's last lane holds the maximum)
        uint64_t best = live ? ((uint64_t)len << 32) | (ref_mix(g, gc, gd, gl + 1u) & 0xFFFFFF00u) | gl : 0ull;
        const uint32_t gs = live ? g : gl;
#pragma unroll
        for (uint32_t o = 1; o < (uint32_t)W; o <<= 1) {
            const uint64_t y = __shfl_up_sync(SSS_FULL, best, o, W);
            if (gl >= gs + o) best = y > best ? y : best;
        }
        best = __shfl_sync(SSS_FULL, best, gb + (live ? g + gc - 1u : gl));
        const uint32_t rlane = (uint32_t)best & 0xFFu;
        const uint32_t r = __shfl_sync(SSS_FULL, e, gb + rlane);
        const uint32_t rl = __shfl_sync(SSS_FULL, len, gb + rlane);
        const uint32_t f = key_fmt(rl, gd);
        uint64_t hi, lo;
        if (!done) {
            const uint8_t* rs = chars + offs[r];
            uint64_t w;
            uint32_t v;
            if (gl == rlane) {
                v = rl > gd ? rl - gd : 0u;
                v = v < VCAP ? v : VCAP;
                w = load_word_be(rs, rl, gd + v);
            } else {
                v = lcp_full_w(chars + offs[e], len, rs, rl, gd, &w);
            }
            uint64_t k = ref_key(v, w, (uint32_t)(load_word_be(rs, rl, gd + v) >> 56), f);
            hi = ((uint64_t)g << 48) | (k >> 16);
            lo = (k << 48) | (uint64_t)e;
        } else if (live) {
            hi = (uint64_t)gl << 48;  // a finished string is the only member of group `gl`
            lo = DONE_BIT | (uint64_t)e;
        } else {
            hi = ~0ull;
            lo = ~0ull;
        }
        for (uint32_t kk = 2; kk <= span; kk <<= 1) {
            const bool up = (gl & kk) == 0 || kk == span;
            for (uint32_t j = kk >> 1; j > 0; j >>= 1) warp_cas128(hi, lo, gl, j, up);
        }
        // lane j of the group now holds position j; groups kept their ranges
        const uint32_t gg = (uint32_t)(hi >> 48);
        const uint64_t k = (hi << 16) | (lo >> 48);
        const bool fin = !live || (lo & DONE_BIT);
        e = (uint32_t)lo;
        len = live ? lens[e] : 0u;
        const uint64_t hp = __shfl_up_sync(SSS_FULL, hi, 1, W), lp = __shfl_up_sync(SSS_FULL, lo, 1, W);
        const uint32_t gp = (uint32_t)(hp >> 48);
        const uint64_t kp = (hp << 16) | (lp >> 48);
        bool bnd = true;
        if (gl > 0 && !fin && gp == gg && !(lp & DONE_BIT)) {
            bnd = (kp != k);
            if (bnd) lcp[sg.start + gl] = gd + key_lcp(kp, k, f);
        }
        // new group start: inclusive max-scan of boundary positions
        uint32_t ng = bnd ? gl : 0u;
#pragma unroll
        for (uint32_t o = 1; o < (uint32_t)W; o <<= 1) {
            uint32_t y = __shfl_up_sync(SSS_FULL, ng, o, W);
            if (gl >= o) ng = ng > y ? ng : y;
        }
        const unsigned bm = (__ballot_sync(SSS_FULL, bnd) >> gb) & WMASK;
        const unsigned after = gl < (uint32_t)W - 1u ? (bm & (~0u << (gl + 1))) : 0u;
        const uint32_t end = after ? (uint32_t)(__ffs(after) - 1) : m;
        const uint32_t cnt = (end > ng ? end : ng + 1) - ng;
        if (!fin) {
            if (cnt == 1) {
                done = true;
            } else if (key_ended(k, f)) {
                done = true;
                if (gl != ng) lcp[sg.start + gl] = len;
            } else {
                done = false;
                g = ng;
                gc = cnt;
                gd = gd + key_v(k, f) + fmt_chars(f);
            }
        } else {
            done = true;
            g = gl;
            gc = 1;
        }
    }
    if (live) perm[sg.start + gl] = e;
}

// Short segments, 32 / W per warp: segment i is segs[i] (top == 0) or
// segs[top - 1 - i] (a list filled from the top of its array); count from the
// device when d_count is given, clamped to count.  d_other, when given, is the
// count of the list that fills the same array from the other end: the two must
// not overlap.
template <int W>
__global__ void __launch_bounds__(32 * WF_WARPS) k_finish_group(const Seg* __restrict__ segs,
                                                                const uint32_t* __restrict__ d_count,
                                                                const uint32_t* __restrict__ d_other, uint32_t count,
                                                                uint32_t top, uint32_t* work,
                                                                const uint8_t* __restrict__ chars,
                                                                const uint64_t* __restrict__ offs,
                                                                const uint32_t* __restrict__ lens,
                                                                uint32_t* __restrict__ perm,
                                                                uint32_t* __restrict__ lcp, unsigned* err) {
    constexpr uint32_t G = 32u / W;
    uint32_t nseg = d_count ? min(*d_count, count) : count;
    if (d_count && d_other && (uint64_t)*d_count + *d_other > count) {
        if (threadIdx.x == 0) atomicOr(err, ERRBIT_OVERFLOW);
        nseg = 0;
    }
    const uint32_t lane = threadIdx.x & 31;
    for (;;) {
        uint32_t i0 = 0;
        if (lane == 0) i0 = atomicAdd(work, G);
        i0 = __shfl_sync(SSS_FULL, i0, 0);
        if (i0 >= nseg) break;
        const uint32_t i = i0 + lane / W;
        const bool has = i < nseg;
        const Seg sg = has ? segs[top ? top - 1u - i : i] : Seg{0, 0, 0, 0};
        finish_group_segment<W>(sg, has, chars, offs, lens, perm, lcp, err);
    }
}

constexpr size_t finish_smem(int cap) { return (size_t)cap * (8 + 8 + 4 * 7); }
// sort_emit: keys, values (64-bit), two 32-bit arrays
constexpr size_t emit_smem(int, int cap) { return (size_t)cap * (8 + 8 + 4 + 4); }

// ---------------------------------------------------------------------------
// Large path.
// the uncached LCP scan, kept out of line: it is the rare path of k_lg_ext
// (shared prefixes longer than the 512 cached reference characters)
__device__ __noinline__ uint32_t lcp_full_w_outline(const uint8_t* a, uint32_t la, const uint8_t* b, uint32_t lb,
                                                    uint32_t d, uint64_t* w) {
    return lcp_full_w(a, la, b, lb, d, w);
}

__device__ __forceinline__ void lg_ext_tile(const LgTile tl, const LgSegInfo* __restrict__ info,
                                            const uint8_t* __restrict__ chars, const uint64_t* __restrict__ offs,
                                            const uint32_t* __restrict__ lens, const uint32_t* __restrict__ perm,
                                            uint64_t* __restrict__ K, uint32_t* __restrict__ segfmt) {
    constexpr uint32_t NREF = 68;  // 64 words (512 chars) plus a 4-word block of slack
    __shared__ uint64_t refw[NREF];
    __shared__ uint32_t s_refpos;
    LgSegInfo si = info[tl.s];
    const uint32_t d = si.seg.depth;
    // The reference of a large segment: the longest of REF_CAND pseudo-random
    // members (the earliest candidate on ties).  A member's LCP with the
    // reference is capped by the reference's length, so a short reference
    // leaves every longer member that shares its whole remainder in one group,
    // and an input whose shared prefixes grow with the length (nested copies of
    // one template) then sheds only a fraction of the segment per round.
    if (threadIdx.x < 32) {
        constexpr uint32_t REF_CAND = 8;
        const uint32_t t = threadIdx.x;
        uint64_t best = 0;
        uint32_t pos = si.seg.start;
        if (t < REF_CAND) {
            pos = si.seg.start + ref_pick(si.seg.start, si.seg.size, d, t);
            best = ((uint64_t)lens[perm[pos]] << 32) | (uint64_t)(REF_CAND - t);
        }
#pragma unroll
        for (uint32_t o = 16; o > 0; o >>= 1) {
            uint64_t ob = __shfl_xor_sync(SSS_FULL, best, o);
            best = ob > best ? ob : best;
        }
        const uint32_t win = REF_CAND - (uint32_t)best;  // the winning candidate's t
        const uint32_t wpos = __shfl_sync(SSS_FULL, pos, win);
        if (t == 0) s_refpos = wpos;
    }
    __syncthreads();
    const uint32_t refpos = s_refpos;
    uint32_t r = perm[refpos];
    const uint8_t* rs = chars + offs[r];
    uint32_t rl = lens[r];
    const uint32_t f = key_fmt(rl, d);
    if (threadIdx.x == 0 && tl.begin == si.seg.start) segfmt[tl.s] = f;
    for (uint32_t i = threadIdx.x; i < NREF; i += LG_T) refw[i] = load_word_be(rs, rl, d + 8 * i);
    __syncthreads();
    for (uint32_t q = tl.begin + threadIdx.x; q < tl.end; q += LG_T) {
        uint64_t w;
        uint32_t v;
        if (q == refpos) {
            v = rl > d ? rl - d : 0u;
            v = v < VCAP ? v : VCAP;
            w = load_word_be(rs, rl, d + v);
        } else {
            uint32_t e = perm[q];
            uint32_t le = lens[e];
            uint32_t mlen = le < rl ? le : rl;
            v = (mlen <= d + 8 * (NREF - 4)) ? lcp_full_w_ref(chars + offs[e], le, rl, refw, d, &w)
                                             : lcp_full_w_outline(chars + offs[e], le, rs, rl, d, &w);
        }
        uint32_t rho = (v >> 3) < NREF ? (uint32_t)(refw[v >> 3] >> (56 - 8 * (v & 7))) & 0xFFu
                                       : (uint32_t)(load_word_be(rs, rl, d + v) >> 56);
        K[q] = ref_key(v, w, rho, f);
    }
}

__global__ void __launch_bounds__(LG_T, 6) k_lg_ext(const LsPlan* __restrict__ plan, const LgTile* __restrict__ tiles,
                                                 const LgSegInfo* __restrict__ info,
                                                 const uint8_t* __restrict__ chars, const uint64_t* __restrict__ offs,
                                                 const uint32_t* __restrict__ lens, const uint32_t* __restrict__ perm,
                                                 uint64_t* __restrict__ K, uint32_t* __restrict__ segfmt) {
    const uint32_t nt = plan->ntiles;
    for (uint32_t g = blockIdx.x; g < nt; g += gridDim.x) {
        __syncthreads();
        lg_ext_tile(tiles[g], info, chars, offs, lens, perm, K, segfmt);
    }
}

// Sort positions [bs, bs+m) (m <= CAP) by (key, index) in one CTA, write the
// keys and indices back, set the LCP at every key change (d + key_lcp) and emit
// the groups of equal keys: runs of equal strings get lcp = length, other groups
// become segments at depth d + v + C.  The first position's LCP is left alone.
// Reads srcK/srcV fully before writing K/perm.
template <int THREADS, int CAP>
__device__ void sort_emit(unsigned char* smem, uint32_t bs, uint32_t m, uint32_t d, uint32_t f, const uint64_t* srcK,
                          const uint32_t* srcV, const uint32_t* __restrict__ lens, uint64_t* K, uint32_t* perm,
                          uint32_t* __restrict__ lcp, const SegLists& L, unsigned* err) {
    constexpr int ITEMS = CAP / THREADS;
    uint64_t* sHi = reinterpret_cast<uint64_t*>(smem);
    uint64_t* sLo = sHi + CAP;
    uint32_t* sA = reinterpret_cast<uint32_t*>(sLo + CAP);
    uint32_t* sN = sA + CAP;
    __shared__ uint32_t sh_warp[32];
    for (uint32_t i = threadIdx.x; i < m; i += THREADS) {
        sHi[i] = srcK[bs + i];
        sA[i] = srcV[bs + i];
    }
    __syncthreads();
    // A segment's members arrive in index order (every sort of an earlier round
    // breaks ties by index, and the partition scatter keeps the order): then a
    // stable sort by the key alone yields (key, index) order.  Checked; the
    // 128-bit merge sort of (key, index) otherwise.
    bool ordered = true;
    for (uint32_t i = threadIdx.x + 1; i < m; i += THREADS) ordered = ordered && sA[i - 1] < sA[i];
    if (__syncthreads_and(ordered)) {
        block_merge_sort_kv_fit<THREADS, ITEMS>(sHi, sA, m);
        for (uint32_t i = threadIdx.x; i < m; i += THREADS) sLo[i] = sA[i];
        __syncthreads();
    } else {
        for (uint32_t i = threadIdx.x; i < m; i += THREADS) sLo[i] = sA[i];
        __syncthreads();
        block_merge_sort128_fit<THREADS, ITEMS>(sHi, sLo, m);
    }
    for (uint32_t i = threadIdx.x; i < CAP; i += THREADS) {
        uint32_t v = 0;
        if (i < m) {
            uint64_t k = sHi[i];
            K[bs + i] = k;
            perm[bs + i] = (uint32_t)sLo[i];
            bool bnd = (i == 0) || (sHi[i - 1] != k);
            if (bnd && i > 0) lcp[bs + i] = d + key_lcp(sHi[i - 1], k, f);
            v = bnd ? i : 0u;
        }
        sA[i] = v;
    }
    __syncthreads();
    block_inclusive_max_inplace<THREADS, ITEMS>(sA, m, sh_warp);  // sA[i] = first index of i's group
    // group sizes at the group's first index, written by the group's last member
    // (no atomics: a group of equal keys may hold the whole segment)
    for (uint32_t i = threadIdx.x; i < m; i += THREADS)
        if (i + 1 == m || sA[i + 1] == i + 1) sN[sA[i]] = i + 1 - sA[i];
    __syncthreads();
    for (uint32_t i0 = 0; i0 < m; i0 += THREADS) {  // uniform trip count: push_seg_warp needs whole warps
        const uint32_t i = i0 + threadIdx.x;
        bool want = false;
        uint32_t c = 0, dn = 0;
        if (i < m) {
            const uint32_t g = sA[i];
            c = sN[g];
            if (c >= 2) {
                const uint64_t k = sHi[i];
                if (key_ended(k, f)) {
                    if (i != g) lcp[bs + i] = lens[(uint32_t)sLo[i]];
                } else if (i == g) {
                    want = true;
                    dn = d + key_v(k, f) + fmt_chars(f);
                }
            }
        }
        push_seg_warp(L, want, bs + i, c, dn, err);
    }
}

// One CTA per (segment, bucket).  Range buckets are sorted in shared memory;
// groups of equal keys become new segments at depth d + v + C.
template <int THREADS, int CAP>
__device__ __forceinline__ void lg_bucket(uint32_t g, uint32_t ns, const LgSegInfo* __restrict__ info,
                                          const uint32_t* __restrict__ bst, const uint32_t* __restrict__ segfmt,
                                          const uint64_t* __restrict__ tK, const uint32_t* __restrict__ tV,
                                          const uint32_t* __restrict__ lens, uint64_t* __restrict__ K,
                                          uint32_t* __restrict__ perm, uint32_t* __restrict__ lcp, const SegLists& L,
                                          unsigned* err, uint8_t* __restrict__ fixmark) {
    extern __shared__ __align__(16) unsigned char smem[];
    const uint32_t sidx = segment_of_bucket(info, ns, g);
    LgSegInfo si = info[sidx];
    uint32_t b = g - si.bk_base;
    uint32_t nbk = 2 * si.nb - 1;
    if (b >= nbk) return;
    uint32_t bs = bst[si.bst_base + b], be = bst[si.bst_base + b + 1];
    if (bs < si.seg.start || be > si.seg.start + si.seg.size || be < bs) {
        if (threadIdx.x == 0) atomicOr(err, ERRBIT_OVERFLOW);
        return;
    }
    uint32_t m = be - bs;
    if (m == 0) return;
    uint32_t d = si.seg.depth;
    const uint32_t f = segfmt[sidx];
    bool eq = (b & 1u) != 0;
    if (eq || m > (uint32_t)CAP) {
        for (uint32_t q = bs + threadIdx.x; q < be; q += THREADS) {
            K[q] = tK[q];
            perm[q] = tV[q];
        }
        if (threadIdx.x == 0) {
            if (eq) {
                uint64_t k = tK[bs];
                if (m >= 2 && !key_ended(k, f)) push_seg(L, bs, m, d + key_v(k, f) + fmt_chars(f), err);
            } else {
                // oversized range bucket: another round at this depth.  Its members
                // have distinct keys, so the LCPs across its two ends depend on which
                // members end up first and last: recomputed after the last round.
                push_seg(L, bs, m, d, err);
                if (bs > si.seg.start) fixmark[bs] = 1;
                if (be < si.seg.start + si.seg.size) fixmark[be] = 1;
            }
        }
        if (eq && m >= 2 && key_ended(tK[bs], f)) {
            // a run of equal strings: lcp = length inside the run
            for (uint32_t q = bs + 1 + threadIdx.x; q < be; q += THREADS) lcp[q] = lens[tV[q]];
        }
        return;
    }
    sort_emit<THREADS, CAP>(smem, bs, m, d, f, tK, tV, lens, K, perm, lcp, L, err);
}

template <int THREADS, int CAP>
__global__ void __launch_bounds__(THREADS, 65536 / (64 * THREADS)) k_lg_buckets(const LsPlan* __restrict__ plan,
                                                     const LgSegInfo* __restrict__ info,
                                                     const uint32_t* __restrict__ bst,
                                                     const uint32_t* __restrict__ segfmt,
                                                     const uint64_t* __restrict__ tK, const uint32_t* __restrict__ tV,
                                                     const uint32_t* __restrict__ lens, uint64_t* __restrict__ K,
                                                     uint32_t* __restrict__ perm, uint32_t* __restrict__ lcp,
                                                     SegLists L, unsigned* err, uint8_t* __restrict__ fixmark,
                                                     uint32_t* work) {
    const uint32_t nb = plan->pbuckets, npart = plan->npart;
    for (uint32_t g = cta_next_unit(work); g < nb; g = cta_next_unit(work))
        lg_bucket<THREADS, CAP>(g, npart, info, bst, segfmt, tK, tV, lens, K, perm, lcp, L, err, fixmark);
}

// Large segments of at most DIRECT_CAP strings: one CTA sorts the whole segment
// by its keys (no sampling, classification or scatter).
// (segments of more than min_size strings; CAP bounds the size)
template <int THREADS, int CAP>
__global__ void __launch_bounds__(THREADS) k_lg_direct(const LsPlan* __restrict__ plan,
                                                       const LgSegInfo* __restrict__ info,
                                                       const uint32_t* __restrict__ segfmt,
                                                       const uint32_t* __restrict__ lens, uint64_t* __restrict__ K,
                                                       uint32_t* __restrict__ perm, uint32_t* __restrict__ lcp,
                                                       SegLists L, unsigned* err, uint32_t* work, uint32_t min_size) {
    extern __shared__ __align__(16) unsigned char smem[];
    const uint32_t ns = plan->ns, npart = plan->npart;
    for (uint32_t sidx = npart + cta_next_unit(work); sidx < ns; sidx = npart + cta_next_unit(work)) {
        const LgSegInfo si = info[sidx];
        if (si.seg.size <= min_size || si.seg.size > (uint32_t)CAP) continue;
        sort_emit<THREADS, CAP>(smem, si.seg.start, si.seg.size, si.seg.depth, segfmt[sidx], K, perm, lens, K, perm,
                                lcp, L, err);
    }
}

// LCP at the first position of every non-first, non-empty bucket.
__global__ void __launch_bounds__(512) k_lg_seams(const LsPlan* __restrict__ plan, const LgSegInfo* __restrict__ info,
                                                  const uint32_t* __restrict__ bst, const uint32_t* __restrict__ segfmt,
                                                  const uint64_t* __restrict__ K, uint32_t* __restrict__ lcp) {
    const uint32_t npart = plan->npart;
    for (uint32_t s = blockIdx.x; s < npart; s += gridDim.x) {
        LgSegInfo si = info[s];
        uint32_t nbk = 2 * si.nb - 1;
        uint32_t d = si.seg.depth;
        const uint32_t f = segfmt[s];
        for (uint32_t b = threadIdx.x; b < nbk; b += 512) {
            uint32_t bs = bst[si.bst_base + b], be = bst[si.bst_base + b + 1];
            if (be > bs && bs > si.seg.start && be <= si.seg.start + si.seg.size)
                lcp[bs] = d + key_lcp(K[bs - 1], K[bs], f);
        }
    }
}

// LCP with the predecessor at the positions marked by k_lg_buckets, from the
// final order (full comparison; there are at most two per oversized bucket).
__global__ void k_fix_seams(const uint8_t* __restrict__ fixmark, uint32_t n, const uint8_t* __restrict__ chars,
                            const uint64_t* __restrict__ offs, const uint32_t* __restrict__ lens,
                            const uint32_t* __restrict__ perm, uint32_t* __restrict__ lcp) {
    for (uint32_t q = blockIdx.x * blockDim.x + threadIdx.x; q < n; q += gridDim.x * blockDim.x) {
        if (!fixmark[q] || q == 0) continue;
        uint32_t a = perm[q - 1], b = perm[q];
        uint32_t la = lens[a], lb = lens[b];
        uint32_t m = la < lb ? la : lb;
        WordStream A, B;
        A.init(chars + offs[a], la, 0);
        B.init(chars + offs[b], lb, 0);
        uint32_t r = m;
        for (uint32_t k = 0; k < m; k += 8) {
            uint64_t x = A.next() ^ B.next();
            if (x) {
                uint32_t c = k + ((uint32_t)__clzll((long long)x) >> 3);
                r = c < m ? c : m;
                break;
            }
        }
        lcp[q] = r;
    }
}

__global__ void k_dist(const uint32_t* __restrict__ lens, uint32_t n, const uint32_t* __restrict__ perm,
                       const uint32_t* __restrict__ lcp, uint32_t* __restrict__ dist) {
    uint32_t r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    uint32_t left = r > 0 ? lcp[r] : 0;
    uint32_t right = r + 1 < n ? lcp[r + 1] : 0;
    uint32_t m = left > right ? left : right;
    uint32_t i = perm[r];
    uint64_t d = (uint64_t)m + 1;
    dist[i] = d < lens[i] ? (uint32_t)d : lens[i];
}

__global__ void k_check_input(const uint8_t* __restrict__ chars, uint64_t n_chars, const uint64_t* __restrict__ offs,
                              const uint32_t* __restrict__ lens, uint32_t n, unsigned* err) {
    uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    uint64_t o = offs[i];
    uint32_t l = lens[i];
    if (o > n_chars || (uint64_t)l > n_chars - o || l >= 0x80000000u) {
        atomicOr(err, ERRBIT_CHECK);
        return;
    }
    for (uint32_t k = 0; k < l; ++k)
        if (chars[o + k] == 0) {
            atomicOr(err, ERRBIT_CHECK);
            return;
        }
}

// Work memory layout of the local sort.
struct LsBufs {
    uint64_t* K;
    uint64_t* tK;
    uint32_t* tV;
    Seg* warp;
    Seg* tiny;
    Seg* small;
    Seg* med;
    Seg* large;
    uint32_t* cnt;
    uint32_t* work;  // dynamic work counters: [0] warp, [1] tiny, [2] med, [3] buckets, [4] direct
    uint32_t* segfmt;
    uint8_t* fixmark;
    SpBufs sp;
    uint32_t cap_warp, cap_tiny, cap_small, cap_med, cap_large;
};

// The size-class knobs of the local sort; 0 (e.g. internal callers passing
// sss_params{}) means the default.  Values are clamped by the API already.
struct LsKnobs {
    uint32_t warp_cap, cta_cap, direct_cap, bucket_target;
};
static LsKnobs ls_knobs(const sss_params& prm) {
    LsKnobs k;
    k.warp_cap = prm.warp_cap ? std::min(prm.warp_cap, 32u) : 32u;
    k.cta_cap = prm.cta_cap ? std::min(std::max(prm.cta_cap, (uint32_t)TINY_CAP), (uint32_t)MED_CAP) : (uint32_t)MED_CAP;
    k.direct_cap = prm.direct_cap ? std::min(std::max(prm.direct_cap, k.cta_cap), (uint32_t)DIRECT_CAP)
                                  : (uint32_t)DIRECT_CAP;
    k.bucket_target = prm.bucket_target ? std::min(std::max(prm.bucket_target, 256u), (uint32_t)BK_CAP) : 2048u;
    return k;
}

void carve_ls(Arena& ar, uint32_t n, uint32_t p, const sss_params& prm, LsBufs& b) {
    const LsKnobs kn = ls_knobs(prm);
    b.cap_warp = n / 2 + 2;
    b.cap_tiny = n / (kn.warp_cap + 1) + 2;
    b.cap_small = n / (TINY_CAP + 1) + 2;
    b.cap_med = n / (SM_CAP + 1) + 2;
    b.cap_large = n / (kn.cta_cap + 1) + p + 2;  // every large segment holds > cta_cap strings
    b.K = ar.take<uint64_t>(n);
    b.tK = ar.take<uint64_t>(n);
    b.tV = ar.take<uint32_t>(n);
    b.warp = ar.take<Seg>(b.cap_warp);
    b.tiny = ar.take<Seg>(b.cap_tiny);
    b.small = ar.take<Seg>(b.cap_small);
    b.med = ar.take<Seg>(b.cap_med);
    b.large = ar.take<Seg>(b.cap_large);
    b.cnt = ar.take<uint32_t>(8);
    b.work = ar.take<uint32_t>(8);
    b.segfmt = ar.take<uint32_t>(b.cap_large);
    b.fixmark = ar.take<uint8_t>(n);
    carve_sp(ar, n, b.cap_large, b.sp);
}

// The finishers over their lists: host counts, or (d_cnt != NULL) the device
// counters of the round that just ran (d_cnt[5] quad, [3] warp, [0] tiny,
// [4] small, [1] med).
sss_status run_finishers(sss_ctx* ctx, const LsBufs& B, const uint32_t* d_cnt, uint32_t nquad, uint32_t nwarp,
                         uint32_t ntiny, uint32_t nsmall, uint32_t nmed, const StrIn& in, uint32_t* perm,
                         uint32_t* lcp) {
    const uint32_t sm = (uint32_t)std::max(1, ctx->sm_count);
    uint32_t gq, gw, gt, gs, gm;
    if (d_cnt) {
        nquad = nwarp = B.cap_warp;
        ntiny = B.cap_tiny;
        nsmall = B.cap_small;
        nmed = B.cap_med;
        gq = sm * 8;
        gw = sm * 8;
        gt = sm * 16;
        gs = sm * 8;
        gm = sm * 2;
    } else {
        if ((uint64_t)nquad + nwarp > B.cap_warp) return sss_fail(ctx, SSS_ERR_CUDA, "local sort: internal capacity exceeded");
        const uint32_t qpb = WF_WARPS * (32 / QUAD_W);  // quad segments per CTA step
        gq = std::min((nquad + qpb - 1) / qpb, sm * 8);
        gw = std::min((nwarp + WF_WARPS - 1) / WF_WARPS, sm * 16);
        gt = std::min(ntiny, sm * 32);
        gs = std::min(nsmall, sm * 16);
        gm = std::min(nmed, sm * 4);
    }
    SSS_TRY(sss_launch(ctx, "ls_finish_quad", k_finish_group<QUAD_W>, dim3(gq), dim3(32 * WF_WARPS), 0,
                       (const Seg*)B.warp, d_cnt ? d_cnt + 5 : (const uint32_t*)nullptr,
                       d_cnt ? d_cnt + 3 : (const uint32_t*)nullptr, nquad, 0u, B.work + 4, in.chars, in.offs,
                       in.lens, perm, lcp, ctx->d_err));
    SSS_TRY(sss_launch(ctx, "ls_finish_warp", k_finish_group<32>, dim3(gw), dim3(32 * WF_WARPS), 0,
                       (const Seg*)B.warp, d_cnt ? d_cnt + 3 : (const uint32_t*)nullptr,
                       (const uint32_t*)nullptr, nwarp, B.cap_warp, B.work + 0, in.chars, in.offs, in.lens, perm,
                       lcp, ctx->d_err));
    SSS_TRY(sss_launch(ctx, "ls_finish_tiny", k_finish<TINY_T, TINY_CAP>, dim3(gt), dim3(TINY_T),
                       finish_smem(TINY_CAP), (const Seg*)B.tiny, d_cnt ? d_cnt + 0 : (const uint32_t*)nullptr, ntiny,
                       B.work + 1, in.chars, in.offs, in.lens, perm, lcp, ctx->d_err));
    SSS_TRY(sss_launch(ctx, "ls_finish_small", k_finish<SM_T, SM_CAP>, dim3(gs), dim3(SM_T), finish_smem(SM_CAP),
                       (const Seg*)B.small, d_cnt ? d_cnt + 4 : (const uint32_t*)nullptr, nsmall, B.work + 6, in.chars,
                       in.offs, in.lens, perm, lcp, ctx->d_err));
    SSS_TRY(sss_launch(ctx, "ls_finish_cta", k_finish2<MED_T, MED_CAP>, dim3(gm), dim3(MED_T), finish_smem(MED_CAP),
                       (const Seg*)B.med, d_cnt ? d_cnt + 1 : (const uint32_t*)nullptr, nmed, B.work + 2, in.chars,
                       in.offs, in.lens, perm, lcp, ctx->d_err));
    return SSS_OK;
}

}  // namespace

size_t need_local_sort(uint32_t n, uint32_t p, const sss_params& prm) {
    Arena ar;
    LsBufs b;
    carve_ls(ar, n, p, prm, b);
    return ar.off + 256;
}

static bool g_attr_done[64];

static sss_status set_ls_attributes(sss_ctx* ctx) {
    if (!g_attr_done[ctx->device & 63]) {
        SSS_CUDA(cudaFuncSetAttribute(k_finish2<MED_T, MED_CAP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)finish_smem(MED_CAP)));
        SSS_CUDA(cudaFuncSetAttribute(k_finish<TINY_T, TINY_CAP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)finish_smem(TINY_CAP)));
        SSS_CUDA(cudaFuncSetAttribute(k_finish<SM_T, SM_CAP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)finish_smem(SM_CAP)));
        SSS_CUDA(cudaFuncSetAttribute(k_lg_buckets<BK_T, BK_CAP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)emit_smem(BK_T, BK_CAP)));
        SSS_CUDA(cudaFuncSetAttribute(k_lg_buckets<BKS_T, BKS_CAP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)emit_smem(BKS_T, BKS_CAP)));
        SSS_CUDA(cudaFuncSetAttribute(k_lg_direct<DIRECT_T, DIRECT_CAP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)emit_smem(DIRECT_T, DIRECT_CAP)));
        g_attr_done[ctx->device & 63] = true;
    }
    return SSS_OK;
}

sss_status impl_local_sort(sss_ctx* ctx, Arena& ar, const StrIn& in, uint32_t p, const sss_params& prm,
                           uint32_t* perm, uint32_t* lcp) {
    std::vector<Seg> init;
    for (uint32_t i = 0; i < p; ++i) {
        uint32_t lo = part_lo(in.n, p, i), hi = part_lo(in.n, p, i + 1);
        init.push_back(Seg{lo, hi - lo, 0, 0});
    }
    return impl_sort_segments(ctx, ar, in, init, prm, perm, lcp);
}

// One round of the multi-CTA path, planned on the device from the segments the
// previous round pushed: keys, partition of the large segments, bucket sorts,
// seams, whole-segment sorts, then the finishers of every segment pushed.
static sss_status launch_round(sss_ctx* ctx, const LsBufs& B, const LsKnobs& kn, const SegLists& L,
                               const StrIn& in, uint32_t* perm, uint32_t* lcp) {
    const uint32_t sm = (uint32_t)std::max(1, ctx->sm_count);
    SSS_TRY(sss_launch(ctx, "ls_lg_plan", k_lg_plan, dim3(1), dim3(1024), 0, (const Seg*)B.large, B.cnt, B.work,
                       kn.direct_cap, kn.bucket_target, B.sp.cap_segs, B.sp.cap_tiles, B.sp.cap_hist, B.sp.info,
                       B.sp.plan, ctx->d_err));
    SSS_TRY(sss_launch(ctx, "ls_lg_tiles", k_lg_tiles, dim3(sm * 4), dim3(256), 0, (const LsPlan*)B.sp.plan,
                       (const LgSegInfo*)B.sp.info, B.sp.tiles));
    SSS_TRY(sss_launch(ctx, "ls_lg_ext", k_lg_ext, dim3(sm * 6), dim3(LG_T), 0, (const LsPlan*)B.sp.plan,
                       (const LgTile*)B.sp.tiles, (const LgSegInfo*)B.sp.info, in.chars, in.offs, in.lens,
                       (const uint32_t*)perm, B.K, B.segfmt));
    SSS_TRY(launch_sp(ctx, B.sp, B.K, perm, B.tK, B.tV, "ls_lg_samples", "ls_lg_classify", "ls_lg_offsets",
                      "ls_lg_scatter"));
    if (kn.bucket_target <= (uint32_t)BKS_CAP / 2) {
        SSS_TRY(sss_launch(ctx, "ls_lg_buckets", k_lg_buckets<BKS_T, BKS_CAP>, dim3(sm * 4), dim3(BKS_T),
                           emit_smem(BKS_T, BKS_CAP), (const LsPlan*)B.sp.plan, (const LgSegInfo*)B.sp.info,
                           (const uint32_t*)B.sp.bst, (const uint32_t*)B.segfmt, (const uint64_t*)B.tK,
                           (const uint32_t*)B.tV, in.lens, B.K, perm, lcp, L, ctx->d_err, B.fixmark, B.work + 3));
    } else {
        SSS_TRY(sss_launch(ctx, "ls_lg_buckets", k_lg_buckets<BK_T, BK_CAP>, dim3(sm * 2), dim3(BK_T),
                           emit_smem(BK_T, BK_CAP), (const LsPlan*)B.sp.plan, (const LgSegInfo*)B.sp.info,
                           (const uint32_t*)B.sp.bst, (const uint32_t*)B.segfmt, (const uint64_t*)B.tK,
                           (const uint32_t*)B.tV, in.lens, B.K, perm, lcp, L, ctx->d_err, B.fixmark, B.work + 3));
    }
    SSS_TRY(sss_launch(ctx, "ls_lg_seams", k_lg_seams, dim3(sm * 2), dim3(512), 0, (const LsPlan*)B.sp.plan,
                       (const LgSegInfo*)B.sp.info, (const uint32_t*)B.sp.bst, (const uint32_t*)B.segfmt,
                       (const uint64_t*)B.K, lcp));
    SSS_TRY(sss_launch(ctx, "ls_lg_direct", k_lg_direct<DIRECT_T, DIRECT_CAP>, dim3(sm), dim3(DIRECT_T),
                       emit_smem(DIRECT_T, DIRECT_CAP), (const LsPlan*)B.sp.plan, (const LgSegInfo*)B.sp.info,
                       (const uint32_t*)B.segfmt, in.lens, B.K, perm, lcp, L, ctx->d_err, B.work + 5, 0u));
    return run_finishers(ctx, B, B.cnt, 0, 0, 0, 0, 0, in, perm, lcp);
}

// Loop condition of the captured round loop: another round while segments were
// pushed, the round limit is not reached and no capacity error occurred.
__global__ void k_ls_cond(const uint32_t* __restrict__ cnt, uint32_t* rounds, uint32_t limit, unsigned* err,
                          cudaGraphConditionalHandle h) {
    const uint32_t r = ++*rounds;
    bool more = cnt[2] > 0;
    if (more && r >= limit) {
        atomicOr(err, ERRBIT_OVERFLOW);
        more = false;
    }
    if (*(volatile unsigned*)err & ERRBIT_OVERFLOW) more = false;
    cudaGraphSetConditional(h, more ? 1u : 0u);
}

// The round loop as one graph launch: a while node whose body is one round plus
// k_ls_cond.  Built on first use and kept in the context (a few graphs, least
// recently used replaced) under a key of every pointer and size its kernels take.
static sss_status run_rounds_graph(sss_ctx* ctx, const LsBufs& B, const LsKnobs& kn, const SegLists& L,
                                   const StrIn& in, uint32_t* perm, uint32_t* lcp, uint32_t limit) {
    char keyb[512];
    std::snprintf(keyb, sizeof(keyb), "%p %p %p %u %p %p %p %p %p %u %u %u %u %d %u", (const void*)in.chars,
                  (const void*)in.offs, (const void*)in.lens, in.n, (void*)perm, (void*)lcp, (void*)B.K,
                  (void*)B.large, (void*)B.sp.plan, kn.warp_cap, kn.cta_cap, kn.direct_cap, kn.bucket_target,
                  ctx->sm_count, limit);
    uint32_t* rounds = reinterpret_cast<uint32_t*>(ctx->d_err) + 1;  // a spare word of the context
    sss_ctx::LsGraph* slot = nullptr;
    for (auto& lg : ctx->ls_graphs)
        if (lg.exec && lg.key == keyb) slot = &lg;
    if (!slot) {
        slot = &ctx->ls_graphs[0];  // an empty entry, else the least recently used
        for (auto& lg : ctx->ls_graphs)
            if (!lg.exec ? slot->exec != nullptr : (slot->exec && lg.used < slot->used)) slot = &lg;
        if (slot->exec) cudaGraphExecDestroy(slot->exec);
        if (slot->graph) cudaGraphDestroy(slot->graph);
        slot->exec = nullptr;
        slot->graph = nullptr;
        slot->key.clear();
        if (!ctx->cap_stream) SSS_CUDA(cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking));
        cudaGraph_t g;
        SSS_CUDA(cudaGraphCreate(&g, 0));
        cudaGraphConditionalHandle h;
        SSS_CUDA(cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault));
        cudaGraphNodeParams cp{};
        cp.type = cudaGraphNodeTypeConditional;
        cp.conditional.handle = h;
        cp.conditional.type = cudaGraphCondTypeWhile;
        cp.conditional.size = 1;
        cudaGraphNode_t node;
        SSS_CUDA(cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &cp));
        cudaGraph_t body = cp.conditional.phGraph_out[0];
        cudaStream_t saved = ctx->stream;
        ctx->stream = ctx->cap_stream;
        ctx->capturing = true;
        sss_status st = SSS_OK;
        cudaError_t ce = cudaStreamBeginCaptureToGraph(ctx->cap_stream, body, nullptr, nullptr, 0,
                                                       cudaStreamCaptureModeThreadLocal);
        if (ce == cudaSuccess) {
            st = launch_round(ctx, B, kn, L, in, perm, lcp);
            if (st == SSS_OK)
                st = sss_launch(ctx, "ls_cond", k_ls_cond, dim3(1), dim3(1), 0, (const uint32_t*)B.cnt, rounds, limit,
                                ctx->d_err, h);
            cudaGraph_t out = body;
            cudaError_t ee = cudaStreamEndCapture(ctx->cap_stream, &out);
            if (ce == cudaSuccess) ce = ee;
        }
        ctx->capturing = false;
        ctx->stream = saved;
        if (st != SSS_OK || ce != cudaSuccess) {
            cudaGetLastError();
            cudaGraphDestroy(g);
            return st != SSS_OK ? st : sss_fail(ctx, SSS_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(ce));
        }
        cudaGraphExec_t ex;
        ce = cudaGraphInstantiate(&ex, g, 0);
        if (ce != cudaSuccess) {
            cudaGetLastError();
            cudaGraphDestroy(g);
            return sss_fail(ctx, SSS_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(ce));
        }
        slot->graph = g;
        slot->exec = ex;
        slot->key = keyb;
    }
    slot->used = ++ctx->ls_clock;
    SSS_CUDA(cudaMemsetAsync(rounds, 0, sizeof(uint32_t), ctx->stream));
    return sss_graph_launch(ctx, ctx->graph_tag, slot->exec);
}

sss_status impl_sort_segments(sss_ctx* ctx, Arena& ar, const StrIn& in, const std::vector<Seg>& init,
                              const sss_params& prm, uint32_t* perm, uint32_t* lcp) {
    return impl_sort_segments_range(ctx, ar, in, init, prm, perm, lcp, 0, in.n);
}

sss_status impl_sort_segments_range(sss_ctx* ctx, Arena& ar, const StrIn& in, const std::vector<Seg>& init,
                                    const sss_params& prm, uint32_t* perm, uint32_t* lcp, uint32_t q0, uint32_t q1) {
    const uint32_t n = in.n;
    if (n == 0 || q1 <= q0) return SSS_OK;
    const uint32_t nr = q1 - q0;
    LsBufs B;
    carve_ls(ar, n, 1, prm, B);
    const LsKnobs kn = ls_knobs(prm);
    const uint32_t warp_max = kn.warp_cap, med_max = kn.cta_cap;
    SSS_TRY(set_ls_attributes(ctx));
    SSS_TRY(sss_launch(ctx, "ls_init", k_init_perm, dim3((nr + 255) / 256), dim3(256), 0, perm + q0, lcp + q0, nr,
                       q0));

    // initial segments (partitions or instances), by size class
    std::vector<Seg> quad, warp, tiny, small, med, large;
    for (const Seg& s : init) {
        if (s.size < 2) continue;
        if (s.size <= warp_max && s.size <= (uint32_t)QUAD_W) quad.push_back(s);
        else if (s.size <= warp_max) warp.push_back(s);
        else if (s.size <= (uint32_t)TINY_CAP) tiny.push_back(s);
        else if (s.size <= (uint32_t)SM_CAP && s.size <= med_max) small.push_back(s);
        else if (s.size <= med_max) med.push_back(s);
        else large.push_back(s);
    }
    if (large.size() > B.cap_large || quad.size() + warp.size() > B.cap_warp)
        return sss_fail(ctx, SSS_ERR_CUDA, "local sort: internal capacity exceeded");
    // the warp class fills its array from the top: segment i at cap_warp - 1 - i
    std::reverse(warp.begin(), warp.end());
    // pinned staging: counters, then the initial lists
    void* pin;
    SSS_TRY(sss_pinned(ctx, 64 + sizeof(Seg) * (init.size() + 4), &pin));
    uint32_t* h_cnt = reinterpret_cast<uint32_t*>(pin);
    Seg* hq = reinterpret_cast<Seg*>(reinterpret_cast<char*>(pin) + 64);
    Seg* hw = hq + quad.size();
    Seg* ht = hw + warp.size();
    Seg* hs = ht + tiny.size();
    Seg* hm = hs + small.size();
    Seg* hl = hm + med.size();
    std::copy(quad.begin(), quad.end(), hq);
    std::copy(warp.begin(), warp.end(), hw);
    std::copy(tiny.begin(), tiny.end(), ht);
    std::copy(small.begin(), small.end(), hs);
    std::copy(med.begin(), med.end(), hm);
    std::copy(large.begin(), large.end(), hl);
    for (int k = 0; k < 8; ++k) h_cnt[k] = 0;
    h_cnt[2] = (uint32_t)large.size();
    SSS_TRY(sss_upload(ctx, B.warp, hq, sizeof(Seg) * quad.size()));
    SSS_TRY(sss_upload(ctx, B.warp + (B.cap_warp - warp.size()), hw, sizeof(Seg) * warp.size()));
    SSS_TRY(sss_upload(ctx, B.tiny, ht, sizeof(Seg) * tiny.size()));
    SSS_TRY(sss_upload(ctx, B.small, hs, sizeof(Seg) * small.size()));
    SSS_TRY(sss_upload(ctx, B.med, hm, sizeof(Seg) * med.size()));
    SSS_TRY(sss_upload(ctx, B.large, hl, sizeof(Seg) * large.size()));
    SSS_TRY(sss_upload(ctx, B.cnt, h_cnt, sizeof(uint32_t) * 8));
    SSS_CUDA(cudaMemsetAsync(B.work, 0, sizeof(uint32_t) * 8, ctx->stream));
    SSS_TRY(run_finishers(ctx, B, nullptr, (uint32_t)quad.size(), (uint32_t)warp.size(), (uint32_t)tiny.size(),
                          (uint32_t)small.size(), (uint32_t)med.size(), in, perm, lcp));
    if (large.empty()) return SSS_OK;

    SSS_CUDA(cudaMemsetAsync(B.fixmark + q0, 0, nr, ctx->stream));
    SegLists L{B.tiny, B.med, B.large, B.cnt, B.cap_tiny, B.cap_med, B.cap_large, B.warp, B.cap_warp, B.small,
               B.cap_small, warp_max, med_max};
    if (prm.flags & SSS_FLAG_GRAPH) {
        SSS_TRY(run_rounds_graph(ctx, B, kn, L, in, perm, lcp, 100000u));
    } else {
    uint32_t* h_next = reinterpret_cast<uint32_t*>(ctx->h_small);
    for (uint32_t rounds = 1;; ++rounds) {
        if (rounds > 100000u) return sss_fail(ctx, SSS_ERR_CUDA, "local sort: round limit exceeded");
        SSS_TRY(launch_round(ctx, B, kn, L, in, perm, lcp));
        // segments pushed for the next round, and the sticky error word
        SSS_CUDA(cudaMemcpyAsync(h_next, B.cnt + 2, sizeof(uint32_t), cudaMemcpyDeviceToHost, ctx->stream));
        SSS_CUDA(cudaMemcpyAsync(h_next + 1, ctx->d_err, sizeof(uint32_t), cudaMemcpyDeviceToHost, ctx->stream));
        SSS_CUDA(cudaStreamSynchronize(ctx->stream));
        if (h_next[1] & ERRBIT_OVERFLOW) return sss_fail(ctx, SSS_ERR_CUDA, "local sort: device capacity check failed");
        if (h_next[0] == 0) break;
    }
    }
    // (over the sorted range only; its first position keeps lcp 0)
    SSS_TRY(sss_launch(ctx, "ls_fix_seams", k_fix_seams, dim3(std::min((nr + 255) / 256, 4096u)), dim3(256), 0,
                       (const uint8_t*)(B.fixmark + q0), nr, in.chars, in.offs, in.lens,
                       (const uint32_t*)(perm + q0), lcp + q0));
    return SSS_OK;
}

// ---------------------------------------------------------------------------
// The batched sort as one graph launch (sss_sort_batch with SSS_FLAG_GRAPH).
// The instances are classified into the size-class lists on the device, so no
// step needs the host: identity order, classification, the first finishers,
// the round loop (a conditional WHILE node around one planned round) and the
// instance-local permutation are all nodes of one graph, kept in the context
// under a key of every pointer and size its kernels take.

// every instance of >= 2 strings becomes a segment of its size class
__global__ void k_batch_classify(const Seg* __restrict__ inst, uint32_t m, SegLists L, unsigned* err) {
    for (uint32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < m; k += gridDim.x * blockDim.x) {
        const Seg s = inst[k];
        if (s.size >= 2) push_seg(L, s.start, s.size, 0, err);
    }
}

// the round loop runs at least once only if an instance is large
__global__ void k_ls_cond0(const uint32_t* __restrict__ cnt, cudaGraphConditionalHandle h) {
    cudaGraphSetConditional(h, cnt[2] > 0 ? 1u : 0u);
}

sss_status impl_sort_batch_graph(sss_ctx* ctx, Arena& ar, const StrIn& in, const Seg* d_inst, uint32_t m,
                                 const sss_params& prm, uint32_t* perm, uint32_t* lcp, uint32_t* dist) {
    const uint32_t n = in.n;
    if (n == 0 || m == 0) return SSS_OK;
    LsBufs B;
    carve_ls(ar, n, 1, prm, B);
    const LsKnobs kn = ls_knobs(prm);
    SSS_TRY(set_ls_attributes(ctx));
    const SegLists L{B.tiny, B.med, B.large, B.cnt, B.cap_tiny, B.cap_med, B.cap_large, B.warp, B.cap_warp, B.small,
                     B.cap_small, kn.warp_cap, kn.cta_cap};
    const uint32_t limit = 100000u;
    char keyb[512];
    std::snprintf(keyb, sizeof(keyb), "batch %p %p %p %u %p %p %p %p %u %p %p %p %u %u %u %u %d", (const void*)in.chars,
                  (const void*)in.offs, (const void*)in.lens, n, (void*)perm, (void*)lcp, (void*)dist,
                  (const void*)d_inst, m, (void*)B.K, (void*)B.large, (void*)B.sp.plan, kn.warp_cap, kn.cta_cap,
                  kn.direct_cap, kn.bucket_target, ctx->sm_count);
    uint32_t* rounds = reinterpret_cast<uint32_t*>(ctx->d_err) + 1;  // a spare word of the context
    sss_ctx::LsGraph* slot = nullptr;
    for (auto& lg : ctx->ls_graphs)
        if (lg.exec && lg.key == keyb) slot = &lg;
    if (!slot) {
        slot = &ctx->ls_graphs[0];  // an empty entry, else the least recently used
        for (auto& lg : ctx->ls_graphs)
            if (!lg.exec ? slot->exec != nullptr : (slot->exec && lg.used < slot->used)) slot = &lg;
        if (slot->exec) cudaGraphExecDestroy(slot->exec);
        if (slot->graph) cudaGraphDestroy(slot->graph);
        slot->exec = nullptr;
        slot->graph = nullptr;
        slot->key.clear();
        if (!ctx->cap_stream) SSS_CUDA(cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking));
        if (!ctx->cap_stream2) SSS_CUDA(cudaStreamCreateWithFlags(&ctx->cap_stream2, cudaStreamNonBlocking));
        cudaGraph_t g;
        SSS_CUDA(cudaGraphCreate(&g, 0));
        cudaGraphConditionalHandle h;
        SSS_CUDA(cudaGraphConditionalHandleCreate(&h, g, 0, cudaGraphCondAssignDefault));
        const uint32_t sm = (uint32_t)std::max(1, ctx->sm_count);
        cudaStream_t saved = ctx->stream;
        ctx->capturing = true;
        sss_status st = SSS_OK;
        cudaError_t ce = cudaStreamBeginCaptureToGraph(ctx->cap_stream, g, nullptr, nullptr, 0,
                                                       cudaStreamCaptureModeThreadLocal);
        if (ce == cudaSuccess) {
            ctx->stream = ctx->cap_stream;
            // A: identity order, the instances' segments by size class, their finishers
            ce = cudaMemsetAsync(rounds, 0, sizeof(uint32_t), ctx->stream);
            if (ce == cudaSuccess) ce = cudaMemsetAsync(B.cnt, 0, sizeof(uint32_t) * 8, ctx->stream);
            if (ce == cudaSuccess) ce = cudaMemsetAsync(B.work, 0, sizeof(uint32_t) * 8, ctx->stream);
            if (ce == cudaSuccess) ce = cudaMemsetAsync(B.fixmark, 0, n, ctx->stream);
            if (ce == cudaSuccess) {
                st = sss_launch(ctx, "ls_init", k_init_perm, dim3((n + 255) / 256), dim3(256), 0, perm, lcp, n, 0u);
                if (st == SSS_OK)
                    st = sss_launch(ctx, "batch_classify", k_batch_classify, dim3(std::min((m + 255) / 256, sm * 4)),
                                    dim3(256), 0, d_inst, m, L, ctx->d_err);
                if (st == SSS_OK) st = run_finishers(ctx, B, B.cnt, 0, 0, 0, 0, 0, in, perm, lcp);
                if (st == SSS_OK)
                    st = sss_launch(ctx, "ls_cond", k_ls_cond0, dim3(1), dim3(1), 0, (const uint32_t*)B.cnt, h);
            }
            // B: the round loop, a while node after everything captured so far
            cudaGraphNode_t wnode = nullptr;
            if (st == SSS_OK && ce == cudaSuccess) {
                cudaStreamCaptureStatus cs;
                cudaGraph_t cg;
                const cudaGraphNode_t* deps = nullptr;
                size_t ndeps = 0;
                ce = cudaStreamGetCaptureInfo(ctx->cap_stream, &cs, nullptr, &cg, &deps, nullptr, &ndeps);
                cudaGraphNodeParams cp{};
                cp.type = cudaGraphNodeTypeConditional;
                cp.conditional.handle = h;
                cp.conditional.type = cudaGraphCondTypeWhile;
                cp.conditional.size = 1;
                if (ce == cudaSuccess) ce = cudaGraphAddNode(&wnode, cg, deps, nullptr, ndeps, &cp);
                if (ce == cudaSuccess)
                    ce = cudaStreamUpdateCaptureDependencies(ctx->cap_stream, &wnode, nullptr, 1,
                                                             cudaStreamSetCaptureDependencies);
                if (ce == cudaSuccess) {
                    cudaGraph_t body = cp.conditional.phGraph_out[0];
                    ce = cudaStreamBeginCaptureToGraph(ctx->cap_stream2, body, nullptr, nullptr, 0,
                                                       cudaStreamCaptureModeThreadLocal);
                    if (ce == cudaSuccess) {
                        ctx->stream = ctx->cap_stream2;
                        st = launch_round(ctx, B, kn, L, in, perm, lcp);
                        if (st == SSS_OK)
                            st = sss_launch(ctx, "ls_cond", k_ls_cond, dim3(1), dim3(1), 0, (const uint32_t*)B.cnt,
                                            rounds, limit, ctx->d_err, h);
                        cudaGraph_t out = body;
                        cudaError_t ee = cudaStreamEndCapture(ctx->cap_stream2, &out);
                        if (ce == cudaSuccess) ce = ee;
                        ctx->stream = ctx->cap_stream;
                    }
                }
            }
            // C: LCPs across re-sorted buckets, instance-local order, dist
            if (st == SSS_OK && ce == cudaSuccess) {
                st = sss_launch(ctx, "ls_fix_seams", k_fix_seams, dim3(std::min((n + 255) / 256, 4096u)), dim3(256), 0,
                                (const uint8_t*)B.fixmark, n, in.chars, in.offs, in.lens, (const uint32_t*)perm, lcp);
                if (st == SSS_OK) st = impl_batch_finish(ctx, d_inst, m, in.lens, perm, lcp, dist);
            }
            cudaGraph_t out = g;
            cudaError_t ee = cudaStreamEndCapture(ctx->cap_stream, &out);
            if (ce == cudaSuccess) ce = ee;
        }
        ctx->capturing = false;
        ctx->stream = saved;
        if (st != SSS_OK || ce != cudaSuccess) {
            cudaGetLastError();
            cudaGraphDestroy(g);
            return st != SSS_OK ? st : sss_fail(ctx, SSS_ERR_CUDA, std::string("batch graph: ") + cudaGetErrorString(ce));
        }
        cudaGraphExec_t ex;
        ce = cudaGraphInstantiate(&ex, g, 0);
        if (ce != cudaSuccess) {
            cudaGetLastError();
            cudaGraphDestroy(g);
            return sss_fail(ctx, SSS_ERR_CUDA, std::string("batch graph instantiate: ") + cudaGetErrorString(ce));
        }
        slot->graph = g;
        slot->exec = ex;
        slot->key = keyb;
    }
    slot->used = ++ctx->ls_clock;
    return sss_graph_launch(ctx, "batch_graph", slot->exec);
}

sss_status impl_finish_segments(sss_ctx* ctx, const Seg* tiny, uint32_t ntiny, const Seg* med, uint32_t nmed,
                                const StrIn& in, uint32_t* perm, uint32_t* lcp) {
    SSS_TRY(set_ls_attributes(ctx));
    const uint32_t sm = (uint32_t)std::max(1, ctx->sm_count);
    uint32_t* work = reinterpret_cast<uint32_t*>(ctx->d_err) + 2;  // two spare words of the context
    SSS_CUDA(cudaMemsetAsync(work, 0, sizeof(uint32_t) * 2, ctx->stream));
    SSS_TRY(sss_launch(ctx, "ls_finish_tiny", k_finish<TINY_T, TINY_CAP>, dim3(std::min(ntiny, sm * 32)), dim3(TINY_T),
                       finish_smem(TINY_CAP), tiny, (const uint32_t*)nullptr, ntiny, work, in.chars, in.offs, in.lens,
                       perm, lcp, ctx->d_err));
    SSS_TRY(sss_launch(ctx, "ls_finish_cta", k_finish2<MED_T, MED_CAP>, dim3(std::min(nmed, sm * 4)), dim3(MED_T),
                       finish_smem(MED_CAP), med, (const uint32_t*)nullptr, nmed, work + 1, in.chars, in.offs, in.lens,
                       perm, lcp, ctx->d_err));
    return SSS_OK;
}

// Smallest offset and largest end of every partition's strings: blocks of
// 4096 positions over the whole grid, each block reducing within one partition
// and folding its result into out[2i] (min) and out[2i+1] (max) with atomics
// (out pre-set by k_part_extents_init).
__global__ void k_part_extents_init(uint32_t p, unsigned long long* __restrict__ out) {
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < p; i += gridDim.x * blockDim.x) {
        out[2 * i] = ~0ull;
        out[2 * i + 1] = 0ull;
    }
}

__global__ void __launch_bounds__(256) k_part_extents(const uint64_t* __restrict__ offs,
                                                      const uint32_t* __restrict__ lens, uint32_t n, uint32_t p,
                                                      unsigned long long* __restrict__ out) {
    constexpr uint32_t SPAN = 4096;
    __shared__ unsigned long long s_lo[8], s_hi[8];
    for (uint64_t c = blockIdx.x; c * SPAN < n; c += gridDim.x) {
        const uint32_t a = (uint32_t)(c * SPAN);
        const uint32_t b = (uint32_t)min((uint64_t)n, (uint64_t)a + SPAN);
        // partitions are contiguous: handle the part of [a, b) in each partition it touches
        uint32_t i = (uint32_t)(((uint64_t)a * p) / n);
        while (i + 1 < p && part_lo(n, p, i + 1) <= a) ++i;
        for (uint32_t q0 = a; q0 < b; ++i) {
            const uint32_t q1 = min(b, part_lo(n, p, i + 1));
            unsigned long long lo = ~0ull, hi = 0ull;
            for (uint32_t q = q0 + threadIdx.x; q < q1; q += 256) {
                const unsigned long long o = offs[q];
                lo = o < lo ? o : lo;
                const unsigned long long e = o + lens[q];
                hi = e > hi ? e : hi;
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const unsigned long long ol = __shfl_xor_sync(SSS_FULL, lo, o), oh = __shfl_xor_sync(SSS_FULL, hi, o);
                lo = ol < lo ? ol : lo;
                hi = oh > hi ? oh : hi;
            }
            if ((threadIdx.x & 31) == 0) {
                s_lo[threadIdx.x >> 5] = lo;
                s_hi[threadIdx.x >> 5] = hi;
            }
            __syncthreads();
            if (threadIdx.x == 0) {
                for (int w = 1; w < 8; ++w) {
                    lo = s_lo[w] < lo ? s_lo[w] : lo;
                    hi = s_hi[w] > hi ? s_hi[w] : hi;
                }
                if (q1 > q0) {
                    atomicMin(&out[2 * i], lo);
                    atomicMax(&out[2 * i + 1], hi);
                }
            }
            __syncthreads();
            q0 = q1;
        }
    }
}

sss_status impl_part_extents(sss_ctx* ctx, const StrIn& in, uint32_t p, unsigned long long* out) {
    const uint32_t sm = (uint32_t)std::max(1, ctx->sm_count);
    SSS_TRY(sss_launch(ctx, "part_extents", k_part_extents_init, dim3((p + 255) / 256), dim3(256), 0, p, out));
    const uint32_t blocks = std::min((in.n + 4095u) / 4096u, sm * 8);
    return sss_launch(ctx, "part_extents", k_part_extents, dim3(blocks), dim3(256), 0, in.offs, in.lens, in.n, p,
                      out);
}

uint32_t finish_cap_tiny() { return TINY_CAP; }
uint32_t finish_cap_med() { return MED_CAP; }

// Suffix views of a text: string i is text[i .. i + min(n - i, max_len)).
__global__ void k_suffix_views(uint32_t n, uint32_t max_len, uint64_t* __restrict__ offs,
                               uint32_t* __restrict__ lens) {
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        uint32_t r = n - i;
        offs[i] = i;
        lens[i] = r < max_len ? r : max_len;
    }
}

sss_status impl_suffix_views(sss_ctx* ctx, uint32_t n, uint32_t max_len, uint64_t* offs, uint32_t* lens) {
    return sss_launch(ctx, "sfx_views", k_suffix_views, dim3(std::min((n + 255) / 256, 65535u)), dim3(256), 0, n,
                      max_len, offs, lens);
}

// Batched sorts: one CTA per instance turns table positions into
// instance-local indices and (optionally) computes the instance's dist.
__global__ void k_batch_finish(const Seg* __restrict__ inst, uint32_t m, const uint32_t* __restrict__ lens,
                               uint32_t* __restrict__ perm, const uint32_t* __restrict__ lcp,
                               uint32_t* __restrict__ dist) {
    for (uint32_t k = blockIdx.x; k < m; k += gridDim.x) {
        const Seg s = inst[k];
        for (uint32_t r = threadIdx.x; r < s.size; r += blockDim.x) {
            uint32_t q = s.start + r;
            uint32_t g = perm[q];
            if (dist) {
                uint32_t left = r > 0 ? lcp[q] : 0;
                uint32_t right = r + 1 < s.size ? lcp[q + 1] : 0;
                uint32_t mx = left > right ? left : right;
                uint64_t d = (uint64_t)mx + 1;
                dist[g] = d < lens[g] ? (uint32_t)d : lens[g];
            }
        }
        __syncthreads();
        for (uint32_t r = threadIdx.x; r < s.size; r += blockDim.x) perm[s.start + r] -= s.start;
        __syncthreads();
    }
}

sss_status impl_batch_finish(sss_ctx* ctx, const Seg* d_inst, uint32_t m, const uint32_t* lens, uint32_t* perm,
                             const uint32_t* lcp, uint32_t* dist) {
    return sss_launch(ctx, "batch_finish", k_batch_finish, dim3(std::min<uint32_t>(m, 65535u)), dim3(256), 0, d_inst,
                      m, lens, perm, lcp, dist);
}

sss_status impl_dist(sss_ctx* ctx, const uint32_t* lens, uint32_t n, const uint32_t* perm, const uint32_t* lcp,
                     uint32_t* dist) {
    return sss_launch(ctx, "dist", k_dist, dim3((n + 255) / 256), dim3(256), 0, lens, n, perm, lcp, dist);
}

sss_status impl_check_input(sss_ctx* ctx, const StrIn& in) {
    return sss_launch(ctx, "check_input", k_check_input, dim3((in.n + 255) / 256), dim3(256), 0, in.chars,
                      in.n_chars, in.offs, in.lens, in.n, ctx->d_err);
}
