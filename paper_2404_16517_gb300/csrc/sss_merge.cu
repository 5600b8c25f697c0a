// Stage C: string-based regular sampling, splitters and bucket bounds
// (Section 3.1.1 "Local Sampling" / "Splitter Computation"; bucket rule of
// Section 3 step 1).  Stage D: LCP-compressed exchange into buckets (Section 3
// step 2 with the LCP compression of Section 2) and LCP-aware merging of every
// bucket (Section 3 step 3; LCP merging of Section 2).
//
// GB300 design of the merge.  Bucket j holds one sorted piece from every run;
// the pieces are merged by a tree of pairwise merges (log2 p levels).  A merge
// of runs A and B is split into independent segments at every S-th element of
// A and of B: each such sample is located in the other run by an LCP-aware
// binary search on the original strings, which also yields its LCPs with its
// neighbours there.  One thread then merges one segment sequentially with the
// LCP merge rule (the head sharing the longer prefix with the last output is
// smaller; equal LCPs compare characters from that LCP on).  Those character
// comparisons always start at or beyond the LCP a record was stored with, so
// they read only the compressed records: records of one bucket are contiguous
// and small enough to stay in L2.
#include <algorithm>
#include <vector>

#include "sss_device.cuh"
#include "sss_internal.cuh"

namespace {

constexpr uint32_t MINF = 0xFFFFFFFFu;  // "minus infinity" splitter
constexpr uint32_t PINF = 0xFFFFFFFEu;  // no upper splitter: "plus infinity"
constexpr uint32_t MS_DEFAULT = 32;      // merge segment sample spacing (default)

// ---------------------------------------------------------------------------
// string comparison helpers on (truncated) original strings
struct Strs {
    const uint8_t* chars;
    const uint64_t* offs;
    const uint32_t* lens;
    const uint32_t* trunc;  // nullable
};

__device__ __forceinline__ uint32_t tlen(const Strs& S, uint32_t i) { return S.trunc ? S.trunc[i] : S.lens[i]; }

// compare strings a and b from character d on (both share [0, d)); returns the
// LCP in *l and -1/0/1
__device__ __forceinline__ int cmp_from(const uint8_t* a, uint32_t la, const uint8_t* b, uint32_t lb, uint32_t d,
                                        uint32_t* l) {
    uint32_t m = la < lb ? la : lb;
    uint32_t k = d;
    while (k < m) {
        uint64_t x = load_word_be(a, la, k), y = load_word_be(b, lb, k);
        if (x != y) {
            uint32_t c = k + word_lcp(x, y);
            if (c >= m) break;
            *l = c;
            return x < y ? -1 : 1;
        }
        k += 8;
    }
    *l = m;
    return la < lb ? -1 : (la > lb ? 1 : 0);
}

// cmp_from over at most 4 words (32 characters) from d: *dec = false when the
// strings agree on all of them with characters of both left (undecided).
__device__ __forceinline__ int cmp_from4(const uint8_t* a, uint32_t la, const uint8_t* b, uint32_t lb, uint32_t d,
                                         bool* dec) {
    const uint32_t m = la < lb ? la : lb;
    uint32_t k = d;
    for (int w = 0; w < 4 && k < m; ++w, k += 8) {
        const uint64_t x = load_word_be(a, la, k), y = load_word_be(b, lb, k);
        if (x != y) {
            *dec = true;
            if (k + word_lcp(x, y) >= m) return la < lb ? -1 : (la > lb ? 1 : 0);  // one ends first
            return x < y ? -1 : 1;
        }
    }
    *dec = k >= m;  // both agree up to the shorter's end: decided by the lengths
    return la < lb ? -1 : (la > lb ? 1 : 0);
}

// The same comparison by a whole warp: lane k tests the word at d + 256*i + 8k,
// a ballot finds the first differing word.  Every lane gets the result.
__device__ __forceinline__ int warp_cmp_from(const uint8_t* a, uint32_t la, const uint8_t* b, uint32_t lb, uint32_t d,
                                             uint32_t* l) {
    const int lane = threadIdx.x & 31;
    uint32_t m = la < lb ? la : lb;
    for (uint32_t k = d; k < m; k += 256) {
        uint32_t pos = k + 8 * lane;
        uint64_t x = 0, y = 0;
        if (pos < m) {
            x = load_word_be(a, la, pos);
            y = load_word_be(b, lb, pos);
        }
        uint32_t ne = __ballot_sync(SSS_FULL, x != y);
        if (ne) {
            int f = __ffs(ne) - 1;
            uint64_t xf = __shfl_sync(SSS_FULL, x, f), yf = __shfl_sync(SSS_FULL, y, f);
            uint32_t c = k + 8 * f + word_lcp(xf, yf);
            if (c >= m) break;
            *l = c;
            return xf < yf ? -1 : 1;
        }
    }
    *l = m;
    return la < lb ? -1 : (la > lb ? 1 : 0);
}

__device__ __forceinline__ int cmp_str_from(const Strs& S, uint32_t a, uint32_t b, uint32_t d, uint32_t* l) {
    return cmp_from(S.chars + S.offs[a], tlen(S, a), S.chars + S.offs[b], tlen(S, b), d, l);
}

// ---------------------------------------------------------------------------
// Stage C
__global__ void k_c_samples(const uint32_t* __restrict__ run_perm, uint32_t n, uint32_t p, uint32_t v, Strs S,
                            uint32_t* __restrict__ smp, uint64_t* __restrict__ s_offs, uint32_t* __restrict__ s_lens,
                            uint32_t* __restrict__ cnt) {
    // one thread per (partition, t); compacted in (partition, t) order by a
    // prefix count of non-empty partitions
    uint32_t g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= p * (v + 1)) return;
    uint32_t i = g / (v + 1), t = g % (v + 1) + 1;
    uint32_t lo = part_lo(n, p, i), hi = part_lo(n, p, i + 1);
    uint64_t ni = hi - lo;
    if (ni == 0) return;
    // number of non-empty partitions before i
    uint32_t ne = 0;
    for (uint32_t k = 0; k < i; ++k) ne += part_lo(n, p, k + 1) > part_lo(n, p, k) ? 1u : 0u;
    uint64_t rank = (t * ni + v) / (v + 1) - 1;
    uint32_t s = run_perm[lo + rank];
    uint32_t o = ne * (v + 1) + (t - 1);
    smp[o] = s;
    s_offs[o] = S.offs[s];
    s_lens[o] = tlen(S, s);
    if (g == 0) *cnt = 0;
}

__global__ void k_c_splitters(const uint32_t* __restrict__ smp, const uint32_t* __restrict__ sperm, uint32_t ns,
                              uint32_t p, uint32_t* __restrict__ spl) {
    uint32_t j = blockIdx.x * blockDim.x + threadIdx.x + 1;
    if (j >= p) return;
    int64_t k = (int64_t)(((uint64_t)j * ns) / p) - 1;
    spl[j - 1] = k < 0 ? MINF : smp[sperm[k]];
}

// ---- character-based regular sampling (Section 3.1.2) ----------------------
// C_i = characters (truncated lengths) of partition i: input indices [lo_i, hi_i)
__global__ void k_c_chartot(Strs S, uint32_t n, uint32_t p, unsigned long long* __restrict__ tot) {
    const uint32_t i = blockIdx.y;
    const uint32_t lo = part_lo(n, p, i), hi = part_lo(n, p, i + 1);
    uint64_t v = 0;
    for (uint32_t q = lo + blockIdx.x * blockDim.x + threadIdx.x; q < hi; q += gridDim.x * blockDim.x) v += tlen(S, q);
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(SSS_FULL, v, o);
    if ((threadIdx.x & 31) == 0 && v) atomicAdd(&tot[i], (unsigned long long)v);
}

// P[q] = characters of the run positions before q (runs in position order), in
// three passes over chunks of CP_CHUNK positions
constexpr uint32_t CP_T = 256, CP_PER = 16, CP_CHUNK = CP_T * CP_PER;

__device__ __forceinline__ uint64_t cp_block_excl(uint64_t v, uint64_t* wt, uint64_t* total) {
    const uint32_t lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    uint64_t x = v;
    for (int d = 1; d < 32; d <<= 1) {
        uint64_t y = __shfl_up_sync(SSS_FULL, x, d);
        if (lane >= (uint32_t)d) x += y;
    }
    if (lane == 31) wt[w] = x;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint64_t run = 0;
        for (uint32_t k = 0; k < CP_T / 32; ++k) {
            uint64_t t = wt[k];
            wt[k] = run;
            run += t;
        }
        *total = run;
    }
    __syncthreads();
    return wt[w] + x - v;
}

__global__ void __launch_bounds__(CP_T) k_c_psum(Strs S, const uint32_t* __restrict__ run_perm, uint32_t n,
                                                  uint64_t* __restrict__ csum) {
    __shared__ uint64_t wt[CP_T / 32], tot;
    const uint64_t q0 = (uint64_t)blockIdx.x * CP_CHUNK + (uint64_t)threadIdx.x * CP_PER;
    uint64_t v = 0;
    for (uint32_t k = 0; k < CP_PER; ++k)
        if (q0 + k < n) v += tlen(S, run_perm[q0 + k]);
    cp_block_excl(v, wt, &tot);
    if (threadIdx.x == 0) csum[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(CP_T) k_c_pscan(uint64_t* __restrict__ csum, uint32_t nc) {
    __shared__ uint64_t wt[CP_T / 32], tot;
    uint64_t carry = 0;
    for (uint32_t b0 = 0; b0 < nc; b0 += CP_T) {
        const uint32_t i = b0 + threadIdx.x;
        uint64_t v = i < nc ? csum[i] : 0;
        uint64_t e = cp_block_excl(v, wt, &tot);
        if (i < nc) csum[i] = carry + e;
        carry += tot;
        __syncthreads();
    }
}

__global__ void __launch_bounds__(CP_T) k_c_pwrite(Strs S, const uint32_t* __restrict__ run_perm, uint32_t n,
                                                    const uint64_t* __restrict__ csum, uint64_t* __restrict__ P) {
    __shared__ uint64_t wt[CP_T / 32], tot;
    const uint64_t q0 = (uint64_t)blockIdx.x * CP_CHUNK + (uint64_t)threadIdx.x * CP_PER;
    uint32_t l[CP_PER];
    uint64_t v = 0;
#pragma unroll
    for (uint32_t k = 0; k < CP_PER; ++k) {
        l[k] = q0 + k < n ? tlen(S, run_perm[q0 + k]) : 0u;
        v += l[k];
    }
    uint64_t run = csum[blockIdx.x] + cp_block_excl(v, wt, &tot);
#pragma unroll
    for (uint32_t k = 0; k < CP_PER; ++k) {
        if (q0 + k < n) P[q0 + k] = run;
        run += l[k];
        if (q0 + k + 1 == n) P[n] = run;
    }
}

// sample g of partition i: the string of run i that covers character position
// floor(t N / want) of the run's character array, t = g - so[i] + 1 (t <= cnt[i]),
// else the run's last string (the additional sample of the first partitions)
__global__ void k_c_csamples(const uint32_t* __restrict__ run_perm, uint32_t n, uint32_t p, Strs S,
                             const uint64_t* __restrict__ P, const uint32_t* __restrict__ so,
                             const uint32_t* __restrict__ cnt, uint64_t N, uint64_t want, uint32_t* __restrict__ smp,
                             uint64_t* __restrict__ s_offs, uint32_t* __restrict__ s_lens) {
    const uint32_t g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= so[p]) return;
    uint32_t a = 0, b = p;  // last i with so[i] <= g
    while (b - a > 1) {
        uint32_t mid = (a + b) >> 1;
        if (so[mid] <= g) a = mid; else b = mid;
    }
    const uint32_t i = a;
    const uint32_t lo = part_lo(n, p, i), hi = part_lo(n, p, i + 1);
    const uint64_t t = (uint64_t)(g - so[i]) + 1;
    uint32_t q;
    if (t <= cnt[i]) {
        const uint64_t X = P[lo] + (t * N) / want;
        uint32_t x0 = lo, x1 = hi;  // last q in [lo, hi) with P[q] <= X
        while (x1 - x0 > 1) {
            uint32_t mid = (x0 + x1) >> 1;
            if (P[mid] <= X) x0 = mid; else x1 = mid;
        }
        q = x0;
    } else {
        q = hi - 1;
    }
    const uint32_t s = run_perm[q];
    smp[g] = s;
    s_offs[g] = S.offs[s];
    s_lens[g] = tlen(S, s);
}

// bounds[i*(p+1)+j] = #{ s in run i : s <= f_j }, LCP-aware binary search (one
// warp per search, warp-wide comparisons)
__global__ void k_c_bounds(const uint32_t* __restrict__ run_perm, uint32_t n, uint32_t p, Strs S,
                           const uint32_t* __restrict__ spl, uint32_t* __restrict__ bounds) {
    uint32_t g = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (g >= p * (p + 1)) return;
    uint32_t i = g / (p + 1), j = g % (p + 1);
    uint32_t lo = part_lo(n, p, i), hi = part_lo(n, p, i + 1);
    uint32_t res;
    if (j == 0) res = 0;
    else if (j == p) res = hi - lo;
    else if (spl[j - 1] == MINF) res = 0;
    else {
        uint32_t f = spl[j - 1];
        const uint8_t* fs = S.chars + S.offs[f];
        uint32_t fl = tlen(S, f);
        uint32_t a = 0, b = hi - lo, la = 0, lb = 0;  // run[a-1] <= f < run[b]
        while (a < b) {
            uint32_t mid = (a + b) >> 1;
            uint32_t e = run_perm[lo + mid];
            uint32_t d = la < lb ? la : lb, l;
            int c = warp_cmp_from(S.chars + S.offs[e], tlen(S, e), fs, fl, d, &l);
            if (c <= 0) {
                a = mid + 1;
                la = l;
            } else {
                b = mid;
                lb = l;
            }
        }
        res = a;
    }
    if ((threadIdx.x & 31) == 0) bounds[g] = res;
}

// ---------------------------------------------------------------------------
// Stage D1: records.  Record r (bucket order, pieces in run order) keeps
// idx, h = LCP with its predecessor in the piece (0 for the piece's first),
// tl = truncated length, base = offset such that its character c (h <= c < tl)
// is recchars[base + c].
struct Recs {
    uint32_t* idx;
    uint32_t* h;
    uint32_t* tl;
    uint64_t* base;
    uint8_t* chars;
    uint64_t* head;  // the first 8 characters past h (two-level merge)
};

// position q of the run layout -> record index; also the record's h and length
__global__ void k_d_records(const uint32_t* __restrict__ run_perm, const uint32_t* __restrict__ run_lcp, uint32_t n,
                            uint32_t p, Strs S, const uint32_t* __restrict__ bounds,
                            const uint32_t* __restrict__ piece_off, Recs R, uint32_t* __restrict__ clen,
                            unsigned* err) {
    uint32_t q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n) return;
    // partition i of q
    uint32_t i = (uint32_t)(((uint64_t)(q + 1) * p + n - 1) / n - 1);
    uint32_t lo = part_lo(n, p, i);
    uint32_t t = q - lo;
    const uint32_t* b = bounds + (size_t)i * (p + 1);
    // bucket j: b[j] <= t < b[j+1]
    uint32_t a = 0, c = p;  // find largest j with b[j] <= t
    while (a + 1 < c) {
        uint32_t mid = (a + c) >> 1;
        if (b[mid] <= t) a = mid; else c = mid;
    }
    uint32_t j = a;
    while (j + 1 < p && b[j + 1] <= t) ++j;  // skip empty buckets at equal bounds
    uint32_t r = piece_off[(size_t)j * p + i] + (t - b[j]);
    if (r >= n) {
        atomicOr(err, ERRBIT_OVERFLOW);
        return;
    }
    uint32_t s = run_perm[q];
    uint32_t tl = tlen(S, s);
    uint32_t h = 0;
    if (t > b[j]) {
        uint32_t prev_tl = tlen(S, run_perm[q - 1]);
        h = run_lcp[q];
        h = h < tl ? h : tl;
        h = h < prev_tl ? h : prev_tl;
    }
    R.idx[r] = s;
    R.h[r] = h;
    R.tl[r] = tl;
    clen[r] = tl - h;
}

// exclusive scan of u32 lengths into u64 offsets: per-block totals
__global__ void __launch_bounds__(1024) k_scan_blocks(const uint32_t* __restrict__ in, uint32_t n,
                                                      uint64_t* __restrict__ out, uint64_t* __restrict__ btot) {
    constexpr int ITEMS = 4;
    __shared__ uint64_t sw[32];
    uint32_t base = blockIdx.x * 1024 * ITEMS + threadIdx.x * ITEMS;
    uint64_t loc[ITEMS];
    uint64_t sum = 0;
#pragma unroll
    for (int k = 0; k < ITEMS; ++k) {
        uint32_t v = base + k < n ? in[base + k] : 0;
        loc[k] = sum;
        sum += v;
    }
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    uint64_t x = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint64_t y = __shfl_up_sync(SSS_FULL, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) sw[w] = x;
    __syncthreads();
    if (w == 0) {
        uint64_t t = sw[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint64_t y = __shfl_up_sync(SSS_FULL, t, o);
            if (lane >= o) t += y;
        }
        sw[lane] = t;
    }
    __syncthreads();
    uint64_t off = (w > 0 ? sw[w - 1] : 0) + x - sum;
#pragma unroll
    for (int k = 0; k < ITEMS; ++k)
        if (base + k < n) out[base + k] = off + loc[k];
    if (threadIdx.x == 1023) btot[blockIdx.x] = sw[31];
}

// scan of the block totals by one CTA in chunks of 1024 (carry between chunks)
__global__ void __launch_bounds__(1024) k_scan_totals(uint64_t* __restrict__ btot, uint32_t nb) {
    __shared__ uint64_t sw[32];
    __shared__ uint64_t carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (uint32_t base = 0; base < nb; base += 1024) {
        uint32_t b = base + threadIdx.x;
        uint64_t v = b < nb ? btot[b] : 0;
        uint64_t x = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint64_t y = __shfl_up_sync(SSS_FULL, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) sw[w] = x;
        __syncthreads();
        if (w == 0) {
            uint64_t t = sw[lane];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                uint64_t y = __shfl_up_sync(SSS_FULL, t, o);
                if (lane >= o) t += y;
            }
            sw[lane] = t;
        }
        __syncthreads();
        uint64_t c0 = carry;
        uint64_t ex = c0 + (w > 0 ? sw[w - 1] : 0) + x - v;
        if (b < nb) btot[b] = ex;
        __syncthreads();
        if (threadIdx.x == 1023) carry = c0 + sw[31];
        __syncthreads();
    }
    if (threadIdx.x == 0) btot[nb] = carry;
}

__global__ void k_scan_add(uint64_t* __restrict__ out, uint32_t n, const uint64_t* __restrict__ btot) {
    uint32_t q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q < n) out[q] += btot[q / 4096];
}

// copy every record's characters [h, tl) into the record area
__global__ void k_d_copy(Strs S, Recs R, const uint64_t* __restrict__ coff, uint32_t nrec) {
    uint32_t r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= nrec) return;
    uint32_t s = R.idx[r], h = R.h[r], tl = R.tl[r];
    uint64_t co = coff[r];
    R.base[r] = co - h;
    const uint8_t* src = S.chars + S.offs[s];
    uint8_t* dst = R.chars + co;
    for (uint32_t c = h; c < tl; c += 8) {
        uint64_t w = load_word_be(src, tl, c);
        uint32_t m = tl - c < 8 ? tl - c : 8;
        for (uint32_t k = 0; k < m; ++k) dst[c - h + k] = (uint8_t)(w >> (56 - 8 * k));
    }
}

// ---------------------------------------------------------------------------
// Stage D2
struct Pair {
    uint32_t a0, na, b0, nb;  // run A = [a0, a0+na), run B = [b0, b0+nb), b0 = a0+na
    uint32_t sa, sb;          // first sample index of A's and of B's samples
    uint32_t pad[2];
};

// compare two records from character d on using the record characters
__device__ __forceinline__ int rec_cmp_from(const Recs& R, uint32_t ra, uint32_t rb, uint32_t d, uint32_t* l) {
    uint32_t la = R.tl[ra], lb = R.tl[rb];
    uint32_t m = la < lb ? la : lb;
    const uint8_t* sa = R.chars + R.base[ra];
    const uint8_t* sb = R.chars + R.base[rb];
    for (uint32_t k = d; k < m; k += 8) {
        uint64_t x = load_word_be(sa, la, k), y = load_word_be(sb, lb, k);
        if (x != y) {
            uint32_t c = k + word_lcp(x, y);
            if (c >= m) break;
            *l = c;
            return x < y ? -1 : 1;
        }
    }
    *l = m;
    return la < lb ? -1 : (la > lb ? 1 : 0);
}

// Locate record rp within run X = RX[x0, x0+nx): number of elements < P
// (strict) or <= P; returns also LCP(P, X[pos-1]) and LCP(P, X[pos]).
__device__ __forceinline__ uint32_t lcp_search(const Strs& S, const Recs& R, const uint32_t* RX, uint32_t x0,
                                               uint32_t nx, uint32_t rp, bool strict, uint32_t* l_before,
                                               uint32_t* l_at) {
    uint32_t ip = R.idx[rp];
    const uint8_t* ps = S.chars + S.offs[ip];
    uint32_t pl = R.tl[rp];
    uint32_t lo = 0, hi = nx, llo = 0, lhi = 0;
    while (lo < hi) {
        uint32_t mid = (lo + hi) >> 1;
        uint32_t rm = RX[x0 + mid];
        uint32_t im = R.idx[rm];
        uint32_t d = llo < lhi ? llo : lhi, l;
        int c = cmp_from(S.chars + S.offs[im], R.tl[rm], ps, pl, d, &l);
        bool left = strict ? (c < 0) : (c <= 0);  // X[mid] goes before P
        if (left) {
            lo = mid + 1;
            llo = l;
        } else {
            hi = mid;
            lhi = l;
        }
    }
    *l_before = llo;
    *l_at = lhi;
    return lo;
}

// one thread per sample: rank in the other run and LCPs with the neighbours there
__global__ void k_d_search(Strs S, Recs R, const uint32_t* __restrict__ Rin, const Pair* __restrict__ pairs,
                           uint32_t npairs, uint32_t nsamp, uint32_t* __restrict__ srank,
                           uint32_t* __restrict__ sl0, uint32_t* __restrict__ sl1, uint32_t MS) {
    uint32_t g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= nsamp) return;
    // pair of sample g: last pair with sa <= g
    uint32_t a = 0, c = npairs;
    while (a + 1 < c) {
        uint32_t mid = (a + c) >> 1;
        if (pairs[mid].sa <= g) a = mid; else c = mid;
    }
    Pair pr = pairs[a];
    uint32_t rank, l0, l1;
    if (g < pr.sb) {  // sample of A, searched in B (A wins ties: strict)
        uint32_t x = (g - pr.sa) * MS;
        rank = lcp_search(S, R, Rin, pr.b0, pr.nb, Rin[pr.a0 + x], true, &l0, &l1);
    } else {  // sample of B, searched in A (A elements equal to it go first)
        uint32_t y = (g - pr.sb) * MS;
        rank = lcp_search(S, R, Rin, pr.a0, pr.na, Rin[pr.b0 + y], false, &l0, &l1);
    }
    srank[g] = rank;
    sl0[g] = l0;
    sl1[g] = l1;
}

// one thread per sample: merge from its split point to the next split point
__global__ void k_d_merge(Strs S, Recs R, const uint32_t* __restrict__ Rin, const uint32_t* __restrict__ Hin,
                          uint32_t* __restrict__ Rout, uint32_t* __restrict__ Hout, const Pair* __restrict__ pairs,
                          uint32_t npairs, uint32_t nsamp, const uint32_t* __restrict__ srank,
                          const uint32_t* __restrict__ sl0, const uint32_t* __restrict__ sl1, uint32_t MS) {
    uint32_t g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= nsamp) return;
    uint32_t a = 0, c = npairs;
    while (a + 1 < c) {
        uint32_t mid = (a + c) >> 1;
        if (pairs[mid].sa <= g) a = mid; else c = mid;
    }
    const Pair pr = pairs[a];
    const uint32_t nsa = pr.sb - pr.sa;
    const uint32_t nsb = (a + 1 < npairs ? pairs[a + 1].sa : nsamp) - pr.sb;
    const uint32_t* RA = Rin + pr.a0;
    const uint32_t* RB = Rin + pr.b0;
    const uint32_t* HA = Hin + pr.a0;
    const uint32_t* HB = Hin + pr.b0;
    uint32_t x, y, ha, hb;
    // split point and LCP state
    if (g < pr.sb) {
        uint32_t k = g - pr.sa;
        x = k * MS;
        y = srank[g];
        uint32_t l1 = sl0[g], l2 = sl1[g];  // LCP(P, B[y-1]), LCP(P, B[y])
        uint32_t hP = x > 0 ? HA[x] : 0;     // LCP(A[x-1], P)
        if (x == 0 && y == 0) {
            ha = hb = 0;
        } else if (x == 0) {
            ha = l1;
            hb = HB[y];
        } else if (y == 0) {
            ha = hP;
            hb = l2 < hP ? l2 : hP;
        } else {
            bool prevA;
            if (hP != l1) prevA = hP > l1;
            else {
                uint32_t l;
                int cc = cmp_str_from(S, R.idx[RA[x - 1]], R.idx[RB[y - 1]], hP, &l);
                prevA = cc > 0;  // equal: A[x-1] goes first, so B[y-1] is the later one
            }
            if (prevA) {
                ha = hP;
                hb = l2 < hP ? l2 : hP;
            } else {
                ha = l1;
                hb = HB[y];
            }
        }
        if (y >= pr.nb) hb = 0;
    } else {
        uint32_t k = g - pr.sb;
        y = k * MS;
        x = srank[g];
        uint32_t m1 = sl0[g], m2 = sl1[g];  // LCP(Q, A[x-1]), LCP(Q, A[x])
        uint32_t hQ = y > 0 ? HB[y] : 0;     // LCP(B[y-1], Q)
        if (x == 0 && y == 0) {
            ha = hb = 0;
        } else if (x == 0) {
            hb = hQ;
            ha = m2 < hQ ? m2 : hQ;
        } else if (y == 0) {
            hb = m1;
            ha = HA[x];
        } else {
            bool prevB;
            if (hQ != m1) prevB = hQ > m1;
            else {
                uint32_t l;
                int cc = cmp_str_from(S, R.idx[RA[x - 1]], R.idx[RB[y - 1]], hQ, &l);
                prevB = cc <= 0;  // A[x-1] <= B[y-1]: B[y-1] is the later output
            }
            if (prevB) {
                hb = hQ;
                ha = m2 < hQ ? m2 : hQ;
            } else {
                hb = m1;
                ha = HA[x];
            }
        }
        if (x >= pr.na) ha = 0;
    }
    // end point: the next split point in output order
    uint32_t xe, ye;
    {
        // candidate from the next sample of A (the first A sample with index*MS >= x, excluding ours)
        uint32_t ka = g < pr.sb ? (g - pr.sa) + 1 : (x + MS - 1) / MS;
        uint32_t kb = g >= pr.sb ? (g - pr.sb) + 1 : (y + MS - 1) / MS;
        uint64_t posA = ~0ull, posB = ~0ull;
        uint32_t xa = pr.na, ya = pr.nb, xb = pr.na, yb = pr.nb;
        if (ka < nsa) {
            xa = ka * MS;
            ya = srank[pr.sa + ka];
            posA = (uint64_t)xa + ya;
        }
        if (kb < nsb) {
            yb = kb * MS;
            xb = srank[pr.sb + kb];
            posB = (uint64_t)xb + yb;
        }
        if (posA == ~0ull && posB == ~0ull) {
            xe = pr.na;
            ye = pr.nb;
        } else if (posA <= posB) {
            xe = xa;
            ye = ya;
        } else {
            xe = xb;
            ye = yb;
        }
    }
    uint32_t o = pr.a0 + x + y;
    while (x < xe || y < ye) {
        bool takeA;
        if (y >= ye) takeA = true;
        else if (x >= xe) takeA = false;
        else if (ha != hb) takeA = ha > hb;
        else {
            uint32_t l;
            int cc = rec_cmp_from(R, RA[x], RB[y], ha, &l);
            takeA = cc <= 0;
            // the head not taken now shares l characters with the new last output
            if (takeA) hb = l; else ha = l;
        }
        if (takeA) {
            Rout[o] = RA[x];
            Hout[o] = ha;
            ++x;
            ha = x < pr.na ? HA[x] : 0;
        } else {
            Rout[o] = RB[y];
            Hout[o] = hb;
            ++y;
            hb = y < pr.nb ? HB[y] : 0;
        }
        ++o;
    }
}

// D3: LCP at bucket seams, then the outputs
__global__ void k_d_seams(Strs S, const Recs R, const uint32_t* __restrict__ Rfin, uint32_t* __restrict__ Hfin,
                          const uint32_t* __restrict__ bstart, uint32_t p) {
    uint32_t j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= p) return;
    uint32_t s0 = bstart[j], s1 = bstart[j + 1];
    if (s1 == s0 || s0 == 0) return;
    uint32_t l;
    cmp_str_from(S, R.idx[Rfin[s0 - 1]], R.idx[Rfin[s0]], 0, &l);
    Hfin[s0] = l;
}

__global__ void k_d_out(const Recs R, const uint32_t* __restrict__ Rfin, const uint32_t* __restrict__ Hfin, uint32_t n,
                        uint32_t* __restrict__ out_perm, uint32_t* __restrict__ out_lcp) {
    uint32_t q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n) return;
    out_perm[q] = R.idx[Rfin[q]];
    out_lcp[q] = Hfin[q];
}

// ---------------------------------------------------------------------------
// Stage D, second level (the multi-level idea of Section 3 on one GPU): every
// level-1 bucket is split again by regular sampling into sub-buckets of at most
// D2_CAP strings, and each sub-bucket's p slices are merged inside one CTA.
constexpr uint32_t D2_CAP = 2048;  // strings merged by one CTA (<= the stage-A CTA finisher)
constexpr uint32_t D2_OVS = 16;    // samples per sub-bucket
constexpr int D2_T = 512;
constexpr int D2_T_SMALL = 128;    // CTA of the small sub-buckets
constexpr uint32_t D2_SMALL = 512; // largest small sub-bucket
constexpr uint32_t D2_MAXP = 256;  // slices a CTA merges as runs (more: a full sort)
static_assert(D2_MAXP <= 2 * D2_T, "block_merge_runs128 takes at most 2*THREADS runs");

struct BucketInfo {
    uint32_t sbase;  // first sorted-sample index of the bucket
    uint32_t nsmp;   // samples drawn in the bucket
    uint32_t sb0;    // first global sub-bucket
    uint32_t nsb;    // sub-buckets
    uint32_t ss0;    // first global sub-splitter
    uint32_t fref;   // the bucket's lower splitter (MINF: none)
    uint32_t uref;   // the bucket's upper splitter (PINF: none)
    uint32_t pad;
};

__device__ __forceinline__ uint32_t last_le(const uint32_t* a, uint32_t n, uint32_t g, uint32_t stride, uint32_t off) {
    // last index i < n with a[i*stride+off] <= g (a non-decreasing, a[off] <= g)
    uint32_t lo = 0, hi = n;
    while (lo + 1 < hi) {
        uint32_t mid = (lo + hi) >> 1;
        if (a[mid * stride + off] <= g) lo = mid; else hi = mid;
    }
    return lo;
}

__global__ void k_d2_samples(const uint32_t* __restrict__ run_perm, Strs S, const uint32_t* __restrict__ pso,
                             const uint32_t* __restrict__ pstart, uint32_t npieces, uint32_t S2, uint32_t step,
                             uint32_t* __restrict__ smp, uint64_t* __restrict__ s_offs,
                             uint32_t* __restrict__ s_lens) {
    uint32_t g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= S2) return;
    // last piece with pso <= g (pso has npieces+1 entries, pso[npieces] = S2)
    uint32_t lo = 0, hi = npieces;
    while (lo + 1 < hi) {
        uint32_t mid = (lo + hi) >> 1;
        if (pso[mid] <= g) lo = mid; else hi = mid;
    }
    uint32_t k = g - pso[lo];
    uint32_t q = pstart[lo] + (k + 1) * step - 1;
    uint32_t s = run_perm[q];
    smp[g] = s;
    s_offs[g] = S.offs[s];
    s_lens[g] = tlen(S, s);
}

__global__ void k_d2_subspl(const BucketInfo* __restrict__ bi, uint32_t p, uint32_t nss,
                            const uint32_t* __restrict__ smp, const uint32_t* __restrict__ sperm,
                            uint32_t* __restrict__ subspl) {
    uint32_t m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= nss) return;
    uint32_t j = last_le(&bi[0].ss0, p, m, sizeof(BucketInfo) / 4, 0);
    // skip buckets without sub-splitters that share ss0
    while (j + 1 < p && bi[j + 1].ss0 <= m) ++j;
    uint32_t k = m - bi[j].ss0;
    subspl[m] = smp[sperm[bi[j].sbase + D2_OVS * (k + 1) - 1]];
}

// Sorted rank of every second-level sample: srank[sperm[x]] = x.
__global__ void k_d2_srank(const uint32_t* __restrict__ sperm, uint32_t S2, uint32_t* __restrict__ srank) {
    const uint32_t x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x < S2) srank[sperm[x]] = x;
}

// sb[m*p+i] = number of strings of piece (bucket of m, i) that are <= subspl[m],
// one warp per (sub-splitter, piece).  Sub-splitter m is the sorted sample at
// rank R of its bucket; the piece's own samples sit at piece positions
// (t+1)*step - 1 in string order, and the sample sort (ties by sample index)
// keeps them in that order.  So with a = the number of the piece's samples
// ranked at or before R_end (R extended over the following samples equal to
// the sub-splitter, which are <= it too), sample a - 1 is <= the sub-splitter
// and sample a is larger: the count lies in [a*step, (a+1)*step - 1] (or up to
// the piece's end past its last sample).  A binary search over the samples'
// ranks finds a; then a window of at most 32 strings is compared a lane per
// string, a wider one searched.
__global__ void k_d2_bounds(const uint32_t* __restrict__ run_perm, Strs S, const BucketInfo* __restrict__ bi,
                            uint32_t p, uint32_t nss, const uint32_t* __restrict__ pstart,
                            const uint32_t* __restrict__ psz, const uint32_t* __restrict__ pso,
                            const uint32_t* __restrict__ subspl, const uint32_t* __restrict__ sperm,
                            const uint32_t* __restrict__ srank, const uint32_t* __restrict__ s2lcp,
                            const uint32_t* __restrict__ s2lens, uint32_t step, uint32_t* __restrict__ sb) {
    uint32_t g = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (g >= nss * p) return;
    uint32_t m = g / p, i = g % p;
    uint32_t j = last_le(&bi[0].ss0, p, m, sizeof(BucketInfo) / 4, 0);
    while (j + 1 < p && bi[j + 1].ss0 <= m) ++j;
    const BucketInfo B = bi[j];
    const uint32_t k = m - B.ss0;
    const uint32_t f = subspl[m];
    const uint8_t* fs = S.chars + S.offs[f];
    const uint32_t fl = tlen(S, f);
    // R_end: the sub-splitter's sorted rank, past the samples equal to it
    uint32_t rend = B.sbase + D2_OVS * (k + 1) - 1;
    const uint32_t rlim = B.sbase + B.nsmp;
    while (rend + 1 < rlim && s2lcp[rend + 1] >= fl && s2lens[sperm[rend + 1]] == fl) ++rend;
    // a: the piece's samples ranked <= R_end (their ranks grow with their
    // positions): 32 evenly spaced samples per ballot narrow the range until it
    // fits one ballot
    const uint32_t lane = threadIdx.x & 31;
    const uint32_t g0 = pso[j * p + i], c = pso[j * p + i + 1] - g0;
    uint32_t klo = 0, khi = c;
    while (khi - klo > 32) {
        const uint32_t stride = (khi - klo + 31) / 32;
        const uint32_t t = klo + lane * stride;
        const uint32_t k = (uint32_t)__popc(__ballot_sync(SSS_FULL, t < khi && srank[g0 + t] <= rend));
        if (k == 0) {
            khi = klo;
        } else {
            const uint32_t nlo = klo + (k - 1) * stride + 1, nhi = klo + k * stride;
            klo = nlo;
            khi = nhi < khi ? nhi : khi;
        }
    }
    const uint32_t ka =
        klo + (uint32_t)__popc(__ballot_sync(SSS_FULL, klo + lane < khi && srank[g0 + klo + lane] <= rend));
    const uint32_t n_i = psz[j * p + i];
    const uint32_t wa = ka * step, wb = ka < c ? (ka + 1) * step - 1 : n_i;
    const uint32_t q0 = pstart[j * p + i];
    uint32_t cnt = wa;
    if (wb - wa <= 32) {
        // a narrow window (large p: few strings between samples), a lane per
        // string; the strings <= the sub-splitter form a prefix.  First their
        // first 32 characters only: enough when neighbours differ early
        const uint32_t q = wa + lane;
        const uint32_t e = q < wb ? run_perm[q0 + q] : 0u;
        bool le = false, dec = true;
        if (q < wb) le = cmp_from4(S.chars + S.offs[e], tlen(S, e), fs, fl, 0, &dec) <= 0;
        if (__ballot_sync(SSS_FULL, !dec) != 0) {
            // some strings share 32+ characters with the sub-splitter: compare
            // from the LCP that every string between the window's neighbours
            // shares with it (the shorter of the neighbours' LCPs with it)
            uint32_t dl = 0, dh = 0;
            if (wa > 0) {
                const uint32_t en = run_perm[q0 + wa - 1];
                warp_cmp_from(S.chars + S.offs[en], tlen(S, en), fs, fl, 0, &dl);
            }
            if (wb < n_i) {
                const uint32_t en = run_perm[q0 + wb];
                warp_cmp_from(S.chars + S.offs[en], tlen(S, en), fs, fl, 0, &dh);
            }
            const uint32_t d = wa > 0 && wb < n_i ? (dl < dh ? dl : dh) : 0u;
            if (q < wb) {
                uint32_t l;
                le = cmp_from(S.chars + S.offs[e], tlen(S, e), fs, fl, d, &l) <= 0;
            }
        }
        cnt = wa + (uint32_t)__popc(__ballot_sync(SSS_FULL, le));
    } else {
        // a wider window: binary search with warp-wide comparisons that carry the
        // LCP with both ends (fewer strings fetched than a lane per string)
        uint32_t a = wa, b = wb, la = 0, lb = 0;
        while (a < b) {
            const uint32_t mid = (a + b) >> 1;
            const uint32_t e = run_perm[q0 + mid];
            uint32_t l;
            const int cmp = warp_cmp_from(S.chars + S.offs[e], tlen(S, e), fs, fl, la < lb ? la : lb, &l);
            if (cmp <= 0) {
                a = mid + 1;
                la = l;
            } else {
                b = mid;
                lb = l;
            }
        }
        cnt = a;
    }
    if (lane == 0) sb[g] = cnt;
}

__device__ __forceinline__ uint32_t bucket_of_sub(const BucketInfo* bi, uint32_t p, uint32_t b) {
    uint32_t j = last_le(&bi[0].sb0, p, b, sizeof(BucketInfo) / 4, 0);
    while (j + 1 < p && bi[j + 1].sb0 <= b) ++j;
    return j;
}

// slice (sub-bucket b, piece i): [lo, hi) within the piece
__device__ __forceinline__ void slice_range(const BucketInfo& B, uint32_t b, uint32_t i, uint32_t p,
                                            const uint32_t* sb, const uint32_t* psz, uint32_t j, uint32_t* lo,
                                            uint32_t* hi) {
    uint32_t k = b - B.sb0;
    *lo = k == 0 ? 0u : sb[(B.ss0 + k - 1) * p + i];
    *hi = k + 1 == B.nsb ? psz[j * p + i] : sb[(B.ss0 + k) * p + i];
}

__global__ void k_d2_slices(const BucketInfo* __restrict__ bi, uint32_t p, uint32_t nsb,
                            const uint32_t* __restrict__ sb, const uint32_t* __restrict__ psz,
                            uint32_t* __restrict__ ssz) {
    uint32_t g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= nsb * p) return;
    uint32_t b = g / p, i = g % p;
    uint32_t j = bucket_of_sub(bi, p, b);
    uint32_t lo, hi;
    slice_range(bi[j], b, i, p, sb, psz, j, &lo, &hi);
    ssz[g] = hi > lo ? hi - lo : 0u;
}

__global__ void k_d2_oversized(const uint64_t* __restrict__ soff, uint32_t p, uint32_t nsb,
                               uint32_t* __restrict__ list, uint32_t* __restrict__ cnt) {
    uint32_t b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nsb) return;
    if (soff[(uint64_t)(b + 1) * p] - soff[(uint64_t)b * p] > D2_CAP) list[atomicAdd(cnt, 1u)] = b;
}

// D1 at the second level: run position q -> record of its sub-bucket slice.  The
// first string of every slice keeps all its characters (h = 0).
__global__ void k_d2_records(const uint32_t* __restrict__ run_perm, const uint32_t* __restrict__ run_lcp, uint32_t n,
                             uint32_t p, Strs S, const uint32_t* __restrict__ bounds,
                             const BucketInfo* __restrict__ bi, const uint32_t* __restrict__ sb,
                             const uint64_t* __restrict__ soff, Recs R, uint32_t* __restrict__ clen, unsigned* err) {
    uint32_t q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n) return;
    uint32_t i = (uint32_t)(((uint64_t)(q + 1) * p + n - 1) / n - 1);
    uint32_t t = q - part_lo(n, p, i);
    const uint32_t* b1 = bounds + (size_t)i * (p + 1);
    uint32_t a = 0, c = p;
    while (a + 1 < c) {
        uint32_t mid = (a + c) >> 1;
        if (b1[mid] <= t) a = mid; else c = mid;
    }
    const uint32_t j = a;
    const uint32_t tp = t - b1[j];
    const BucketInfo B = bi[j];
    // sub-bucket: number of sub-splitters of bucket j whose bound is <= tp
    uint32_t lo = 0, hi = B.nsb - 1;
    while (lo < hi) {
        uint32_t mid = (lo + hi) >> 1;
        if (sb[(B.ss0 + mid) * p + i] <= tp) lo = mid + 1; else hi = mid;
    }
    const uint32_t k = lo;
    const uint32_t slo = k == 0 ? 0u : sb[(B.ss0 + k - 1) * p + i];
    const uint64_t r64 = soff[(uint64_t)(B.sb0 + k) * p + i] + (tp - slo);
    if (r64 >= n) {
        atomicOr(err, ERRBIT_OVERFLOW);
        return;
    }
    const uint32_t r = (uint32_t)r64;
    uint32_t s = run_perm[q];
    uint32_t tl = tlen(S, s);
    uint32_t h = 0;
    if (tp > slo) {
        uint32_t prev_tl = tlen(S, run_perm[q - 1]);
        h = run_lcp[q];
        h = h < tl ? h : tl;
        h = h < prev_tl ? h : prev_tl;
    }
    R.idx[r] = s;
    R.h[r] = h;
    R.tl[r] = tl;
    R.head[r] = load_word_be<true>(S.chars + S.offs[s], tl, h);
    clen[r] = tl - h;
}

// the lower reference string of sub-bucket b (MINF: the empty string)
__device__ __forceinline__ uint32_t sub_ref(const BucketInfo& B, uint32_t b, const uint32_t* subspl) {
    uint32_t k = b - B.sb0;
    return k == 0 ? B.fref : subspl[B.ss0 + k - 1];
}
// the upper reference string of sub-bucket b (PINF: none)
__device__ __forceinline__ uint32_t sub_uref(const BucketInfo& B, uint32_t b, const uint32_t* subspl) {
    uint32_t k = b - B.sb0;
    return k + 1 < B.nsb ? subspl[B.ss0 + k] : B.uref;
}

// Key sides of a sub-bucket's records (every record x lies in (L, U], L and U
// the sub-bucket's lower and upper reference strings, c = lcp(L, U); with
// r = lcp(x, L) and u = lcp(x, U), min(r, u) = c):
//   0: r > c, x agrees with L past c: (r descending, the 8 characters at r)
//   1: r = u = c:                    (the 8 characters at c)
//   2: r = c < u, x agrees with U:    (u ascending, the 8 characters at u)
// Side 0 members come before side 1, side 1 before side 2; members of
// different sides have lcp c.

// c = lcp(L, U) of every sub-bucket (one thread each): between two sub-splitters
// of a bucket, the minimum of the sorted samples' LCP array over the samples
// from one to the other; next to a level-1 splitter, a direct comparison; 0
// next to a missing splitter.
__global__ void k_d2_cb(Strs S, const BucketInfo* __restrict__ bi, uint32_t p, uint32_t nsb,
                        const uint32_t* __restrict__ subspl, const uint32_t* __restrict__ s2lcp,
                        uint32_t* __restrict__ cb) {
    const uint32_t b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nsb) return;
    const uint32_t j = bucket_of_sub(bi, p, b);
    const BucketInfo B = bi[j];
    const uint32_t k = b - B.sb0;
    const uint32_t L = sub_ref(B, b, subspl), U = sub_uref(B, b, subspl);
    uint32_t c = 0;
    if (L == MINF || U == PINF || U == MINF) {
        c = 0;
    } else if (k >= 1 && k + 1 < B.nsb) {
        // sub-splitters k-1 and k: sorted samples sbase + D2_OVS*k - 1 and sbase + D2_OVS*(k+1) - 1
        const uint32_t t0 = B.sbase + D2_OVS * k - 1, t1 = B.sbase + D2_OVS * (k + 1) - 1;
        c = 0xFFFFFFFFu;
        for (uint32_t t = t0 + 1; t <= t1; ++t) c = s2lcp[t] < c ? s2lcp[t] : c;
    } else {
        cmp_from(S.chars + S.offs[L], tlen(S, L), S.chars + S.offs[U], tlen(S, U), 0, &c);
    }
    cb[b] = c;
}

// Decode each slice once, one warp per slice, 32 records at a time:
//  * r = lcp with L: r(first) by a direct comparison from c = lcp(L, U) on
//    (every record of the sub-bucket shares c characters with L and U), then r(e) = min(r(prev),
//    h(e)) -- a prefix minimum of the stored LCPs;
//  * the 8 characters at r: record e agrees with its predecessor below h(e) and
//    stores its own 8 characters at h(e) (head).  Where r drops (h(e) <= r(prev))
//    the key restarts as e's head; elsewhere e's head overwrites the key's bytes
//    from h(e) - r on.  "Later head overwrites the bytes it covers" is
//    associative, so the keys of a chunk are a segmented scan over the warp;
//  * u = lcp with U: u(last) = c when r(last) > c (min(r, u) = c), else by a
//    direct comparison from c on; then u(e) = min(h(next), u(next)) -- a
//    suffix minimum;
//  * side 0 / 1 / 2 from r, u and c; at side 2 the characters at u are read
//    from the string.
// Writes rv (r, c or u), rs (side), rk (characters) per record.
__device__ __forceinline__ uint64_t d2_mask_from(uint32_t off) { return off == 0 ? ~0ull : (~0ull >> (8 * off)); }

// The two-sided path builds a slice's records and decodes them in one warp
// (k_d2_recdec): the slice's positions are walked in run order (coalesced reads
// of the run, no search for the slice, the predecessor's length by a shuffle),
// every record is written for the merge and the fallback, and the forward walk
// of the decode runs on the values still in registers.
__global__ void __launch_bounds__(256) k_d2_recdec(const uint32_t* __restrict__ run_perm,
                                                   const uint32_t* __restrict__ run_lcp, Strs S,
                                                   const BucketInfo* __restrict__ bi, uint32_t p, uint32_t nsb,
                                                   const uint32_t* __restrict__ pstart,
                                                   const uint32_t* __restrict__ psz, const uint32_t* __restrict__ sb,
                                                   const uint64_t* __restrict__ soff,
                                                   const uint32_t* __restrict__ subspl,
                                                   const uint32_t* __restrict__ cb, Recs R, uint32_t* clen,
                                                   uint32_t* rv, uint8_t* rs, uint64_t* rk) {
    const uint32_t lane = threadIdx.x & 31;
    const uint32_t g = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;  // the warp's slice (b, i)
    if (g >= nsb * p) return;
    const uint32_t b = g / p, i = g % p;
    const uint32_t j = bucket_of_sub(bi, p, b);
    const BucketInfo B = bi[j];
    uint32_t lo, hi;
    slice_range(B, b, i, p, sb, psz, j, &lo, &hi);
    if (lo >= hi) return;
    const uint32_t len = hi - lo;
    const uint32_t s0 = (uint32_t)soff[g], s1 = s0 + len;
    const uint32_t q0 = pstart[j * p + i] + lo;  // run position of the slice's first string
    const uint32_t ref = sub_ref(B, b, subspl), uref = sub_uref(B, b, subspl);
    const uint32_t c = cb[b];
    const uint32_t ef = run_perm[q0];
    const uint32_t tlf = tlen(S, ef);
    uint32_t r0 = 0, ul = 0;
    if (ref != MINF) warp_cmp_from(S.chars + S.offs[ref], tlen(S, ref), S.chars + S.offs[ef], tlf, c, &r0);
    const uint64_t key0 = load_word_be(S.chars + S.offs[ef], tlf, r0);
    // forwards: the records, then r and the characters at r
    uint32_t carry_r = 0xFFFFFFFFu, carry_tl = 0;
    uint64_t carry_key = 0;
    for (uint32_t o0 = 0; o0 < len; o0 += 32) {
        const uint32_t o = o0 + lane;
        const bool valid = o < len;
        const uint32_t t = s0 + o;
        uint32_t e = 0, tl = 0;
        if (valid) {
            e = run_perm[q0 + o];
            tl = tlen(S, e);
        }
        uint32_t prev_tl = __shfl_up_sync(SSS_FULL, tl, 1);
        if (lane == 0) prev_tl = carry_tl;
        carry_tl = __shfl_sync(SSS_FULL, tl, 31);
        uint32_t h = 0xFFFFFFFFu;
        uint64_t hw = 0ull;
        if (valid) {
            uint32_t hr = 0;  // the record's LCP with its predecessor (0 for the slice's first)
            if (o > 0) {
                hr = run_lcp[q0 + o];
                hr = hr < tl ? hr : tl;
                hr = hr < prev_tl ? hr : prev_tl;
            }
            const uint64_t head = load_word_be<true>(S.chars + S.offs[e], tl, hr);
            R.idx[t] = e;
            R.h[t] = hr;
            R.tl[t] = tl;
            R.head[t] = head;
            clen[t] = tl - hr;
            h = o == 0 ? r0 : hr;
            hw = o == 0 ? key0 : head;
        }
        uint32_t r = h;
#pragma unroll
        for (uint32_t sh = 1; sh < 32; sh <<= 1) {
            const uint32_t y = __shfl_up_sync(SSS_FULL, r, sh);
            if (lane >= sh) r = y < r ? y : r;
        }
        r = carry_r < r ? carry_r : r;
        uint32_t rp = __shfl_up_sync(SSS_FULL, r, 1);  // r after the previous record
        if (lane == 0) rp = carry_r;
        // scan element: (segment starts here, bytes written, their values)
        bool f = valid && h <= rp;
        uint64_t m = 0, w = 0;
        if (f) {
            m = ~0ull;
            w = hw;
        } else if (valid && h - r < 8) {
            m = d2_mask_from(h - r);
            w = hw >> (8 * (h - r));
        }
#pragma unroll
        for (uint32_t sh = 1; sh < 32; sh <<= 1) {
            const uint32_t lf = __shfl_up_sync(SSS_FULL, (uint32_t)f, sh);
            const uint64_t lm = __shfl_up_sync(SSS_FULL, m, sh), lw = __shfl_up_sync(SSS_FULL, w, sh);
            if (lane >= sh && !f) {
                w = (lw & ~m) | (w & m);
                m |= lm;
                f = lf != 0;
            }
        }
        const uint64_t key = f ? w : ((carry_key & ~m) | (w & m));
        if (valid) {
            rv[t] = r;
            rk[t] = key;
        }
        carry_r = __shfl_sync(SSS_FULL, r, 31);
        carry_key = __shfl_sync(SSS_FULL, key, 31);
    }
    __syncwarp();  // the records and r written above are read back below
    const uint32_t el = R.idx[s1 - 1];
    // u of the last record: c when its r (the last chunk's lane 31 holds it:
    // lanes past the slice's end leave the minimum alone) is larger, as
    // min(r, u) = c; else compared from c on
    if (uref != PINF && uref != MINF) {
        if (carry_r > c) ul = c;
        else warp_cmp_from(S.chars + S.offs[uref], tlen(S, uref), S.chars + S.offs[el], tlen(S, el), c, &ul);
    }
    // backwards
    uint32_t carry_u = ul;
    const uint32_t nch = (len + 31) / 32;
    for (uint32_t ci = nch; ci-- > 0;) {
        const uint32_t t = s0 + 32 * ci + lane;
        const bool valid = t < s1;
        uint32_t u = valid && t + 1 < s1 ? R.h[t + 1] : 0xFFFFFFFFu;  // h of the next record
#pragma unroll
        for (uint32_t sh = 1; sh < 32; sh <<= 1) {
            const uint32_t y = __shfl_down_sync(SSS_FULL, u, sh);
            if (lane + sh < 32) u = y < u ? y : u;
        }
        u = carry_u < u ? carry_u : u;
        carry_u = __shfl_sync(SSS_FULL, u, 0);
        if (valid) {
            const uint32_t rt = rv[t];
            if (rt > c) {
                rs[t] = 0;  // rv and rk hold r and the characters at r
            } else if (u > c) {
                rs[t] = 2;
                rv[t] = u;
                const uint32_t e = R.idx[t];
                rk[t] = load_word_be(S.chars + S.offs[e], R.tl[t], u);
            } else {
                rs[t] = 1;  // r = c: rk holds the characters at c
            }
        }
    }
}

// One-sided decode, one thread per slice (slices of a few records, large p):
// r and the characters at r by the forward walk only, every record on side 0
// (r > 0) or 1 (r = 0), as if U were missing (c = 0): keys relative to L, and
// runs of equal keys go to the CTA finisher.
__global__ void k_d2_decode1(Strs S, Recs R, const BucketInfo* __restrict__ bi, uint32_t p, uint32_t nsb,
                             const uint64_t* __restrict__ soff, const uint32_t* __restrict__ subspl,
                             uint32_t* __restrict__ rv, uint8_t* __restrict__ rs, uint64_t* __restrict__ rk) {
    uint32_t g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= nsb * p) return;
    uint32_t b = g / p;
    uint32_t s0 = (uint32_t)soff[g], s1 = (uint32_t)soff[g + 1];
    if (s0 >= s1) return;
    uint32_t j = bucket_of_sub(bi, p, b);
    uint32_t ref = sub_ref(bi[j], b, subspl);
    uint32_t r = 0;
    uint32_t e0 = R.idx[s0];
    if (ref != MINF) cmp_from(S.chars + S.offs[ref], tlen(S, ref), S.chars + S.offs[e0], tlen(S, e0), 0, &r);
    uint64_t key = load_word_be(S.chars + S.offs[e0], R.tl[s0], r);
    rv[s0] = r;
    rk[s0] = key;
    rs[s0] = r > 0 ? 0 : 1;
    // the walk is serial, so the records are read 8 at a time ahead of it
    for (uint32_t u0 = s0 + 1; u0 < s1; u0 += 8) {
        uint32_t hb[8];
        uint64_t wb[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            hb[i] = u0 + i < s1 ? R.h[u0 + i] : 0u;
            wb[i] = u0 + i < s1 ? R.head[u0 + i] : 0ull;  // characters [h, h+8) of the string
        }
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            if (u0 + i >= s1) break;
            const uint32_t h = hb[i];
            const uint64_t hw = wb[i];
            if (h <= r) {
                r = h;
                key = hw;
            } else if (h - r < 8) {
                uint32_t d = h - r;
                key = (key & (~0ull << (64 - 8 * d))) | (hw >> (8 * d));
            }
            rv[u0 + i] = r;
            rk[u0 + i] = key;
            rs[u0 + i] = r > 0 ? 0 : 1;
        }
    }
}

// One CTA per sub-bucket: merge its slices by (side, lcp value, next 8
// characters, run order).  A run of equal keys whose strings go on shares their
// first v+8 characters: it becomes a segment for the CTA finisher, which orders
// it from there (equal strings by index).
struct TieLists {
    Seg* tiny;
    Seg* med;
    uint32_t* cnt;  // [0] tiny, [1] med
    uint32_t cap_tiny, cap_med, lim_tiny;
};

// 128-bit merge key: side (2 bits) | field (31) | characters (64) | position (31);
// field = 2^31 - 1 - r at side 0 (r descending), v at sides 1 and 2
__device__ __forceinline__ void d2_key(uint32_t side, uint32_t v, uint64_t k, uint32_t pos, uint64_t* hi,
                                       uint64_t* lo) {
    const uint64_t field = side == 0 ? (uint64_t)(0x7FFFFFFFu - v) : (uint64_t)v;
    *hi = ((uint64_t)side << 62) | (field << 31) | (k >> 33);
    *lo = (k << 31) | pos;
}
__device__ __forceinline__ uint32_t d2_side(uint64_t hi) { return (uint32_t)(hi >> 62); }
__device__ __forceinline__ uint32_t d2_v(uint64_t hi) {
    const uint32_t f = (uint32_t)(hi >> 31) & 0x7FFFFFFFu;
    return (hi >> 62) == 0 ? 0x7FFFFFFFu - f : f;
}
__device__ __forceinline__ uint64_t d2_chars(uint64_t hi, uint64_t lo) { return (hi << 33) | (lo >> 31); }
__device__ __forceinline__ bool d2_same_key(uint64_t ha, uint64_t la, uint64_t hb, uint64_t lb) {
    return ha == hb && (la >> 31) == (lb >> 31);
}

// THREADS/CAP: the CTA's size and the largest sub-bucket it takes; sub-buckets
// of at most minsz records are left to a smaller instance.
template <int THREADS, int CAP>
__global__ void __launch_bounds__(THREADS) k_d2_cta(Strs S, Recs R, const uint64_t* __restrict__ soff, uint32_t p,
                                                    const uint32_t* __restrict__ rv, const uint8_t* __restrict__ rs,
                                                    const uint64_t* __restrict__ rk, const uint32_t* __restrict__ cb,
                                                    uint32_t* __restrict__ out_perm, uint32_t* __restrict__ out_lcp,
                                                    TieLists T, unsigned* err, uint32_t minsz) {
    extern __shared__ __align__(16) unsigned char smem[];
    uint64_t* sHi = reinterpret_cast<uint64_t*>(smem);
    uint64_t* sLo = sHi + CAP;
    const uint32_t b = blockIdx.x;
    const uint32_t base = (uint32_t)soff[(uint64_t)b * p];
    const uint32_t m = (uint32_t)soff[(uint64_t)(b + 1) * p] - base;
    if (m <= minsz || m > (uint32_t)CAP) return;
    const uint32_t c = cb[b];
    // slice i (one sorted run of the merge) is [rb[i], rb[i+1])
    __shared__ uint32_t s_rb[D2_MAXP + 1];
    const bool runs = p <= D2_MAXP;
    if (runs)
        for (uint32_t i = threadIdx.x; i <= p; i += THREADS) s_rb[i] = (uint32_t)soff[(uint64_t)b * p + i] - base;
    for (uint32_t u = threadIdx.x; u < m; u += THREADS)
        d2_key(rs[base + u], rv[base + u], rk[base + u], u, &sHi[u], &sLo[u]);
    __syncthreads();
    // every slice is ascending in these keys (along a sorted slice r never grows
    // and u never falls, so the sides come in order 0, 1, 2; within a side the
    // field does not fall, and at an equal field neither do the characters), so a
    // merge of the p slices sorts the sub-bucket
    if (!runs) block_merge_sort128_fit<THREADS, CAP / THREADS>(sHi, sLo, m);
    else if (m <= (uint32_t)CAP / 2) block_merge_runs128<THREADS, CAP / THREADS / 2>(sHi, sLo, m, s_rb, p);
    else block_merge_runs128<THREADS, CAP / THREADS>(sHi, sLo, m, s_rb, p);
    for (uint32_t t = threadIdx.x; t < m; t += THREADS) {
        const uint32_t u = (uint32_t)(sLo[t] & 0x7FFFFFFFu);
        out_perm[base + t] = R.idx[base + u];
        const uint64_t hb = sHi[t], lb = sLo[t];
        const uint32_t sideb = d2_side(hb), vb = d2_v(hb);
        const uint64_t kb = d2_chars(hb, lb);
        const bool tie_next = t + 1 < m && d2_same_key(sHi[t + 1], sLo[t + 1], hb, lb);
        bool tie_prev = false;
        if (t > 0) {
            const uint64_t ha = sHi[t - 1], la = sLo[t - 1];
            tie_prev = d2_same_key(ha, la, hb, lb);
            const uint32_t sidea = d2_side(ha), va = d2_v(ha);
            const uint64_t ka = d2_chars(ha, la);
            uint32_t l;
            if (sidea != sideb) l = c;
            else if (va != vb) l = va < vb ? va : vb;
            else if (ka != kb) l = va + word_lcp(ka, kb);
            else l = word_has_zero(kb) ? R.tl[base + u] : vb + 8;  // equal strings / set by the finisher
            out_lcp[base + t] = l;  // t == 0: overwritten by k_d2_seams
        }
        if (tie_next && !tie_prev && !word_has_zero(kb)) {
            uint32_t t1 = t + 1;
            while (t1 < m && d2_same_key(sHi[t1], sLo[t1], hb, lb)) ++t1;
            Seg sg{base + t, t1 - t, vb + 8, 0};
            if (sg.size <= T.lim_tiny) {
                uint32_t i = atomicAdd(&T.cnt[0], 1u);
                if (i < T.cap_tiny) T.tiny[i] = sg; else atomicOr(err, ERRBIT_OVERFLOW);
            } else {
                uint32_t i = atomicAdd(&T.cnt[1], 1u);
                if (i < T.cap_med) T.med[i] = sg; else atomicOr(err, ERRBIT_OVERFLOW);
            }
        }
    }
}

// LCP across sub-bucket boundaries (all outputs written); one warp per seam
__global__ void k_d2_seams(Strs S, const uint64_t* __restrict__ soff, uint32_t p, uint32_t nsb,
                           const uint32_t* __restrict__ out_perm, uint32_t* __restrict__ out_lcp) {
    uint32_t b = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (b >= nsb) return;
    uint32_t s0 = (uint32_t)soff[(uint64_t)b * p], s1 = (uint32_t)soff[(uint64_t)(b + 1) * p];
    if (s1 == s0) return;
    uint32_t l = 0;
    if (s0 > 0) {
        uint32_t a = out_perm[s0 - 1], c = out_perm[s0];
        warp_cmp_from(S.chars + S.offs[a], tlen(S, a), S.chars + S.offs[c], tlen(S, c), 0, &l);
    }
    if ((threadIdx.x & 31) == 0) out_lcp[s0] = l;
}

// fallback for oversized sub-buckets: the pairwise merge tree over their slices
__global__ void k_d2_fb_init(const uint64_t* __restrict__ soff, uint32_t p, const uint32_t* __restrict__ list,
                             uint32_t cnt, const uint32_t* __restrict__ rec_h, uint32_t* __restrict__ RA,
                             uint32_t* __restrict__ HA) {
    for (uint32_t w = blockIdx.x; w < cnt; w += gridDim.x) {
        uint32_t b = list[w];
        uint32_t s0 = (uint32_t)soff[(uint64_t)b * p], s1 = (uint32_t)soff[(uint64_t)(b + 1) * p];
        for (uint32_t u = s0 + threadIdx.x; u < s1; u += blockDim.x) {
            RA[u] = u;
            HA[u] = rec_h[u];
        }
    }
}

__global__ void k_d2_fb_out(const uint64_t* __restrict__ soff, uint32_t p, const uint32_t* __restrict__ list,
                            uint32_t cnt, const uint32_t* __restrict__ rec_idx, const uint32_t* __restrict__ RA,
                            const uint32_t* __restrict__ HA, uint32_t* __restrict__ out_perm,
                            uint32_t* __restrict__ out_lcp) {
    for (uint32_t w = blockIdx.x; w < cnt; w += gridDim.x) {
        uint32_t b = list[w];
        uint32_t s0 = (uint32_t)soff[(uint64_t)b * p], s1 = (uint32_t)soff[(uint64_t)(b + 1) * p];
        for (uint32_t u = s0 + threadIdx.x; u < s1; u += blockDim.x) {
            out_perm[u] = rec_idx[RA[u]];
            out_lcp[u] = HA[u];
        }
    }
}

struct MgBufs {
    uint32_t* smp;
    uint64_t* s_offs;
    uint32_t* s_lens;
    uint32_t* s_perm;
    uint32_t* s_lcp;
    uint32_t* spl;
    uint32_t* bounds;
    uint32_t* piece_off;
    uint32_t* bstart;
    uint32_t* clen;
    uint64_t* coff;
    uint64_t* btot;
    Recs R;
    uint32_t* RA[2];
    uint32_t* HA[2];
    Pair* pairs;
    uint32_t* srank;
    uint32_t* sl0;
    uint32_t* sl1;
    uint32_t* cnt;
    unsigned long long* ctot;  // character totals of the partitions (character-based sampling)
    uint64_t* cpre;            // character prefix over run positions, n + 1
    uint64_t* csum;            // chunk sums of cpre
    uint32_t* so;              // sample offsets per partition, p + 1
    uint32_t* scnt;            // equally spaced samples per partition
    Arena sub;  // work memory for sorting the samples
    // second level
    uint32_t cap_s2, cap_nsb;
    uint32_t* smp2;
    uint64_t* s2offs;
    uint32_t* s2lens;
    uint32_t* s2perm;
    uint32_t* s2lcp;
    uint32_t* s2rank;  // sorted rank of every second-level sample
    uint32_t* subspl;
    uint32_t* sb;
    uint32_t* ssz;
    uint64_t* soff;
    uint32_t* olist;
    BucketInfo* binfo;
    uint32_t* pstart;
    uint32_t* psz;
    uint32_t* pso;
    uint32_t* rr;
    uint8_t* rs;
    uint64_t* rk;
    uint32_t* cb;
    Seg* tie_tiny;
    Seg* tie_med;
    Arena sub2;  // work memory for sorting the second-level samples
    uint32_t max_pairs;
};

void carve_mg_small(Arena& ar, uint32_t n, uint32_t p, uint32_t v, MgBufs& b) {
    uint32_t ns = p * (v + 1);
    b.smp = ar.take<uint32_t>(ns);
    b.s_offs = ar.take<uint64_t>(ns);
    b.s_lens = ar.take<uint32_t>(ns);
    b.s_perm = ar.take<uint32_t>(ns);
    b.s_lcp = ar.take<uint32_t>(ns);
    b.spl = ar.take<uint32_t>(p);
    b.bounds = ar.take<uint32_t>((size_t)p * (p + 1));
    b.cnt = ar.take<uint32_t>(4);
    b.ctot = ar.take<unsigned long long>(p);
    b.cpre = ar.take<uint64_t>((size_t)n + 1);
    b.csum = ar.take<uint64_t>((size_t)n / CP_CHUNK + 2);
    b.so = ar.take<uint32_t>(p + 1);
    b.scnt = ar.take<uint32_t>(p);
    size_t sub = need_local_sort(ns, 1, sss_params{});
    char* base = ar.take<char>(sub);
    b.sub = Arena{base, sub, 0};
}

constexpr uint32_t MAX_P_TWO_LEVEL = 256;

void carve_mg(Arena& ar, uint32_t n, uint32_t p, uint32_t v, uint64_t nrecchars, MgBufs& b) {
    const uint32_t MS = 8;  // smallest spacing: sample arrays sized for it
    carve_mg_small(ar, n, p, v, b);
    b.piece_off = ar.take<uint32_t>((size_t)p * p);
    b.bstart = ar.take<uint32_t>(p + 1);
    b.clen = ar.take<uint32_t>(n);
    b.coff = ar.take<uint64_t>(n + 1);
    b.R.idx = ar.take<uint32_t>(n);
    b.R.h = ar.take<uint32_t>(n);
    b.R.tl = ar.take<uint32_t>(n);
    b.R.base = ar.take<uint64_t>(n);
    b.R.head = ar.take<uint64_t>(n);
    b.R.chars = ar.take<uint8_t>(nrecchars + 16);
    b.RA[0] = ar.take<uint32_t>(n);
    b.RA[1] = ar.take<uint32_t>(n);
    b.HA[0] = ar.take<uint32_t>(n);
    b.HA[1] = ar.take<uint32_t>(n);
    // second level (sized for the smallest sample step, 16)
    b.cap_s2 = n / 16 + 16;
    b.cap_nsb = b.cap_s2 / D2_OVS + p + 1;
    uint32_t pp = p <= MAX_P_TWO_LEVEL ? p : 1;
    size_t nslices = (size_t)b.cap_nsb * pp;
    // pairwise-tree pairs over all levels: the level-1 tree has fewer than p*p + p
    // (every level halves the runs of a bucket, and a pair needs a non-empty run);
    // the oversized-sub-bucket tree fewer than its slices
    uint32_t lg = 1;
    while ((1u << lg) < p) ++lg;
    size_t tree1 = std::min<size_t>((size_t)p * p + p, (size_t)n * (lg + 1));
    b.max_pairs = (uint32_t)(std::max<size_t>(tree1, (p <= MAX_P_TWO_LEVEL ? nslices : 0)) + 64);
    b.pairs = ar.take<Pair>(b.max_pairs);
    uint32_t maxs = n / MS + b.max_pairs * 2 + 2;
    b.srank = ar.take<uint32_t>(maxs);
    b.sl0 = ar.take<uint32_t>(maxs);
    b.sl1 = ar.take<uint32_t>(maxs);
    b.btot = ar.take<uint64_t>((std::max<size_t>(n, nslices) + 1) / 4096 + 4);
    b.smp2 = ar.take<uint32_t>(b.cap_s2);
    b.s2offs = ar.take<uint64_t>(b.cap_s2);
    b.s2lens = ar.take<uint32_t>(b.cap_s2);
    b.s2perm = ar.take<uint32_t>(b.cap_s2);
    b.s2lcp = ar.take<uint32_t>(b.cap_s2);
    b.s2rank = ar.take<uint32_t>(b.cap_s2);
    b.subspl = ar.take<uint32_t>(b.cap_nsb);
    b.sb = ar.take<uint32_t>(nslices);
    b.ssz = ar.take<uint32_t>(nslices);
    b.soff = ar.take<uint64_t>(nslices + 1);
    b.olist = ar.take<uint32_t>(b.cap_nsb);
    b.binfo = ar.take<BucketInfo>(p);
    b.pstart = ar.take<uint32_t>((size_t)p * p);
    b.psz = ar.take<uint32_t>((size_t)p * p);
    b.pso = ar.take<uint32_t>((size_t)p * p + 1);
    b.rr = ar.take<uint32_t>(n);
    b.rs = ar.take<uint8_t>(n);
    b.rk = ar.take<uint64_t>(n);
    b.cb = ar.take<uint32_t>(b.cap_nsb);
    b.tie_tiny = ar.take<Seg>(n / 2 + 2);
    b.tie_med = ar.take<Seg>(n / 65 + 2);
    size_t sub2 = need_local_sort(b.cap_s2, 1, sss_params{});
    char* base2 = ar.take<char>(sub2);
    b.sub2 = Arena{base2, sub2, 0};
}

__global__ void __launch_bounds__(256) k_sum_tlen(Strs S, uint32_t n, unsigned long long* out) {
    __shared__ uint64_t sw[8];
    uint64_t v = 0;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) v += tlen(S, i);
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(SSS_FULL, v, o);
    if ((threadIdx.x & 31) == 0) sw[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint64_t t = 0;
        for (int w = 0; w < 8; ++w) t += sw[w];
        if (t) atomicAdd(out, (unsigned long long)t);
    }
}

__global__ void k_iota(uint32_t* a, uint32_t n) {
    uint32_t q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q < n) a[q] = q;
}

}  // namespace

// Stage C into b (splitters and bounds on the device).
// Character-based samples (Section 3.1.2) into b.smp/s_offs/s_lens; *ns_out =
// their count, or 0 when the strings hold no characters (string-based then).
static sss_status char_samples(sss_ctx* ctx, const uint32_t* run_perm, uint32_t n, uint32_t p, uint32_t v,
                               const Strs& S, MgBufs& b, uint32_t* ns_out) {
    *ns_out = 0;
    SSS_CUDA(cudaMemsetAsync(b.ctot, 0, sizeof(unsigned long long) * p, ctx->stream));
    const uint32_t per_part = (n / p + 1 + 8191) / 8192;
    SSS_TRY(sss_launch(ctx, "c_chartot", k_c_chartot, dim3(std::max(1u, std::min(per_part, 1024u)), p), dim3(256), 0,
                       S, n, p, b.ctot));
    const uint32_t nc = (n + CP_CHUNK - 1) / CP_CHUNK;
    SSS_TRY(sss_launch(ctx, "c_psum", k_c_psum, dim3(nc), dim3(CP_T), 0, S, run_perm, n, b.csum));
    SSS_TRY(sss_launch(ctx, "c_pscan", k_c_pscan, dim3(1), dim3(CP_T), 0, b.csum, nc));
    SSS_TRY(sss_launch(ctx, "c_pwrite", k_c_pwrite, dim3(nc), dim3(CP_T), 0, S, run_perm, n, (const uint64_t*)b.csum,
                       b.cpre));
    void* pin;
    SSS_TRY(sss_pinned(ctx, sizeof(uint64_t) * p + sizeof(uint32_t) * (2 * p + 2), &pin));
    uint64_t* hc = static_cast<uint64_t*>(pin);
    SSS_CUDA(cudaMemcpyAsync(hc, b.ctot, sizeof(uint64_t) * p, cudaMemcpyDeviceToHost, ctx->stream));
    SSS_CUDA(cudaStreamSynchronize(ctx->stream));
    uint64_t N = 0;
    for (uint32_t i = 0; i < p; ++i) N += hc[i];
    if (N == 0) return SSS_OK;
    const uint64_t want = (uint64_t)p * (v + 1);
    if (N > UINT64_MAX / want) return sss_fail(ctx, SSS_ERR_UNIMPLEMENTED, "character-based sampling: too many characters");
    uint32_t* hso = reinterpret_cast<uint32_t*>(hc + p);
    uint32_t* hcnt = hso + p + 1;
    uint64_t total = 0;
    for (uint32_t i = 0; i < p; ++i) {
        uint64_t c = (hc[i] * want + N - 1) / N;  // ceil(C_i / w), w = N / want
        hcnt[i] = (uint32_t)(c ? c - 1 : 0);
        total += hcnt[i];
    }
    uint64_t extra = total < want ? want - total : 0;
    uint32_t o = 0;
    for (uint32_t i = 0; i < p; ++i) {
        hso[i] = o;
        o += hcnt[i];
        if (extra > 0 && part_lo(n, p, i + 1) > part_lo(n, p, i)) {  // the first partitions' extra sample
            ++o;
            --extra;
        }
    }
    hso[p] = o;
    if (o > want) return sss_fail(ctx, SSS_ERR_CUDA, "character-based sampling: sample count");
    SSS_TRY(sss_upload(ctx, b.so, hso, sizeof(uint32_t) * (p + 1)));
    SSS_TRY(sss_upload(ctx, b.scnt, hcnt, sizeof(uint32_t) * p));
    SSS_TRY(sss_launch(ctx, "c_csamples", k_c_csamples, dim3((o + 127) / 128), dim3(128), 0, run_perm, n, p, S,
                       (const uint64_t*)b.cpre, (const uint32_t*)b.so, (const uint32_t*)b.scnt, N, want, b.smp,
                       b.s_offs, b.s_lens));
    *ns_out = o;
    return SSS_OK;
}

static sss_status run_partition(sss_ctx* ctx, const StrIn& in, const uint32_t* trunc, const uint32_t* run_perm,
                                uint32_t p, uint32_t v, uint32_t flags, MgBufs& b) {
    const uint32_t n = in.n;
    Strs S{in.chars, in.offs, in.lens, trunc};
    uint32_t ne = 0;
    for (uint32_t i = 0; i < p; ++i) ne += part_lo(n, p, i + 1) > part_lo(n, p, i) ? 1u : 0u;
    uint32_t ns = 0;
    if ((flags & SSS_FLAG_CHAR_SAMPLING) && n > 0) SSS_TRY(char_samples(ctx, run_perm, n, p, v, S, b, &ns));
    if (ns == 0) {
        ns = ne * (v + 1);
        uint32_t tot = p * (v + 1);
        SSS_TRY(sss_launch(ctx, "c_samples", k_c_samples, dim3((tot + 127) / 128), dim3(128), 0, run_perm, n, p, v, S,
                           b.smp, b.s_offs, b.s_lens, b.cnt));
    }
    // sort the samples (views of the same characters, truncated) with stage A;
    // equal truncated samples keep sample order, which is input-index order
    StrIn sin{in.chars, in.n_chars, b.s_offs, b.s_lens, ns};
    Arena sub = b.sub;
    SSS_TRY(impl_local_sort(ctx, sub, sin, 1, sss_params{}, b.s_perm, b.s_lcp));
    SSS_TRY(sss_launch(ctx, "c_splitters", k_c_splitters, dim3((p + 127) / 128), dim3(128), 0, (const uint32_t*)b.smp,
                       (const uint32_t*)b.s_perm, ns, p, b.spl));
    uint32_t nb = p * (p + 1);
    SSS_TRY(sss_launch(ctx, "c_bounds", k_c_bounds, dim3((nb * 32 + 127) / 128), dim3(128), 0, run_perm, n, p, S,
                       (const uint32_t*)b.spl, b.bounds));
    return SSS_OK;
}

size_t need_partition(uint32_t n, uint32_t p, uint32_t v) {
    Arena ar;
    MgBufs b;
    carve_mg_small(ar, n, p, v, b);
    return ar.off + 256;
}

sss_status impl_partition(sss_ctx* ctx, Arena& ar, const StrIn& in, const uint32_t* trunc, const uint32_t* run_perm,
                          uint32_t p, uint32_t v, uint32_t flags, uint32_t* out_spl, uint32_t* out_bounds) {
    MgBufs b;
    carve_mg_small(ar, in.n, p, v, b);
    SSS_TRY(run_partition(ctx, in, trunc, run_perm, p, v, flags, b));
    if (p > 1 && out_spl)
        SSS_CUDA(cudaMemcpyAsync(out_spl, b.spl, sizeof(uint32_t) * (p - 1), cudaMemcpyDeviceToDevice, ctx->stream));
    SSS_CUDA(cudaMemcpyAsync(out_bounds, b.bounds, sizeof(uint32_t) * p * (p + 1), cudaMemcpyDeviceToDevice,
                             ctx->stream));
    return SSS_OK;
}

size_t need_merge(uint32_t n, uint32_t p, uint32_t v, uint64_t nrecchars) {
    Arena ar;
    MgBufs b;
    carve_mg(ar, n, p, v, nrecchars, b);
    return ar.off + 256;
}

// Stages C and D.  The record-character bound (sum of truncated lengths) is
// needed to size the work memory, so it is computed first by the caller.
// exclusive scan of count u32 values into u64 offsets (out[count] is not written)
static sss_status scan_u32_u64(sss_ctx* ctx, const uint32_t* in, uint32_t count, uint64_t* out, uint64_t* btot) {
    if (count == 0) return SSS_OK;
    uint32_t nblk = (count + 4095) / 4096;
    SSS_TRY(sss_launch(ctx, "d_scan", k_scan_blocks, dim3(nblk), dim3(1024), 0, in, count, out, btot));
    SSS_TRY(sss_launch(ctx, "d_scan_tot", k_scan_totals, dim3(1), dim3(1024), 0, btot, nblk));
    SSS_TRY(sss_launch(ctx, "d_scan_add", k_scan_add, dim3((count + 255) / 256), dim3(256), 0, out, count,
                       (const uint64_t*)btot));
    return SSS_OK;
}

sss_status impl_scan_u32_u64(sss_ctx* ctx, const uint32_t* in, uint32_t count, uint64_t* out, uint64_t* btot) {
    return scan_u32_u64(ctx, in, count, out, btot);
}

// Pairwise merge tree over groups of runs: group g occupies [base_g, ...) with
// run sizes sizes_g; every level's pairs are planned at once.
struct TreePlan {
    std::vector<Pair> pairs;
    std::vector<uint32_t> first, np, ns;
};

static void plan_tree(std::vector<std::pair<uint32_t, std::vector<uint32_t>>> groups, uint32_t MS, TreePlan& T) {
    for (;;) {
        bool more = false;
        for (auto& g : groups) more |= g.second.size() > 1;
        if (!more) break;
        uint32_t np = 0, ns = 0;
        T.first.push_back((uint32_t)T.pairs.size());
        for (auto& g : groups) {
            uint32_t pos = g.first;
            std::vector<uint32_t> next;
            for (size_t k = 0; k < g.second.size(); k += 2) {
                uint32_t na = g.second[k], nb = k + 1 < g.second.size() ? g.second[k + 1] : 0;
                if (na + nb > 0) {
                    Pair pr{};
                    pr.a0 = pos;
                    pr.na = na;
                    pr.b0 = pos + na;
                    pr.nb = nb;
                    pr.sa = ns;
                    ns += (na + MS - 1) / MS;
                    pr.sb = ns;
                    ns += (nb + MS - 1) / MS;
                    T.pairs.push_back(pr);
                    ++np;
                }
                pos += na + nb;
                next.push_back(na + nb);
            }
            g.second = next;
        }
        T.np.push_back(np);
        T.ns.push_back(ns);
    }
}

static sss_status run_tree(sss_ctx* ctx, MgBufs& b, const Strs& S, const TreePlan& T, Pair* hpairs, int* cur_io,
                           uint32_t MS) {
    const uint32_t nlev = (uint32_t)T.np.size();
    if (nlev == 0) return SSS_OK;
    if (T.pairs.size() > b.max_pairs) return sss_fail(ctx, SSS_ERR_CUDA, "merge: pair table overflow");
    std::copy(T.pairs.begin(), T.pairs.end(), hpairs);
    SSS_TRY(sss_upload(ctx, b.pairs, hpairs, sizeof(Pair) * T.pairs.size()));
    int cur = *cur_io;
    for (uint32_t lv = 0; lv < nlev; ++lv) {
        const Pair* pr = b.pairs + T.first[lv];
        uint32_t np = T.np[lv], ns = T.ns[lv];
        SSS_TRY(sss_launch(ctx, "d_search", k_d_search, dim3((ns + 127) / 128), dim3(128), 0, S, b.R,
                           (const uint32_t*)b.RA[cur], pr, np, ns, b.srank, b.sl0, b.sl1, MS));
        SSS_TRY(sss_launch(ctx, "d_merge", k_d_merge, dim3((ns + 127) / 128), dim3(128), 0, S, b.R,
                           (const uint32_t*)b.RA[cur], (const uint32_t*)b.HA[cur], b.RA[cur ^ 1], b.HA[cur ^ 1],
                           pr, np, ns, (const uint32_t*)b.srank, (const uint32_t*)b.sl0, (const uint32_t*)b.sl1,
                           MS));
        cur ^= 1;
    }
    *cur_io = cur;
    return SSS_OK;
}

static bool g_mg_attr[64];

sss_status impl_merge(sss_ctx* ctx, char* ws, size_t ws_bytes, const StrIn& in, const uint32_t* trunc,
                      const uint32_t* run_perm, const uint32_t* run_lcp, uint32_t p, uint32_t v, uint32_t ms_param,
                      uint32_t flags, uint64_t nrecchars, uint32_t* out_perm, uint32_t* out_lcp) {
    uint32_t MS = MS_DEFAULT;
    if (ms_param >= 8 && ms_param <= 1024 && (ms_param & (ms_param - 1)) == 0) MS = ms_param;
    const uint32_t n = in.n;
    if (p == 1) {  // one sorted run: it is the result
        SSS_CUDA(cudaMemcpyAsync(out_perm, run_perm, sizeof(uint32_t) * n, cudaMemcpyDeviceToDevice, ctx->stream));
        SSS_CUDA(cudaMemcpyAsync(out_lcp, run_lcp, sizeof(uint32_t) * n, cudaMemcpyDeviceToDevice, ctx->stream));
        return SSS_OK;
    }
    if (!g_mg_attr[ctx->device & 63]) {
        SSS_CUDA(cudaFuncSetAttribute(k_d2_cta<D2_T, D2_CAP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)(D2_CAP * (8 + 8))));
        g_mg_attr[ctx->device & 63] = true;
    }
    Arena ar{ws, ws_bytes, 0};
    MgBufs b;
    carve_mg(ar, n, p, v, nrecchars, b);
    Strs S{in.chars, in.offs, in.lens, trunc};
    SSS_TRY(run_partition(ctx, in, trunc, run_perm, p, v, flags, b));
    const bool two_level = p <= MAX_P_TWO_LEVEL && !(flags & SSS_FLAG_MERGE_TREE);

    // level-1 bounds and splitters to the host
    void* pin;
    const size_t npieces = (size_t)p * p;
    size_t pin_need = sizeof(uint32_t) * ((size_t)p * (p + 1) + p + 4 * npieces + 16) + sizeof(BucketInfo) * p +
                      sizeof(Pair) * (b.max_pairs + 16) + 4096;
    SSS_TRY(sss_pinned(ctx, pin_need, &pin));
    uint32_t* hb = static_cast<uint32_t*>(pin);
    uint32_t* hspl = hb + (size_t)p * (p + 1);
    uint32_t* hpo = hspl + p;             // piece_off   [p*p]
    uint32_t* hpst = hpo + npieces;       // pstart      [p*p]
    uint32_t* hpsz = hpst + npieces;      // psz         [p*p]
    uint32_t* hpso = hpsz + npieces;      // pso         [p*p+1]
    uint32_t* hbs = hpso + npieces + 1;   // bstart      [p+1]
    BucketInfo* hbi = reinterpret_cast<BucketInfo*>(reinterpret_cast<uintptr_t>(hbs + p + 1 + 15) & ~uintptr_t(15));
    uint64_t* hn = reinterpret_cast<uint64_t*>(hbi + p);
    uint32_t* hcnt = reinterpret_cast<uint32_t*>(hn + 2);
    Pair* hpairs = reinterpret_cast<Pair*>(reinterpret_cast<uintptr_t>(hcnt + 8 + 15) & ~uintptr_t(15));
    SSS_CUDA(cudaMemcpyAsync(hb, b.bounds, sizeof(uint32_t) * p * (p + 1), cudaMemcpyDeviceToHost, ctx->stream));
    SSS_CUDA(cudaMemcpyAsync(hspl, b.spl, sizeof(uint32_t) * (p - 1), cudaMemcpyDeviceToHost, ctx->stream));
    SSS_CUDA(cudaStreamSynchronize(ctx->stream));
    uint32_t acc = 0;
    for (uint32_t j = 0; j < p; ++j) {
        hbs[j] = acc;
        for (uint32_t i = 0; i < p; ++i) {
            uint32_t sz = hb[(size_t)i * (p + 1) + j + 1] - hb[(size_t)i * (p + 1) + j];
            hpsz[(size_t)j * p + i] = sz;
            hpst[(size_t)j * p + i] = part_lo(n, p, i) + hb[(size_t)i * (p + 1) + j];
            hpo[(size_t)j * p + i] = acc;
            acc += sz;
        }
    }
    hbs[p] = acc;
    if (acc != n) return sss_fail(ctx, SSS_ERR_CUDA, "merge: bucket bounds do not cover the input");
    int cur = 0;

    if (!two_level) {
        // D1 into level-1 buckets, then the pairwise merge tree per bucket
        SSS_TRY(sss_upload(ctx, b.piece_off, hpo, sizeof(uint32_t) * npieces));
        SSS_TRY(sss_upload(ctx, b.bstart, hbs, sizeof(uint32_t) * (p + 1)));
        SSS_TRY(sss_launch(ctx, "d_records", k_d_records, dim3((n + 255) / 256), dim3(256), 0, run_perm, run_lcp, n,
                           p, S, (const uint32_t*)b.bounds, (const uint32_t*)b.piece_off, b.R, b.clen, ctx->d_err));
        SSS_TRY(scan_u32_u64(ctx, b.clen, n, b.coff, b.btot));
        SSS_TRY(sss_launch(ctx, "d_copy", k_d_copy, dim3((n + 127) / 128), dim3(128), 0, S, b.R,
                           (const uint64_t*)b.coff, n));
        SSS_TRY(sss_launch(ctx, "d_iota", k_iota, dim3((n + 255) / 256), dim3(256), 0, b.RA[0], n));
        SSS_CUDA(cudaMemcpyAsync(b.HA[0], b.R.h, sizeof(uint32_t) * n, cudaMemcpyDeviceToDevice, ctx->stream));
        std::vector<std::pair<uint32_t, std::vector<uint32_t>>> groups(p);
        for (uint32_t j = 0; j < p; ++j) {
            groups[j].first = hbs[j];
            groups[j].second.assign(hpsz + (size_t)j * p, hpsz + (size_t)(j + 1) * p);
        }
        TreePlan T;
        plan_tree(groups, MS, T);
        SSS_TRY(run_tree(ctx, b, S, T, hpairs, &cur, MS));
        SSS_TRY(sss_launch(ctx, "d_seams", k_d_seams, dim3((p + 127) / 128), dim3(128), 0, S, b.R,
                           (const uint32_t*)b.RA[cur], b.HA[cur], (const uint32_t*)b.bstart, p));
        return sss_launch(ctx, "d_out", k_d_out, dim3((n + 255) / 256), dim3(256), 0, b.R,
                          (const uint32_t*)b.RA[cur], (const uint32_t*)b.HA[cur], n, out_perm, out_lcp);
    }

    // second-level plan: regular samples every `step` strings of every piece
    const uint32_t step = std::max<uint32_t>(16u, D2_CAP / (D2_OVS + p));
    uint32_t S2 = 0, NSB = 0, NSS = 0, sbase = 0;
    for (uint32_t j = 0; j < p; ++j) {
        uint32_t nsmp = 0;
        for (uint32_t i = 0; i < p; ++i) {
            hpso[(size_t)j * p + i] = S2;
            uint32_t c = hpsz[(size_t)j * p + i] / step;
            S2 += c;
            nsmp += c;
        }
        BucketInfo bi{};
        bi.sbase = sbase;
        bi.nsmp = nsmp;
        bi.nsb = nsmp / D2_OVS + 1;
        bi.sb0 = NSB;
        bi.ss0 = NSS;
        bi.fref = j == 0 ? MINF : hspl[j - 1];
        bi.uref = j + 1 < p ? hspl[j] : PINF;
        hbi[j] = bi;
        sbase += nsmp;
        NSB += bi.nsb;
        NSS += bi.nsb - 1;
    }
    hpso[npieces] = S2;
    if (S2 > b.cap_s2 || NSB > b.cap_nsb) return sss_fail(ctx, SSS_ERR_CUDA, "merge: second-level capacity");
    *hn = n;
    SSS_TRY(sss_upload(ctx, b.binfo, hbi, sizeof(BucketInfo) * p));
    SSS_TRY(sss_upload(ctx, b.pstart, hpst, sizeof(uint32_t) * npieces));
    SSS_TRY(sss_upload(ctx, b.psz, hpsz, sizeof(uint32_t) * npieces));
    SSS_TRY(sss_upload(ctx, b.pso, hpso, sizeof(uint32_t) * (npieces + 1)));
    const uint32_t nslices = NSB * p;
    SSS_TRY(sss_upload(ctx, b.soff + nslices, hn, sizeof(uint64_t)));
    if (S2 > 0) {
        SSS_TRY(sss_launch(ctx, "d2_samples", k_d2_samples, dim3((S2 + 255) / 256), dim3(256), 0, run_perm, S,
                           (const uint32_t*)b.pso, (const uint32_t*)b.pstart, (uint32_t)npieces, S2, step, b.smp2,
                           b.s2offs, b.s2lens));
        StrIn sin{in.chars, in.n_chars, b.s2offs, b.s2lens, S2};
        Arena sub = b.sub2;
        // the samples' round loop as a cached graph: a sort this small is bound by
        // the host's launches and per-round synchronisation otherwise
        sss_params sp{};
        sp.flags = SSS_FLAG_GRAPH;
        const char* tag = ctx->graph_tag;
        ctx->graph_tag = "d2_sample_sort";  // stage D's time in the statistics
        const sss_status ss = impl_local_sort(ctx, sub, sin, 1, sp, b.s2perm, b.s2lcp);
        ctx->graph_tag = tag;
        SSS_TRY(ss);
    }
    if (NSS > 0) {
        SSS_TRY(sss_launch(ctx, "d2_subspl", k_d2_subspl, dim3((NSS + 255) / 256), dim3(256), 0,
                           (const BucketInfo*)b.binfo, p, NSS, (const uint32_t*)b.smp2, (const uint32_t*)b.s2perm,
                           b.subspl));
        SSS_TRY(sss_launch(ctx, "d2_srank", k_d2_srank, dim3((S2 + 255) / 256), dim3(256), 0,
                           (const uint32_t*)b.s2perm, S2, b.s2rank));
        SSS_TRY(sss_launch(ctx, "d2_bounds", k_d2_bounds, dim3((NSS * p * 32 + 127) / 128), dim3(128), 0, run_perm,
                           S, (const BucketInfo*)b.binfo, p, NSS, (const uint32_t*)b.pstart, (const uint32_t*)b.psz,
                           (const uint32_t*)b.pso, (const uint32_t*)b.subspl, (const uint32_t*)b.s2perm,
                           (const uint32_t*)b.s2rank, (const uint32_t*)b.s2lcp, (const uint32_t*)b.s2lens, step,
                           b.sb));
    }
    SSS_TRY(sss_launch(ctx, "d2_slices", k_d2_slices, dim3((nslices + 255) / 256), dim3(256), 0,
                       (const BucketInfo*)b.binfo, p, NSB, (const uint32_t*)b.sb, (const uint32_t*)b.psz, b.ssz));
    SSS_TRY(scan_u32_u64(ctx, b.ssz, nslices, b.soff, b.btot));
    SSS_CUDA(cudaMemsetAsync(b.cnt, 0, sizeof(uint32_t), ctx->stream));
    SSS_TRY(sss_launch(ctx, "d2_oversized", k_d2_oversized, dim3((NSB + 255) / 256), dim3(256), 0,
                       (const uint64_t*)b.soff, p, NSB, b.olist, b.cnt));
    // D1 (LCP-compressed records of every sub-bucket slice) and the decode of D2.
    // Slices of 16 or more records on average: the two-sided decode, a warp per
    // slice, which also builds the slice's records; shorter slices (large p):
    // the records by position, then the one-sided forward walk, a thread per
    // slice, with c = 0 for every sub-bucket.
    const bool two_sided = (uint64_t)n >= 16ull * nslices;
    if (!two_sided) {
        SSS_TRY(sss_launch(ctx, "d2_records", k_d2_records, dim3((n + 255) / 256), dim3(256), 0, run_perm, run_lcp, n,
                           p, S, (const uint32_t*)b.bounds, (const BucketInfo*)b.binfo, (const uint32_t*)b.sb,
                           (const uint64_t*)b.soff, b.R, b.clen, ctx->d_err));
        SSS_CUDA(cudaMemsetAsync(b.cb, 0, sizeof(uint32_t) * NSB, ctx->stream));
        SSS_TRY(sss_launch(ctx, "d2_decode", k_d2_decode1, dim3((nslices + 127) / 128), dim3(128), 0, S, b.R,
                           (const BucketInfo*)b.binfo, p, NSB, (const uint64_t*)b.soff, (const uint32_t*)b.subspl,
                           b.rr, b.rs, b.rk));
    } else {
        SSS_TRY(sss_launch(ctx, "d2_cb", k_d2_cb, dim3((NSB + 255) / 256), dim3(256), 0, S,
                           (const BucketInfo*)b.binfo, p, NSB, (const uint32_t*)b.subspl, (const uint32_t*)b.s2lcp,
                           b.cb));
        SSS_TRY(sss_launch(ctx, "d2_recdec", k_d2_recdec, dim3((nslices * 32 + 255) / 256), dim3(256), 0, run_perm,
                           run_lcp, S, (const BucketInfo*)b.binfo, p, NSB, (const uint32_t*)b.pstart,
                           (const uint32_t*)b.psz, (const uint32_t*)b.sb, (const uint64_t*)b.soff,
                           (const uint32_t*)b.subspl, (const uint32_t*)b.cb, b.R, b.clen, b.rr, b.rs, b.rk));
    }
    TieLists TL{b.tie_tiny, b.tie_med, b.cnt + 1, n / 2 + 2, n / 65 + 2, finish_cap_tiny()};
    SSS_CUDA(cudaMemsetAsync(b.cnt + 1, 0, sizeof(uint32_t) * 2, ctx->stream));
    // when sub-buckets are small (large p: their mean is D2_OVS * step), those of
    // at most D2_SMALL records go to 128-thread CTAs, the others to 512-thread CTAs
    const bool small = D2_OVS * step <= D2_SMALL;
    if (small)
        SSS_TRY(sss_launch(ctx, "d2_cta", k_d2_cta<D2_T_SMALL, D2_SMALL>, dim3(NSB), dim3(D2_T_SMALL),
                           (size_t)D2_SMALL * (8 + 8), S, b.R, (const uint64_t*)b.soff, p, (const uint32_t*)b.rr,
                           (const uint8_t*)b.rs, (const uint64_t*)b.rk, (const uint32_t*)b.cb, out_perm, out_lcp, TL,
                           ctx->d_err, 0u));
    SSS_TRY(sss_launch(ctx, "d2_cta", k_d2_cta<D2_T, D2_CAP>, dim3(NSB), dim3(D2_T), (size_t)D2_CAP * (8 + 8), S,
                       b.R, (const uint64_t*)b.soff, p, (const uint32_t*)b.rr, (const uint8_t*)b.rs,
                       (const uint64_t*)b.rk, (const uint32_t*)b.cb, out_perm, out_lcp, TL, ctx->d_err,
                       small ? D2_SMALL : 0u));
    // oversized sub-buckets (many equal strings): pairwise merge tree over their slices.
    // (the sample sort above may have grown the pinned staging: re-derive pointers)
    {
        const size_t off_cnt = reinterpret_cast<char*>(hcnt) - static_cast<char*>(pin);
        const size_t off_pairs = reinterpret_cast<char*>(hpairs) - static_cast<char*>(pin);
        SSS_TRY(sss_pinned(ctx, pin_need, &pin));
        hcnt = reinterpret_cast<uint32_t*>(static_cast<char*>(pin) + off_cnt);
        hpairs = reinterpret_cast<Pair*>(static_cast<char*>(pin) + off_pairs);
    }
    SSS_CUDA(cudaMemcpyAsync(hcnt, b.cnt, sizeof(uint32_t) * 3, cudaMemcpyDeviceToHost, ctx->stream));
    SSS_CUDA(cudaStreamSynchronize(ctx->stream));
    const uint32_t nover = hcnt[0];
    if (hcnt[1] > n / 2 + 2 || hcnt[2] > n / 65 + 2) return sss_fail(ctx, SSS_ERR_CUDA, "merge: tie list overflow");
    if (hcnt[1] + hcnt[2] > 0) {
        // strings compared as their truncated prefixes
        StrIn tin{in.chars, in.n_chars, in.offs, trunc ? trunc : in.lens, n};
        SSS_TRY(impl_finish_segments(ctx, b.tie_tiny, hcnt[1], b.tie_med, hcnt[2], tin, out_perm, out_lcp));
    }
    if (nover > 0) {
        std::vector<uint32_t> olist(nover);
        std::vector<uint32_t> sizes((size_t)nover * p);
        std::vector<uint64_t> base(nover);
        SSS_CUDA(cudaMemcpy(olist.data(), b.olist, sizeof(uint32_t) * nover, cudaMemcpyDeviceToHost));
        std::vector<std::pair<uint32_t, std::vector<uint32_t>>> groups(nover);
        for (uint32_t w = 0; w < nover; ++w) {
            uint32_t sbk = olist[w];
            SSS_CUDA(cudaMemcpy(&base[w], b.soff + (size_t)sbk * p, sizeof(uint64_t), cudaMemcpyDeviceToHost));
            SSS_CUDA(cudaMemcpy(sizes.data() + (size_t)w * p, b.ssz + (size_t)sbk * p, sizeof(uint32_t) * p,
                                cudaMemcpyDeviceToHost));
            groups[w].first = (uint32_t)base[w];
            groups[w].second.assign(sizes.begin() + (size_t)w * p, sizes.begin() + (size_t)(w + 1) * p);
        }
        // the pairwise tree compares record characters: materialise them
        SSS_TRY(scan_u32_u64(ctx, b.clen, n, b.coff, b.btot));
        SSS_TRY(sss_launch(ctx, "d_copy", k_d_copy, dim3((n + 127) / 128), dim3(128), 0, S, b.R,
                           (const uint64_t*)b.coff, n));
        SSS_TRY(sss_launch(ctx, "d2_fb_init", k_d2_fb_init, dim3(std::min<uint32_t>(nover, 1024)), dim3(256), 0,
                           (const uint64_t*)b.soff, p, (const uint32_t*)b.olist, nover, (const uint32_t*)b.R.h,
                           b.RA[0], b.HA[0]));
        TreePlan T;
        plan_tree(groups, MS, T);
        cur = 0;
        SSS_TRY(run_tree(ctx, b, S, T, hpairs, &cur, MS));
        SSS_TRY(sss_launch(ctx, "d2_fb_out", k_d2_fb_out, dim3(std::min<uint32_t>(nover, 1024)), dim3(256), 0,
                           (const uint64_t*)b.soff, p, (const uint32_t*)b.olist, nover, (const uint32_t*)b.R.idx,
                           (const uint32_t*)b.RA[cur], (const uint32_t*)b.HA[cur], out_perm, out_lcp));
    }
    // D3
    return sss_launch(ctx, "d2_seams", k_d2_seams, dim3((NSB * 32 + 255) / 256), dim3(256), 0, S, (const uint64_t*)b.soff,
                      p, NSB, (const uint32_t*)out_perm, out_lcp);
}

// Sum of the (truncated) lengths: an upper bound on the record characters.
sss_status impl_sum_tlen(sss_ctx* ctx, const StrIn& in, const uint32_t* trunc, uint64_t* out) {
    void* pin;
    SSS_TRY(sss_pinned(ctx, 64, &pin));
    unsigned long long* d = ctx->d_small;
    SSS_CUDA(cudaMemsetAsync(d, 0, sizeof(unsigned long long), ctx->stream));
    Strs S{in.chars, in.offs, in.lens, trunc};
    uint32_t grid = std::min<uint32_t>((in.n + 255) / 256, 4u * (uint32_t)ctx->sm_count);
    SSS_TRY(sss_launch(ctx, "sum_tlen", k_sum_tlen, dim3(grid), dim3(256), 0, S, in.n, d));
    SSS_CUDA(cudaMemcpyAsync(pin, d, sizeof(unsigned long long), cudaMemcpyDeviceToHost, ctx->stream));
    SSS_CUDA(cudaStreamSynchronize(ctx->stream));
    *out = *static_cast<unsigned long long*>(pin);
    return SSS_OK;
}
