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

// bounds[i*(p+1)+j] = #{ s in run i : s <= f_j }, LCP-aware binary search
__global__ void k_c_bounds(const uint32_t* __restrict__ run_perm, uint32_t n, uint32_t p, Strs S,
                           const uint32_t* __restrict__ spl, uint32_t* __restrict__ bounds) {
    uint32_t g = blockIdx.x * blockDim.x + threadIdx.x;
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
            int c = cmp_from(S.chars + S.offs[e], tlen(S, e), fs, fl, d, &l);
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
    bounds[g] = res;
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
    Arena sub;  // work memory for sorting the samples
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
    size_t sub = need_local_sort(ns, 1, sss_params{});
    char* base = ar.take<char>(sub);
    b.sub = Arena{base, sub, 0};
    (void)n;
}

void carve_mg(Arena& ar, uint32_t n, uint32_t p, uint32_t v, uint64_t nrecchars, MgBufs& b) {
    const uint32_t MS = 8;  // smallest spacing: sample arrays sized for it
    carve_mg_small(ar, n, p, v, b);
    b.piece_off = ar.take<uint32_t>((size_t)p * p);
    b.bstart = ar.take<uint32_t>(p + 1);
    b.clen = ar.take<uint32_t>(n);
    b.coff = ar.take<uint64_t>(n + 1);
    b.btot = ar.take<uint64_t>(n / 4096 + 2);
    b.R.idx = ar.take<uint32_t>(n);
    b.R.h = ar.take<uint32_t>(n);
    b.R.tl = ar.take<uint32_t>(n);
    b.R.base = ar.take<uint64_t>(n);
    b.R.chars = ar.take<uint8_t>(nrecchars + 16);
    b.RA[0] = ar.take<uint32_t>(n);
    b.RA[1] = ar.take<uint32_t>(n);
    b.HA[0] = ar.take<uint32_t>(n);
    b.HA[1] = ar.take<uint32_t>(n);
    uint32_t maxpairs = p * ((p + 1) / 2) + 1;
    b.pairs = ar.take<Pair>((size_t)p * p + 16);  // every level's pairs (< p per bucket in total)
    uint32_t maxs = n / MS + maxpairs * 2 + 2;
    b.srank = ar.take<uint32_t>(maxs);
    b.sl0 = ar.take<uint32_t>(maxs);
    b.sl1 = ar.take<uint32_t>(maxs);
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
static sss_status run_partition(sss_ctx* ctx, const StrIn& in, const uint32_t* trunc, const uint32_t* run_perm,
                                uint32_t p, uint32_t v, MgBufs& b) {
    const uint32_t n = in.n;
    Strs S{in.chars, in.offs, in.lens, trunc};
    uint32_t ne = 0;
    for (uint32_t i = 0; i < p; ++i) ne += part_lo(n, p, i + 1) > part_lo(n, p, i) ? 1u : 0u;
    uint32_t ns = ne * (v + 1);
    uint32_t tot = p * (v + 1);
    SSS_TRY(sss_launch(ctx, "c_samples", k_c_samples, dim3((tot + 127) / 128), dim3(128), 0, run_perm, n, p, v, S,
                       b.smp, b.s_offs, b.s_lens, b.cnt));
    // sort the samples (views of the same characters, truncated) with stage A;
    // equal truncated samples keep sample order, which is input-index order
    StrIn sin{in.chars, in.n_chars, b.s_offs, b.s_lens, ns};
    Arena sub = b.sub;
    SSS_TRY(impl_local_sort(ctx, sub, sin, 1, sss_params{}, b.s_perm, b.s_lcp));
    SSS_TRY(sss_launch(ctx, "c_splitters", k_c_splitters, dim3((p + 127) / 128), dim3(128), 0, (const uint32_t*)b.smp,
                       (const uint32_t*)b.s_perm, ns, p, b.spl));
    uint32_t nb = p * (p + 1);
    SSS_TRY(sss_launch(ctx, "c_bounds", k_c_bounds, dim3((nb + 127) / 128), dim3(128), 0, run_perm, n, p, S,
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
                          uint32_t p, uint32_t v, uint32_t* out_spl, uint32_t* out_bounds) {
    MgBufs b;
    carve_mg_small(ar, in.n, p, v, b);
    SSS_TRY(run_partition(ctx, in, trunc, run_perm, p, v, b));
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
sss_status impl_merge(sss_ctx* ctx, char* ws, size_t ws_bytes, const StrIn& in, const uint32_t* trunc,
                      const uint32_t* run_perm, const uint32_t* run_lcp, uint32_t p, uint32_t v, uint32_t ms_param,
                      uint64_t nrecchars, uint32_t* out_perm, uint32_t* out_lcp) {
    uint32_t MS = MS_DEFAULT;
    if (ms_param >= 8 && ms_param <= 1024 && (ms_param & (ms_param - 1)) == 0) MS = ms_param;
    const uint32_t n = in.n;
    Arena ar{ws, ws_bytes, 0};
    MgBufs b;
    carve_mg(ar, n, p, v, nrecchars, b);
    Strs S{in.chars, in.offs, in.lens, trunc};
    SSS_TRY(run_partition(ctx, in, trunc, run_perm, p, v, b));

    // bounds to the host: piece sizes, bucket starts, piece offsets
    void* pin;
    size_t pin_need = sizeof(uint32_t) * ((size_t)p * (p + 1) + (size_t)p * p + p + 1) + sizeof(Pair) * (p * p + 16);
    SSS_TRY(sss_pinned(ctx, pin_need + 256, &pin));
    uint32_t* hb = static_cast<uint32_t*>(pin);
    uint32_t* hpo = hb + (size_t)p * (p + 1);
    uint32_t* hbs = hpo + (size_t)p * p;
    Pair* hpairs = reinterpret_cast<Pair*>(reinterpret_cast<uintptr_t>(hbs + p + 1 + 15) & ~uintptr_t(15));
    SSS_CUDA(cudaMemcpyAsync(hb, b.bounds, sizeof(uint32_t) * p * (p + 1), cudaMemcpyDeviceToHost, ctx->stream));
    SSS_CUDA(cudaStreamSynchronize(ctx->stream));
    std::vector<std::vector<uint32_t>> psz(p, std::vector<uint32_t>(p));  // psz[j][i]
    uint32_t acc = 0;
    for (uint32_t j = 0; j < p; ++j) {
        hbs[j] = acc;
        for (uint32_t i = 0; i < p; ++i) {
            uint32_t sz = hb[(size_t)i * (p + 1) + j + 1] - hb[(size_t)i * (p + 1) + j];
            psz[j][i] = sz;
            hpo[(size_t)j * p + i] = acc;
            acc += sz;
        }
    }
    hbs[p] = acc;
    if (acc != n) return sss_fail(ctx, SSS_ERR_CUDA, "merge: bucket bounds do not cover the input");
    SSS_TRY(sss_upload(ctx, b.piece_off, hpo, sizeof(uint32_t) * p * p));
    SSS_TRY(sss_upload(ctx, b.bstart, hbs, sizeof(uint32_t) * (p + 1)));

    // D1: records and their characters
    SSS_TRY(sss_launch(ctx, "d_records", k_d_records, dim3((n + 255) / 256), dim3(256), 0, run_perm, run_lcp, n, p, S,
                       (const uint32_t*)b.bounds, (const uint32_t*)b.piece_off, b.R, b.clen, ctx->d_err));
    uint32_t nblk = (n + 4095) / 4096;
    SSS_TRY(sss_launch(ctx, "d_scan", k_scan_blocks, dim3(nblk), dim3(1024), 0, (const uint32_t*)b.clen, n, b.coff,
                       b.btot));
    SSS_TRY(sss_launch(ctx, "d_scan_tot", k_scan_totals, dim3(1), dim3(1024), 0, b.btot, nblk));
    SSS_TRY(sss_launch(ctx, "d_scan_add", k_scan_add, dim3((n + 255) / 256), dim3(256), 0, b.coff, n,
                       (const uint64_t*)b.btot));
    SSS_TRY(sss_launch(ctx, "d_copy", k_d_copy, dim3((n + 127) / 128), dim3(128), 0, S, b.R, (const uint64_t*)b.coff,
                       n));
    SSS_TRY(sss_launch(ctx, "d_iota", k_iota, dim3((n + 255) / 256), dim3(256), 0, b.RA[0], n));
    SSS_CUDA(cudaMemcpyAsync(b.HA[0], b.R.h, sizeof(uint32_t) * n, cudaMemcpyDeviceToDevice, ctx->stream));

    // D2: pairwise merge levels; runs of bucket j at level 0 are its pieces.
    // All levels' pair tables are planned on the host and uploaded at once.
    std::vector<std::vector<uint32_t>> runs(p);  // run sizes per bucket
    for (uint32_t j = 0; j < p; ++j) runs[j] = psz[j];
    std::vector<Pair> all_pairs;
    std::vector<uint32_t> lvl_first, lvl_np, lvl_ns;
    for (;;) {
        bool more = false;
        for (uint32_t j = 0; j < p; ++j) more |= runs[j].size() > 1;
        if (!more) break;
        uint32_t np = 0, ns = 0;
        lvl_first.push_back((uint32_t)all_pairs.size());
        for (uint32_t j = 0; j < p; ++j) {
            uint32_t pos = hbs[j];
            std::vector<uint32_t> next;
            for (size_t k = 0; k < runs[j].size(); k += 2) {
                uint32_t na = runs[j][k], nb = k + 1 < runs[j].size() ? runs[j][k + 1] : 0;
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
                    all_pairs.push_back(pr);
                    ++np;
                }
                pos += na + nb;
                next.push_back(na + nb);
            }
            runs[j] = next;
        }
        lvl_np.push_back(np);
        lvl_ns.push_back(ns);
    }
    const uint32_t nlev = (uint32_t)lvl_np.size();
    Pair* d_pairs = nullptr;
    if (nlev > 0) {
        // the pinned region after the bucket tables was reserved for the pairs
        if (all_pairs.size() > (size_t)p * p + 16) return sss_fail(ctx, SSS_ERR_CUDA, "merge: pair table overflow");
        std::copy(all_pairs.begin(), all_pairs.end(), hpairs);
        d_pairs = b.pairs;
        SSS_TRY(sss_upload(ctx, d_pairs, hpairs, sizeof(Pair) * all_pairs.size()));
    }
    int cur = 0;
    for (uint32_t lv = 0; lv < nlev; ++lv) {
        const Pair* pr = d_pairs + lvl_first[lv];
        uint32_t np = lvl_np[lv], ns = lvl_ns[lv];
        SSS_TRY(sss_launch(ctx, "d_search", k_d_search, dim3((ns + 127) / 128), dim3(128), 0, S, b.R,
                           (const uint32_t*)b.RA[cur], pr, np, ns, b.srank, b.sl0, b.sl1, MS));
        SSS_TRY(sss_launch(ctx, "d_merge", k_d_merge, dim3((ns + 127) / 128), dim3(128), 0, S, b.R,
                           (const uint32_t*)b.RA[cur], (const uint32_t*)b.HA[cur], b.RA[cur ^ 1], b.HA[cur ^ 1],
                           pr, np, ns, (const uint32_t*)b.srank, (const uint32_t*)b.sl0, (const uint32_t*)b.sl1,
                           MS));
        cur ^= 1;
    }
    // D3
    SSS_TRY(sss_launch(ctx, "d_seams", k_d_seams, dim3((p + 127) / 128), dim3(128), 0, S, b.R,
                       (const uint32_t*)b.RA[cur], b.HA[cur], (const uint32_t*)b.bstart, p));
    SSS_TRY(sss_launch(ctx, "d_out", k_d_out, dim3((n + 255) / 256), dim3(256), 0, b.R, (const uint32_t*)b.RA[cur],
                       (const uint32_t*)b.HA[cur], n, out_perm, out_lcp));
    return SSS_OK;
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
