// Stage B: distinguishing-prefix approximation by prefix doubling (Section 4;
// round schedule in the appendix "Distinguishing Prefix Approximation via
// Doubling"; duplicate detection by sorting hash values as in the appendix
// "Duplicate Detection with Atomic Hypercube Quicksort").
//
// Round k tests prefixes of length L = 2^k.  With the local sorted runs of the
// partitions available, positions whose LCP with their local predecessor is >= L
// share that predecessor's L-prefix: they are duplicates without hashing, and a
// group of such positions needs one key (its first position, the "rep") for the
// global check.  A string retires when its group is a single string whose key
// occurs once among all reps, or when L covers the whole string.  The result is
// identical to hashing every active string.
//
// Hash of a prefix of length l (the same definition as the oracle):
//   P = 2^61 - 1, B = 2 + (SplitMix64(seed) mod (P - 3)); the l characters form
//   big-endian 64-bit words (bytes at or past l zero); h folds every word's high
//   then low 32-bit limb as h <- (h*B + limb) mod P; key = smix(h ^ (l * G)).
// Horner's rule resumes from the stored h of the L/2-prefix, so a string that
// was hashed in the previous round reads only characters [L/2, L).
//
// Work per round: position q starts a group from the round whose L exceeds its
// local LCP, k*(q) = bit length of lcp[q]; positions are bucketed once by k*
// (and equal strings by the round that covers their length), so a round only
// touches its reps, the positions that become reps next round and the equal
// strings that end this round -- not all n positions.
//
// Duplicate detection, two exact variants:
//  * sort (the appendix's route): the (key, rep) pairs are bucketed by the key's
//    top bits (keys are uniform), each bucket is sorted in shared memory and
//    equal neighbours mark duplicates; a bucket larger than shared memory (only
//    with many equal keys) is sorted in chunks and cross-checked by binary search.
//  * hash table (default; the single-shot filter of the appendix with the full
//    64-bit key stored, so there are no false positives): keys are inserted into
//    an open-addressing table of >= 2x slots with atomicCAS, a second insert of a
//    key marks its slot, and each rep reads its slot's mark.
#include <algorithm>
#include <mutex>
#include <vector>

#include "sss_device.cuh"
#include "sss_internal.cuh"

namespace {

constexpr uint64_t P61 = (1ull << 61) - 1;
constexpr uint64_t GAMMA = 0x9E3779B97F4A7C15ull;
constexpr uint32_t ACTIVE = 0xFFFFFFFFu;
constexpr int DD_T = 512, DD_CAP = 4096;  // dedupe bucket CTA
constexpr int HB_MAX = 13;                // max top bits for bucketing (8192 buckets)
constexpr int KBINS = 34;                 // rounds 0..33 for the per-position round buckets
constexpr int PD_T = 256;                 // threads of the per-rep kernels

__host__ __device__ __forceinline__ uint64_t smix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// (a * b) mod (2^61 - 1) for a, b < 2^61: 2^61 == 1 (mod P), so the 122-bit
// product hi*2^64 + lo folds to 8*hi + (lo >> 61) + (lo & P).
__device__ __forceinline__ uint64_t mulmod61(uint64_t a, uint64_t b) {
    uint64_t lo = a * b, hi = __umul64hi(a, b);
    uint64_t s = (hi << 3) + (lo >> 61) + (lo & P61);
    s = (s & P61) + (s >> 61);
    return s >= P61 ? s - P61 : s;
}

__device__ __forceinline__ uint64_t fold_limb(uint64_t h, uint64_t B, uint64_t limb) {
    uint64_t t = mulmod61(h, B) + limb;
    return t >= P61 ? t - P61 : t;
}

// Both 32-bit limbs of the word x at once: fold_limb(fold_limb(h, B, x_hi), B,
// x_lo) = (h*B^2 + x_hi*B + x_lo) mod P, with B2 = B^2 mod P.  The 128-bit sum
// of the two products and the low limb is reduced once: h*B2 < 2^122 and
// x_hi*B < 2^93, so the high word stays below 2^59.
__device__ __forceinline__ uint64_t fold_word(uint64_t h, uint64_t B, uint64_t B2, uint64_t x) {
    const uint64_t xh = x >> 32, xl = x & 0xFFFFFFFFull;
    const uint64_t a_lo = h * B2, a_hi = __umul64hi(h, B2);
    const uint64_t b_lo = xh * B, b_hi = __umul64hi(xh, B);
    const uint64_t s1 = a_lo + b_lo;
    const uint64_t s2 = s1 + xl;
    const uint64_t s_hi = a_hi + b_hi + (s1 < a_lo ? 1u : 0u) + (s2 < s1 ? 1u : 0u);
    uint64_t s = (s_hi << 3) + (s2 >> 61) + (s2 & P61);
    s = (s & P61) + (s >> 61);
    return s >= P61 ? s - P61 : s;
}

struct PdIn {
    const uint8_t* chars;
    const uint64_t* offs;
    const uint32_t* run_perm;  // nullable: identity order
    const uint32_t* run_lcp;   // nullable: no local groups
    uint32_t n, p;
};

__device__ __forceinline__ uint32_t ord_of(const PdIn& in, uint32_t q) { return in.run_perm ? in.run_perm[q] : q; }

// end of the partition that holds position q
__device__ __forceinline__ uint32_t part_end_of(uint32_t q, uint32_t n, uint32_t p) {
    uint64_t i = ((uint64_t)(q + 1) * p + n - 1) / n - 1;
    return (uint32_t)(((i + 1) * n) / p);
}
__device__ __forceinline__ bool is_part_start(uint32_t q, uint32_t n, uint32_t p) {
    uint64_t i = ((uint64_t)q * p + n - 1) / n;  // smallest i with floor(i*n/p) >= q
    return (uint32_t)((i * n) / p) == q;
}

// Block-aggregated append of q to list[] (counter *cnt): one atomic per block
// and call instead of one per warp, which matters when millions of positions
// append to one counter.  Every thread of the block calls it; sh holds
// THREADS / 32 words.
template <int THREADS>
__device__ __forceinline__ void block_append(bool want, uint32_t q, uint32_t* list, uint32_t* cnt, uint32_t* sh) {
    constexpr int NW = THREADS / 32;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const unsigned m = __ballot_sync(SSS_FULL, want);
    if (lane == 0) sh[w] = (uint32_t)__popc(m);
    __syncthreads();
    if (w == 0) {
        const uint32_t c = lane < NW ? sh[lane] : 0u;
        uint32_t x = c;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(SSS_FULL, x, o);
            if (lane >= o) x += y;
        }
        const uint32_t tot = __shfl_sync(SSS_FULL, x, 31);
        uint32_t base = 0;
        if (lane == 0 && tot) base = atomicAdd(cnt, tot);
        base = __shfl_sync(SSS_FULL, base, 0);
        if (lane < NW) sh[lane] = base + x - c;
    }
    __syncthreads();
    if (want) list[sh[w] + (uint32_t)__popc(m & ((1u << lane) - 1u))] = q;
    __syncthreads();
}

// block sum of v added to *cnt with one atomic (every thread calls it)
template <int THREADS>
__device__ __forceinline__ void block_count(uint32_t v, uint32_t* cnt, uint32_t* sh) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    v = __reduce_add_sync(SSS_FULL, v);
    if (lane == 0) sh[w] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t t = 0;
        for (int i = 0; i < THREADS / 32; ++i) t += sh[i];
        if (t) atomicAdd(cnt, t);
    }
    __syncthreads();
}

// round from which q starts a group (lcp[q] < 2^k), at least kmin
__device__ __forceinline__ uint32_t kstar_of(const PdIn& in, uint32_t q, uint32_t kmin) {
    uint32_t k = 0;
    if (in.run_lcp && !is_part_start(q, in.n, in.p)) {
        uint32_t l = in.run_lcp[q];
        k = l ? 32u - (uint32_t)__clz(l) : 0u;
    }
    return k > kmin ? k : kmin;
}
// first round whose L covers the whole string (2^k >= len), at least kmin
__device__ __forceinline__ uint32_t klen_of(uint32_t len, uint32_t kmin) {
    uint32_t k = len <= 1 ? 0u : 32u - (uint32_t)__clz(len - 1);
    return k > kmin ? k : kmin;
}

// per-position state; counts of the round buckets
__global__ void k_pd_init(PdIn in, const uint32_t* __restrict__ lens, uint32_t* __restrict__ apos,
                          uint32_t* __restrict__ lpos, uint32_t* __restrict__ hlen, uint32_t* __restrict__ cnt_ks,
                          uint32_t* __restrict__ cnt_kl, uint32_t kmin) {
    __shared__ uint32_t hs[KBINS], hl[KBINS];
    for (int i = threadIdx.x; i < KBINS; i += blockDim.x) hs[i] = hl[i] = 0;
    __syncthreads();
    const uint32_t q = blockIdx.x * blockDim.x + threadIdx.x;
    const bool live = q < in.n;
    uint32_t ks = 0, kl = 0;
    if (live) {
        uint32_t len = lens[ord_of(in, q)];
        apos[q] = ACTIVE;
        lpos[q] = len;
        hlen[q] = 0;
        ks = kstar_of(in, q, kmin);
        kl = klen_of(len, kmin);
    }
    // neighbouring positions mostly share their bins: one shared atomic per
    // (warp, bin), adding the number of lanes with that bin
    const uint32_t lane = threadIdx.x & 31;
    const unsigned ms = __ballot_sync(SSS_FULL, live);
    if (live) {
        const unsigned peers = __match_any_sync(ms, ks);
        if (lane == (uint32_t)(__ffs(peers) - 1)) atomicAdd(&hs[ks], (uint32_t)__popc(peers));
    }
    const bool below = live && kl < ks;
    const unsigned ml = __ballot_sync(SSS_FULL, below);
    if (below) {
        const unsigned peers = __match_any_sync(ml, kl);
        if (lane == (uint32_t)(__ffs(peers) - 1)) atomicAdd(&hl[kl], (uint32_t)__popc(peers));
    }
    __syncthreads();
    for (int i = threadIdx.x; i < KBINS; i += blockDim.x) {
        if (hs[i]) atomicAdd(&cnt_ks[i], hs[i]);
        if (hl[i]) atomicAdd(&cnt_kl[i], hl[i]);
    }
}

// Reserve a slot of bin b among the lanes that call it with `active`: lanes with
// the same bin share one shared-memory atomic (the bins of neighbouring
// positions are mostly equal).  Every lane of the warp calls it.
__device__ __forceinline__ uint32_t warp_bin_reserve(uint32_t* bins, uint32_t b, bool active) {
    const unsigned am = __ballot_sync(SSS_FULL, active);
    uint32_t r = 0;
    if (active) {
        const uint32_t lane = threadIdx.x & 31;
        const unsigned peers = __match_any_sync(am, b);
        const int leader = __ffs(peers) - 1;
        uint32_t base = 0;
        if (lane == (uint32_t)leader) base = atomicAdd(&bins[b], (uint32_t)__popc(peers));
        base = __shfl_sync(peers, base, leader);
        r = base + (uint32_t)__popc(peers & ((1u << lane) - 1u));
    }
    return r;
}

// scatter positions into their round buckets, PL_ITEMS positions per thread:
// lanes with equal buckets share a shared-memory atomic, and one global
// reservation per (CTA, bucket) keeps the cursors uncontended (the order
// within a bucket is free: a bucket is a set)
constexpr int PL_ITEMS = 4;
__global__ void __launch_bounds__(256) k_pd_lists(PdIn in, const uint32_t* __restrict__ lpos,
                                                  uint32_t* __restrict__ cur_ks, uint32_t* __restrict__ cur_kl,
                                                  uint32_t* __restrict__ list_ks, uint32_t* __restrict__ list_kl,
                                                  uint32_t kmin) {
    __shared__ uint32_t cs[KBINS], cl[KBINS];
    for (int i = threadIdx.x; i < KBINS; i += blockDim.x) cs[i] = cl[i] = 0;
    __syncthreads();
    uint32_t ks[PL_ITEMS], kl[PL_ITEMS], rs[PL_ITEMS], rl[PL_ITEMS];
    const uint32_t q0 = blockIdx.x * blockDim.x * PL_ITEMS + threadIdx.x;
#pragma unroll
    for (int i = 0; i < PL_ITEMS; ++i) {
        const uint32_t q = q0 + i * blockDim.x;
        ks[i] = kl[i] = 0;
        if (q < in.n) {
            ks[i] = kstar_of(in, q, kmin);
            kl[i] = klen_of(lpos[q], kmin);
        }
    }
#pragma unroll
    for (int i = 0; i < PL_ITEMS; ++i) {
        const uint32_t q = q0 + i * blockDim.x;
        rs[i] = warp_bin_reserve(cs, ks[i], q < in.n);
        rl[i] = warp_bin_reserve(cl, kl[i], q < in.n && kl[i] < ks[i]);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < KBINS; i += blockDim.x) {
        cs[i] = cs[i] ? atomicAdd(&cur_ks[i], cs[i]) : 0u;
        cl[i] = cl[i] ? atomicAdd(&cur_kl[i], cl[i]) : 0u;
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < PL_ITEMS; ++i) {
        const uint32_t q = q0 + i * blockDim.x;
        if (q < in.n) {
            list_ks[cs[ks[i]] + rs[i]] = q;
            if (kl[i] < ks[i]) list_kl[cl[kl[i]] + rl[i]] = q;
        }
    }
}

// Fold words wa..wb-1 of the prefix of s (le characters: a last partial word is
// zero-padded) into h, read as aligned 8-byte loads issued in batches of 8
// (only words that hold a character of the prefix are loaded).
__device__ __forceinline__ uint64_t fold_words(uint64_t h, const uint8_t* s, uint32_t wa, uint32_t wb, uint32_t le,
                                               uint64_t B, uint64_t B2) {
    if (wa >= wb) return h;
    uintptr_t a0 = (uintptr_t)(s + 8 * wa);
    const uint64_t* pw = reinterpret_cast<const uint64_t*>(a0 & ~uintptr_t(7));
    const uint32_t sh = (uint32_t)(a0 & 7) * 8;
    const uint32_t lim = le < 8 * wb ? le : 8 * wb;
    const uint8_t* end = s + lim;
    uint64_t prev = bswap64(__ldg(pw));
    for (uint32_t w = wa; w < wb; w += 8) {
        uint64_t buf[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const uint64_t* pi = pw + 1 + i;
            buf[i] = reinterpret_cast<const uint8_t*>(pi) < end ? bswap64(__ldg(pi)) : 0ull;
        }
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            if (w + i >= wb) break;
            uint64_t x = sh ? ((prev << sh) | (buf[i] >> (64 - sh))) : prev;
            prev = buf[i];
            uint32_t left = le - 8 * (w + i);
            if (left < 8) x &= ~0ull << (8 * (8 - left));
            h = fold_word(h, B, B2, x);
        }
        pw += 8;
    }
    return h;
}

// B1: the key of rep q.  Horner resumes from the L/2-prefix state of the
// previous round: the rep's own state, or (for a position that starts a group
// only from this round on) the state of its previous group start q', which
// shares that prefix.  Such a position also shares its first minlcp[q]
// characters with q': the whole words among them are read from q''s string,
// which every member of the group reads (so from L2), and only the rest from
// its own.  States are double-buffered by round parity.  prevstart and minlcp
// are optional (a new rep then hashes its prefix from the first word).
// (The state pointers carry no __restrict__: k_pd_cta_rounds reads in one
// round the states it wrote in the previous one, so they must not take the
// read-only cache path.)
__device__ __forceinline__ uint64_t pd_rep_key(const PdIn& in, uint32_t q, const uint32_t* __restrict__ lpos,
                                               const uint64_t* hst_in, const uint32_t* hlen_in, uint64_t* hst_out,
                                               uint32_t* hlen_out, const uint32_t* __restrict__ prevstart,
                                               const uint32_t* __restrict__ minlcp, uint64_t L, uint64_t B) {
    uint32_t s = ord_of(in, q);
    uint32_t len = lpos[q];
    uint32_t le = L < len ? (uint32_t)L : len;
    const uint8_t* str = in.chars + in.offs[s];
    uint64_t h = 0;
    uint32_t w0 = 0, wsh = 0;
    const uint8_t* sstr = str;
    if (L >= 16) {
        uint32_t src = q;
        if (hlen_in[q] != (uint32_t)(L / 2) && prevstart) src = prevstart[q];
        if (hlen_in[src] == (uint32_t)(L / 2)) {
            h = hst_in[src];
            w0 = (uint32_t)(L / 16);
        }
        if (src != q && minlcp) {
            const uint32_t ml = minlcp[q];
            wsh = (ml < le ? ml : le) / 8;
            sstr = in.chars + in.offs[ord_of(in, src)];
        }
    }
    wsh = wsh > w0 ? wsh : w0;
    uint32_t nw = (le + 7) / 8;
    const uint64_t B2 = mulmod61(B, B);
    h = fold_words(h, sstr, w0, wsh, 8 * wsh, B, B2);  // whole words shared with the group start
    h = fold_words(h, str, wsh, nw, le, B, B2);
    hst_out[q] = h;
    hlen_out[q] = le;
    return smix64(h ^ ((uint64_t)le * GAMMA));
}

// (a - b) mod P for a, b < P
__device__ __forceinline__ uint64_t submod61(uint64_t a, uint64_t b) { return a >= b ? a - b : a + P61 - b; }

// The hash of a new rep q from its group start's finished hash (same tested
// length le): the two prefixes agree on their first wsh whole words, so their
// Horner values differ by the Horner fold of the limb differences over words
// wsh .. nw-1 alone (the polynomial is linear in the limbs, and every limb
// keeps its power of B).
__device__ __forceinline__ uint64_t pd_key_from_start(const uint8_t* str, const uint8_t* sstr, uint32_t le,
                                                      uint32_t wsh, uint64_t hsrc, uint64_t B, uint64_t B2) {
    const uint32_t nw = (le + 7) / 8;
    uint64_t D = 0;
    for (uint32_t w = wsh; w < nw; ++w) {
        const uint64_t x = load_word_be(str, le, 8 * w), y = load_word_be(sstr, le, 8 * w);
        const uint64_t dh = submod61(x >> 32, y >> 32), dl = submod61(x & 0xFFFFFFFFull, y & 0xFFFFFFFFull);
        uint64_t t = mulmod61(D, B2) + mulmod61(dh, B);
        t = t >= P61 ? t - P61 : t;
        t += dl;
        D = t >= P61 ? t - P61 : t;
    }
    const uint64_t h = hsrc + D;
    return h >= P61 ? h - P61 : h;
}

// Phase 0: every rep.  When new reps resume from their group starts (prevstart
// given), phase 1 hashes the reps that resume their own L/2 state (the group
// starts that are still reps) and phase 2 the others; a rep of phase 2 whose
// group start has just been hashed to the same length finishes from that hash
// (pd_key_from_start) instead of folding the words they share.
__global__ void k_pd_hash(PdIn in, const uint32_t* __restrict__ reps, uint32_t nreps, const uint32_t* __restrict__ lpos,
                          const uint64_t* __restrict__ hst_in, const uint32_t* __restrict__ hlen_in,
                          uint64_t* hst_out, uint32_t* hlen_out, const uint32_t* __restrict__ prevstart,
                          const uint32_t* __restrict__ minlcp, uint64_t* __restrict__ K, uint32_t* __restrict__ V,
                          uint64_t L, uint64_t B, int phase) {
    uint32_t j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= nreps) return;
    uint32_t q = reps[j];
    if (phase != 0) {
        const bool own = L >= 16 && hlen_in[q] == (uint32_t)(L / 2);
        if ((phase == 1) != own) return;
        if (phase == 2 && prevstart && minlcp) {
            const uint32_t src = prevstart[q];
            const uint32_t len = lpos[q];
            const uint32_t le = L < len ? (uint32_t)L : len;
            if (src != q && hlen_out[src] == le) {
                const uint32_t ml = minlcp[q];
                const uint32_t wsh = (ml < le ? ml : le) / 8;
                const uint64_t B2 = mulmod61(B, B);
                const uint64_t h = pd_key_from_start(in.chars + in.offs[ord_of(in, q)],
                                                     in.chars + in.offs[ord_of(in, src)], le, wsh, hst_out[src], B,
                                                     B2);
                hst_out[q] = h;
                hlen_out[q] = le;
                K[j] = smix64(h ^ ((uint64_t)le * GAMMA));
                V[j] = q;
                return;
            }
        }
    }
    K[j] = pd_rep_key(in, q, lpos, hst_in, hlen_in, hst_out, hlen_out, prevstart, minlcp, L, B);
    V[j] = q;
}

// prevstart[q] = last position q' <= q that starts a group in round k-1
// (kstar(q') <= k-1), and minlcp[q] = min of run_lcp over (q', q], the number
// of characters q shares with q' (all ones when q' = q).  One scan over the
// pairs (last start + 1, min since it) with the operator
//     (s1, m1) then (s2, m2) = s2 ? (s2, m2) : (s1, min(m1, m2)):
// tiles of 4096 positions (4 per thread, warp shuffles, warp totals in shared
// memory), then the carry of earlier tiles.
struct PsPair {
    uint32_t s;  // last group start + 1 (0: none yet)
    uint32_t m;  // min run_lcp since it
};
__device__ __forceinline__ PsPair ps_then(PsPair a, PsPair b) {
    return b.s ? b : PsPair{a.s, a.m < b.m ? a.m : b.m};
}

__global__ void __launch_bounds__(1024) k_pd_ps_tiles(PdIn in, uint32_t kprev, uint32_t kmin,
                                                      uint32_t* __restrict__ out_s, uint32_t* __restrict__ out_m,
                                                      PsPair* __restrict__ tagg) {
    constexpr int ITEMS = 4;
    __shared__ PsPair sh_w[32];
    const uint32_t base = blockIdx.x * 4096 + threadIdx.x * ITEMS;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    PsPair loc[ITEMS];
    PsPair t{0u, ~0u};
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) {
        const uint32_t q = base + i;
        if (q < in.n) {
            const bool start = kstar_of(in, q, kmin) <= kprev;
            t = start ? PsPair{q + 1, ~0u} : ps_then(t, PsPair{0u, in.run_lcp[q]});
        }
        loc[i] = t;
    }
    // inclusive scan of the thread totals within the warp
    PsPair x = t;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        PsPair y{__shfl_up_sync(SSS_FULL, x.s, o), __shfl_up_sync(SSS_FULL, x.m, o)};
        if (lane >= o) x = ps_then(y, x);
    }
    PsPair ex{__shfl_up_sync(SSS_FULL, x.s, 1), __shfl_up_sync(SSS_FULL, x.m, 1)};
    if (lane == 0) ex = PsPair{0u, ~0u};
    if (lane == 31) sh_w[w] = x;
    __syncthreads();
    if (w == 0) {
        PsPair v = sh_w[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            PsPair y{__shfl_up_sync(SSS_FULL, v.s, o), __shfl_up_sync(SSS_FULL, v.m, o)};
            if (lane >= o) v = ps_then(y, v);
        }
        sh_w[lane] = v;  // inclusive over warps
    }
    __syncthreads();
    const PsPair pre = w > 0 ? ps_then(sh_w[w - 1], ex) : ex;
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) {
        const uint32_t q = base + i;
        if (q < in.n) {
            const PsPair r = ps_then(pre, loc[i]);
            out_s[q] = r.s;
            out_m[q] = r.m;
        }
    }
    if (threadIdx.x == 0) tagg[blockIdx.x] = sh_w[31];
}

// exclusive carry of the tile totals: one CTA scans them 1024 at a time
__global__ void __launch_bounds__(1024) k_pd_ps_carry(PsPair* __restrict__ tagg, uint32_t nt) {
    __shared__ PsPair sh_w[32];
    __shared__ PsPair s_run;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const PsPair id{0u, ~0u};
    if (threadIdx.x == 0) s_run = id;
    __syncthreads();
    for (uint32_t c0 = 0; c0 < nt; c0 += 1024) {
        const uint32_t t = c0 + threadIdx.x;
        PsPair x = t < nt ? tagg[t] : id;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            PsPair y{__shfl_up_sync(SSS_FULL, x.s, o), __shfl_up_sync(SSS_FULL, x.m, o)};
            if (lane >= o) x = ps_then(y, x);
        }
        PsPair ex{__shfl_up_sync(SSS_FULL, x.s, 1), __shfl_up_sync(SSS_FULL, x.m, 1)};
        if (lane == 0) ex = id;
        if (lane == 31) sh_w[w] = x;
        __syncthreads();
        if (w == 0) {
            PsPair v = sh_w[lane];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                PsPair y{__shfl_up_sync(SSS_FULL, v.s, o), __shfl_up_sync(SSS_FULL, v.m, o)};
                if (lane >= o) v = ps_then(y, v);
            }
            sh_w[lane] = v;  // inclusive over warps
        }
        __syncthreads();
        const PsPair pre = w > 0 ? ps_then(s_run, sh_w[w - 1]) : s_run;
        if (t < nt) tagg[t] = ps_then(pre, ex);  // exclusive: the earlier tiles
        __syncthreads();
        if (threadIdx.x == 0) s_run = ps_then(s_run, sh_w[31]);
        __syncthreads();
    }
}

__global__ void k_pd_ps_apply(uint32_t n, uint32_t* __restrict__ out_s, uint32_t* __restrict__ out_m,
                              const PsPair* __restrict__ tagg) {
    const uint32_t q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n) return;
    const PsPair r = ps_then(tagg[q / 4096], PsPair{out_s[q], out_m[q]});
    out_s[q] = r.s ? r.s - 1 : q;  // no earlier start (cannot happen): itself
    out_m[q] = r.s ? r.m : 0u;
}

// B2: bucket the keys by their top bits
__global__ void k_pd_hist(const uint64_t* __restrict__ K, uint32_t m, uint32_t bits, uint32_t* __restrict__ hist) {
    __shared__ uint32_t sh[1u << HB_MAX];
    uint32_t nb = 1u << bits;
    for (uint32_t i = threadIdx.x; i < nb; i += blockDim.x) sh[i] = 0;
    __syncthreads();
    for (uint32_t j = blockIdx.x * blockDim.x + threadIdx.x; j < m; j += gridDim.x * blockDim.x) {
        uint32_t b = bits ? (uint32_t)(K[j] >> (64 - bits)) : 0u;
        atomicAdd(&sh[b], 1u);
    }
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < nb; i += blockDim.x)
        if (sh[i]) atomicAdd(&hist[i], sh[i]);
}

// exclusive scan of nb <= 8192 counts in one CTA; writes bucket starts and
// resets the scatter cursors
__global__ void __launch_bounds__(1024) k_pd_scan(uint32_t* __restrict__ hist, uint32_t nb,
                                                  uint32_t* __restrict__ bstart, uint32_t* __restrict__ cursor) {
    constexpr int ITEMS = (1 << HB_MAX) / 1024;
    __shared__ uint32_t sh_warp[32];
    uint32_t loc[ITEMS];
    uint32_t sum = 0;
    uint32_t b0 = threadIdx.x * ITEMS;
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) {
        uint32_t v = b0 + i < nb ? hist[b0 + i] : 0;
        loc[i] = sum;
        sum += v;
    }
    uint32_t total;
    uint32_t off = BlockScan<1024>::exclusive_sum(sum, sh_warp, &total);
#pragma unroll
    for (int i = 0; i < ITEMS; ++i)
        if (b0 + i < nb) {
            bstart[b0 + i] = off + loc[i];
            cursor[b0 + i] = 0;
        }
    if (threadIdx.x == 0) bstart[nb] = total;
}

__global__ void k_pd_scatter(const uint64_t* __restrict__ K, const uint32_t* __restrict__ V, uint32_t m, uint32_t bits,
                             const uint32_t* __restrict__ bstart, uint32_t* __restrict__ cursor,
                             uint64_t* __restrict__ tK, uint32_t* __restrict__ tV) {
    uint32_t j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= m) return;
    uint64_t k = K[j];
    uint32_t b = bits ? (uint32_t)(k >> (64 - bits)) : 0u;
    uint32_t dst = bstart[b] + atomicAdd(&cursor[b], 1u);
    tK[dst] = k;
    tV[dst] = V[j];
}

__device__ __forceinline__ bool bsearch64(const uint64_t* a, uint32_t m, uint64_t k) {
    uint32_t lo = 0, hi = m;
    while (lo < hi) {
        uint32_t mid = (lo + hi) >> 1;
        uint64_t x = a[mid];
        if (x == k) return true;
        if (x < k) lo = mid + 1; else hi = mid;
    }
    return false;
}

// B3: one CTA per bucket; dupf[rep position] = key occurs more than once
__global__ void __launch_bounds__(DD_T) k_pd_buckets(const uint32_t* __restrict__ bstart, uint64_t* __restrict__ tK,
                                                     uint32_t* __restrict__ tV, uint8_t* __restrict__ dupf) {
    extern __shared__ __align__(16) unsigned char smem[];
    uint64_t* sK = reinterpret_cast<uint64_t*>(smem);
    uint64_t* sV = sK + DD_CAP;
    uint8_t* sF = reinterpret_cast<uint8_t*>(sV + DD_CAP);
    uint32_t bs = bstart[blockIdx.x], be = bstart[blockIdx.x + 1];
    uint32_t m = be - bs;
    if (m == 0) return;
    if (m == 1) {
        if (threadIdx.x == 0) dupf[tV[bs]] = 0;
        return;
    }
    if (m <= (uint32_t)DD_CAP) {
        for (uint32_t i = threadIdx.x; i < m; i += DD_T) {
            sK[i] = tK[bs + i];
            sV[i] = tV[bs + i];
        }
        __syncthreads();
        block_merge_sort128_fit<DD_T, DD_CAP / DD_T>(sK, sV, m);
        for (uint32_t i = threadIdx.x; i < m; i += DD_T) {
            uint64_t k = sK[i];
            bool d = (i > 0 && sK[i - 1] == k) || (i + 1 < m && sK[i + 1] == k);
            dupf[(uint32_t)sV[i]] = d ? 1 : 0;
        }
        return;
    }
    // oversized bucket: sort chunks in place, then check runs across chunks
    uint32_t nch = (m + DD_CAP - 1) / DD_CAP;
    for (uint32_t c = 0; c < nch; ++c) {
        uint32_t c0 = bs + c * DD_CAP, cm = min((uint32_t)DD_CAP, be - c0);
        for (uint32_t i = threadIdx.x; i < cm; i += DD_T) {
            sK[i] = tK[c0 + i];
            sV[i] = tV[c0 + i];
        }
        __syncthreads();
        block_merge_sort128_fit<DD_T, DD_CAP / DD_T>(sK, sV, cm);
        for (uint32_t i = threadIdx.x; i < cm; i += DD_T) {
            tK[c0 + i] = sK[i];
            tV[c0 + i] = (uint32_t)sV[i];
        }
        __syncthreads();
    }
    __threadfence_block();
    __syncthreads();
    for (uint32_t c = 0; c < nch; ++c) {
        uint32_t c0 = bs + c * DD_CAP, cm = min((uint32_t)DD_CAP, be - c0);
        for (uint32_t i = threadIdx.x; i < cm; i += DD_T) sK[i] = tK[c0 + i];
        __syncthreads();
        for (uint32_t i = threadIdx.x; i < cm; i += DD_T) {
            uint64_t k = sK[i];
            if (i > 0 && sK[i - 1] == k) continue;  // not the first of its run in this chunk
            bool d = (i + 1 < cm && sK[i + 1] == k);
            for (uint32_t c2 = 0; c2 < nch && !d; ++c2) {
                if (c2 == c) continue;
                uint32_t o0 = bs + c2 * DD_CAP, om = min((uint32_t)DD_CAP, be - o0);
                d = bsearch64(tK + o0, om, k);
            }
            sF[i] = d ? 1 : 0;
        }
        __syncthreads();
        for (uint32_t i = threadIdx.x; i < cm; i += DD_T) {
            // first position of i's run
            uint32_t lo = 0, hi = i;
            uint64_t k = sK[i];
            while (lo < hi) {
                uint32_t mid = (lo + hi) >> 1;
                if (sK[mid] < k) lo = mid + 1; else hi = mid;
            }
            dupf[tV[c0 + i]] = sF[lo];
        }
        __syncthreads();
    }
}

// B2/B3, hash-table variant: insert every rep key; a second copy marks the slot
__global__ void k_pd_ht_insert(const uint64_t* __restrict__ K, uint32_t m, unsigned long long* __restrict__ tab,
                               uint8_t* __restrict__ mark, uint32_t tmask, uint32_t* __restrict__ zero_cnt,
                               unsigned* err) {
    uint32_t j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= m) return;
    uint64_t k = K[j];
    if (k == 0) {  // 0 marks an empty slot: count zero keys apart
        atomicAdd(zero_cnt, 1u);
        return;
    }
    uint32_t h = (uint32_t)k & tmask;
    for (uint32_t i = 0; i <= tmask; ++i) {
        unsigned long long old = atomicCAS(&tab[h], 0ull, (unsigned long long)k);
        if (old == 0ull) return;
        if (old == k) {
            mark[h] = 1;
            return;
        }
        h = (h + 1) & tmask;
    }
    atomicOr(err, ERRBIT_OVERFLOW);
}

__device__ __forceinline__ bool ht_dup(const unsigned long long* tab, const uint8_t* mark, uint32_t tmask,
                                       uint32_t zero_cnt, uint64_t k) {
    if (k == 0) return zero_cnt > 1;
    uint32_t h = (uint32_t)k & tmask;
    for (uint32_t i = 0; i <= tmask; ++i) {
        uint64_t t = tab[h];
        if (t == k) return mark[h] != 0;
        if (t == 0) return false;  // not reachable: every key was inserted
        h = (h + 1) & tmask;
    }
    return true;
}

// B4: retire the reps whose group is one string with a unique key (or whose
// length <= L); survivors stay reps next round.
__global__ void __launch_bounds__(PD_T) k_pd_retire(PdIn in, const uint32_t* __restrict__ reps, uint32_t nreps,
                            const uint32_t* __restrict__ lpos, const uint64_t* __restrict__ K,
                            const uint8_t* __restrict__ dupf, const unsigned long long* __restrict__ tab,
                            const uint8_t* __restrict__ mark, uint32_t tmask, const uint32_t* __restrict__ zero_cnt,
                            uint32_t* __restrict__ apos, uint32_t* __restrict__ reps_next,
                            uint32_t* __restrict__ cnt, uint64_t L, int use_ht) {
    uint32_t j = blockIdx.x * blockDim.x + threadIdx.x;
    bool keep = false;
    uint32_t q = 0, retired = 0;
    if (j < nreps) {
        q = reps[j];
        uint32_t len = lpos[q];
        bool single = true;
        if (in.run_lcp) {
            uint32_t pe = part_end_of(q, in.n, in.p);
            single = !(q + 1 < pe && in.run_lcp[q + 1] >= L);
        }
        bool dup = !single;
        if (!dup) dup = use_ht ? ht_dup(tab, mark, tmask, *zero_cnt, K[j]) : (dupf[q] != 0);
        if (!dup || (uint64_t)len <= L) {
            apos[q] = (uint64_t)len < L ? len : (uint32_t)L;
            retired = 1;
        } else {
            keep = true;
        }
    }
    __shared__ uint32_t sh[PD_T / 32];
    block_append<PD_T>(keep, q, reps_next, &cnt[0], sh);
    block_count<PD_T>(retired, &cnt[1], sh);
}

// strings equal to their local predecessor whose whole length is tested this
// round: duplicates that retire with approx = len
__global__ void __launch_bounds__(PD_T) k_pd_retire_equal(const uint32_t* __restrict__ list, uint32_t m, const uint32_t* __restrict__ lpos,
                                  uint32_t* __restrict__ apos, uint32_t* __restrict__ cnt) {
    uint32_t j = blockIdx.x * blockDim.x + threadIdx.x;
    uint32_t retired = 0;
    if (j < m) {
        uint32_t q = list[j];
        if (apos[q] == ACTIVE) {
            apos[q] = lpos[q];
            retired = 1;
        }
    }
    __shared__ uint32_t sh[PD_T / 32];
    block_count<PD_T>(retired, &cnt[1], sh);
}

// positions that start a group from the next round on become reps (if active)
__global__ void __launch_bounds__(PD_T) k_pd_newreps(const uint32_t* __restrict__ list, uint32_t m, const uint32_t* __restrict__ apos,
                             uint32_t* __restrict__ reps_next, uint32_t* __restrict__ cnt) {
    uint32_t j = blockIdx.x * blockDim.x + threadIdx.x;
    bool want = false;
    uint32_t q = 0;
    if (j < m) {
        q = list[j];
        want = apos[q] == ACTIVE;
    }
    __shared__ uint32_t sh[PD_T / 32];
    block_append<PD_T>(want, q, reps_next, &cnt[0], sh);
}

__global__ void k_pd_final(PdIn in, const uint32_t* __restrict__ apos, const uint32_t* __restrict__ lpos,
                           uint32_t* __restrict__ approx) {
    uint32_t q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= in.n) return;
    uint32_t a = apos[q];
    approx[ord_of(in, q)] = a == ACTIVE ? lpos[q] : a;
}

// Offsets of the per-position round buckets (by the round a position starts a
// group, and by the round that covers an equal string's length).
struct PdOffs {
    uint32_t ks[KBINS + 1];
    uint32_t kl[KBINS + 1];
};

// Rounds k0..k1 in one CTA, for rounds whose reps number at most CR_CAP: the
// same steps as k_pd_hash, k_pd_ht_insert, k_pd_retire, k_pd_retire_equal and
// k_pd_newreps, with the hash table, the keys and the rep lists in shared
// memory and __syncthreads between the steps instead of kernel boundaries and a
// host round trip.  The host picks k1 so that no round holds more than CR_CAP
// reps (the reps of round k are at most the reps of round k0 plus the
// positions whose group starts in rounds k0+1..k).  On return the next round's
// reps are in reps_out, their count in cnt[0], and cnt[1] has grown by the
// strings retired.  States are read and written in the global double buffers
// with the same round parity as the per-round kernels.
constexpr int CR_T = 1024, CR_CAP = 4096;
constexpr size_t CR_SMEM = (size_t)CR_CAP * 8 + (size_t)2 * CR_CAP * 8 + (size_t)2 * CR_CAP * 4 + (size_t)2 * CR_CAP;

__global__ void __launch_bounds__(CR_T) k_pd_cta_rounds(PdIn in, const uint32_t* __restrict__ reps0, uint32_t nreps0,
                                                         uint32_t k0, uint32_t k1, uint32_t kmin, uint32_t kmax,
                                                         const PdOffs off, const uint32_t* __restrict__ list_ks,
                                                         const uint32_t* __restrict__ list_kl,
                                                         const uint32_t* __restrict__ lpos, uint64_t* hst,
                                                         uint32_t* hlen, uint64_t* hst2, uint32_t* hlen2,
                                                         uint32_t* apos, uint32_t* __restrict__ reps_out,
                                                         uint32_t* __restrict__ cnt, uint64_t B, unsigned* err) {
    extern __shared__ __align__(16) unsigned char smem[];
    uint64_t* sK = reinterpret_cast<uint64_t*>(smem);                                // CR_CAP keys
    unsigned long long* tab = reinterpret_cast<unsigned long long*>(sK + CR_CAP);    // 2 CR_CAP slots
    uint32_t* lst0 = reinterpret_cast<uint32_t*>(tab + 2 * CR_CAP);                  // CR_CAP
    uint32_t* lst1 = lst0 + CR_CAP;                                                  // CR_CAP
    uint8_t* mark = reinterpret_cast<uint8_t*>(lst1 + CR_CAP);                       // 2 CR_CAP
    __shared__ uint32_t s_n[2], s_zero, s_ret, s_ovf;
    const uint32_t tid = threadIdx.x;
    const uint32_t n0 = nreps0 < (uint32_t)CR_CAP ? nreps0 : (uint32_t)CR_CAP;
    for (uint32_t i = tid; i < n0; i += CR_T) lst0[i] = reps0[i];
    if (tid == 0) {
        s_n[0] = n0;
        s_ret = 0;
        s_ovf = nreps0 > (uint32_t)CR_CAP;
    }
    __syncthreads();
    uint32_t cur = 0;
    for (uint32_t k = k0; k <= k1; ++k) {
        const uint64_t L = 1ull << k;
        uint32_t* lc = cur ? lst1 : lst0;
        uint32_t* ln = cur ? lst0 : lst1;
        const uint32_t nr = s_n[cur];
        uint32_t T = 1024;
        while (T < 2u * nr) T <<= 1;
        const uint32_t tmask = T - 1;
        for (uint32_t i = tid; i < T; i += CR_T) {
            tab[i] = 0ull;
            mark[i] = 0;
        }
        if (tid == 0) {
            s_zero = 0;
            s_n[cur ^ 1] = 0;
        }
        __syncthreads();
        const bool odd = ((k - kmin) & 1u) != 0;
        const uint64_t* hs_in = odd ? hst2 : hst;
        const uint32_t* hl_in = odd ? hlen2 : hlen;
        uint64_t* hs_out = odd ? hst : hst2;
        uint32_t* hl_out = odd ? hlen : hlen2;
        // keys of the reps, inserted into the table (a second copy marks its slot)
        for (uint32_t j = tid; j < nr; j += CR_T) {
            const uint64_t key =
                pd_rep_key(in, lc[j], lpos, hs_in, hl_in, hs_out, hl_out, nullptr, nullptr, L, B);
            sK[j] = key;
            if (key == 0) {
                atomicAdd(&s_zero, 1u);
                continue;
            }
            uint32_t h = (uint32_t)key & tmask;
            for (uint32_t i = 0; i <= tmask; ++i) {
                const unsigned long long old = atomicCAS(&tab[h], 0ull, (unsigned long long)key);
                if (old == 0ull) break;
                if (old == key) {
                    mark[h] = 1;
                    break;
                }
                h = (h + 1) & tmask;
            }
        }
        __syncthreads();
        // retire the reps whose group is one string with a unique key (or whose
        // length <= L); the others stay reps
        for (uint32_t j = tid; j < nr; j += CR_T) {
            const uint32_t q = lc[j];
            const uint32_t len = lpos[q];
            bool dup = false;
            if (in.run_lcp) {
                const uint32_t pe = part_end_of(q, in.n, in.p);
                dup = q + 1 < pe && in.run_lcp[q + 1] >= L;
            }
            if (!dup) {
                const uint64_t key = sK[j];
                if (key == 0) {
                    dup = s_zero > 1;
                } else {
                    uint32_t h = (uint32_t)key & tmask;
                    for (uint32_t i = 0; i <= tmask; ++i) {
                        const uint64_t t = tab[h];
                        if (t == key) {
                            dup = mark[h] != 0;
                            break;
                        }
                        h = (h + 1) & tmask;
                    }
                }
            }
            if (!dup || (uint64_t)len <= L) {
                apos[q] = (uint64_t)len < L ? len : (uint32_t)L;
                atomicAdd(&s_ret, 1u);
            } else {
                const uint32_t at = atomicAdd(&s_n[cur ^ 1], 1u);
                if (at < (uint32_t)CR_CAP) ln[at] = q;
                else s_ovf = 1;
            }
        }
        // strings equal to their local predecessor whose whole length is tested now
        for (uint32_t j = off.kl[k] + tid; j < off.kl[k + 1]; j += CR_T) {
            const uint32_t q = list_kl[j];
            if (apos[q] == ACTIVE) {
                apos[q] = lpos[q];
                atomicAdd(&s_ret, 1u);
            }
        }
        __syncthreads();
        // positions that start a group from the next round on become reps
        // (after the last round k1 the host appends them)
        if (k < k1) {
            for (uint32_t j = off.ks[k + 1] + tid; j < off.ks[k + 2]; j += CR_T) {
                const uint32_t q = list_ks[j];
                if (apos[q] == ACTIVE) {
                    const uint32_t at = atomicAdd(&s_n[cur ^ 1], 1u);
                    if (at < (uint32_t)CR_CAP) ln[at] = q;
                    else s_ovf = 1;
                }
            }
        }
        __syncthreads();
        cur ^= 1;
    }
    const uint32_t nr = s_n[cur] < (uint32_t)CR_CAP ? s_n[cur] : (uint32_t)CR_CAP;
    const uint32_t* lc = cur ? lst1 : lst0;
    for (uint32_t j = tid; j < nr; j += CR_T) reps_out[j] = lc[j];
    if (tid == 0) {
        cnt[0] = nr;
        cnt[1] += s_ret;
        if (s_ovf) atomicOr(err, ERRBIT_OVERFLOW);
    }
}

struct PdBufs {
    uint32_t* apos;
    uint32_t* lpos;
    uint32_t* hlen;
    uint64_t* hst;
    uint32_t* hlen2;
    uint64_t* hst2;
    uint32_t* prevstart;
    uint32_t* minlcp;
    PsPair* tagg;
    uint32_t* list_ks;
    uint32_t* list_kl;
    uint32_t* reps[2];
    unsigned long long* tab;
    uint8_t* mark;
    uint32_t tcap;
    uint64_t* K;
    uint32_t* V;
    uint64_t* tK;
    uint32_t* tV;
    uint8_t* dupf;
    uint32_t* hist;
    uint32_t* bstart;
    uint32_t* cursor;
    uint32_t* cnt;
};

void carve_pd(Arena& ar, uint32_t n, PdBufs& b) {
    b.apos = ar.take<uint32_t>(n);
    b.lpos = ar.take<uint32_t>(n);
    b.hlen = ar.take<uint32_t>(n);
    b.hst = ar.take<uint64_t>(n);
    b.hlen2 = ar.take<uint32_t>(n);
    b.hst2 = ar.take<uint64_t>(n);
    b.prevstart = ar.take<uint32_t>(n);
    b.minlcp = ar.take<uint32_t>(n);
    b.tagg = ar.take<PsPair>(n / 4096 + 2);
    b.list_ks = ar.take<uint32_t>(n);
    b.list_kl = ar.take<uint32_t>(n);
    b.reps[0] = ar.take<uint32_t>(n);
    b.reps[1] = ar.take<uint32_t>(n);
    b.K = ar.take<uint64_t>(n);
    b.V = ar.take<uint32_t>(n);
    b.tK = ar.take<uint64_t>(n);
    b.tV = ar.take<uint32_t>(n);
    b.dupf = ar.take<uint8_t>(n);
    b.hist = ar.take<uint32_t>((1u << HB_MAX) + 1);
    b.bstart = ar.take<uint32_t>((1u << HB_MAX) + 1);
    b.cursor = ar.take<uint32_t>((1u << HB_MAX) + 1);
    b.cnt = ar.take<uint32_t>(8 + 4 * KBINS);
    b.tcap = 1024;
    while (b.tcap < 2ull * n) b.tcap <<= 1;
    b.tab = ar.take<unsigned long long>(b.tcap);
    b.mark = ar.take<uint8_t>(b.tcap);
}

uint64_t host_smix(uint64_t z) { return smix64(z); }

}  // namespace

size_t need_dist_prefix(uint32_t n) {
    Arena ar;
    PdBufs b;
    carve_pd(ar, n, b);
    return ar.off + 256;
}

static bool g_pd_attr[64];
static bool g_cr_attr[64];

sss_status impl_dist_prefix(sss_ctx* ctx, Arena& ar, const StrIn& sin, const uint32_t* run_perm,
                            const uint32_t* run_lcp, uint32_t p, const sss_params& prm, uint32_t* approx) {
    const uint32_t n = sin.n;
    if (n == 0) return SSS_OK;
    PdBufs B;
    carve_pd(ar, n, B);
    if (!g_pd_attr[ctx->device & 63]) {
        SSS_CUDA(cudaFuncSetAttribute(k_pd_buckets, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)(DD_CAP * (8 + 8 + 1))));
        g_pd_attr[ctx->device & 63] = true;
    }
    PdIn in{sin.chars, sin.offs, run_perm, run_lcp, n, run_perm ? p : 1u};
    const uint32_t kmin = std::min<uint32_t>(prm.kmin, 31u);
    uint32_t kmax = prm.kmax == SSS_KMAX_AUTO ? 31u : std::min<uint32_t>(prm.kmax, 31u);
    const bool use_ht = !(prm.flags & SSS_FLAG_DEDUPE_SORT);
    const uint64_t Bh = 2 + host_smix(prm.hash_seed + GAMMA) % (P61 - 3);

    void* pin;
    SSS_TRY(sss_pinned(ctx, sizeof(uint32_t) * (8 + 4 * KBINS), &pin));
    uint32_t* h = static_cast<uint32_t*>(pin);
    uint32_t* cnt = B.cnt;                  // [0] reps next, [1] retired, [2] zero keys
    uint32_t* cnt_ks = B.cnt + 8;           // KBINS
    uint32_t* cnt_kl = cnt_ks + KBINS;      // KBINS
    uint32_t* cur_ks = cnt_kl + KBINS;      // KBINS
    uint32_t* cur_kl = cur_ks + KBINS;      // KBINS

    SSS_CUDA(cudaMemsetAsync(B.cnt, 0, sizeof(uint32_t) * (8 + 4 * KBINS), ctx->stream));
    SSS_CUDA(cudaMemsetAsync(B.hlen2, 0, sizeof(uint32_t) * n, ctx->stream));
    SSS_TRY(sss_launch(ctx, "pd_init", k_pd_init, dim3((n + 255) / 256), dim3(256), 0, in, sin.lens, B.apos, B.lpos,
                       B.hlen, cnt_ks, cnt_kl, kmin));
    if (kmin > kmax) {
        return sss_launch(ctx, "pd_final", k_pd_final, dim3((n + 255) / 256), dim3(256), 0, in,
                          (const uint32_t*)B.apos, (const uint32_t*)B.lpos, approx);
    }
    SSS_CUDA(cudaMemcpyAsync(h, cnt_ks, sizeof(uint32_t) * 2 * KBINS, cudaMemcpyDeviceToHost, ctx->stream));
    SSS_CUDA(cudaStreamSynchronize(ctx->stream));
    uint32_t ks_off[KBINS + 1], kl_off[KBINS + 1];
    ks_off[0] = kl_off[0] = 0;
    for (int i = 0; i < KBINS; ++i) {
        ks_off[i + 1] = ks_off[i] + h[i];
        kl_off[i + 1] = kl_off[i] + h[KBINS + i];
    }
    // list cursors start at the bucket offsets
    for (int i = 0; i < KBINS; ++i) {
        h[i] = ks_off[i];
        h[KBINS + i] = kl_off[i];
    }
    SSS_TRY(sss_upload(ctx, cur_ks, h, sizeof(uint32_t) * 2 * KBINS));
    SSS_TRY(sss_launch(ctx, "pd_lists", k_pd_lists, dim3((n + 256 * PL_ITEMS - 1) / (256 * PL_ITEMS)), dim3(256), 0,
                       in, (const uint32_t*)B.lpos, cur_ks, cur_kl, B.list_ks, B.list_kl, kmin));
    // the first round's reps are the positions that start a group at L = 2^kmin
    const uint32_t* reps = B.list_ks + ks_off[kmin];
    uint32_t nreps = ks_off[kmin + 1] - ks_off[kmin];
    uint32_t retired = 0;
    int nxt = 0;
    PdOffs offs;
    for (int i = 0; i <= KBINS; ++i) {
        offs.ks[i] = ks_off[i];
        offs.kl[i] = kl_off[i];
    }
    const bool cta_rounds = use_ht && !(prm.flags & SSS_FLAG_NO_CTA_ROUNDS);
    for (uint32_t k = kmin; k <= kmax && retired < n; ++k) {
        const uint64_t L = 1ull << k;
        uint32_t tmask = 0;
        if (cta_rounds && nreps <= (uint32_t)CR_CAP) {
            // this round and the following ones while their reps stay few: one
            // CTA; the reps that join in the round after the last one are
            // appended by k_pd_newreps (they may be many)
            uint32_t k1 = k;
            while (k1 < kmax && (uint64_t)nreps + (ks_off[k1 + 2] - ks_off[k + 1]) <= (uint64_t)CR_CAP) ++k1;
            if (!g_cr_attr[ctx->device & 63]) {
                SSS_CUDA(cudaFuncSetAttribute(k_pd_cta_rounds, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                              (int)CR_SMEM));
                g_cr_attr[ctx->device & 63] = true;
            }
            SSS_TRY(sss_launch(ctx, "pd_cta_rounds", k_pd_cta_rounds, dim3(1), dim3(CR_T), CR_SMEM, in, reps, nreps,
                               k, k1, kmin, kmax, offs, (const uint32_t*)B.list_ks, (const uint32_t*)B.list_kl,
                               (const uint32_t*)B.lpos, B.hst, B.hlen, B.hst2, B.hlen2, B.apos, B.reps[nxt], cnt, Bh,
                               ctx->d_err));
            if (k1 < kmax) {
                const uint32_t nn = ks_off[k1 + 2] - ks_off[k1 + 1];
                SSS_TRY(sss_launch(ctx, "pd_newreps", k_pd_newreps, dim3((nn + PD_T - 1) / PD_T), dim3(PD_T), 0,
                                   (const uint32_t*)(B.list_ks + ks_off[k1 + 1]), nn, (const uint32_t*)B.apos,
                                   B.reps[nxt], cnt));
            }
            SSS_CUDA(cudaMemcpyAsync(h, cnt, sizeof(uint32_t) * 2, cudaMemcpyDeviceToHost, ctx->stream));
            SSS_CUDA(cudaStreamSynchronize(ctx->stream));
            nreps = h[0];
            retired = h[1];
            reps = B.reps[nxt];
            nxt ^= 1;
            k = k1;
            continue;
        }
        if (nreps > 0) {
            // many positions start a group only from this round on: locate their
            // previous group start, whose L/2-prefix state they share
            const uint32_t nnew = k > kmin ? ks_off[k + 1] - ks_off[k] : 0;
            const uint32_t* ps = nullptr;
            if (run_lcp && k >= 4 && k > kmin && nnew > n / 16) {
                uint32_t nt = (n + 4095) / 4096;
                SSS_TRY(sss_launch(ctx, "pd_prevstart", k_pd_ps_tiles, dim3(nt), dim3(1024), 0, in, k - 1, kmin,
                                   B.prevstart, B.minlcp, B.tagg));
                SSS_TRY(sss_launch(ctx, "pd_prevstart_carry", k_pd_ps_carry, dim3(1), dim3(1024), 0, B.tagg, nt));
                SSS_TRY(sss_launch(ctx, "pd_prevstart_apply", k_pd_ps_apply, dim3((n + 255) / 256), dim3(256), 0, n,
                                   B.prevstart, B.minlcp, (const PsPair*)B.tagg));
                ps = B.prevstart;
            }
            const bool odd = ((k - kmin) & 1u) != 0;
            uint64_t* hs_in = odd ? B.hst2 : B.hst;
            uint32_t* hl_in = odd ? B.hlen2 : B.hlen;
            uint64_t* hs_out = odd ? B.hst : B.hst2;
            uint32_t* hl_out = odd ? B.hlen : B.hlen2;
            // with previous starts: the surviving group starts first, then the new
            // reps, which can finish from their start's hash
            for (int phase = ps ? 1 : 0; phase <= (ps ? 2 : 0); ++phase)
                SSS_TRY(sss_launch(ctx, "pd_hash", k_pd_hash, dim3((nreps + 255) / 256), dim3(256), 0, in, reps,
                                   nreps, (const uint32_t*)B.lpos, (const uint64_t*)hs_in, (const uint32_t*)hl_in,
                                   hs_out, hl_out, ps, ps ? (const uint32_t*)B.minlcp : (const uint32_t*)nullptr,
                                   B.K, B.V, L, Bh, phase));
            if (use_ht) {
                uint32_t T = 1024;
                while (T < 2ull * nreps) T <<= 1;
                tmask = T - 1;
                SSS_CUDA(cudaMemsetAsync(B.tab, 0, sizeof(unsigned long long) * T, ctx->stream));
                SSS_CUDA(cudaMemsetAsync(B.mark, 0, T, ctx->stream));
                SSS_CUDA(cudaMemsetAsync(&cnt[2], 0, sizeof(uint32_t), ctx->stream));
                SSS_TRY(sss_launch(ctx, "pd_ht_insert", k_pd_ht_insert, dim3((nreps + 255) / 256), dim3(256), 0,
                                   (const uint64_t*)B.K, nreps, B.tab, B.mark, tmask, &cnt[2], ctx->d_err));
            } else {
                uint32_t bits = 0;
                while (bits < (uint32_t)HB_MAX && ((uint64_t)nreps >> bits) > 1024) ++bits;
                uint32_t nb = 1u << bits;
                SSS_CUDA(cudaMemsetAsync(B.hist, 0, sizeof(uint32_t) * (nb + 1), ctx->stream));
                uint32_t hgrid = std::min<uint32_t>((nreps + 4095) / 4096, 2u * (uint32_t)ctx->sm_count);
                SSS_TRY(sss_launch(ctx, "pd_hist", k_pd_hist, dim3(hgrid), dim3(512), 0, (const uint64_t*)B.K, nreps,
                                   bits, B.hist));
                SSS_TRY(sss_launch(ctx, "pd_scan", k_pd_scan, dim3(1), dim3(1024), 0, B.hist, nb, B.bstart,
                                   B.cursor));
                SSS_TRY(sss_launch(ctx, "pd_scatter", k_pd_scatter, dim3((nreps + 255) / 256), dim3(256), 0,
                                   (const uint64_t*)B.K, (const uint32_t*)B.V, nreps, bits,
                                   (const uint32_t*)B.bstart, B.cursor, B.tK, B.tV));
                SSS_TRY(sss_launch(ctx, "pd_buckets", k_pd_buckets, dim3(nb), dim3(DD_T),
                                   (size_t)DD_CAP * (8 + 8 + 1), (const uint32_t*)B.bstart, B.tK, B.tV, B.dupf));
            }
        }
        SSS_CUDA(cudaMemsetAsync(&cnt[0], 0, sizeof(uint32_t), ctx->stream));
        SSS_TRY(sss_launch(ctx, "pd_retire", k_pd_retire, dim3((nreps + PD_T - 1) / PD_T), dim3(PD_T), 0, in, reps, nreps,
                           (const uint32_t*)B.lpos, (const uint64_t*)B.K, (const uint8_t*)B.dupf,
                           (const unsigned long long*)B.tab, (const uint8_t*)B.mark, tmask,
                           (const uint32_t*)&cnt[2], B.apos, B.reps[nxt], cnt, L, (int)use_ht));
        uint32_t ne = kl_off[k + 1] - kl_off[k];
        SSS_TRY(sss_launch(ctx, "pd_retire_equal", k_pd_retire_equal, dim3((ne + PD_T - 1) / PD_T), dim3(PD_T), 0,
                           (const uint32_t*)(B.list_kl + kl_off[k]), ne, (const uint32_t*)B.lpos, B.apos, cnt));
        if (k < kmax) {
            uint32_t nn = ks_off[k + 2] - ks_off[k + 1];
            SSS_TRY(sss_launch(ctx, "pd_newreps", k_pd_newreps, dim3((nn + PD_T - 1) / PD_T), dim3(PD_T), 0,
                               (const uint32_t*)(B.list_ks + ks_off[k + 1]), nn, (const uint32_t*)B.apos,
                               B.reps[nxt], cnt));
        }
        SSS_CUDA(cudaMemcpyAsync(h, cnt, sizeof(uint32_t) * 2, cudaMemcpyDeviceToHost, ctx->stream));
        SSS_CUDA(cudaStreamSynchronize(ctx->stream));
        nreps = h[0];
        retired = h[1];
        reps = B.reps[nxt];
        nxt ^= 1;
    }
    return sss_launch(ctx, "pd_final", k_pd_final, dim3((n + 255) / 256), dim3(256), 0, in, (const uint32_t*)B.apos,
                      (const uint32_t*)B.lpos, approx);
}

// ---------------------------------------------------------------------------
// Allocation-free variant of stage B for small sets (sss_dist_prefix_noalloc).
//
// Some callers cannot allocate device memory when they need this result: a host
// framework that owns the whole device budget and hands out no allocator, or a
// latency-critical request loop where a cudaMalloc could block, fail or
// fragment memory at an arbitrary moment.  This entry point therefore needs no
// context and no work memory: its per-string state and its hash table live in
// the fixed array below, which every GPU that loads the library holds until the
// process exits.  One CTA runs all rounds (plain doubling, no local runs).
namespace {

constexpr uint32_t NA_MAXN = SSS_NOALLOC_MAX_STRINGS;  // strings per call
constexpr uint32_t NA_TSLOTS = 2 * NA_MAXN;            // hash-table slots
constexpr size_t NA_OFF_APOS = 0;
constexpr size_t NA_OFF_HLEN = NA_OFF_APOS + sizeof(uint32_t) * NA_MAXN;
constexpr size_t NA_OFF_HST = NA_OFF_HLEN + sizeof(uint32_t) * NA_MAXN;
constexpr size_t NA_OFF_KEY = NA_OFF_HST + sizeof(uint64_t) * NA_MAXN;
constexpr size_t NA_OFF_TAB = NA_OFF_KEY + sizeof(uint64_t) * NA_MAXN;
constexpr size_t NA_OFF_MARK = NA_OFF_TAB + sizeof(uint64_t) * NA_TSLOTS;
constexpr size_t NA_BYTES = NA_OFF_MARK + NA_TSLOTS;
constexpr int NA_T = 1024;
static_assert((NA_TSLOTS & (NA_TSLOTS - 1)) == 0, "the fixed hash table must have a power-of-two slot count");

// The scratch shared by every call on a device (contents persist between calls).
static __device__ __align__(256) unsigned char g_pd_noalloc_scratch[NA_BYTES];

__global__ void __launch_bounds__(NA_T) k_pd_noalloc(const uint8_t* __restrict__ chars,
                                                     const uint64_t* __restrict__ offs,
                                                     const uint32_t* __restrict__ lens, uint32_t n, uint32_t kmin,
                                                     uint32_t kmax, uint64_t B, uint32_t tslots,
                                                     uint32_t* __restrict__ out_approx,
                                                     unsigned char* __restrict__ scratch) {
    uint32_t* apos = reinterpret_cast<uint32_t*>(scratch + NA_OFF_APOS);
    uint32_t* hlen = reinterpret_cast<uint32_t*>(scratch + NA_OFF_HLEN);
    uint64_t* hst = reinterpret_cast<uint64_t*>(scratch + NA_OFF_HST);
    uint64_t* key = reinterpret_cast<uint64_t*>(scratch + NA_OFF_KEY);
    unsigned long long* tab = reinterpret_cast<unsigned long long*>(scratch + NA_OFF_TAB);
    uint8_t* mark = scratch + NA_OFF_MARK;
    __shared__ uint32_t sh_zero, sh_active;
    // the table in use: tslots = the power of two >= 2n (<= NA_TSLOTS), so the
    // per-round clear touches only the slots this call can fill
    const uint32_t tmask = tslots - 1;
    // every call starts from a clean state: the array keeps the previous call's contents
    for (uint32_t i = threadIdx.x; i < n; i += NA_T) {
        apos[i] = ACTIVE;
        hlen[i] = 0;
    }
    __syncthreads();
    for (uint32_t k = kmin; k <= kmax; ++k) {
        const uint64_t L = 1ull << k;
        for (uint32_t t = threadIdx.x; t < tslots; t += NA_T) {
            tab[t] = 0ull;
            mark[t] = 0;
        }
        if (threadIdx.x == 0) {
            sh_zero = 0;
            sh_active = 0;
        }
        __syncthreads();
        // hash every active string's prefix of length min(L, len) and insert its key
        for (uint32_t i = threadIdx.x; i < n; i += NA_T) {
            if (apos[i] != ACTIVE) continue;
            uint32_t len = lens[i];
            uint32_t le = L < len ? (uint32_t)L : len;
            const uint8_t* str = chars + offs[i];
            uint64_t h = 0;
            uint32_t w0 = 0;
            if (L >= 16 && hlen[i] == (uint32_t)(L / 2)) {
                h = hst[i];
                w0 = (uint32_t)(L / 16);
            }
            for (uint32_t w = w0; w < (le + 7) / 8; ++w) {
                uint64_t x = load_word_be(str, le, 8 * w);
                h = fold_limb(h, B, x >> 32);
                h = fold_limb(h, B, x & 0xFFFFFFFFull);
            }
            hst[i] = h;
            hlen[i] = le;
            uint64_t kk = smix64(h ^ ((uint64_t)le * GAMMA));
            key[i] = kk;
            if (kk == 0) {
                atomicAdd(&sh_zero, 1u);
                continue;
            }
            uint32_t hs = (uint32_t)kk & tmask;
            for (uint32_t probe = 0; probe <= tmask; ++probe) {
                unsigned long long old = atomicCAS(&tab[hs], 0ull, (unsigned long long)kk);
                if (old == 0ull) break;
                if (old == kk) {
                    mark[hs] = 1;
                    break;
                }
                hs = (hs + 1) & tmask;
            }
        }
        __syncthreads();
        // retire strings whose key is unique or whose whole length was tested
        for (uint32_t i = threadIdx.x; i < n; i += NA_T) {
            if (apos[i] != ACTIVE) continue;
            uint32_t len = lens[i];
            bool dup = ht_dup(tab, mark, tmask, sh_zero, key[i]);
            if (!dup || (uint64_t)len <= L) apos[i] = (uint64_t)len < L ? len : (uint32_t)L;
            else atomicAdd(&sh_active, 1u);
        }
        __syncthreads();
        if (sh_active == 0) break;
        __syncthreads();
    }
    for (uint32_t i = threadIdx.x; i < n; i += NA_T) {
        uint32_t a = apos[i];
        out_approx[i] = a == ACTIVE ? lens[i] : a;
    }
}

std::mutex g_na_mu;
unsigned char* g_na_ptr[64];

}  // namespace

extern "C" sss_status sss_dist_prefix_noalloc(const uint8_t* chars, uint64_t n_chars, const uint64_t* offsets,
                                              const uint32_t* lengths, uint32_t n, const sss_params* params,
                                              uint32_t* out_approx, void* cuda_stream) {
    (void)n_chars;
    if (n > NA_MAXN) return SSS_ERR_INVALID_ARG;  // beyond the fixed capacity
    if (n == 0) return SSS_OK;
    if (!chars || !offsets || !lengths || !out_approx) return SSS_ERR_INVALID_ARG;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return SSS_ERR_CUDA;
    unsigned char* scratch;
    {
        // first call on this device: look up the device address of the fixed array
        // (host code may not use the array's name as a device pointer)
        std::lock_guard<std::mutex> lk(g_na_mu);
        if (!g_na_ptr[dev]) {
            void* ptr = nullptr;
            if (cudaGetSymbolAddress(&ptr, g_pd_noalloc_scratch) != cudaSuccess || ptr == nullptr) {
                cudaGetLastError();
                return SSS_ERR_CUDA;
            }
            g_na_ptr[dev] = static_cast<unsigned char*>(ptr);
        }
        scratch = g_na_ptr[dev];
    }
    sss_params prm;
    sss_params_default(&prm);
    if (params) prm = *params;
    const uint32_t kmin = std::min<uint32_t>(prm.kmin, 31u);
    const uint32_t kmax = prm.kmax == SSS_KMAX_AUTO ? 31u : std::min<uint32_t>(prm.kmax, 31u);
    const uint64_t Bh = 2 + host_smix(prm.hash_seed + GAMMA) % (P61 - 3);
    if (kmin > kmax) {
        // no rounds: every string keeps approx = len
        return cudaMemcpyAsync(out_approx, lengths, sizeof(uint32_t) * n, cudaMemcpyDeviceToDevice,
                               static_cast<cudaStream_t>(cuda_stream)) == cudaSuccess
                   ? SSS_OK
                   : SSS_ERR_CUDA;
    }
    uint32_t tslots = 64;
    while (tslots < 2 * n) tslots *= 2;  // n <= NA_MAXN, so tslots <= NA_TSLOTS
    k_pd_noalloc<<<1, NA_T, 0, static_cast<cudaStream_t>(cuda_stream)>>>(chars, offsets, lengths, n, kmin, kmax, Bh,
                                                                         tslots, out_approx, scratch);
    return cudaGetLastError() == cudaSuccess ? SSS_OK : SSS_ERR_CUDA;
}
