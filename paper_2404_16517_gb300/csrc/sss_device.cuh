// Device-side helpers: character words, LCP extension, block scans, bitonic sort.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#define SSS_FULL 0xFFFFFFFFu

__device__ __forceinline__ uint64_t bswap64(uint64_t x) {
    uint32_t lo = (uint32_t)x, hi = (uint32_t)(x >> 32);
    return ((uint64_t)__byte_perm(lo, 0, 0x0123) << 32) | (uint64_t)__byte_perm(hi, 0, 0x0123);
}

// Character loads.  STREAM = true marks a word read once from a scattered
// string (one word per string in a pass over many strings): the load allocates
// its lines with evict-first priority in L1 and L2 (ld.global.cs), so they give
// way before the lines other strings' gathers still need.  Not for a window a
// thread streams through: there the next loads use the rest of the same lines.
template <bool STREAM>
__device__ __forceinline__ uint64_t ld_chars8(const uint64_t* p) {
    const unsigned long long* q = reinterpret_cast<const unsigned long long*>(p);
    if constexpr (STREAM) return (uint64_t)__ldcs(q);
    else return (uint64_t)__ldg(q);
}

// The 8 characters s[d .. d+8) as a big-endian word, bytes at or past `len` zero
// (the implicit sentinel sorts below every character, so word order == string
// order on these 8 characters).  Reads only 8-byte-aligned words that contain at
// least one character of the string, so it never touches a page the string does
// not touch.
template <bool STREAM = false>
__device__ __forceinline__ uint64_t load_word_be(const uint8_t* __restrict__ s, uint32_t len, uint32_t d) {
    if (d >= len) return 0;
    uintptr_t ai = (uintptr_t)(s + d);
    const uint64_t* base = reinterpret_cast<const uint64_t*>(ai & ~uintptr_t(7));
    uint32_t sh = (uint32_t)(ai & 7);
    uint32_t rem = len - d;
    uint64_t x = bswap64(ld_chars8<STREAM>(base)) << (8 * sh);
    if (sh != 0 && rem > 8 - sh) x |= bswap64(ld_chars8<STREAM>(base + 1)) >> (64 - 8 * sh);
    if (rem < 8) x &= ~0ull << (8 * (8 - rem));
    return x;
}

// Consecutive big-endian 8-character words of s[d .. len), zero past len, with
// one aligned 8-byte load per word.  Only aligned words that hold at least one
// character of the string are loaded.
struct WordStream {
    const uint64_t* p;  // next aligned word to load
    const uint8_t* end;
    uint64_t cur;       // current aligned word, big-endian
    uint32_t sh;        // misalignment in bits
    uint32_t rem;       // characters left from the current position
    __device__ __forceinline__ void init(const uint8_t* __restrict__ s, uint32_t len, uint32_t d) {
        rem = len > d ? len - d : 0;
        uintptr_t a = (uintptr_t)(s + d);
        p = reinterpret_cast<const uint64_t*>(a & ~uintptr_t(7));
        sh = (uint32_t)(a & 7) * 8;
        end = s + len;
        cur = rem ? bswap64(__ldg(p)) : 0;
        ++p;
    }
    // the characters at the current position that came with the first load:
    // returns them left-aligned, *nb = how many (>= 1 when rem > 0)
    __device__ __forceinline__ uint64_t head(uint32_t* nb) const {
        const uint32_t av = 8u - sh / 8u;
        *nb = av < rem ? av : rem;
        return cur << sh;
    }
    // the next 4 words (32 characters), with the 4 aligned loads issued together
    __device__ __forceinline__ void next4(uint64_t* w) {
        uint64_t nx[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const uint64_t* pi = p + i;
            nx[i] = (rem > 8u * i && reinterpret_cast<const uint8_t*>(pi) < end) ? bswap64(__ldg(pi)) : 0ull;
        }
        p += 4;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            uint64_t x = sh ? ((cur << sh) | (nx[i] >> (64 - sh))) : cur;
            cur = nx[i];
            if (rem < 8) {
                x = rem ? (x & (~0ull << (8 * (8 - rem)))) : 0ull;
                rem = 0;
            } else {
                rem -= 8;
            }
            w[i] = x;
        }
    }
    __device__ __forceinline__ uint64_t next() {
        if (rem == 0) return 0;
        uint64_t nx = (reinterpret_cast<const uint8_t*>(p) < end) ? bswap64(__ldg(p)) : 0;
        ++p;
        uint64_t w = sh ? ((cur << sh) | (nx >> (64 - sh))) : cur;
        cur = nx;
        if (rem < 8) {
            w &= ~0ull << (8 * (8 - rem));
            rem = 0;
        } else {
            rem -= 8;
        }
        return w;
    }
};

// WordStream with 16-byte loads: the next 4 words cost two aligned 16-byte
// loads (half the load instructions, and half the L1 wavefronts of a gather
// where every lane reads its own string).  A 16-byte-aligned chunk never
// crosses a page, and only chunks that start before the string's end are
// loaded, so it touches no memory the string's own pages do not hold.
struct WordStream16 {
    const ulonglong2* p;  // next aligned chunk to load
    const uint8_t* end;
    uint64_t a0;          // current aligned word (big-endian)
    uint64_t a1;          // the word after it, when it came with a0's chunk (hi == 0)
    uint32_t hi;          // 0: a0 is the low half of its chunk (a1 valid); 1: the high half
    uint32_t sh;          // misalignment in bits
    uint32_t rem;         // characters left from the current position
    __device__ __forceinline__ void init(const uint8_t* __restrict__ s, uint32_t len, uint32_t d) {
        rem = len > d ? len - d : 0;
        uintptr_t a = (uintptr_t)(s + d);
        const ulonglong2* c = reinterpret_cast<const ulonglong2*>(a & ~uintptr_t(15));
        sh = (uint32_t)(a & 7) * 8;
        hi = (uint32_t)((a >> 3) & 1);
        end = s + len;
        ulonglong2 v = rem ? __ldg(c) : make_ulonglong2(0ull, 0ull);
        a0 = bswap64(hi ? v.y : v.x);
        a1 = bswap64(v.y);
        p = c + 1;
    }
    // the next 4 words (32 characters)
    __device__ __forceinline__ void next4(uint64_t* w) {
        ulonglong2 c1 = make_ulonglong2(0ull, 0ull), c2 = make_ulonglong2(0ull, 0ull);
        if (rem > 0 && reinterpret_cast<const uint8_t*>(p) < end) c1 = __ldg(p);
        if (rem > 16 - 8 * hi && reinterpret_cast<const uint8_t*>(p + 1) < end) c2 = __ldg(p + 1);
        p += 2;
        uint64_t x[5];
        x[0] = a0;
        if (hi) {  // a0 was the high half: the next words are c1.x, c1.y, c2.x, c2.y
            x[1] = bswap64(c1.x);
            x[2] = bswap64(c1.y);
            x[3] = bswap64(c2.x);
            x[4] = bswap64(c2.y);
            a0 = x[4];
        } else {   // a0 was the low half: a1 came with it
            x[1] = a1;
            x[2] = bswap64(c1.x);
            x[3] = bswap64(c1.y);
            x[4] = bswap64(c2.x);
            a0 = x[4];
            a1 = bswap64(c2.y);
        }
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            uint64_t v = sh ? ((x[i] << sh) | (x[i + 1] >> (64 - sh))) : x[i];
            if (rem < 8) {
                v = rem ? (v & (~0ull << (8 * (8 - rem)))) : 0ull;
                rem = 0;
            } else {
                rem -= 8;
            }
            w[i] = v;
        }
    }
};

// Full LCP of a[d..] and b[d..] (capped at min(la, lb) - d and at VCAP), in
// blocks of 32 characters with independent loads; *w = the 8 characters of `a`
// at d + v (zero past its end).
constexpr uint32_t VCAP = (1u << 30) - 1;

// the first nb (0..8) bytes of a big-endian word
__device__ __forceinline__ uint64_t top_bytes_mask(uint32_t nb) {
    return nb >= 8u ? ~0ull : (nb ? ~0ull << (8u * (8u - nb)) : 0ull);
}

__device__ __forceinline__ uint32_t lcp_full_w(const uint8_t* __restrict__ a, uint32_t la,
                                               const uint8_t* __restrict__ b, uint32_t lb, uint32_t d,
                                               uint64_t* w) {
    uint32_t m = la < lb ? la : lb;
    uint32_t r = 0;
    if (d < m) {
        uint32_t cap = m - d;
        WordStream A, B;
        A.init(a, la, d);
        B.init(b, lb, d);
        r = cap;
        // most pairs differ within the characters of the first loads: only
        // then stream on
        uint32_t na, nb;
        const uint64_t ha = A.head(&na), hb = B.head(&nb);
        const uint64_t x0 = (ha ^ hb) & top_bytes_mask(na < nb ? na : nb);
        if (x0) {
            const uint32_t c = (uint32_t)__clzll((long long)x0) >> 3;
            r = c < cap ? c : cap;
        }
        for (uint32_t k = 0; !x0 && k < cap && k < VCAP; k += 32) {
            uint64_t xa[4], xb[4];
            A.next4(xa);
            B.next4(xb);
            bool hit = false;
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                uint64_t x = xa[i] ^ xb[i];
                if (!hit && x) {
                    uint32_t c = k + 8 * i + ((uint32_t)__clzll((long long)x) >> 3);
                    r = c < cap ? c : cap;
                    hit = true;
                }
            }
            if (hit) break;
        }
    }
    if (r > VCAP) r = VCAP;
    *w = load_word_be(a, la, d + r);
    return r;
}

// lcp_full_w with the reference's words [d, d + 8*nref) already in shared memory
// (refw, zero past the reference's end); only used when min(la, lb) - d <=
// 8*nref, so every reference word it needs is there.
__device__ __forceinline__ uint32_t lcp_full_w_ref(const uint8_t* __restrict__ a, uint32_t la, uint32_t lb,
                                                   const uint64_t* refw, uint32_t d, uint64_t* w) {
    uint32_t m = la < lb ? la : lb;
    uint32_t r = 0;
    if (d < m) {
        uint32_t cap = m - d;
        WordStream16 A;
        A.init(a, la, d);
        r = cap;
        for (uint32_t k = 0; k < cap; k += 32) {
            uint64_t xa[4];
            A.next4(xa);
            bool hit = false;
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                uint64_t x = xa[i] ^ refw[(k >> 3) + i];
                if (!hit && x) {
                    uint32_t c = k + 8 * i + ((uint32_t)__clzll((long long)x) >> 3);
                    r = c < cap ? c : cap;
                    hit = true;
                }
            }
            if (hit) break;
        }
    }
    *w = load_word_be(a, la, d + r);
    return r;
}

// ---------------------------------------------------------------------------
// Reference-split keys.  All members of a segment share their first d
// characters; r is the segment's reference member.  For a member s let v =
// lcp(s[d..], r[d..]), c = s[d+v] and rho = r[d+v] (0 past an end).  Then s < r
// when c < rho, s > r when c > rho, and c == rho only when s equals r (both
// ended).  Among the members below r a larger v means closer to r; among those
// above, a larger v means smaller.  So the 64-bit key
//     side  (2 bits: 0 below, 1 equal, 2 above)
//   | vk    (vb bits: v below and equal, vcap - v above)
//   | chars (8*C bits: s[d+v .. d+v+C), zero past the end)
// orders the members by string order on their first d + v + C characters.  Two
// members with equal keys share d + v + C characters (or are equal strings when
// the chars hold a zero byte); two adjacent distinct keys have lcp d + v + (first
// differing byte of the chars) when side and v agree, else d + min(v, v').  Every
// member advances by its own v, so a segment whose members leave a shared prefix
// one by one (a staircase) splits in a few rounds instead of one round per word.
//
// The field widths depend on the reference's remaining length W = |r| - d,
// which bounds v: vb = bit length of W (at most 30), C = 6, 5 or 4 characters
// for vb <= 14, 22, 30.  When W >= 2^30 a member agreeing with r on 2^30 - 1
// characters gets side 1 and v = vcap (its group continues from there).  The
// format is packed as vb | C << 8.
__device__ __forceinline__ uint32_t key_fmt(uint32_t rlen, uint32_t d) {
    uint32_t w = rlen > d ? rlen - d : 0u;
    uint32_t vb = w ? 32u - (uint32_t)__clz((int)w) : 1u;
    vb = vb < 30u ? vb : 30u;
    uint32_t c = vb <= 14u ? 6u : (vb <= 22u ? 5u : 4u);
    return vb | (c << 8);
}
__device__ __forceinline__ uint32_t fmt_chars(uint32_t f) { return f >> 8; }

__device__ __forceinline__ uint64_t ref_key(uint32_t v, uint64_t w, uint32_t rho, uint32_t f) {
    const uint32_t vb = f & 31u, cb = 8u * (f >> 8);
    const uint32_t vcap = (1u << vb) - 1u;
    uint32_t c = (uint32_t)(w >> 56);
    uint64_t side, vk;
    if (v >= vcap || c == rho) {
        side = 1;
        vk = v < vcap ? v : vcap;
    } else if (c < rho) {
        side = 0;
        vk = v;
    } else {
        side = 2;
        vk = vcap - v;
    }
    return (side << 62) | (vk << (62 - vb)) | ((w >> (64 - cb)) << (62 - vb - cb));
}

__device__ __forceinline__ uint32_t key_v(uint64_t k, uint32_t f) {
    const uint32_t vb = f & 31u;
    const uint32_t vcap = (1u << vb) - 1u;
    uint32_t vk = (uint32_t)(k >> (62 - vb)) & vcap;
    return (k >> 62) == 2 ? vcap - vk : vk;
}

// lcp beyond the segment depth of two distinct keys of one segment
__device__ __forceinline__ uint32_t key_lcp(uint64_t a, uint64_t b, uint32_t f) {
    const uint32_t vb = f & 31u;
    if ((a >> (62 - vb)) == (b >> (62 - vb))) {
        uint64_t x = (a ^ b) << (2 + vb);
        return key_v(a, f) + (x ? ((uint32_t)__clzll((long long)x) >> 3) : fmt_chars(f));
    }
    uint32_t va = key_v(a, f), vbb = key_v(b, f);
    return va < vbb ? va : vbb;
}

// the strings of a key ended inside its characters (equal keys = equal strings)
__device__ __forceinline__ bool key_ended(uint64_t k, uint32_t f) {
    const uint32_t vb = f & 31u, cb = 8u * (f >> 8);
    uint64_t x = (k << (2 + vb)) | (~0ull >> cb);
    return ((x - 0x0101010101010101ull) & ~x & 0x8080808080808080ull) != 0;
}

// First differing character of two distinct words, counted from the word start.
__device__ __forceinline__ uint32_t word_lcp(uint64_t a, uint64_t b) {
    uint64_t x = a ^ b;
    return x ? ((uint32_t)__clzll((long long)x) >> 3) : 8u;
}

// True if the word contains a zero byte, i.e. the string ended inside it.
__device__ __forceinline__ bool word_has_zero(uint64_t k) {
    return ((k - 0x0101010101010101ull) & ~k & 0x8080808080808080ull) != 0;
}

// ---------------------------------------------------------------------------
// Block-wide scans over THREADS threads, each owning one value.
template <int THREADS>
struct BlockScan {
    static constexpr int WARPS = (THREADS + 31) / 32;
    // exclusive sum; *total receives the block sum (all threads)
    __device__ static uint32_t exclusive_sum(uint32_t v, uint32_t* sh_warp, uint32_t* total) {
        int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
        uint32_t x = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(SSS_FULL, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) sh_warp[w] = x;
        __syncthreads();
        if (w == 0) {
            uint32_t t = lane < WARPS ? sh_warp[lane] : 0;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                uint32_t y = __shfl_up_sync(SSS_FULL, t, o);
                if (lane >= o) t += y;
            }
            if (lane < WARPS) sh_warp[lane] = t;  // inclusive warp prefix
        }
        __syncthreads();
        uint32_t base = w > 0 ? sh_warp[w - 1] : 0;
        uint32_t tot = sh_warp[WARPS - 1];
        __syncthreads();
        if (total) *total = tot;
        return base + x - v;
    }
    // inclusive max
    __device__ static uint32_t inclusive_max(uint32_t v, uint32_t* sh_warp) {
        int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
        uint32_t x = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(SSS_FULL, x, o);
            if (lane >= o) x = x > y ? x : y;
        }
        if (lane == 31) sh_warp[w] = x;
        __syncthreads();
        if (w == 0) {
            uint32_t t = lane < WARPS ? sh_warp[lane] : 0;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                uint32_t y = __shfl_up_sync(SSS_FULL, t, o);
                if (lane >= o) t = t > y ? t : y;
            }
            if (lane < WARPS) sh_warp[lane] = t;
        }
        __syncthreads();
        uint32_t base = w > 0 ? sh_warp[w - 1] : 0;
        __syncthreads();
        return x > base ? x : base;
    }
};

// Exclusive sum over `count` items held ITEMS-per-thread in a contiguous blocked
// layout of an smem array (in place); returns the total.
template <int THREADS, int ITEMS>
__device__ uint32_t block_exclusive_sum_inplace(uint32_t* a, uint32_t count, uint32_t* sh_warp) {
    uint32_t loc[ITEMS];
    uint32_t sum = 0;
    int b = threadIdx.x * ITEMS;
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) {
        uint32_t v = (uint32_t)(b + i) < count ? a[b + i] : 0;
        loc[i] = sum;
        sum += v;
    }
    uint32_t total;
    uint32_t off = BlockScan<THREADS>::exclusive_sum(sum, sh_warp, &total);
#pragma unroll
    for (int i = 0; i < ITEMS; ++i)
        if ((uint32_t)(b + i) < count) a[b + i] = off + loc[i];
    __syncthreads();
    return total;
}

// Inclusive max over a blocked smem array (in place).
template <int THREADS, int ITEMS>
__device__ void block_inclusive_max_inplace(uint32_t* a, uint32_t count, uint32_t* sh_warp) {
    uint32_t loc[ITEMS];
    uint32_t m = 0;
    int b = threadIdx.x * ITEMS;
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) {
        uint32_t v = (uint32_t)(b + i) < count ? a[b + i] : 0;
        m = v > m ? v : m;
        loc[i] = m;
    }
    // exclusive max of thread totals = inclusive max of previous threads
    uint32_t incl = BlockScan<THREADS>::inclusive_max(m, sh_warp);
    uint32_t prev = __shfl_up_sync(SSS_FULL, incl, 1);
    // thread 0 of each warp needs the previous warp's inclusive value
    __shared__ uint32_t sh_last[(THREADS + 31) / 32];
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 31) sh_last[w] = incl;
    __syncthreads();
    if (lane == 0) prev = w > 0 ? sh_last[w - 1] : 0;
    if (threadIdx.x == 0) prev = 0;
#pragma unroll
    for (int i = 0; i < ITEMS; ++i)
        if ((uint32_t)(b + i) < count) a[b + i] = loc[i] > prev ? loc[i] : prev;
    __syncthreads();
}

// ---------------------------------------------------------------------------
// In-shared-memory bitonic sort of `count` 128-bit keys (hi, lo), ascending,
// padded to the next power of two with all-ones keys (count <= CAP).
__device__ __forceinline__ bool key128_less(uint64_t ah, uint64_t al, uint64_t bh, uint64_t bl) {
    return ah < bh || (ah == bh && al < bl);
}

template <int THREADS>
__device__ void bitonic_sort128(uint64_t* hi, uint64_t* lo, uint32_t count) {
    uint32_t P = 1;
    while (P < count) P <<= 1;
    for (uint32_t i = count + threadIdx.x; i < P; i += THREADS) {
        hi[i] = ~0ull;
        lo[i] = ~0ull;
    }
    __syncthreads();
    for (uint32_t k = 2; k <= P; k <<= 1) {
        for (uint32_t j = k >> 1; j > 0; j >>= 1) {
            for (uint32_t t = threadIdx.x; t < P / 2; t += THREADS) {
                // t-th compare-exchange pair of this stage
                uint32_t i = 2 * j * (t / j) + (t % j);
                uint32_t ixj = i + j;
                bool up = (i & k) == 0;
                uint64_t ah = hi[i], al = lo[i], bh = hi[ixj], bl = lo[ixj];
                bool sw = up ? key128_less(bh, bl, ah, al) : key128_less(ah, al, bh, bl);
                if (sw) {
                    hi[i] = bh;
                    lo[i] = bl;
                    hi[ixj] = ah;
                    lo[ixj] = al;
                }
            }
            __syncthreads();
        }
    }
}

template <int THREADS>
__device__ void bitonic_sort64(uint64_t* a, uint32_t count) {
    uint32_t P = 1;
    while (P < count) P <<= 1;
    for (uint32_t i = count + threadIdx.x; i < P; i += THREADS) a[i] = ~0ull;
    __syncthreads();
    for (uint32_t k = 2; k <= P; k <<= 1) {
        for (uint32_t j = k >> 1; j > 0; j >>= 1) {
            for (uint32_t t = threadIdx.x; t < P / 2; t += THREADS) {
                uint32_t i = 2 * j * (t / j) + (t % j);
                uint32_t ixj = i + j;
                bool up = (i & k) == 0;
                uint64_t x = a[i], y = a[ixj];
                if (up ? (y < x) : (x < y)) {
                    a[i] = y;
                    a[ixj] = x;
                }
            }
            __syncthreads();
        }
    }
}

// ---------------------------------------------------------------------------
// Shared-memory swizzle for the merge sort's blocked layout: thread t owns the
// ITEMS logical slots t*ITEMS .. t*ITEMS+ITEMS-1, and when all threads access
// their i-th slot at once a plain layout puts 16 lanes of a half-warp on the
// same few 8-byte bank pairs.  XOR-ing the slot with a few bits of the thread
// index spreads them over all 16; consecutive logical indices stay
// conflict-free too.  A bijection on every block of ITEMS slots.
template <int ITEMS>
__device__ __forceinline__ uint32_t swz(uint32_t j) {
    constexpr uint32_t PER_ROW = ITEMS >= 16 ? 1u : 16u / ITEMS;  // blocks per 128-byte row
    return j ^ (((j / ITEMS) / PER_ROW) & (ITEMS - 1));
}

// The merge rounds' barrier: while a pair of runs spans at most 32 threads
// (2w <= 32, runs of w threads' outputs), the pair's slots are written and read
// by that warp alone (the swizzle permutes within blocks of ITEMS slots, and a
// thread writes only its own block), so the warp's barrier suffices.
__device__ __forceinline__ void merge_round_sync(uint32_t w) {
    if (2 * w <= 32) __syncwarp();
    else __syncthreads();
}

// Block merge sort of `count` 128-bit keys (hi, lo) held in shared memory arrays
// of THREADS*ITEMS entries, ascending; input and output in plain index order.
// Each thread sorts ITEMS keys in registers (odd-even transposition), then
// log2(THREADS) rounds merge pairs of sorted lists: every thread finds its ITEMS
// outputs with a merge-path binary search and merges them serially.  Inside, the
// arrays use the swizzled layout (swz), entered and left through striped passes,
// so no register<->shared transfer has bank conflicts.  Slots past `count` are
// padded with all-ones keys (the arrays are fully overwritten).
template <int THREADS, int ITEMS>
__device__ void block_merge_sort128(uint64_t* sHi, uint64_t* sLo, uint32_t count) {
    static_assert(THREADS % 32 == 0, "whole warps: the in-warp merge rounds use the warp barrier");
    const uint32_t tid = threadIdx.x;
    uint64_t h[ITEMS], l[ITEMS];
    // plain -> swizzled, padding the tail
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) {
        uint32_t j = tid + i * THREADS;
        h[i] = j < count ? sHi[j] : ~0ull;
        l[i] = j < count ? sLo[j] : ~0ull;
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) {
        uint32_t j = swz<ITEMS>(tid + i * THREADS);
        sHi[j] = h[i];
        sLo[j] = l[i];
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) {
        uint32_t j = swz<ITEMS>(tid * ITEMS + i);
        h[i] = sHi[j];
        l[i] = sLo[j];
    }
#pragma unroll
    for (int r = 0; r < ITEMS; ++r) {
#pragma unroll
        for (int i = (r & 1); i + 1 < ITEMS; i += 2) {
            if (key128_less(h[i + 1], l[i + 1], h[i], l[i])) {
                uint64_t th = h[i], tl = l[i];
                h[i] = h[i + 1];
                l[i] = l[i + 1];
                h[i + 1] = th;
                l[i + 1] = tl;
            }
        }
    }
    const uint32_t used = (count + ITEMS - 1) / ITEMS;  // threads holding real keys
    for (uint32_t w = 1; w < used; w <<= 1) {
        merge_round_sync(w);
#pragma unroll
        for (int i = 0; i < ITEMS; ++i) {
            uint32_t j = swz<ITEMS>(tid * ITEMS + i);
            sHi[j] = h[i];
            sLo[j] = l[i];
        }
        merge_round_sync(w);
        const uint32_t L = w * ITEMS;
        const uint32_t g0 = (tid / (2 * w)) * (2 * L);
        if (g0 >= count) continue;  // a pair of padding lists stays as it is
        const uint32_t diag = (tid % (2 * w)) * ITEMS;
        const uint32_t A0 = g0, B0 = g0 + L;
        uint32_t lo = diag > L ? diag - L : 0, hi = diag < L ? diag : L;
        while (lo < hi) {
            uint32_t mid = (lo + hi) >> 1;
            uint32_t bj = swz<ITEMS>(B0 + diag - 1 - mid), aj = swz<ITEMS>(A0 + mid);
            if (!key128_less(sHi[bj], sLo[bj], sHi[aj], sLo[aj])) lo = mid + 1;
            else hi = mid;
        }
        uint32_t a = lo, b = diag - lo;
        // the heads of both lists stay in registers; each output step loads
        // only the new head of the list it took from (address chosen without a
        // branch, so the warp does not diverge)
        uint64_t ah = ~0ull, al = ~0ull, bh = ~0ull, bl = ~0ull;
        if (a < L) {
            const uint32_t aj = swz<ITEMS>(A0 + a);
            ah = sHi[aj];
            al = sLo[aj];
        }
        if (b < L) {
            const uint32_t bj = swz<ITEMS>(B0 + b);
            bh = sHi[bj];
            bl = sLo[bj];
        }
#pragma unroll
        for (int i = 0; i < ITEMS; ++i) {
            const bool takeA = a < L && (b >= L || !key128_less(bh, bl, ah, al));
            h[i] = takeA ? ah : bh;
            l[i] = takeA ? al : bl;
            a += takeA ? 1u : 0u;
            b += takeA ? 0u : 1u;
            if (i + 1 < ITEMS) {
                const uint32_t nx = takeA ? a : b;
                uint64_t nh = ~0ull, nl = ~0ull;
                if (nx < L) {
                    const uint32_t nj = swz<ITEMS>((takeA ? A0 : B0) + nx);
                    nh = sHi[nj];
                    nl = sLo[nj];
                }
                ah = takeA ? nh : ah;
                al = takeA ? nl : al;
                bh = takeA ? bh : nh;
                bl = takeA ? bl : nl;
            }
        }
    }
    // swizzled -> plain
    __syncthreads();
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) {
        uint32_t j = swz<ITEMS>(tid * ITEMS + i);
        sHi[j] = h[i];
        sLo[j] = l[i];
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) {
        uint32_t j = swz<ITEMS>(tid + i * THREADS);
        h[i] = sHi[j];
        l[i] = sLo[j];
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) {
        uint32_t j = tid + i * THREADS;
        sHi[j] = h[i];
        sLo[j] = l[i];
    }
    __syncthreads();
}

// Stable block merge sort of `count` (64-bit key, 32-bit value) pairs in shared
// memory by the key alone: pairs with equal keys keep their input order (the
// per-thread odd-even sort swaps only strictly smaller keys, and every merge
// takes the first list's element on ties).  Same structure as
// block_merge_sort128: per-thread sorts of ITEMS pairs, then log2(THREADS)
// merge-path rounds over the swizzled layout; a third less shared-memory
// traffic and 64-bit instead of 128-bit comparisons.  Input and output in plain
// index order; slots past `count` are overwritten with padding.
template <int THREADS, int ITEMS>
__device__ void block_merge_sort_kv(uint64_t* sK, uint32_t* sV, uint32_t count) {
    static_assert(THREADS % 32 == 0, "whole warps: the in-warp merge rounds use the warp barrier");
    const uint32_t tid = threadIdx.x;
    uint64_t k[ITEMS];
    uint32_t v[ITEMS];
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) {
        uint32_t j = tid + i * THREADS;
        k[i] = j < count ? sK[j] : ~0ull;
        v[i] = j < count ? sV[j] : ~0u;
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) {
        uint32_t j = swz<ITEMS>(tid + i * THREADS);
        sK[j] = k[i];
        sV[j] = v[i];
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) {
        uint32_t j = swz<ITEMS>(tid * ITEMS + i);
        k[i] = sK[j];
        v[i] = sV[j];
    }
    // padding (all-ones keys) sits at the end of the thread order, so stability
    // among real pairs is not disturbed by it
#pragma unroll
    for (int r = 0; r < ITEMS; ++r) {
#pragma unroll
        for (int i = (r & 1); i + 1 < ITEMS; i += 2) {
            if (k[i + 1] < k[i]) {
                const uint64_t tk = k[i];
                const uint32_t tv = v[i];
                k[i] = k[i + 1];
                v[i] = v[i + 1];
                k[i + 1] = tk;
                v[i + 1] = tv;
            }
        }
    }
    const uint32_t used = (count + ITEMS - 1) / ITEMS;  // threads holding real pairs
    for (uint32_t w = 1; w < used; w <<= 1) {
        merge_round_sync(w);
#pragma unroll
        for (int i = 0; i < ITEMS; ++i) {
            uint32_t j = swz<ITEMS>(tid * ITEMS + i);
            sK[j] = k[i];
            sV[j] = v[i];
        }
        merge_round_sync(w);
        const uint32_t L = w * ITEMS;
        const uint32_t g0 = (tid / (2 * w)) * (2 * L);
        if (g0 >= count) continue;
        const uint32_t diag = (tid % (2 * w)) * ITEMS;
        const uint32_t A0 = g0, B0 = g0 + L;
        uint32_t lo = diag > L ? diag - L : 0, hi = diag < L ? diag : L;
        while (lo < hi) {
            uint32_t mid = (lo + hi) >> 1;
            if (!(sK[swz<ITEMS>(B0 + diag - 1 - mid)] < sK[swz<ITEMS>(A0 + mid)])) lo = mid + 1;
            else hi = mid;
        }
        uint32_t a = lo, b = diag - lo;
        uint64_t ak = ~0ull, bk = ~0ull;
        uint32_t av = ~0u, bv = ~0u;
        if (a < L) {
            const uint32_t aj = swz<ITEMS>(A0 + a);
            ak = sK[aj];
            av = sV[aj];
        }
        if (b < L) {
            const uint32_t bj = swz<ITEMS>(B0 + b);
            bk = sK[bj];
            bv = sV[bj];
        }
#pragma unroll
        for (int i = 0; i < ITEMS; ++i) {
            const bool takeA = a < L && (b >= L || !(bk < ak));
            k[i] = takeA ? ak : bk;
            v[i] = takeA ? av : bv;
            a += takeA ? 1u : 0u;
            b += takeA ? 0u : 1u;
            if (i + 1 < ITEMS) {
                const uint32_t nx = takeA ? a : b;
                uint64_t nk = ~0ull;
                uint32_t nv = ~0u;
                if (nx < L) {
                    const uint32_t nj = swz<ITEMS>((takeA ? A0 : B0) + nx);
                    nk = sK[nj];
                    nv = sV[nj];
                }
                ak = takeA ? nk : ak;
                av = takeA ? nv : av;
                bk = takeA ? bk : nk;
                bv = takeA ? bv : nv;
            }
        }
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) {
        uint32_t j = swz<ITEMS>(tid * ITEMS + i);
        sK[j] = k[i];
        sV[j] = v[i];
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) {
        uint32_t j = swz<ITEMS>(tid + i * THREADS);
        k[i] = sK[j];
        v[i] = sV[j];
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) {
        uint32_t j = tid + i * THREADS;
        sK[j] = k[i];
        sV[j] = v[i];
    }
    __syncthreads();
}

// block_merge_sort_kv with half the items per thread when they suffice
template <int THREADS, int ITEMS>
__device__ void block_merge_sort_kv_fit(uint64_t* sK, uint32_t* sV, uint32_t count) {
    if constexpr (ITEMS >= 4) {
        if (count <= (uint32_t)(THREADS * ITEMS / 2)) {
            block_merge_sort_kv<THREADS, ITEMS / 2>(sK, sV, count);
            return;
        }
    }
    block_merge_sort_kv<THREADS, ITEMS>(sK, sV, count);
}

// Merge nr sorted runs of 128-bit keys held in shared memory (run k = slots
// [rb[k], rb[k+1]), rb[0] = 0, rb[nr] = count; plain order in and out) into one
// ascending list: ceil(log2 nr) rounds that merge adjacent pairs of runs, where a
// full sort takes log2(THREADS) rounds plus the per-thread sorts.  Every thread
// produces the ITEMS consecutive outputs from tid*ITEMS on, crossing into the
// next pair of runs where its range does; layout and merge steps as in
// block_merge_sort128.  rb (nr + 1 shared words) is overwritten; nr <= 2*THREADS.
template <int THREADS, int ITEMS>
__device__ void block_merge_runs128(uint64_t* sHi, uint64_t* sLo, uint32_t count, uint32_t* rb, uint32_t nr) {
    const uint32_t tid = threadIdx.x;
    uint64_t h[ITEMS], l[ITEMS];
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) {
        const uint32_t j = tid + i * THREADS;
        h[i] = j < count ? sHi[j] : ~0ull;
        l[i] = j < count ? sLo[j] : ~0ull;
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) {
        const uint32_t j = swz<ITEMS>(tid + i * THREADS);
        sHi[j] = h[i];
        sLo[j] = l[i];
    }
    while (nr > 1) {
        __syncthreads();
        const uint32_t npair = (nr + 1) / 2;
        const uint32_t j0 = tid * ITEMS;
        if (j0 < count) {
            // the pair of runs holding output j0: the last q with rb[2q] <= j0
            uint32_t q = 0, qe = npair;
            while (qe - q > 1) {
                const uint32_t mid = (q + qe) >> 1;
                if (rb[2 * mid] <= j0) q = mid;
                else qe = mid;
            }
            uint32_t A0 = rb[2 * q], B0 = 2 * q + 1 <= nr ? rb[2 * q + 1] : count;
            uint32_t E = 2 * q + 2 <= nr ? rb[2 * q + 2] : count;
            uint32_t LA = B0 - A0, LB = E - B0;
            const uint32_t diag = j0 - A0;
            uint32_t lo = diag > LB ? diag - LB : 0, hi = diag < LA ? diag : LA;
            while (lo < hi) {
                const uint32_t mid = (lo + hi) >> 1;
                const uint32_t bj = swz<ITEMS>(B0 + diag - 1 - mid), aj = swz<ITEMS>(A0 + mid);
                if (!key128_less(sHi[bj], sLo[bj], sHi[aj], sLo[aj])) lo = mid + 1;
                else hi = mid;
            }
            uint32_t a = lo, b = diag - lo;
            uint64_t ah = ~0ull, al = ~0ull, bh = ~0ull, bl = ~0ull;
            if (a < LA) {
                ah = sHi[swz<ITEMS>(A0 + a)];
                al = sLo[swz<ITEMS>(A0 + a)];
            }
            if (b < LB) {
                bh = sHi[swz<ITEMS>(B0 + b)];
                bl = sLo[swz<ITEMS>(B0 + b)];
            }
#pragma unroll
            for (int i = 0; i < ITEMS; ++i) {
                if (j0 + i >= count) {
                    h[i] = ~0ull;
                    l[i] = ~0ull;
                    continue;
                }
                while (a >= LA && b >= LB) {  // this pair is done: on to the next
                    ++q;
                    A0 = E;
                    B0 = 2 * q + 1 <= nr ? rb[2 * q + 1] : count;
                    E = 2 * q + 2 <= nr ? rb[2 * q + 2] : count;
                    LA = B0 - A0;
                    LB = E - B0;
                    a = b = 0;
                    if (LA) {
                        ah = sHi[swz<ITEMS>(A0)];
                        al = sLo[swz<ITEMS>(A0)];
                    }
                    if (LB) {
                        bh = sHi[swz<ITEMS>(B0)];
                        bl = sLo[swz<ITEMS>(B0)];
                    }
                }
                const bool takeA = a < LA && (b >= LB || !key128_less(bh, bl, ah, al));
                h[i] = takeA ? ah : bh;
                l[i] = takeA ? al : bl;
                a += takeA ? 1u : 0u;
                b += takeA ? 0u : 1u;
                const uint32_t nx = takeA ? a : b;
                if (nx < (takeA ? LA : LB)) {
                    const uint32_t nj = swz<ITEMS>((takeA ? A0 : B0) + nx);
                    const uint64_t nh = sHi[nj], nl = sLo[nj];
                    ah = takeA ? nh : ah;
                    al = takeA ? nl : al;
                    bh = takeA ? bh : nh;
                    bl = takeA ? bl : nl;
                }
            }
        }
        // the merged pairs are the next round's runs
        uint32_t nb = 0;
        if (tid < npair) nb = rb[2 * tid];
        __syncthreads();
#pragma unroll
        for (int i = 0; i < ITEMS; ++i) {
            const uint32_t j = tid * ITEMS + i;
            if (j < count) {
                sHi[swz<ITEMS>(j)] = h[i];
                sLo[swz<ITEMS>(j)] = l[i];
            }
        }
        if (tid < npair) rb[tid] = nb;
        if (tid == 0) rb[npair] = count;
        nr = npair;
    }
    // swizzled -> plain
    __syncthreads();
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) {
        const uint32_t j = tid + i * THREADS;
        h[i] = sHi[swz<ITEMS>(j)];
        l[i] = sLo[swz<ITEMS>(j)];
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) {
        const uint32_t j = tid + i * THREADS;
        if (j < count) {
            sHi[j] = h[i];
            sLo[j] = l[i];
        }
    }
    __syncthreads();
}

// block_merge_sort128 with half the items per thread when `count` fits in half
// the slots: every thread then holds real keys, instead of half of them idling
// through every merge round (one more, shorter round).  `count` is uniform over
// the CTA; both variants are compiled in.
template <int THREADS, int ITEMS>
__device__ void block_merge_sort128_fit(uint64_t* sHi, uint64_t* sLo, uint32_t count) {
    if constexpr (ITEMS >= 4) {
        if (count <= (uint32_t)(THREADS * ITEMS / 2)) {
            block_merge_sort128<THREADS, ITEMS / 2>(sHi, sLo, count);
            return;
        }
    }
    block_merge_sort128<THREADS, ITEMS>(sHi, sLo, count);
}
