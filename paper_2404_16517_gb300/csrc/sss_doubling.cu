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
// Duplicate detection: the (key, rep) pairs are bucketed by the key's top bits
// (keys are uniform), each bucket is sorted in shared memory and equal
// neighbours mark duplicates.  A bucket larger than shared memory (only with
// many equal keys) is sorted in chunks and cross-checked by binary search.
#include <algorithm>
#include <vector>

#include "sss_device.cuh"
#include "sss_internal.cuh"

namespace {

constexpr uint64_t P61 = (1ull << 61) - 1;
constexpr uint64_t GAMMA = 0x9E3779B97F4A7C15ull;
constexpr uint32_t ACTIVE = 0xFFFFFFFFu;
constexpr int DD_T = 512, DD_CAP = 4096;  // dedupe bucket CTA
constexpr int HB_MAX = 13;                // max top bits for bucketing (8192 buckets)

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

// position q starts a group of equal L-prefixes in its local run
__device__ __forceinline__ bool group_start(const PdIn& in, uint32_t q, uint64_t L) {
    if (!in.run_lcp) return true;
    return in.run_lcp[q] < L || is_part_start(q, in.n, in.p);
}

// warp-aggregated append of q to list[] (counter *cnt)
__device__ __forceinline__ void warp_append(bool want, uint32_t q, uint32_t* list, uint32_t* cnt) {
    uint32_t m = __ballot_sync(SSS_FULL, want);
    if (!m) return;
    int lane = threadIdx.x & 31;
    int leader = __ffs(m) - 1;
    uint32_t base = 0;
    if (lane == leader) base = atomicAdd(cnt, (uint32_t)__popc(m));
    base = __shfl_sync(SSS_FULL, base, leader);
    if (want) list[base + __popc(m & ((1u << lane) - 1u))] = q;
}

__global__ void k_pd_init(PdIn in, const uint32_t* __restrict__ lens, uint32_t* __restrict__ apos,
                          uint32_t* __restrict__ lpos, uint32_t* __restrict__ hlen, uint32_t* __restrict__ act,
                          uint32_t* __restrict__ reps, uint32_t* __restrict__ cnt, uint64_t L0) {
    uint32_t q = blockIdx.x * blockDim.x + threadIdx.x;
    bool valid = q < in.n;
    bool rep = false;
    if (valid) {
        apos[q] = ACTIVE;
        lpos[q] = lens[ord_of(in, q)];
        hlen[q] = 0;
        act[q] = q;
        rep = group_start(in, q, L0);
    }
    warp_append(rep, q, reps, &cnt[0]);
}

// B1: keys of the reps (incremental Horner from the L/2-prefix when available)
__global__ void k_pd_hash(PdIn in, const uint32_t* __restrict__ reps, uint32_t nreps, const uint32_t* __restrict__ lpos,
                          uint64_t* __restrict__ hst, uint32_t* __restrict__ hlen, uint64_t* __restrict__ K,
                          uint32_t* __restrict__ V, uint64_t L, uint64_t B) {
    uint32_t j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= nreps) return;
    uint32_t q = reps[j];
    uint32_t s = ord_of(in, q);
    uint32_t len = lpos[q];
    uint32_t le = L < len ? (uint32_t)L : len;
    const uint8_t* str = in.chars + in.offs[s];
    uint64_t h = 0;
    uint32_t w0 = 0;
    if (L >= 16 && hlen[q] == (uint32_t)(L / 2)) {
        h = hst[q];
        w0 = (uint32_t)(L / 16);
    }
    uint32_t nw = (le + 7) / 8;
    for (uint32_t w = w0; w < nw; ++w) {
        uint64_t x = load_word_be(str, le, 8 * w);
        h = fold_limb(h, B, x >> 32);
        h = fold_limb(h, B, x & 0xFFFFFFFFull);
    }
    hst[q] = h;
    hlen[q] = le;
    K[j] = smix64(h ^ ((uint64_t)le * GAMMA));
    V[j] = q;
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
        bitonic_sort128<DD_T>(sK, sV, m);
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
        bitonic_sort128<DD_T>(sK, sV, cm);
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

// B4: retire unique / fully tested strings; compact the survivors and the next
// round's reps.
__global__ void k_pd_retire(PdIn in, const uint32_t* __restrict__ act, uint32_t nact,
                            const uint32_t* __restrict__ lpos, const uint8_t* __restrict__ dupf,
                            uint32_t* __restrict__ apos, uint32_t* __restrict__ act_next,
                            uint32_t* __restrict__ reps_next, uint32_t* __restrict__ cnt, uint64_t L, int last) {
    uint32_t j = blockIdx.x * blockDim.x + threadIdx.x;
    bool keep = false, rep_next = false;
    uint32_t q = 0;
    if (j < nact) {
        q = act[j];
        uint32_t len = lpos[q];
        bool dup;
        if (group_start(in, q, L)) {
            bool single = true;
            if (in.run_lcp) {
                uint32_t pe = part_end_of(q, in.n, in.p);
                single = !(q + 1 < pe && in.run_lcp[q + 1] >= L);
            }
            dup = !single || dupf[q] != 0;
        } else {
            dup = true;
        }
        if (!dup || (uint64_t)len <= L) {
            apos[q] = (uint64_t)len < L ? len : (uint32_t)L;
        } else {
            keep = true;
            rep_next = !last && group_start(in, q, 2 * L);
        }
    }
    warp_append(keep, q, act_next, &cnt[1]);
    warp_append(rep_next, q, reps_next, &cnt[0]);
}

__global__ void k_pd_final(PdIn in, const uint32_t* __restrict__ apos, const uint32_t* __restrict__ lpos,
                           uint32_t* __restrict__ approx) {
    uint32_t q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= in.n) return;
    uint32_t a = apos[q];
    approx[ord_of(in, q)] = a == ACTIVE ? lpos[q] : a;
}

struct PdBufs {
    uint32_t* apos;
    uint32_t* lpos;
    uint32_t* hlen;
    uint64_t* hst;
    uint32_t* act[2];
    uint32_t* reps[2];
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
    b.act[0] = ar.take<uint32_t>(n);
    b.act[1] = ar.take<uint32_t>(n);
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
    b.cnt = ar.take<uint32_t>(8);
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
    uint32_t kmin = prm.kmin, kmax = prm.kmax == SSS_KMAX_AUTO ? 31u : prm.kmax;
    if (kmax > 31) kmax = 31;
    const uint64_t Bh = 2 + host_smix(prm.hash_seed + GAMMA) % (P61 - 3);

    void* pin;
    SSS_TRY(sss_pinned(ctx, 64, &pin));
    uint32_t* h_cnt = static_cast<uint32_t*>(pin);

    SSS_CUDA(cudaMemsetAsync(B.cnt, 0, sizeof(uint32_t) * 8, ctx->stream));
    uint32_t nact = n, nreps = 0;
    if (kmin <= kmax) {
        SSS_TRY(sss_launch(ctx, "pd_init", k_pd_init, dim3((n + 255) / 256), dim3(256), 0, in, sin.lens, B.apos,
                           B.lpos, B.hlen, B.act[0], B.reps[0], B.cnt, (uint64_t)1 << kmin));
        SSS_CUDA(cudaMemcpyAsync(h_cnt, B.cnt, sizeof(uint32_t), cudaMemcpyDeviceToHost, ctx->stream));
        SSS_CUDA(cudaStreamSynchronize(ctx->stream));
        nreps = h_cnt[0];
    } else {
        // no rounds: every string keeps approx = len
        SSS_TRY(sss_launch(ctx, "pd_init", k_pd_init, dim3((n + 255) / 256), dim3(256), 0, in, sin.lens, B.apos,
                           B.lpos, B.hlen, B.act[0], B.reps[0], B.cnt, (uint64_t)1));
    }
    int cur = 0;
    for (uint32_t k = kmin; k <= kmax && nact > 0; ++k) {
        const uint64_t L = 1ull << k;
        if (nreps > 0) {
            SSS_TRY(sss_launch(ctx, "pd_hash", k_pd_hash, dim3((nreps + 255) / 256), dim3(256), 0, in,
                               (const uint32_t*)B.reps[cur], nreps, (const uint32_t*)B.lpos, B.hst, B.hlen, B.K, B.V, L,
                               Bh));
            uint32_t bits = 0;
            while (bits < (uint32_t)HB_MAX && ((uint64_t)nreps >> bits) > 1024) ++bits;
            uint32_t nb = 1u << bits;
            SSS_CUDA(cudaMemsetAsync(B.hist, 0, sizeof(uint32_t) * (nb + 1), ctx->stream));
            uint32_t hgrid = std::min<uint32_t>((nreps + 4095) / 4096, 2u * (uint32_t)ctx->sm_count);
            SSS_TRY(sss_launch(ctx, "pd_hist", k_pd_hist, dim3(hgrid), dim3(512), 0, (const uint64_t*)B.K, nreps, bits,
                               B.hist));
            SSS_TRY(sss_launch(ctx, "pd_scan", k_pd_scan, dim3(1), dim3(1024), 0, B.hist, nb, B.bstart, B.cursor));
            SSS_TRY(sss_launch(ctx, "pd_scatter", k_pd_scatter, dim3((nreps + 255) / 256), dim3(256), 0,
                               (const uint64_t*)B.K, (const uint32_t*)B.V, nreps, bits, (const uint32_t*)B.bstart,
                               B.cursor, B.tK, B.tV));
            SSS_TRY(sss_launch(ctx, "pd_buckets", k_pd_buckets, dim3(nb), dim3(DD_T), (size_t)DD_CAP * (8 + 8 + 1),
                               (const uint32_t*)B.bstart, B.tK, B.tV, B.dupf));
        }
        SSS_CUDA(cudaMemsetAsync(B.cnt, 0, sizeof(uint32_t) * 2, ctx->stream));
        SSS_TRY(sss_launch(ctx, "pd_retire", k_pd_retire, dim3((nact + 255) / 256), dim3(256), 0, in,
                           (const uint32_t*)B.act[cur], nact, (const uint32_t*)B.lpos, (const uint8_t*)B.dupf, B.apos,
                           B.act[cur ^ 1], B.reps[cur ^ 1], B.cnt, L, (int)(k == kmax)));
        SSS_CUDA(cudaMemcpyAsync(h_cnt, B.cnt, sizeof(uint32_t) * 2, cudaMemcpyDeviceToHost, ctx->stream));
        SSS_CUDA(cudaStreamSynchronize(ctx->stream));
        nreps = h_cnt[0];
        nact = h_cnt[1];
        cur ^= 1;
    }
    return sss_launch(ctx, "pd_final", k_pd_final, dim3((n + 255) / 256), dim3(256), 0, in, (const uint32_t*)B.apos,
                      (const uint32_t*)B.lpos, approx);
}
