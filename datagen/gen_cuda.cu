// Device implementation of the seeded string-set generator of datagen/__init__.py
// (same counter-based SplitMix64 draws, same template construction), so large
// workloads can be produced directly in device memory.  Input synthesis only:
// nothing here compares, hashes or sorts strings.
#include <cuda_runtime.h>
#include <stdint.h>

namespace {

constexpr uint64_t G = 0x9E3779B97F4A7C15ull;
constexpr uint64_t ST_TEMPLATE = 1, ST_PICK = 2, ST_CHARS = 3;

__host__ __device__ __forceinline__ uint64_t smix(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__host__ __device__ __forceinline__ uint64_t stream_key(uint64_t seed, uint64_t stream) {
    return smix(seed + (stream + 1) * G);
}

__device__ __forceinline__ uint64_t draw(uint64_t key, uint64_t i) { return smix(key + (i + 1) * G); }

__device__ __forceinline__ uint32_t uidx(uint64_t r, uint32_t a) {
    return (uint32_t)(((r >> 32) * (uint64_t)a) >> 32);
}

struct Alpha {
    uint8_t c[64];
    uint32_t n;
};

__global__ void k_template_set(uint8_t* __restrict__ chars, uint64_t* __restrict__ offs, uint32_t* __restrict__ lens,
                               uint64_t kt, uint64_t kp, uint64_t kc, uint32_t length, uint32_t ntmpl,
                               uint32_t shared, Alpha al, uint64_t first, uint64_t count) {
    uint64_t g = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    uint64_t total = count * length;
    for (; g < total; g += (uint64_t)gridDim.x * blockDim.x) {
        uint64_t li = g / length;
        uint32_t j = (uint32_t)(g - li * length);
        uint64_t i = first + li;
        uint8_t c;
        if (j < shared) {
            uint32_t t = uidx(draw(kp, i), ntmpl);
            c = al.c[uidx(draw(kt, (uint64_t)t * length + j), al.n)];
        } else {
            c = al.c[uidx(draw(kc, i * length + j), al.n)];
        }
        chars[g] = c;
        if (j == 0) {
            offs[li] = li * length;
            lens[li] = length;
        }
    }
}

// characters of instance-set strings: string g copies its first cp[g] characters
// from its instance's template, the rest are uniform (counter = offs[g] + j)
// (counters are relative to cbase, so a set placed at any offset of a larger
// buffer gets the same characters; inst == NULL means instance 0 throughout)
// (one warp per string, lanes on consecutive characters, so stores coalesce)
__global__ void k_instance_chars(uint8_t* __restrict__ chars, const uint64_t* __restrict__ offs,
                                 const uint32_t* __restrict__ lens, const uint32_t* __restrict__ cp,
                                 const uint32_t* __restrict__ inst, uint64_t n, uint64_t kt, uint64_t kc, Alpha al,
                                 uint64_t cbase) {
    const uint32_t lane = threadIdx.x & 31;
    const uint64_t warps = (uint64_t)gridDim.x * (blockDim.x >> 5);
    for (uint64_t g = (uint64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); g < n; g += warps) {
        uint64_t o = offs[g];
        uint32_t l = lens[g], c = cp[g];
        uint64_t tb = inst ? (uint64_t)inst[g] << 20 : 0;
        for (uint32_t j = lane; j < l; j += 32) {
            uint64_t r = j < c ? draw(kt, tb + j) : draw(kc, o - cbase + j);
            chars[o + j] = al.c[uidx(r, al.n)];
        }
    }
}

// lengths and template-copy lengths of one request's strings (instance layout
// of datagen.instance_layout for a single instance of ratio r)
__global__ void k_request_layout(uint32_t* __restrict__ lens, uint32_t* __restrict__ cp, uint64_t n, uint64_t kl,
                                 uint32_t len_lo, uint32_t span, double ratio, uint32_t logs) {
    for (uint64_t g = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; g < n; g += (uint64_t)gridDim.x * blockDim.x) {
        uint32_t l = len_lo + uidx(draw(kl, g), span);
        long long c = (long long)rint(ratio * (double)l) - (long long)logs - 1;
        c = c < 0 ? 0 : c;
        c = c > l ? l : c;
        lens[g] = l;
        cp[g] = (uint32_t)c;
    }
}

// offsets = base + exclusive prefix sums of the lengths, in three passes over
// chunks of CHUNK lengths (chunk sums, scan of the chunk sums, write)
constexpr uint32_t SCAN_T = 256, SCAN_PER = 16, CHUNK = SCAN_T * SCAN_PER;

__device__ __forceinline__ uint64_t block_excl_scan(uint64_t v, uint64_t* warp_tot, uint64_t* total) {
    uint32_t lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    uint64_t x = v;
    for (int d = 1; d < 32; d <<= 1) {
        uint64_t y = __shfl_up_sync(0xffffffffu, x, d);
        if (lane >= (uint32_t)d) x += y;
    }
    if (lane == 31) warp_tot[w] = x;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint64_t run = 0;
        for (uint32_t k = 0; k < blockDim.x / 32; ++k) {
            uint64_t t = warp_tot[k];
            warp_tot[k] = run;
            run += t;
        }
        *total = run;
    }
    __syncthreads();
    return warp_tot[w] + x - v;
}

__global__ void k_chunk_sums(const uint32_t* __restrict__ lens, uint64_t n, uint64_t* __restrict__ sums) {
    __shared__ uint64_t wt[SCAN_T / 32], tot;
    uint64_t i0 = (uint64_t)blockIdx.x * CHUNK + (uint64_t)threadIdx.x * SCAN_PER;
    uint64_t s = 0;
    for (uint32_t k = 0; k < SCAN_PER; ++k)
        if (i0 + k < n) s += lens[i0 + k];
    block_excl_scan(s, wt, &tot);
    if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}

__global__ void k_scan_sums(uint64_t* __restrict__ sums, uint64_t nb) {
    __shared__ uint64_t wt[SCAN_T / 32], tot;
    uint64_t carry = 0;
    for (uint64_t b0 = 0; b0 < nb; b0 += SCAN_T) {
        uint64_t i = b0 + threadIdx.x;
        uint64_t v = i < nb ? sums[i] : 0;
        uint64_t e = block_excl_scan(v, wt, &tot);
        if (i < nb) sums[i] = carry + e;
        carry += tot;
        __syncthreads();
    }
}

__global__ void k_write_offs(const uint32_t* __restrict__ lens, uint64_t n, const uint64_t* __restrict__ sums,
                             uint64_t* __restrict__ offs, uint64_t base) {
    __shared__ uint64_t wt[SCAN_T / 32], tot;
    uint64_t i0 = (uint64_t)blockIdx.x * CHUNK + (uint64_t)threadIdx.x * SCAN_PER;
    uint64_t s = 0;
    for (uint32_t k = 0; k < SCAN_PER; ++k)
        if (i0 + k < n) s += lens[i0 + k];
    uint64_t run = base + sums[blockIdx.x] + block_excl_scan(s, wt, &tot);
    for (uint32_t k = 0; k < SCAN_PER; ++k)
        if (i0 + k < n) {
            offs[i0 + k] = run;
            run += lens[i0 + k];
        }
}

// total characters of each of m requests (one block per request)
__global__ void k_request_totals(const uint64_t* __restrict__ seeds, const uint64_t* __restrict__ ns, uint64_t m,
                                 uint32_t len_lo, uint32_t span, uint64_t* __restrict__ out) {
    __shared__ uint64_t wt[SCAN_T / 32], tot;
    for (uint64_t r = blockIdx.x; r < m; r += gridDim.x) {
        uint64_t kl = stream_key(seeds[r], 4), n = ns[r], s = 0;
        for (uint64_t g = threadIdx.x; g < n; g += blockDim.x) s += len_lo + uidx(draw(kl, g), span);
        block_excl_scan(s, wt, &tot);
        if (threadIdx.x == 0) out[r] = tot;
        __syncthreads();
    }
}

// ---- a batch of requests in one table (one launch sequence per batch) -------
struct ReqDesc {
    uint64_t kl, kt, kc;   // stream keys of the request: lengths, template, characters
    uint64_t char_base;    // where the request's characters start
    double ratio;          // template copy ratio
    uint32_t first, n;     // the request's strings in the table
    uint32_t logs, pad;    // ceil(log_a n)
};

__device__ __forceinline__ uint32_t req_of(const ReqDesc* __restrict__ R, uint32_t m, uint64_t g) {
    uint32_t lo = 0, hi = m;  // last request with first <= g
    while (hi - lo > 1) {
        uint32_t mid = (lo + hi) >> 1;
        if (R[mid].first <= g) lo = mid; else hi = mid;
    }
    return lo;
}

__global__ void k_batch_layout(const ReqDesc* __restrict__ R, uint32_t m, uint64_t n, uint32_t* __restrict__ lens,
                               uint32_t* __restrict__ cp, uint32_t len_lo, uint32_t span) {
    for (uint64_t g = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; g < n; g += (uint64_t)gridDim.x * blockDim.x) {
        const ReqDesc& q = R[req_of(R, m, g)];
        uint32_t l = len_lo + uidx(draw(q.kl, g - q.first), span);
        long long c = (long long)rint(q.ratio * (double)l) - (long long)q.logs - 1;
        c = c < 0 ? 0 : c;
        c = c > l ? l : c;
        lens[g] = l;
        cp[g] = (uint32_t)c;
    }
}

// adj[k] = char_base_k - (prefix sum of the table's lengths at first_k)
__global__ void k_batch_adj(const ReqDesc* __restrict__ R, uint32_t m, const uint64_t* __restrict__ P,
                            uint64_t* __restrict__ adj) {
    uint32_t k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < m) adj[k] = R[k].char_base - P[R[k].first];
}

// one warp per string: offs[g] = P[g] + adj[k], then its characters
__global__ void k_batch_chars(const ReqDesc* __restrict__ R, uint32_t m, uint64_t n, const uint64_t* __restrict__ adj,
                              uint64_t* __restrict__ offs, const uint32_t* __restrict__ lens,
                              const uint32_t* __restrict__ cp, uint8_t* __restrict__ chars, Alpha al) {
    const uint32_t lane = threadIdx.x & 31;
    const uint64_t warps = (uint64_t)gridDim.x * (blockDim.x >> 5);
    for (uint64_t g = (uint64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); g < n; g += warps) {
        uint32_t k = req_of(R, m, g);
        const ReqDesc& q = R[k];
        uint64_t o = offs[g] + adj[k];
        uint64_t rel = o - q.char_base;
        uint32_t l = lens[g], c = cp[g];
        __syncwarp();
        if (lane == 0) offs[g] = o;
        for (uint32_t j = lane; j < l; j += 32) {
            uint64_t r = j < c ? draw(q.kt, j) : draw(q.kc, rel + j);
            chars[o + j] = al.c[uidx(r, al.n)];
        }
    }
}

// length-skewed set: first character from the pick stream, the rest uniform
// (counter = offset + j); one warp per string
// (strings of length `lng` whose first letter is the last one copy characters
// 1 .. lng-9 from the template stream)
__global__ void k_skew_chars(uint8_t* __restrict__ chars, const uint64_t* __restrict__ offs,
                             const uint32_t* __restrict__ lens, uint64_t n, uint64_t kp, uint64_t kc, uint64_t kt,
                             uint32_t lng, Alpha al) {
    const uint32_t lane = threadIdx.x & 31;
    const uint64_t warps = (uint64_t)gridDim.x * (blockDim.x >> 5);
    for (uint64_t g = (uint64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); g < n; g += warps) {
        uint64_t o = offs[g];
        uint32_t l = lens[g];
        uint32_t f = uidx(draw(kp, g), al.n);
        bool tm = (f == al.n - 1) && l == lng;
        for (uint32_t j = lane; j < l; j += 32) {
            uint32_t c;
            if (j == 0) c = f;
            else if (tm && j + 8 < lng) c = uidx(draw(kt, j), al.n);
            else c = uidx(draw(kc, o + j), al.n);
            chars[o + j] = al.c[c];
        }
    }
}

}  // namespace

extern "C" int sssgen_skew_chars(uint8_t* chars, const uint64_t* offs, const uint32_t* lens, uint64_t n,
                                 uint64_t seed, uint32_t lng, const uint8_t* alphabet, uint32_t alen, void* stream) {
    if (alen == 0 || alen > 64) return 1;
    if (n == 0) return 0;
    Alpha al{};
    for (uint32_t k = 0; k < alen; ++k) al.c[k] = alphabet[k];
    al.n = alen;
    uint32_t grid = (uint32_t)((n + 7) / 8 < 65536 ? (n + 7) / 8 : 65536);
    k_skew_chars<<<grid, 256, 0, (cudaStream_t)stream>>>(chars, offs, lens, n, stream_key(seed, ST_PICK),
                                                         stream_key(seed, ST_CHARS), stream_key(seed, ST_TEMPLATE),
                                                         lng, al);
    return cudaGetLastError() == cudaSuccess ? 0 : 2;
}

extern "C" uint32_t sssgen_req_desc_bytes() { return (uint32_t)sizeof(ReqDesc); }

// All requests of a batch in one table: request k (desc[k], a DEVICE array of m
// descriptors sorted by `first`, covering [0, n) without gaps) gets the same
// strings as sssgen_request with its seed, n, ratio and char_base.
// cp_scratch: uint32_t[n]; sum_scratch: uint64_t[sssgen_request_scratch_words(n)
// + m].  No host synchronisation.
extern "C" int sssgen_request_batch(uint8_t* chars, uint64_t* offs, uint32_t* lens, uint32_t* cp_scratch,
                                    uint64_t* sum_scratch, const void* desc, uint32_t m, uint64_t n, uint32_t len_lo,
                                    uint32_t len_hi, const uint8_t* alphabet, uint32_t alen, void* stream) {
    if (alen == 0 || alen > 64 || len_hi < len_lo || m == 0) return 1;
    if (n == 0) return 0;
    Alpha al{};
    for (uint32_t k = 0; k < alen; ++k) al.c[k] = alphabet[k];
    al.n = alen;
    const ReqDesc* R = static_cast<const ReqDesc*>(desc);
    cudaStream_t st = (cudaStream_t)stream;
    uint32_t grid = (uint32_t)((n + 255) / 256 < 65536 ? (n + 255) / 256 : 65536);
    k_batch_layout<<<grid, 256, 0, st>>>(R, m, n, lens, cp_scratch, len_lo, len_hi - len_lo + 1);
    uint64_t nb = (n + CHUNK - 1) / CHUNK;
    if (nb > 0x7fffffffull) return 1;
    uint64_t* adj = sum_scratch + nb;
    k_chunk_sums<<<(uint32_t)nb, SCAN_T, 0, st>>>(lens, n, sum_scratch);
    k_scan_sums<<<1, SCAN_T, 0, st>>>(sum_scratch, nb);
    k_write_offs<<<(uint32_t)nb, SCAN_T, 0, st>>>(lens, n, sum_scratch, offs, 0);
    k_batch_adj<<<(m + 255) / 256, 256, 0, st>>>(R, m, offs, adj);
    uint32_t cgrid = (uint32_t)((n + 7) / 8 < 65536 ? (n + 7) / 8 : 65536);
    k_batch_chars<<<cgrid, 256, 0, st>>>(R, m, n, adj, offs, lens, cp_scratch, chars, al);
    return cudaGetLastError() == cudaSuccess ? 0 : 2;
}

extern "C" int sssgen_request_totals(const uint64_t* seeds, const uint64_t* ns, uint64_t m, uint32_t len_lo,
                                     uint32_t len_hi, uint64_t* out, void* stream) {
    if (m == 0) return 0;
    if (len_hi < len_lo) return 1;
    uint32_t grid = (uint32_t)(m < 65536 ? m : 65536);
    k_request_totals<<<grid, SCAN_T, 0, (cudaStream_t)stream>>>(seeds, ns, m, len_lo, len_hi - len_lo + 1, out);
    return cudaGetLastError() == cudaSuccess ? 0 : 2;
}

extern "C" uint64_t sssgen_request_scratch_words(uint64_t n) { return (n + CHUNK - 1) / CHUNK; }

// One request of the serving workload: n strings with lengths uniform over
// len_lo..len_hi, each copying its first max(0, round(ratio*len) - logs - 1)
// characters from the request's template, written at chars[char_base ...] with
// absolute offsets.  cp_scratch: uint32_t[n]; sum_scratch:
// uint64_t[sssgen_request_scratch_words(n)].  No host synchronisation.
extern "C" int sssgen_request(uint8_t* chars, uint64_t* offs, uint32_t* lens, uint32_t* cp_scratch,
                              uint64_t* sum_scratch, uint64_t n, uint64_t seed, uint32_t len_lo, uint32_t len_hi,
                              double ratio, uint32_t logs, const uint8_t* alphabet, uint32_t alen,
                              uint64_t char_base, void* stream) {
    if (alen == 0 || alen > 64 || len_hi < len_lo) return 1;
    if (n == 0) return 0;
    Alpha al{};
    for (uint32_t k = 0; k < alen; ++k) al.c[k] = alphabet[k];
    al.n = alen;
    cudaStream_t st = (cudaStream_t)stream;
    uint32_t grid = (uint32_t)((n + 255) / 256 < 65536 ? (n + 255) / 256 : 65536);
    k_request_layout<<<grid, 256, 0, st>>>(lens, cp_scratch, n, stream_key(seed, 4), len_lo, len_hi - len_lo + 1,
                                           ratio, logs);
    uint64_t nb = (n + CHUNK - 1) / CHUNK;
    if (nb > 0x7fffffffull) return 1;
    k_chunk_sums<<<(uint32_t)nb, SCAN_T, 0, st>>>(lens, n, sum_scratch);
    k_scan_sums<<<1, SCAN_T, 0, st>>>(sum_scratch, nb);
    k_write_offs<<<(uint32_t)nb, SCAN_T, 0, st>>>(lens, n, sum_scratch, offs, char_base);
    uint32_t cgrid = (uint32_t)((n + 7) / 8 < 65536 ? (n + 7) / 8 : 65536);
    k_instance_chars<<<cgrid, 256, 0, st>>>(chars, offs, lens, cp_scratch, nullptr, n, stream_key(seed, ST_TEMPLATE),
                                            stream_key(seed, ST_CHARS), al, char_base);
    return cudaGetLastError() == cudaSuccess ? 0 : 2;
}

extern "C" int sssgen_instance_chars(uint8_t* chars, const uint64_t* offs, const uint32_t* lens, const uint32_t* cp,
                                     const uint32_t* inst, uint64_t n, uint64_t seed, const uint8_t* alphabet,
                                     uint32_t alen, void* stream) {
    if (alen == 0 || alen > 64) return 1;
    Alpha al{};
    for (uint32_t k = 0; k < alen; ++k) al.c[k] = alphabet[k];
    al.n = alen;
    if (n == 0) return 0;
    uint32_t grid = (uint32_t)((n + 7) / 8 < 65536 ? (n + 7) / 8 : 65536);
    k_instance_chars<<<grid, 256, 0, (cudaStream_t)stream>>>(chars, offs, lens, cp, inst, n,
                                                             stream_key(seed, ST_TEMPLATE), stream_key(seed, ST_CHARS),
                                                             al, 0);
    return cudaGetLastError() == cudaSuccess ? 0 : 2;
}

extern "C" int sssgen_template_set(uint8_t* chars, uint64_t* offs, uint32_t* lens, uint64_t seed, uint64_t n,
                                   uint32_t length, uint32_t ntmpl, uint32_t shared, const uint8_t* alphabet,
                                   uint32_t alen, uint64_t first, uint64_t count, void* stream) {
    (void)n;
    if (alen == 0 || alen > 64) return 1;
    Alpha al{};
    for (uint32_t k = 0; k < alen; ++k) al.c[k] = alphabet[k];
    al.n = alen;
    uint64_t total = count * length;
    if (total == 0) return 0;
    uint32_t grid = (uint32_t)((total + 255) / 256 < 65536 * 8 ? (total + 255) / 256 : 65536 * 8);
    k_template_set<<<grid, 256, 0, (cudaStream_t)stream>>>(chars, offs, lens, stream_key(seed, ST_TEMPLATE),
                                                           stream_key(seed, ST_PICK), stream_key(seed, ST_CHARS),
                                                           length, ntmpl, shared, al, first, count);
    return cudaGetLastError() == cudaSuccess ? 0 : 2;
}
