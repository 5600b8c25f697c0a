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
__global__ void k_instance_chars(uint8_t* __restrict__ chars, const uint64_t* __restrict__ offs,
                                 const uint32_t* __restrict__ lens, const uint32_t* __restrict__ cp,
                                 const uint32_t* __restrict__ inst, uint64_t n, uint64_t kt, uint64_t kc, Alpha al) {
    for (uint64_t g = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; g < n; g += (uint64_t)gridDim.x * blockDim.x) {
        uint64_t o = offs[g];
        uint32_t l = lens[g], c = cp[g];
        uint64_t tb = (uint64_t)inst[g] << 20;
        for (uint32_t j = 0; j < l; ++j) {
            uint64_t r = j < c ? draw(kt, tb + j) : draw(kc, o + j);
            chars[o + j] = al.c[uidx(r, al.n)];
        }
    }
}

}  // namespace

extern "C" int sssgen_instance_chars(uint8_t* chars, const uint64_t* offs, const uint32_t* lens, const uint32_t* cp,
                                     const uint32_t* inst, uint64_t n, uint64_t seed, const uint8_t* alphabet,
                                     uint32_t alen, void* stream) {
    if (alen == 0 || alen > 64) return 1;
    Alpha al{};
    for (uint32_t k = 0; k < alen; ++k) al.c[k] = alphabet[k];
    al.n = alen;
    if (n == 0) return 0;
    uint32_t grid = (uint32_t)((n + 255) / 256 < 65536 ? (n + 255) / 256 : 65536);
    k_instance_chars<<<grid, 256, 0, (cudaStream_t)stream>>>(chars, offs, lens, cp, inst, n,
                                                             stream_key(seed, ST_TEMPLATE), stream_key(seed, ST_CHARS),
                                                             al);
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
