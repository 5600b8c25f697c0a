// Suffix sorting as string sorting (the extension named in Section 6,
// "Conclusion and Future Work"): the suffixes of one text are sorted as
// strings, views into the text, without copying characters.
//
// GB300 design: prefix doubling over ranks, on top of the string sort.
//  * First the suffixes truncated to H0 = 64 characters are sorted as strings
//    by the local sort (stage A); equal truncated suffixes share a rank (the
//    number of distinct smaller truncations).  On a text with short repeats
//    every rank is already distinct here, and the result is final.
//  * Otherwise the ranks of length h are doubled: the suffix at i of length
//    next = min(2h, target) is ordered by the pair (rank_h(i), rank_h(i + o)),
//    o = next - h <= h.  The second rank covers characters [o, o + h) of the
//    suffix, so the overlap [o, h) adds nothing and the pair orders the
//    suffixes on their first `next` characters, ending at the text's end
//    (a missing second rank, past the end, is the smallest).  The pairs are
//    sorted as 10-character strings by the same local sort: every rank + 1 is
//    written as five 7-bit digits with the top bit set (no zero byte, order
//    kept).  Equal pairs keep the suffix order (ties by position).
//  * The rounds stop when every rank is distinct or the target length
//    (max_len, else the whole text) is reached, so a text of one repeated
//    character takes log2(n / 64) rounds instead of n^2 / 2 character reads.
//  * The LCP of two adjacent suffixes adds the lengths of the rank levels on
//    which they agree, from the longest level down, then compares the fewer
//    than 64 characters that are left.
#include <algorithm>
#include <vector>

#include "sss_device.cuh"
#include "sss_internal.cuh"

namespace {

constexpr uint32_t SX_H0 = 64;    // characters of the first, direct sort
constexpr uint32_t SX_PAIR = 10;  // characters of a rank-pair string
constexpr int SX_MAXLEV = 34;     // rank levels at most (64 .. 2^32, plus a truncated last)

// rank levels a text of n characters can need: 64, 128, ... up to the first
// length >= n, the last possibly shorter
inline uint32_t sx_levels(uint32_t n) {
    uint32_t c = 1;
    for (uint64_t h = SX_H0; h < n; h <<= 1) ++c;
    return std::min<uint32_t>(c, SX_MAXLEV);
}

struct SxLevels {
    const uint32_t* rank[SX_MAXLEV];
    uint32_t len[SX_MAXLEV];
    uint32_t count;
};

__global__ void k_sx_views(uint32_t n, uint32_t h, uint64_t* __restrict__ offs, uint32_t* __restrict__ lens) {
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const uint32_t r = n - i;
        offs[i] = i;
        lens[i] = r < h ? r : h;
    }
}

__device__ __forceinline__ void sx_put_rank(uint8_t* p, uint32_t v) {
    p[0] = (uint8_t)(0x80u | ((v >> 28) & 0x7Fu));
    p[1] = (uint8_t)(0x80u | ((v >> 21) & 0x7Fu));
    p[2] = (uint8_t)(0x80u | ((v >> 14) & 0x7Fu));
    p[3] = (uint8_t)(0x80u | ((v >> 7) & 0x7Fu));
    p[4] = (uint8_t)(0x80u | (v & 0x7Fu));
}

// pair string of suffix i: rank_h(i) + 1, then rank_h(i + o) + 1 (0 past the end);
// the views of the pair strings
__global__ void k_sx_pairs(const uint32_t* __restrict__ rank, uint32_t n, uint32_t o, uint8_t* __restrict__ P,
                           uint64_t* __restrict__ offs, uint32_t* __restrict__ lens) {
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const uint32_t a = rank[i] + 1u;
        const uint32_t b = (uint64_t)i + o < n ? rank[i + o] + 1u : 0u;
        sx_put_rank(P + (size_t)SX_PAIR * i, a);
        sx_put_rank(P + (size_t)SX_PAIR * i + 5, b);
        offs[i] = (uint64_t)SX_PAIR * i;
        lens[i] = SX_PAIR;
    }
}

// group starts of a sorted order: position k starts a group unless its string
// equals its predecessor's (lcp equal to both lengths)
__global__ void k_sx_flags(const uint32_t* __restrict__ perm, const uint32_t* __restrict__ lcp,
                           const uint32_t* __restrict__ lens, uint32_t n, uint32_t* __restrict__ flag) {
    for (uint32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        uint32_t f = 1;
        if (k > 0) {
            const uint32_t l = lcp[k];
            f = (l == lens[perm[k - 1]] && l == lens[perm[k]]) ? 0u : 1u;
        }
        flag[k] = f;
    }
}

// rank of the suffix at sorted position k: the number of group starts before
// its group (exclusive sum over the starts, plus its own start, minus one)
__global__ void k_sx_ranks(const uint32_t* __restrict__ perm, const uint64_t* __restrict__ excl,
                           const uint32_t* __restrict__ flag, uint32_t n, uint32_t* __restrict__ rank) {
    for (uint32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x)
        rank[perm[k]] = (uint32_t)(excl[k] + flag[k] - 1u);
}

// LCP of the suffixes at sorted positions k-1 and k, truncated to max_len
__global__ void k_sx_lcp(const uint8_t* __restrict__ text, uint32_t n, uint32_t max_len,
                         const uint32_t* __restrict__ sa, SxLevels lv, uint32_t* __restrict__ lcp) {
    for (uint32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        if (k == 0) {
            lcp[0] = 0;
            continue;
        }
        const uint32_t i = sa[k - 1], j = sa[k];
        const uint32_t li = min(n - i, max_len), lj = min(n - j, max_len);
        const uint32_t m = li < lj ? li : lj;
        uint32_t l = 0;
        for (int t = (int)lv.count - 1; t >= 0 && l < m; --t) {
            // equal ranks at length L: equal windows of L characters (both inside the
            // text, as the suffixes differ)
            if ((uint64_t)i + l < n && (uint64_t)j + l < n && lv.rank[t][i + l] == lv.rank[t][j + l]) l += lv.len[t];
        }
        if (l < m) {
            // fewer than the shortest level's characters are left: compare them
            for (;;) {
                const uint64_t x = load_word_be(text + i, li, l), y = load_word_be(text + j, lj, l);
                if (x != y) {
                    l += word_lcp(x, y);
                    break;
                }
                l += 8;
                if (l >= m) break;
            }
        }
        lcp[k] = l < m ? l : m;
    }
}

}  // namespace

size_t need_suffix_sort(uint32_t n, const sss_params& prm) {
    Arena a;
    a.take<uint64_t>(n);                          // views
    a.take<uint32_t>(n);
    a.take<uint8_t>((size_t)SX_PAIR * n);         // pair strings
    a.take<uint32_t>(n);                          // group flags
    a.take<uint64_t>(n);                          // their exclusive sum
    a.take<uint64_t>(n / 4096 + 4);
    for (uint32_t t = 0; t < sx_levels(n); ++t) a.take<uint32_t>(n);  // rank levels
    a.take<char>(need_local_sort(n, 1, prm));
    return a.off + 256;
}

// Work memory: need_suffix_sort(n), with room for the rank levels of whole
// suffixes (the most rounds any max_len can take).
sss_status impl_suffix_sort(sss_ctx* ctx, char* ws, size_t ws_bytes, const uint8_t* text, uint32_t n,
                            uint32_t max_len, const sss_params& prm, uint32_t* out_sa, uint32_t* out_lcp) {
    Arena ar{ws, ws_bytes, 0};
    uint64_t* offs = ar.take<uint64_t>(n);
    uint32_t* lens = ar.take<uint32_t>(n);
    uint8_t* P = ar.take<uint8_t>((size_t)SX_PAIR * n);
    uint32_t* flag = ar.take<uint32_t>(n);
    uint64_t* excl = ar.take<uint64_t>(n);
    uint64_t* btot = ar.take<uint64_t>(n / 4096 + 4);
    const uint32_t nlev = sx_levels(n);
    uint32_t* lvbase[SX_MAXLEV];
    for (uint32_t t = 0; t < nlev; ++t) lvbase[t] = ar.take<uint32_t>(n);
    size_t sort_off = (ar.off + 255) & ~size_t(255);
    const size_t sort_bytes = need_local_sort(n, 1, prm);
    const uint32_t sm = (uint32_t)std::max(1, ctx->sm_count);
    const uint32_t grid = std::min((n + 255) / 256, sm * 16);
    const uint32_t target = max_len ? std::min(max_len, n) : n;

    // ranks of the sorted order in perm/lcp (strings of lengths lens) into level t
    auto rank_level = [&](const uint32_t* slens, uint32_t* rank, uint64_t* groups) -> sss_status {
        SSS_TRY(sss_launch(ctx, "sx_flags", k_sx_flags, dim3(grid), dim3(256), 0, (const uint32_t*)out_sa,
                           (const uint32_t*)out_lcp, slens, n, flag));
        SSS_TRY(impl_scan_u32_u64(ctx, flag, n, excl, btot));
        SSS_TRY(sss_launch(ctx, "sx_ranks", k_sx_ranks, dim3(grid), dim3(256), 0, (const uint32_t*)out_sa,
                           (const uint64_t*)excl, (const uint32_t*)flag, n, rank));
        // groups = the last rank + 1 (the pinned staging is looked up again here:
        // the sorts may have grown it)
        void* pin;
        SSS_TRY(sss_pinned(ctx, 64, &pin));
        uint64_t* h_groups = static_cast<uint64_t*>(pin);
        SSS_CUDA(cudaMemcpyAsync(h_groups, excl + (n - 1), sizeof(uint64_t), cudaMemcpyDeviceToHost, ctx->stream));
        uint32_t* h_flag = reinterpret_cast<uint32_t*>(h_groups + 1);
        SSS_CUDA(cudaMemcpyAsync(h_flag, flag + (n - 1), sizeof(uint32_t), cudaMemcpyDeviceToHost, ctx->stream));
        SSS_CUDA(cudaStreamSynchronize(ctx->stream));
        *groups = h_groups[0] + *h_flag;
        return SSS_OK;
    };

    // the suffixes truncated to H0 characters, sorted as strings
    uint32_t h = std::min(SX_H0, target);
    SSS_TRY(sss_launch(ctx, "sx_views", k_sx_views, dim3(grid), dim3(256), 0, n, h, offs, lens));
    {
        Arena sa{ws + sort_off, sort_bytes, 0};
        StrIn in{text, n, offs, lens, n};
        SSS_TRY(impl_local_sort(ctx, sa, in, 1, prm, out_sa, out_lcp));
    }
    if (h >= target) return SSS_OK;  // the views were the truncated suffixes themselves
    SxLevels lv{};
    uint64_t groups = 0;
    SSS_TRY(rank_level(lens, lvbase[0], &groups));
    lv.rank[0] = lvbase[0];
    lv.len[0] = h;
    lv.count = 1;
    // all distinct within H0 characters: the order and the LCPs (all shorter than
    // H0, or a suffix's whole length at the text's end) are final
    if (groups == n) return SSS_OK;
    while (true) {
        const uint32_t next = (uint32_t)std::min<uint64_t>(2ull * h, target);
        const uint32_t o = next - h;
        if (lv.count >= nlev) return sss_fail(ctx, SSS_ERR_CUDA, "suffix sort: too many rounds");
        SSS_TRY(sss_launch(ctx, "sx_pairs", k_sx_pairs, dim3(grid), dim3(256), 0, lv.rank[lv.count - 1], n, o, P,
                           offs, lens));
        {
            Arena sa{ws + sort_off, sort_bytes, 0};
            StrIn in{P, (uint64_t)SX_PAIR * n, offs, lens, n};
            SSS_TRY(impl_local_sort(ctx, sa, in, 1, prm, out_sa, out_lcp));
        }
        h = next;
        SSS_TRY(rank_level(lens, lvbase[lv.count], &groups));
        lv.rank[lv.count] = lvbase[lv.count];
        lv.len[lv.count] = h;
        ++lv.count;
        if (groups == n || h >= target) break;
    }
    // out_sa holds the order (equal truncated suffixes by position); the LCPs
    return sss_launch(ctx, "sx_lcp", k_sx_lcp, dim3(grid), dim3(256), 0, text, n, target, (const uint32_t*)out_sa,
                      lv, out_lcp);
}
