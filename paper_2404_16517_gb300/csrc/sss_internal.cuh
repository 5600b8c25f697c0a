// Internal host/device declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "sss.h"

// ---------------------------------------------------------------------------
// Device error word bits (sticky until sss_sync).
enum : unsigned {
    ERRBIT_CHECK = 1u,     // SSS_CHECKED validation failed
    ERRBIT_TIMEOUT = 2u,   // a bounded wait ran out
    ERRBIT_OVERFLOW = 4u,  // an internal capacity was exceeded (library bug)
};

// A segment of consecutive positions whose strings share their first `depth`
// characters (and are still to be ordered by the characters from `depth` on).
struct Seg {
    uint32_t start;
    uint32_t size;
    uint32_t depth;
    uint32_t aux;
};

// ---------------------------------------------------------------------------
// Bump allocator over one device buffer.  With base == nullptr it only counts,
// so the same carving code gives the workspace size.
struct Arena {
    char* base = nullptr;
    size_t cap = 0;
    size_t off = 0;
    template <typename T>
    T* take(size_t count) {
        off = (off + 255) & ~size_t(255);
        T* p = base ? reinterpret_cast<T*>(base + off) : nullptr;
        off += count * sizeof(T);
        return p;
    }
};

struct KStat {
    const char* name;
    uint64_t launches;
    double ms;
    uint64_t timed;
};

struct PendingTiming {
    int stat;
    cudaEvent_t a, b;
};

struct sss_ctx {
    int device = 0;
    int sm_count = 0;
    cudaStream_t stream = nullptr;
    // library-owned work memory
    void* ws_own = nullptr;
    size_t ws_own_bytes = 0;
    // caller-supplied work memory
    void* ws_user = nullptr;
    size_t ws_user_bytes = 0;
    // pinned host staging for small counters and segment lists; pin_event is
    // recorded after every upload from it, and waited on before it is reused
    void* h_pin = nullptr;
    size_t h_pin_bytes = 0;
    cudaEvent_t pin_event = nullptr;
    // sticky device error word
    unsigned* d_err = nullptr;
    // small device scratch for counters and reductions (never inside the workspace)
    unsigned long long* d_small = nullptr;
    uint32_t* h_small = nullptr;  // pinned: per-round readbacks (16 words)
    std::string last_error;
    // instrumentation
    KStat stats[SSS_MAX_KERNELS];
    int nstats = 0;
    bool timing = false;
    std::string timing_filter;
    std::vector<PendingTiming> pending;
    std::vector<cudaEvent_t> event_pool;
    // graphs of the local sort's round loop (SSS_FLAG_GRAPH and the merge's sample
    // sorts), each reused while its key (every pointer and size baked into it) is
    // unchanged; the least recently used of LS_GRAPHS is replaced
    bool capturing = false;
    cudaStream_t cap_stream = nullptr;
    cudaStream_t cap_stream2 = nullptr;  // captures a graph's loop body while cap_stream captures the graph
    struct LsGraph {
        std::string key;
        cudaGraph_t graph = nullptr;
        cudaGraphExec_t exec = nullptr;
        uint64_t used = 0;
    };
    static constexpr int LS_GRAPHS = 4;
    LsGraph ls_graphs[LS_GRAPHS];
    uint64_t ls_clock = 0;
    // kernel-statistics name of the next round-loop graph launches (timed like a
    // kernel when timing is on); set by a caller for its own sorts
    const char* graph_tag = "ls_graph";
    // sss_sort_host: the stream that uploads characters while stage A runs, and
    // one event per uploaded chunk
    cudaStream_t copy_stream = nullptr;
    std::vector<cudaEvent_t> chunk_events;
};

// Set ctx->last_error and return the status.
sss_status sss_fail(sss_ctx* c, sss_status s, const std::string& msg);

// Check a CUDA runtime result; on failure record it and return SSS_ERR_CUDA.
#define SSS_CUDA(call)                                                                         \
    do {                                                                                       \
        cudaError_t e_ = (call);                                                               \
        if (e_ != cudaSuccess)                                                                 \
            return sss_fail(ctx, SSS_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

#define SSS_TRY(expr)                 \
    do {                              \
        sss_status s_ = (expr);       \
        if (s_ != SSS_OK) return s_;  \
    } while (0)

// Work memory of at least `bytes`; grows library-owned memory when needed.
sss_status sss_workspace(sss_ctx* ctx, size_t bytes, char** out);
// Pinned host staging of at least `bytes` (waits until earlier uploads from it
// have completed).
sss_status sss_pinned(sss_ctx* ctx, size_t bytes, void** out);
// Asynchronous upload from the pinned staging buffer (tracked by pin_event).
sss_status sss_upload(sss_ctx* ctx, void* dst, const void* src, size_t bytes);

// Instrumentation hooks used by the launch wrapper.
int sss_stat_index(sss_ctx* ctx, const char* name);
bool sss_timing_on(sss_ctx* ctx, int stat);
cudaEvent_t sss_event(sss_ctx* ctx);

// Launch an instantiated graph on the context stream, counted (and timed with
// CUDA events when enabled) under `name` like a kernel.
sss_status sss_graph_launch(sss_ctx* ctx, const char* name, cudaGraphExec_t exec);

// Launch a kernel on the context stream, counting it (and timing it with CUDA
// events when enabled).  Grids with zero blocks launch nothing.
template <typename... KArgs, typename... Args>
sss_status sss_launch(sss_ctx* ctx, const char* name, void (*kernel)(KArgs...), dim3 grid, dim3 block,
                      size_t smem, Args... args) {
    if (grid.x == 0 || grid.y == 0 || grid.z == 0) return SSS_OK;
    int st = sss_stat_index(ctx, name);
    bool timed = !ctx->capturing && sss_timing_on(ctx, st);  // no event nodes inside a captured loop
    cudaEvent_t a = nullptr, b = nullptr;
    if (timed) {
        a = sss_event(ctx);
        b = sss_event(ctx);
        cudaEventRecord(a, ctx->stream);
    }
    kernel<<<grid, block, smem, ctx->stream>>>(static_cast<KArgs>(args)...);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return sss_fail(ctx, SSS_ERR_CUDA, std::string("launch ") + name + ": " + cudaGetErrorString(e));
    if (timed) {
        cudaEventRecord(b, ctx->stream);
        ctx->pending.push_back({st, a, b});
    }
    if (st >= 0) ctx->stats[st].launches++;
    return SSS_OK;
}

__host__ __device__ inline uint32_t part_lo(uint32_t n, uint32_t p, uint32_t i) {
    return (uint32_t)(((uint64_t)i * n) / p);
}

// Stage implementations (one per translation unit).  They enqueue on ctx->stream
// and carve their work memory from `ar` (which may be a counting arena).
struct StrIn {
    const uint8_t* chars;
    uint64_t n_chars;
    const uint64_t* offs;
    const uint32_t* lens;
    uint32_t n;
};

sss_status impl_local_sort(sss_ctx* ctx, Arena& ar, const StrIn& in, uint32_t p, const sss_params& prm,
                           uint32_t* perm, uint32_t* lcp);
size_t need_local_sort(uint32_t n, uint32_t p, const sss_params& prm);
// Sort every given segment of positions (each starting at depth 0) independently.
sss_status impl_sort_segments(sss_ctx* ctx, Arena& ar, const StrIn& in, const std::vector<Seg>& init,
                              const sss_params& prm, uint32_t* perm, uint32_t* lcp);
// The same for segments inside positions [q0, q1): only that range of perm and
// lcp is initialised and written (other positions keep their contents).
sss_status impl_sort_segments_range(sss_ctx* ctx, Arena& ar, const StrIn& in, const std::vector<Seg>& init,
                                    const sss_params& prm, uint32_t* perm, uint32_t* lcp, uint32_t q0, uint32_t q1);
// Character extent [lo, hi) of every partition's strings: out[2i] = smallest
// offset, out[2i+1] = largest offset + length (~0, 0 for an empty partition).
sss_status impl_part_extents(sss_ctx* ctx, const StrIn& in, uint32_t p, unsigned long long* out);
sss_status impl_suffix_views(sss_ctx* ctx, uint32_t n, uint32_t max_len, uint64_t* offs, uint32_t* lens);
sss_status impl_batch_finish(sss_ctx* ctx, const Seg* d_inst, uint32_t m, const uint32_t* lens, uint32_t* perm,
                             const uint32_t* lcp, uint32_t* dist);
// The batched sort of the m instances d_inst (device table) as one graph launch.
sss_status impl_sort_batch_graph(sss_ctx* ctx, Arena& ar, const StrIn& in, const Seg* d_inst, uint32_t m,
                                 const sss_params& prm, uint32_t* perm, uint32_t* lcp, uint32_t* dist);

// Finish segments of positions whose strings share their first `depth`
// characters (stage A's CTA finisher): perm[start..start+size) is sorted by the
// strings (lengths from in.lens, ties by index) and lcp is set inside each segment.
sss_status impl_finish_segments(sss_ctx* ctx, const Seg* tiny, uint32_t ntiny, const Seg* med, uint32_t nmed,
                                const StrIn& in, uint32_t* perm, uint32_t* lcp);
uint32_t finish_cap_tiny();
uint32_t finish_cap_med();

size_t need_dist_prefix(uint32_t n);
sss_status impl_dist_prefix(sss_ctx* ctx, Arena& ar, const StrIn& in, const uint32_t* run_perm,
                            const uint32_t* run_lcp, uint32_t p, const sss_params& prm, uint32_t* approx);

size_t need_partition(uint32_t n, uint32_t p, uint32_t v);
sss_status impl_partition(sss_ctx* ctx, Arena& ar, const StrIn& in, const uint32_t* trunc, const uint32_t* run_perm,
                          uint32_t p, uint32_t v, uint32_t flags, uint32_t* out_spl, uint32_t* out_bounds);
size_t need_merge(uint32_t n, uint32_t p, uint32_t v, uint64_t nrecchars);
sss_status impl_merge(sss_ctx* ctx, char* ws, size_t ws_bytes, const StrIn& in, const uint32_t* trunc,
                      const uint32_t* run_perm, const uint32_t* run_lcp, uint32_t p, uint32_t v, uint32_t ms,
                      uint32_t flags, uint64_t nrecchars, uint32_t* out_perm, uint32_t* out_lcp);
sss_status impl_sum_tlen(sss_ctx* ctx, const StrIn& in, const uint32_t* trunc, uint64_t* out);
// exclusive sum of count u32 values into u64 (btot: count / 4096 + 4 words of scratch)
sss_status impl_scan_u32_u64(sss_ctx* ctx, const uint32_t* in, uint32_t count, uint64_t* out, uint64_t* btot);
// suffix array and LCP array of a text by prefix doubling over the string sort
size_t need_suffix_sort(uint32_t n, const sss_params& prm);
sss_status impl_suffix_sort(sss_ctx* ctx, char* ws, size_t ws_bytes, const uint8_t* text, uint32_t n,
                            uint32_t max_len, const sss_params& prm, uint32_t* out_sa, uint32_t* out_lcp);

sss_status impl_dist(sss_ctx* ctx, const uint32_t* lens, uint32_t n, const uint32_t* perm, const uint32_t* lcp,
                     uint32_t* dist);

sss_status impl_check_input(sss_ctx* ctx, const StrIn& in);
