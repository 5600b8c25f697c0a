// C ABI entry points: context, work memory, instrumentation and the stage calls.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <new>

#include "sss_internal.cuh"

sss_status sss_fail(sss_ctx* c, sss_status s, const std::string& msg) {
    if (c) c->last_error = msg;
    return s;
}

sss_status sss_workspace(sss_ctx* ctx, size_t bytes, char** out) {
    if (ctx->ws_user) {
        if (bytes > ctx->ws_user_bytes)
            return sss_fail(ctx, SSS_ERR_WORKSPACE,
                            "caller workspace too small: need " + std::to_string(bytes) + " bytes");
        *out = static_cast<char*>(ctx->ws_user);
        return SSS_OK;
    }
    if (bytes > ctx->ws_own_bytes) {
        if (ctx->ws_own) {
            cudaStreamSynchronize(ctx->stream);
            cudaFree(ctx->ws_own);
            ctx->ws_own = nullptr;
            ctx->ws_own_bytes = 0;
        }
        size_t want = bytes + bytes / 8;
        if (cudaMalloc(&ctx->ws_own, want) != cudaSuccess) {
            cudaGetLastError();
            ctx->ws_own = nullptr;
            return sss_fail(ctx, SSS_ERR_OOM, "cudaMalloc of " + std::to_string(want) + " bytes failed");
        }
        ctx->ws_own_bytes = want;
    }
    *out = static_cast<char*>(ctx->ws_own);
    return SSS_OK;
}

sss_status sss_upload(sss_ctx* ctx, void* dst, const void* src, size_t bytes) {
    if (bytes == 0) return SSS_OK;
    SSS_CUDA(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, ctx->stream));
    SSS_CUDA(cudaEventRecord(ctx->pin_event, ctx->stream));
    return SSS_OK;
}

sss_status sss_pinned(sss_ctx* ctx, size_t bytes, void** out) {
    SSS_CUDA(cudaEventSynchronize(ctx->pin_event));
    if (bytes > ctx->h_pin_bytes) {
        if (ctx->h_pin) {
            cudaStreamSynchronize(ctx->stream);
            cudaFreeHost(ctx->h_pin);
            ctx->h_pin = nullptr;
            ctx->h_pin_bytes = 0;
        }
        if (cudaMallocHost(&ctx->h_pin, bytes) != cudaSuccess) {
            cudaGetLastError();
            ctx->h_pin = nullptr;
            return sss_fail(ctx, SSS_ERR_OOM, "cudaMallocHost failed");
        }
        ctx->h_pin_bytes = bytes;
    }
    *out = ctx->h_pin;
    return SSS_OK;
}

int sss_stat_index(sss_ctx* ctx, const char* name) {
    for (int i = 0; i < ctx->nstats; ++i)
        if (ctx->stats[i].name == name || std::strcmp(ctx->stats[i].name, name) == 0) return i;
    if (ctx->nstats >= SSS_MAX_KERNELS) return -1;
    ctx->stats[ctx->nstats] = KStat{name, 0, 0.0, 0};
    return ctx->nstats++;
}

sss_status sss_graph_launch(sss_ctx* ctx, const char* name, cudaGraphExec_t exec) {
    int st = sss_stat_index(ctx, name);
    bool timed = sss_timing_on(ctx, st);
    cudaEvent_t a = nullptr, b = nullptr;
    if (timed) {
        a = sss_event(ctx);
        b = sss_event(ctx);
        cudaEventRecord(a, ctx->stream);
    }
    SSS_CUDA(cudaGraphLaunch(exec, ctx->stream));
    if (timed) {
        cudaEventRecord(b, ctx->stream);
        ctx->pending.push_back({st, a, b});
    }
    if (st >= 0) ctx->stats[st].launches++;
    return SSS_OK;
}

bool sss_timing_on(sss_ctx* ctx, int stat) {
    if (!ctx->timing || stat < 0) return false;
    if (ctx->timing_filter.empty()) return true;
    return std::strstr(ctx->stats[stat].name, ctx->timing_filter.c_str()) != nullptr;
}

cudaEvent_t sss_event(sss_ctx* ctx) {
    if (!ctx->event_pool.empty()) {
        cudaEvent_t e = ctx->event_pool.back();
        ctx->event_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

static void collect_timings(sss_ctx* ctx) {
    for (auto& p : ctx->pending) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) {
            ctx->stats[p.stat].ms += ms;
            ctx->stats[p.stat].timed++;
        }
        ctx->event_pool.push_back(p.a);
        ctx->event_pool.push_back(p.b);
    }
    ctx->pending.clear();
    cudaGetLastError();
}

extern "C" {

void sss_params_default(sss_params* p) {
    if (!p) return;
    std::memset(p, 0, sizeof(*p));
    p->kmin = 0;
    p->kmax = SSS_KMAX_AUTO;
    p->v = 2;
}

const char* sss_status_string(sss_status s) {
    switch (s) {
        case SSS_OK: return "ok";
        case SSS_ERR_INVALID_ARG: return "invalid argument";
        case SSS_ERR_OOM: return "out of memory";
        case SSS_ERR_CUDA: return "CUDA error";
        case SSS_ERR_TIMEOUT: return "device wait timed out";
        case SSS_ERR_DEVICE_CHECK: return "input validation failed on the device";
        case SSS_ERR_UNIMPLEMENTED: return "not implemented";
        case SSS_ERR_WORKSPACE: return "workspace too small";
    }
    return "unknown status";
}

const char* sss_last_error(sss_ctx* ctx) { return ctx ? ctx->last_error.c_str() : "no context"; }

sss_status sss_create(sss_ctx** out, int device, void* stream) {
    if (!out) return SSS_ERR_INVALID_ARG;
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
        cudaGetLastError();
        return SSS_ERR_INVALID_ARG;
    }
    if (cudaSetDevice(device) != cudaSuccess) return SSS_ERR_CUDA;
    sss_ctx* ctx = new (std::nothrow) sss_ctx();
    if (!ctx) return SSS_ERR_OOM;
    ctx->device = device;
    ctx->stream = static_cast<cudaStream_t>(stream);
    cudaDeviceGetAttribute(&ctx->sm_count, cudaDevAttrMultiProcessorCount, device);
    if (cudaMalloc(&ctx->d_err, sizeof(unsigned) * 4) != cudaSuccess) {
        delete ctx;
        return SSS_ERR_OOM;
    }
    cudaMemset(ctx->d_err, 0, sizeof(unsigned) * 4);
    if (cudaMalloc(&ctx->d_small, 4096) != cudaSuccess) {
        cudaFree(ctx->d_err);
        delete ctx;
        return SSS_ERR_OOM;
    }
    if (cudaMallocHost(&ctx->h_small, 64) != cudaSuccess) {
        cudaFree(ctx->d_small);
        cudaFree(ctx->d_err);
        delete ctx;
        return SSS_ERR_OOM;
    }
    cudaEventCreateWithFlags(&ctx->pin_event, cudaEventDisableTiming);
    cudaEventRecord(ctx->pin_event, ctx->stream);
    cudaDeviceSynchronize();
    *out = ctx;
    return SSS_OK;
}

sss_status sss_destroy(sss_ctx* ctx) {
    if (!ctx) return SSS_OK;
    cudaSetDevice(ctx->device);
    cudaStreamSynchronize(ctx->stream);
    collect_timings(ctx);
    for (cudaEvent_t e : ctx->event_pool) cudaEventDestroy(e);
    if (ctx->ws_own) cudaFree(ctx->ws_own);
    if (ctx->h_pin) cudaFreeHost(ctx->h_pin);
    if (ctx->d_err) cudaFree(ctx->d_err);
    if (ctx->d_small) cudaFree(ctx->d_small);
    if (ctx->h_small) cudaFreeHost(ctx->h_small);
    for (auto& lg : ctx->ls_graphs) {
        if (lg.exec) cudaGraphExecDestroy(lg.exec);
        if (lg.graph) cudaGraphDestroy(lg.graph);
    }
    if (ctx->cap_stream) cudaStreamDestroy(ctx->cap_stream);
    if (ctx->cap_stream2) cudaStreamDestroy(ctx->cap_stream2);
    if (ctx->copy_stream) cudaStreamDestroy(ctx->copy_stream);
    for (cudaEvent_t e : ctx->chunk_events) cudaEventDestroy(e);
    if (ctx->pin_event) cudaEventDestroy(ctx->pin_event);
    delete ctx;
    return SSS_OK;
}

sss_status sss_set_stream(sss_ctx* ctx, void* stream) {
    if (!ctx) return SSS_ERR_INVALID_ARG;
    ctx->stream = static_cast<cudaStream_t>(stream);
    return SSS_OK;
}

sss_status sss_set_workspace(sss_ctx* ctx, void* dev_ptr, size_t bytes) {
    if (!ctx) return SSS_ERR_INVALID_ARG;
    if (dev_ptr == nullptr || bytes == 0) {
        ctx->ws_user = nullptr;
        ctx->ws_user_bytes = 0;
    } else {
        ctx->ws_user = dev_ptr;
        ctx->ws_user_bytes = bytes;
    }
    return SSS_OK;
}

sss_status sss_sync(sss_ctx* ctx) {
    if (!ctx) return SSS_ERR_INVALID_ARG;
    cudaSetDevice(ctx->device);
    SSS_CUDA(cudaStreamSynchronize(ctx->stream));
    unsigned h = 0;
    SSS_CUDA(cudaMemcpy(&h, ctx->d_err, sizeof(unsigned), cudaMemcpyDeviceToHost));
    if (h) SSS_CUDA(cudaMemset(ctx->d_err, 0, sizeof(unsigned)));
    if (h & ERRBIT_CHECK) return sss_fail(ctx, SSS_ERR_DEVICE_CHECK, "input validation failed (offset/length/0x00)");
    if (h & ERRBIT_TIMEOUT) return sss_fail(ctx, SSS_ERR_TIMEOUT, "a bounded device wait ran out");
    if (h & ERRBIT_OVERFLOW) return sss_fail(ctx, SSS_ERR_CUDA, "internal capacity exceeded on the device");
    return SSS_OK;
}

sss_status sss_set_timing(sss_ctx* ctx, int enable, const char* filter) {
    if (!ctx) return SSS_ERR_INVALID_ARG;
    ctx->timing = enable != 0;
    ctx->timing_filter = filter ? filter : "";
    return SSS_OK;
}

sss_status sss_kernel_stats(sss_ctx* ctx, sss_kernel_stat* out, uint32_t cap, uint32_t* count) {
    if (!ctx || (!out && cap) || !count) return SSS_ERR_INVALID_ARG;
    cudaSetDevice(ctx->device);
    SSS_CUDA(cudaStreamSynchronize(ctx->stream));
    collect_timings(ctx);
    uint32_t k = 0;
    for (int i = 0; i < ctx->nstats && k < cap; ++i) {
        if (ctx->stats[i].launches == 0) continue;
        out[k].name = ctx->stats[i].name;
        out[k].launches = ctx->stats[i].launches;
        out[k].total_ms = ctx->stats[i].ms;
        out[k].timed = ctx->stats[i].timed;
        ++k;
    }
    *count = k;
    return SSS_OK;
}

sss_status sss_reset_stats(sss_ctx* ctx) {
    if (!ctx) return SSS_ERR_INVALID_ARG;
    cudaStreamSynchronize(ctx->stream);
    collect_timings(ctx);
    for (int i = 0; i < ctx->nstats; ++i) {
        ctx->stats[i].launches = 0;
        ctx->stats[i].ms = 0.0;
        ctx->stats[i].timed = 0;
    }
    return SSS_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// argument checks shared by the entry points
static sss_status check_common(sss_ctx* ctx, const uint8_t* chars, const uint64_t* offs, const uint32_t* lens,
                               uint32_t n, uint32_t p) {
    if (!ctx) return SSS_ERR_INVALID_ARG;
    if (n == 0xFFFFFFFFu) return sss_fail(ctx, SSS_ERR_INVALID_ARG, "n must be < 2^32 - 1");
    if (p == 0 || p > 1024) return sss_fail(ctx, SSS_ERR_INVALID_ARG, "p must be in 1..1024");
    if (n > 0 && (!offs || !lens)) return sss_fail(ctx, SSS_ERR_INVALID_ARG, "offsets/lengths must be non-NULL");
    if (n > 0 && !chars) return sss_fail(ctx, SSS_ERR_INVALID_ARG, "chars must be non-NULL");
    return SSS_OK;
}

static sss_status checked_input(sss_ctx* ctx, const StrIn& in) {
    SSS_TRY(impl_check_input(ctx, in));
    return sss_sync(ctx);
}

static uint32_t clamp_or(uint32_t x, uint32_t dflt, uint32_t lo, uint32_t hi) {
    if (x == 0) return dflt;
    return x < lo ? lo : (x > hi ? hi : x);
}

static sss_params resolve_params(const sss_params* p) {
    sss_params r;
    sss_params_default(&r);
    if (p) r = *p;
    if (r.v == 0) r.v = 2;
    r.cta_cap = clamp_or(r.cta_cap, 2048, 64, 2048);
    r.direct_cap = clamp_or(r.direct_cap, 8192, r.cta_cap, 8192);
    r.bucket_target = clamp_or(r.bucket_target, 2048, 256, 4096);
    r.warp_cap = clamp_or(r.warp_cap, 32, 2, 32);
    return r;
}

extern "C" {

// Work memory of the whole path: the runs, LCPs and approx of the partitions
// followed by the largest stage scratch (stages run one after the other).
static size_t need_pipeline(uint32_t n, uint64_t total_len, uint32_t p, const sss_params& prm) {
    size_t stage = need_local_sort(n, p, prm);
    if (p > 1) {
        stage = std::max(stage, need_dist_prefix(n));
        stage = std::max(stage, need_merge(n, p, prm.v, total_len));
    }
    Arena ar;
    ar.take<uint32_t>(n);
    ar.take<uint32_t>(n);
    ar.take<uint32_t>(n);
    ar.take<char>(stage);
    return ar.off + 256;
}

size_t sss_workspace_bytes(uint32_t n, uint64_t total_len, uint32_t p, const sss_params* params) {
    sss_params prm = resolve_params(params);
    if (p == 0) p = 1;
    return need_pipeline(n, total_len, p, prm);
}

static size_t need_batch(uint32_t n_table, uint32_t m, const sss_params& prm) {
    Arena cnt;
    cnt.take<Seg>(m);
    return cnt.off + 256 + need_local_sort(n_table, 1, prm);
}

size_t sss_batch_workspace_bytes(uint32_t n_table, uint32_t m, const sss_params* params) {
    return need_batch(n_table, m, resolve_params(params));
}

sss_status sss_local_sort(sss_ctx* ctx, const uint8_t* chars, uint64_t n_chars, const uint64_t* offsets,
                          const uint32_t* lengths, uint32_t n, uint32_t p, const sss_params* params,
                          uint32_t* out_run_perm, uint32_t* out_run_lcp) {
    SSS_TRY(check_common(ctx, chars, offsets, lengths, n, p));
    if (n > 0 && (!out_run_perm || !out_run_lcp)) return sss_fail(ctx, SSS_ERR_INVALID_ARG, "outputs must be non-NULL");
    if (n == 0) return SSS_OK;
    cudaSetDevice(ctx->device);
    sss_params prm = resolve_params(params);
    StrIn in{chars, n_chars, offsets, lengths, n};
    if (prm.flags & SSS_FLAG_CHECKED) SSS_TRY(checked_input(ctx, in));
    char* ws;
    SSS_TRY(sss_workspace(ctx, need_local_sort(n, p, prm), &ws));
    Arena ar{ws, 0, 0};
    return impl_local_sort(ctx, ar, in, p, prm, out_run_perm, out_run_lcp);
}

sss_status sss_dist(sss_ctx* ctx, const uint32_t* lengths, uint32_t n, const uint32_t* perm, const uint32_t* lcp,
                    uint32_t* out_dist) {
    if (!ctx) return SSS_ERR_INVALID_ARG;
    if (n == 0) return SSS_OK;
    if (!lengths || !perm || !lcp || !out_dist) return sss_fail(ctx, SSS_ERR_INVALID_ARG, "NULL pointer");
    cudaSetDevice(ctx->device);
    return impl_dist(ctx, lengths, n, perm, lcp, out_dist);
}

sss_status sss_dist_prefix(sss_ctx* ctx, const uint8_t* chars, uint64_t n_chars, const uint64_t* offsets,
                           const uint32_t* lengths, uint32_t n, const uint32_t* run_perm, const uint32_t* run_lcp,
                           uint32_t p, const sss_params* params, uint32_t* out_approx) {
    SSS_TRY(check_common(ctx, chars, offsets, lengths, n, p));
    if ((run_perm == nullptr) != (run_lcp == nullptr))
        return sss_fail(ctx, SSS_ERR_INVALID_ARG, "run_perm and run_lcp must both be given or both be NULL");
    if (n > 0 && !out_approx) return sss_fail(ctx, SSS_ERR_INVALID_ARG, "out_approx must be non-NULL");
    if (n == 0) return SSS_OK;
    cudaSetDevice(ctx->device);
    sss_params prm = resolve_params(params);
    StrIn in{chars, n_chars, offsets, lengths, n};
    if (prm.flags & SSS_FLAG_CHECKED) SSS_TRY(checked_input(ctx, in));
    char* ws;
    SSS_TRY(sss_workspace(ctx, need_dist_prefix(n), &ws));
    Arena ar{ws, 0, 0};
    const uint32_t* rp = (prm.flags & SSS_FLAG_NO_LOCAL_LCP_SKIP) ? nullptr : run_perm;
    const uint32_t* rl = (prm.flags & SSS_FLAG_NO_LOCAL_LCP_SKIP) ? nullptr : run_lcp;
    return impl_dist_prefix(ctx, ar, in, rp, rl, p, prm, out_approx);
}

sss_status sss_partition(sss_ctx* ctx, const uint8_t* chars, uint64_t n_chars, const uint64_t* offsets,
                         const uint32_t* lengths, const uint32_t* trunc, const uint32_t* run_perm, uint32_t n,
                         uint32_t p, const sss_params* params, uint32_t* out_splitters, uint32_t* out_bounds) {
    SSS_TRY(check_common(ctx, chars, offsets, lengths, n, p));
    if (!run_perm && n > 0) return sss_fail(ctx, SSS_ERR_INVALID_ARG, "run_perm must be non-NULL");
    if (!out_bounds || (p > 1 && !out_splitters))
        return sss_fail(ctx, SSS_ERR_INVALID_ARG, "outputs must be non-NULL");
    cudaSetDevice(ctx->device);
    sss_params prm = resolve_params(params);
    StrIn in{chars, n_chars, offsets, lengths, n};
    char* ws;
    SSS_TRY(sss_workspace(ctx, need_partition(n, p, prm.v), &ws));
    Arena ar{ws, 0, 0};
    return impl_partition(ctx, ar, in, trunc, run_perm, p, prm.v, prm.flags, out_splitters, out_bounds);
}

sss_status sss_lcp_merge(sss_ctx* ctx, const uint8_t* chars, uint64_t n_chars, const uint64_t* offsets,
                         const uint32_t* lengths, const uint32_t* trunc, const uint32_t* run_perm,
                         const uint32_t* run_lcp, uint32_t n, uint32_t p, const sss_params* params,
                         uint32_t* out_perm, uint32_t* out_lcp) {
    SSS_TRY(check_common(ctx, chars, offsets, lengths, n, p));
    if (n > 0 && (!run_perm || !run_lcp || !out_perm || !out_lcp))
        return sss_fail(ctx, SSS_ERR_INVALID_ARG, "NULL pointer");
    if (n == 0) return SSS_OK;
    cudaSetDevice(ctx->device);
    sss_params prm = resolve_params(params);
    StrIn in{chars, n_chars, offsets, lengths, n};
    uint64_t tot = 0;
    SSS_TRY(impl_sum_tlen(ctx, in, trunc, &tot));
    size_t need = need_merge(n, p, prm.v, tot);
    char* ws;
    SSS_TRY(sss_workspace(ctx, need, &ws));
    return impl_merge(ctx, ws, need, in, trunc, run_perm, run_lcp, p, prm.v, prm.merge_ms, prm.flags, tot, out_perm,
                      out_lcp);
}

}  // extern "C"

// Stages B to D and dist after stage A: the path of sss_sort for p > 1 on a
// workspace laid out as run_perm, run_lcp, approx, then the stage scratch.
// `stage_a` fills run_perm/run_lcp (on the context stream).
template <typename StageA>
static sss_status run_pipeline(sss_ctx* ctx, const StrIn& in, uint32_t p, const sss_params& prm, uint32_t* out_perm,
                               uint32_t* out_lcp, uint32_t* out_dist, uint32_t* out_approx, StageA stage_a) {
    const uint32_t n = in.n;
    uint64_t total_len = 0;
    SSS_TRY(impl_sum_tlen(ctx, in, nullptr, &total_len));
    size_t need = need_pipeline(n, total_len, p, prm);
    char* ws;
    SSS_TRY(sss_workspace(ctx, need, &ws));
    Arena ar{ws, need, 0};
    uint32_t* run_perm = ar.take<uint32_t>(n);
    uint32_t* run_lcp = ar.take<uint32_t>(n);
    uint32_t* approx = ar.take<uint32_t>(n);
    size_t stage_off = (ar.off + 255) & ~size_t(255);
    char* stage = ws + stage_off;
    size_t stage_bytes = need - stage_off;
    {
        Arena sa{stage, stage_bytes, 0};
        SSS_TRY(stage_a(sa, run_perm, run_lcp));
    }
    const uint32_t* trunc = nullptr;
    if (!(prm.flags & SSS_FLAG_MS)) {
        Arena sa{stage, stage_bytes, 0};
        SSS_TRY(impl_dist_prefix(ctx, sa, in, run_perm, run_lcp, p, prm, approx));
        trunc = approx;
    }
    SSS_TRY(impl_merge(ctx, stage, stage_bytes, in, trunc, run_perm, run_lcp, p, prm.v, prm.merge_ms, prm.flags,
                       total_len, out_perm, out_lcp));
    if (out_dist) SSS_TRY(impl_dist(ctx, in.lens, n, out_perm, out_lcp, out_dist));
    if (out_approx)
        SSS_CUDA(cudaMemcpyAsync(out_approx, trunc ? trunc : in.lens, sizeof(uint32_t) * n, cudaMemcpyDeviceToDevice,
                                 ctx->stream));
    return SSS_OK;
}

extern "C" {

sss_status sss_sort(sss_ctx* ctx, const uint8_t* chars, uint64_t n_chars, const uint64_t* offsets,
                    const uint32_t* lengths, uint32_t n, uint32_t p, const sss_params* params, uint32_t* out_perm,
                    uint32_t* out_lcp, uint32_t* out_dist, uint32_t* out_approx) {
    SSS_TRY(check_common(ctx, chars, offsets, lengths, n, p));
    if (n > 0 && (!out_perm || !out_lcp)) return sss_fail(ctx, SSS_ERR_INVALID_ARG, "outputs must be non-NULL");
    if (n == 0) return SSS_OK;
    cudaSetDevice(ctx->device);
    sss_params prm = resolve_params(params);
    StrIn in{chars, n_chars, offsets, lengths, n};
    if (prm.flags & SSS_FLAG_CHECKED) SSS_TRY(checked_input(ctx, in));
    if (p == 1) {
        char* ws;
        SSS_TRY(sss_workspace(ctx, need_local_sort(n, 1, prm), &ws));
        Arena ar{ws, 0, 0};
        SSS_TRY(impl_local_sort(ctx, ar, in, 1, prm, out_perm, out_lcp));
        if (out_dist) SSS_TRY(impl_dist(ctx, lengths, n, out_perm, out_lcp, out_dist));
        if (out_approx)
            SSS_CUDA(cudaMemcpyAsync(out_approx, lengths, sizeof(uint32_t) * n, cudaMemcpyDeviceToDevice, ctx->stream));
        return SSS_OK;
    }
    return run_pipeline(ctx, in, p, prm, out_perm, out_lcp, out_dist, out_approx,
                        [&](Arena& sa, uint32_t* run_perm, uint32_t* run_lcp) {
                            return impl_local_sort(ctx, sa, in, p, prm, run_perm, run_lcp);
                        });
}

sss_status sss_sort_host(sss_ctx* ctx, const uint8_t* h_chars, uint64_t n_chars, const uint64_t* h_offsets,
                         const uint32_t* h_lengths, uint32_t n, uint32_t p, const sss_params* params,
                         uint8_t* d_chars, uint64_t* d_offsets, uint32_t* d_lengths, uint32_t* out_perm,
                         uint32_t* out_lcp, uint32_t* h_out_perm, uint32_t* h_out_lcp) {
    SSS_TRY(check_common(ctx, h_chars, h_offsets, h_lengths, n, p));
    if (n > 0 && (!out_perm || !out_lcp || !d_chars || !d_offsets || !d_lengths))
        return sss_fail(ctx, SSS_ERR_INVALID_ARG, "device buffers and outputs must be non-NULL");
    if (n == 0) return SSS_OK;
    cudaSetDevice(ctx->device);
    sss_params prm = resolve_params(params);
    if (prm.flags & SSS_FLAG_CHECKED)
        return sss_fail(ctx, SSS_ERR_UNIMPLEMENTED, "sss_sort_host: SSS_FLAG_CHECKED needs sss_sort");
    if (!ctx->copy_stream) SSS_CUDA(cudaStreamCreateWithFlags(&ctx->copy_stream, cudaStreamNonBlocking));
    while (ctx->chunk_events.size() < (size_t)p + 1) {
        cudaEvent_t e;
        SSS_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        ctx->chunk_events.push_back(e);
    }
    // views first (12 bytes per string), then every partition's character extent
    SSS_CUDA(cudaMemcpyAsync(d_offsets, h_offsets, sizeof(uint64_t) * n, cudaMemcpyHostToDevice, ctx->stream));
    SSS_CUDA(cudaMemcpyAsync(d_lengths, h_lengths, sizeof(uint32_t) * n, cudaMemcpyHostToDevice, ctx->stream));
    StrIn in{d_chars, n_chars, d_offsets, d_lengths, n};
    unsigned long long* d_ext = ctx->d_small;  // 2p words: the 4 KiB scratch holds them for p <= 256
    std::vector<unsigned long long> ext(2 * (size_t)p);
    if ((size_t)p * 16 <= 4096) {
        SSS_TRY(impl_part_extents(ctx, in, p, d_ext));
        SSS_CUDA(cudaMemcpyAsync(ext.data(), d_ext, 16 * (size_t)p, cudaMemcpyDeviceToHost, ctx->stream));
        SSS_CUDA(cudaStreamSynchronize(ctx->stream));
    } else {
        for (uint32_t i = 0; i < p; ++i) ext[2 * i + 1] = n_chars;  // too many partitions: one chunk
    }
    // Characters on the copy stream, one chunk per partition: chunk i ends where
    // the strings of partitions 0..i end, so partition i may start once chunk i
    // is in (the copies wait for earlier work of the stream on these buffers).
    cudaEvent_t start = ctx->chunk_events[p];
    SSS_CUDA(cudaEventRecord(start, ctx->stream));
    SSS_CUDA(cudaStreamWaitEvent(ctx->copy_stream, start, 0));
    uint64_t done = 0;
    auto copy_chunks = [&](uint32_t i0, uint32_t i1) -> sss_status {
        for (uint32_t i = i0; i < i1; ++i) {
            // an empty partition leaves its extent at (max, 0): nothing to add
            uint64_t end = std::min<uint64_t>(std::max<uint64_t>(done, ext[2 * i + 1]), n_chars);
            if (end > done) {
                SSS_CUDA(cudaMemcpyAsync(d_chars + done, h_chars + done, end - done, cudaMemcpyHostToDevice,
                                         ctx->copy_stream));
                done = end;
            }
            SSS_CUDA(cudaEventRecord(ctx->chunk_events[i], ctx->copy_stream));
        }
        return SSS_OK;
    };
    // Partitions are sorted in groups of halving size (p/2, p/4, ..., 1, 1), each
    // once the chunk of its last partition is in: a local sort has a fixed cost per
    // round, so early groups are large, and only the last, small group's sort is
    // left after the upload ends.  A group's chunks are enqueued just before its
    // sort, behind the previous group's: the small uploads of a sort's segment
    // lists then wait on the copy engine only for chunks that group needs.  The
    // round loops run as the captured graph (SSS_FLAG_GRAPH): no group waits for
    // the host between rounds, and one graph serves every group.
    sss_params prm_a = prm;
    prm_a.flags |= SSS_FLAG_GRAPH;
    auto group_end = [&](uint32_t i0) { return i0 + (p - i0 > 1 ? (p - i0) / 2 : 1u); };
    auto stage_a = [&](Arena& sa, uint32_t* run_perm, uint32_t* run_lcp) -> sss_status {
        uint32_t i0 = 0;
        SSS_TRY(copy_chunks(0, group_end(0)));
        while (i0 < p) {
            const uint32_t i1 = group_end(i0);
            SSS_CUDA(cudaStreamWaitEvent(ctx->stream, ctx->chunk_events[i1 - 1], 0));
            std::vector<Seg> segs;
            for (uint32_t i = i0; i < i1; ++i) {
                const uint32_t lo = part_lo(n, p, i), hi = part_lo(n, p, i + 1);
                segs.push_back(Seg{lo, hi - lo, 0, 0});
            }
            Arena a{sa.base, sa.cap, 0};
            SSS_TRY(impl_sort_segments_range(ctx, a, in, segs, prm_a, run_perm, run_lcp, part_lo(n, p, i0),
                                             part_lo(n, p, i1)));
            if (i1 < p) SSS_TRY(copy_chunks(i1, group_end(i1)));
            i0 = i1;
        }
        return SSS_OK;
    };
    if (p == 1) {
        char* ws;
        SSS_TRY(sss_workspace(ctx, need_local_sort(n, 1, prm), &ws));
        Arena ar{ws, 0, 0};
        SSS_TRY(stage_a(ar, out_perm, out_lcp));
    } else {
        SSS_TRY(run_pipeline(ctx, in, p, prm, out_perm, out_lcp, nullptr, nullptr, stage_a));
    }
    if (h_out_perm)
        SSS_CUDA(cudaMemcpyAsync(h_out_perm, out_perm, sizeof(uint32_t) * n, cudaMemcpyDeviceToHost, ctx->stream));
    if (h_out_lcp)
        SSS_CUDA(cudaMemcpyAsync(h_out_lcp, out_lcp, sizeof(uint32_t) * n, cudaMemcpyDeviceToHost, ctx->stream));
    return SSS_OK;
}

sss_status sss_sort_batch(sss_ctx* ctx, const uint8_t* chars, uint64_t n_chars, const uint64_t* offsets,
                          const uint32_t* lengths, uint32_t n_table, const sss_instance* instances, uint32_t m,
                          const sss_params* params, uint32_t* out_perm, uint32_t* out_lcp, uint32_t* out_dist) {
    SSS_TRY(check_common(ctx, chars, offsets, lengths, n_table, 1));
    if (m > 0 && !instances) return sss_fail(ctx, SSS_ERR_INVALID_ARG, "instances must be non-NULL");
    if (n_table > 0 && (!out_perm || !out_lcp)) return sss_fail(ctx, SSS_ERR_INVALID_ARG, "outputs must be non-NULL");
    if (m == 0 || n_table == 0) return SSS_OK;
    std::vector<Seg> segs(m);
    for (uint32_t k = 0; k < m; ++k) {
        const sss_instance& I = instances[k];
        if (I.p > 1) return sss_fail(ctx, SSS_ERR_UNIMPLEMENTED, "batched instances with p > 1");
        if (I.first > n_table || (uint64_t)I.n > n_table - I.first)
            return sss_fail(ctx, SSS_ERR_INVALID_ARG, "instance " + std::to_string(k) + " exceeds the string table");
        segs[k] = Seg{(uint32_t)I.first, I.n, 0, 0};
    }
    std::vector<Seg> sorted = segs;
    std::sort(sorted.begin(), sorted.end(), [](const Seg& x, const Seg& y) { return x.start < y.start; });
    for (uint32_t k = 1; k < m; ++k)
        if ((uint64_t)sorted[k - 1].start + sorted[k - 1].size > sorted[k].start)
            return sss_fail(ctx, SSS_ERR_INVALID_ARG, "instances overlap");
    cudaSetDevice(ctx->device);
    sss_params prm = resolve_params(params);
    StrIn in{chars, n_chars, offsets, lengths, n_table};
    if (prm.flags & SSS_FLAG_CHECKED) SSS_TRY(checked_input(ctx, in));
    // work memory: the instance table, then the segment sort
    size_t need = need_batch(n_table, m, prm);
    char* ws;
    SSS_TRY(sss_workspace(ctx, need, &ws));
    Arena ar{ws, need, 0};
    Seg* d_inst = ar.take<Seg>(m);
    void* pin;
    SSS_TRY(sss_pinned(ctx, sizeof(Seg) * m, &pin));
    std::copy(segs.begin(), segs.end(), static_cast<Seg*>(pin));
    SSS_TRY(sss_upload(ctx, d_inst, pin, sizeof(Seg) * m));
    size_t off = (ar.off + 255) & ~size_t(255);
    Arena sa{ws + off, need - off, 0};
    if (prm.flags & SSS_FLAG_GRAPH)  // the whole sort as one graph launch
        return impl_sort_batch_graph(ctx, sa, in, d_inst, m, prm, out_perm, out_lcp, out_dist);
    SSS_TRY(impl_sort_segments(ctx, sa, in, segs, prm, out_perm, out_lcp));
    return impl_batch_finish(ctx, d_inst, m, lengths, out_perm, out_lcp, out_dist);
}

size_t sss_suffix_workspace_bytes(uint64_t n_text, const sss_params* params) {
    if (n_text > UINT32_MAX) return 0;
    return need_suffix_sort((uint32_t)n_text, resolve_params(params));
}

sss_status sss_suffix_sort(sss_ctx* ctx, const uint8_t* text, uint64_t n_text, uint32_t max_len,
                           const sss_params* params, uint32_t* out_sa, uint32_t* out_lcp) {
    if (!ctx) return SSS_ERR_INVALID_ARG;
    if (n_text > UINT32_MAX) return sss_fail(ctx, SSS_ERR_INVALID_ARG, "text longer than 2^32 - 1 characters");
    if (n_text == 0) return SSS_OK;
    if (!text || !out_sa || !out_lcp) return sss_fail(ctx, SSS_ERR_INVALID_ARG, "NULL pointer");
    cudaSetDevice(ctx->device);
    sss_params prm = resolve_params(params);
    const uint32_t n = (uint32_t)n_text;
    const size_t need = sss_suffix_workspace_bytes(n_text, &prm);
    char* ws;
    SSS_TRY(sss_workspace(ctx, need, &ws));
    if (prm.flags & SSS_FLAG_CHECKED) {
        Arena ar{ws, need, 0};
        uint64_t* offs = ar.take<uint64_t>(n);
        uint32_t* lens = ar.take<uint32_t>(n);
        SSS_TRY(impl_suffix_views(ctx, n, max_len ? max_len : UINT32_MAX, offs, lens));
        StrIn in{text, n_text, offs, lens, n};
        SSS_TRY(checked_input(ctx, in));
    }
    return impl_suffix_sort(ctx, ws, need, text, n, max_len, prm, out_sa, out_lcp);
}

}  // extern "C"
