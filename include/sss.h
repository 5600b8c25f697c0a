/*
 * sss.h -- C ABI of the GB300 string sorter (libsss.so).
 *
 * The library sorts a string array S = [s_0, ..., s_{n-1}] as defined in the
 * paper's Section 2 ("String Properties and Input Format"): strings are views
 * (offset, length) into one character array, the output is the sorted order
 * ("where to find the i-th smallest string", Section 4) plus the LCP array, and
 * optionally the distinguishing-prefix lengths.  The p "PEs" of the paper's
 * distributed algorithm are p partitions of the input held in one GPU's memory:
 * partition i owns input indices [floor(i*n/p), floor((i+1)*n/p)).
 *
 * Conventions for every call below:
 *  - Pointers named chars/offsets/lengths/... and every out_* pointer are DEVICE
 *    pointers owned by the caller; the library never frees them.
 *      chars    : uint8_t[n_chars]   character data; no string contains 0x00
 *                 (the sentinel of Section 2 is implicit at the string end)
 *      offsets  : uint64_t[n]        string i starts at chars[offsets[i]]
 *      lengths  : uint32_t[n]        string i has lengths[i] chars (no terminator)
 *    Strings may overlap (e.g. suffixes of one text).
 *  - Calls are asynchronous on the context's CUDA stream.  A call returns after
 *    enqueueing its work; some calls synchronise the stream internally to read
 *    small counters (documented per call).  Outputs are valid once the stream has
 *    been synchronised.
 *  - The return value reports argument, allocation and launch errors.  Errors
 *    detected on the device (SSS_CHECKED validation, bounded waits that ran out)
 *    are sticky in the context and returned by sss_sync().
 *  - Work memory is owned by the context: it is allocated with cudaMalloc on
 *    first use and grown when a larger problem arrives, or supplied by the caller
 *    with sss_set_workspace().
 *  - A context is not thread-safe; use one context per host thread.
 *  - Limits: n < 2^32 - 1, 1 <= p <= 1024, string lengths < 2^31.
 */
#ifndef SSS_H
#define SSS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum sss_status {
    SSS_OK = 0,
    SSS_ERR_INVALID_ARG = 1,   /* bad pointer/size/parameter; nothing was enqueued */
    SSS_ERR_OOM = 2,           /* device or pinned host allocation failed */
    SSS_ERR_CUDA = 3,          /* a CUDA runtime call failed (see sss_last_error) */
    SSS_ERR_TIMEOUT = 4,       /* reserved: a bounded device-side wait ran out (no call
                                  of this version waits on the device) */
    SSS_ERR_DEVICE_CHECK = 5,  /* SSS_CHECKED validation found bad input */
    SSS_ERR_UNIMPLEMENTED = 6, /* the requested mode is not built */
    SSS_ERR_WORKSPACE = 7      /* caller-supplied workspace is too small */
} sss_status;

/* sss_params.flags */
#define SSS_FLAG_MS 0x1u       /* p > 1: merge full strings, skip prefix doubling */
#define SSS_FLAG_CHECKED 0x2u  /* validate offsets/lengths against n_chars and
                                  scan strings for 0x00 bytes; errors are sticky */
#define SSS_FLAG_NO_LOCAL_LCP_SKIP 0x4u /* doubling: hash every active string
                                  instead of one per locally-equal prefix group */
#define SSS_FLAG_DEDUPE_SORT 0x8u /* doubling: detect duplicate keys by sorting
                                  them (bucketed shared-memory sorts) instead of
                                  the exact hash table */
#define SSS_FLAG_MERGE_TREE 0x10u /* merge: pairwise LCP-merge tree over whole
                                  buckets instead of second-level sub-buckets
                                  merged inside one CTA each */
#define SSS_FLAG_GRAPH 0x40u /* local sort: run its round loop as one CUDA graph
                                  launch (a conditional while node whose body is a
                                  device-planned round); sss_sort_batch: the whole
                                  call (identity order, device-side classification
                                  of the instances, first finishers, round loop,
                                  instance-local order) is one graph launch after
                                  the instance-table upload.  Graphs are kept in the
                                  context (up to four) and relaunched while the
                                  call's pointers and sizes are unchanged */
#define SSS_FLAG_NO_CTA_ROUNDS 0x80u /* doubling: launch the per-round kernels for
                                  every round instead of running the rounds that
                                  test at most 4096 keys inside one CTA (hash-table
                                  dedupe only; results are identical) */
#define SSS_FLAG_CHAR_SAMPLING 0x20u /* partition: character-based regular sampling
                                  (Section 3.1.2): about p(v+1) samples at equally
                                  spaced character positions of the runs (truncated
                                  lengths), so buckets balance characters rather than
                                  strings; string-based (Section 3.1.1) otherwise */

typedef struct sss_params {
    uint32_t kmin;      /* first doubling round: prefix length 2^kmin (default 0) */
    uint32_t kmax;      /* last doubling round; SSS_KMAX_AUTO = ceil(log2(max len)) */
    uint32_t v;         /* regular-sampling factor (default 2, Section 5) */
    uint32_t flags;     /* SSS_FLAG_* */
    uint64_t hash_seed; /* seed of the prefix hash (default 0) */
    /* Tuning knobs of the local sort and merge: they change speed, never results.
     * 0 selects the default; other values are clamped into the stated range. */
    uint32_t cta_cap;       /* largest segment finished inside one CTA, 64..2048 (default 2048) */
    uint32_t merge_ms;      /* merge segment spacing, a power of two 8..1024 (default 32) */
    uint32_t direct_cap;    /* largest segment of the multi-CTA path sorted whole by one CTA,
                               cta_cap..8192 (default 8192) */
    uint32_t bucket_target; /* target size of a sampled-partition range bucket, 256..4096
                               (default 2048) */
    uint32_t warp_cap;      /* largest segment finished by one warp, 2..32 (default 32) */
    uint32_t reserved[1];
} sss_params;

#define SSS_KMAX_AUTO 0xFFFFFFFFu

typedef struct sss_ctx sss_ctx;

/* Fill *p with the defaults (kmin 0, kmax auto, v 2, flags 0, seed 0). */
void sss_params_default(sss_params* p);

/* Create a context on CUDA device `device` that enqueues on `cuda_stream` (a
 * cudaStream_t; NULL = the legacy default stream).  *out is set on success. */
sss_status sss_create(sss_ctx** out, int device, void* cuda_stream);

/* Destroy a context (synchronises its stream, frees its memory).  NULL is a no-op. */
sss_status sss_destroy(sss_ctx* ctx);

/* Change the stream subsequent calls enqueue on. */
sss_status sss_set_stream(sss_ctx* ctx, void* cuda_stream);

/* Hand the context a caller-owned device buffer to use as work memory instead of
 * its own allocations (NULL/0 returns to library-owned memory).  The buffer must
 * stay valid while calls that use it run; sss_workspace_bytes() gives the size. */
sss_status sss_set_workspace(sss_ctx* ctx, void* dev_ptr, size_t bytes);

/* Upper bound on the work memory any call with these sizes needs (bytes):
 * n strings with total_len = sum of lengths (an upper bound is fine), p partitions. */
size_t sss_workspace_bytes(uint32_t n, uint64_t total_len, uint32_t p, const sss_params* params);

/* Synchronise the context's stream and return the sticky device status
 * (SSS_OK, SSS_ERR_DEVICE_CHECK, SSS_ERR_TIMEOUT or SSS_ERR_CUDA); clears it. */
sss_status sss_sync(sss_ctx* ctx);

const char* sss_status_string(sss_status s);

/* Human-readable text of the last error raised by this context (never NULL). */
const char* sss_last_error(sss_ctx* ctx);

/* ------------------------------------------------------------------------ */
/* Stage A -- local string sort with LCP output (Section 3, "Initialization":
 * each PE sorts its local array; the LCP array is a by-product of sorting).
 * MSD string sort by reference-split keys: every member of a segment (strings
 * sharing `depth` characters) is keyed by its LCP with the segment's reference
 * member, the side of the reference it falls on and its next 4-6 characters;
 * large segments are split by sampled key splitters into range and equality
 * buckets sorted in shared memory, segments of up to cta_cap strings are
 * finished inside one CTA (or one warp / 4-lane group when tiny), and equal
 * keys form the next round's segments.
 *
 * out_run_perm : uint32_t[n]; positions [lo_i, hi_i) hold partition i's input
 *                indices in sorted order (equal strings by index).
 * out_run_lcp  : uint32_t[n]; out_run_lcp[q] = lcp(run[q-1], run[q]) within a
 *                partition, 0 at every partition start.
 * Synchronises the stream once per round of segments larger than cta_cap
 * (never with SSS_FLAG_GRAPH, whose round loop runs on the device). */
sss_status sss_local_sort(sss_ctx* ctx, const uint8_t* chars, uint64_t n_chars,
                          const uint64_t* offsets, const uint32_t* lengths, uint32_t n,
                          uint32_t p, const sss_params* params,
                          uint32_t* out_run_perm, uint32_t* out_run_lcp);

/* Stage A6 -- exact distinguishing prefixes (Section 2: the characters needed to
 * rank a string): out_dist[perm[r]] = min(len, 1 + max(lcp[r], lcp[r+1])) for a
 * GLOBAL sorted order perm/lcp of all n strings (missing neighbours count 0). */
sss_status sss_dist(sss_ctx* ctx, const uint32_t* lengths, uint32_t n,
                    const uint32_t* perm, const uint32_t* lcp, uint32_t* out_dist);

/* Stage B -- prefix doubling (Section 4): for k = kmin..kmax the prefixes of
 * length L = 2^k of the still-active strings are hashed to 64-bit keys; keys
 * that occur once (or strings with length <= L) retire with
 * approx = min(L, len); duplicates are found by counting the full 64-bit keys
 * in an exact open-addressing hash table (a single-shot filter without false
 * positives), or with SSS_FLAG_DEDUPE_SORT by sorting them (the appendix's
 * route, "Duplicate Detection with Atomic Hypercube Quicksort").  Survivors of round
 * kmax get approx = len.  approx >= dist always.
 * run_perm/run_lcp (nullable together): the local sorted runs of p partitions
 * (as from sss_local_sort); when given, strings whose L-prefix equals a local
 * neighbour's are known duplicates and one key per such group is hashed -- the
 * result is identical.  out_approx: uint32_t[n] by input index.
 * Consecutive rounds that each test at most 4096 keys run inside one CTA (see
 * SSS_FLAG_NO_CTA_ROUNDS).  Synchronises the stream once per round, or once per
 * such run of rounds. */
sss_status sss_dist_prefix(sss_ctx* ctx, const uint8_t* chars, uint64_t n_chars,
                           const uint64_t* offsets, const uint32_t* lengths, uint32_t n,
                           const uint32_t* run_perm, const uint32_t* run_lcp, uint32_t p,
                           const sss_params* params, uint32_t* out_approx);

/* Stage C -- string-based regular sampling and splitters (Section 3.1.1) and
 * bucket bounds (Section 3, step 1).  Partition i draws v+1 samples at local
 * ranks ceil(t*n_i/(v+1)) - 1 (t = 1..v+1); the samples are sorted (truncated
 * strings, then index) and f_j = V[floor(j*|V|/p) - 1] for 0 < j < p
 * (UINT32_MAX = minus infinity when the index is negative).
 * With SSS_FLAG_CHAR_SAMPLING (Section 3.1.2): with N the total truncated
 * length and want = p(v+1), partition i (C_i characters in its run) draws
 * ceil(C_i*want/N) - 1 samples, the strings of its run covering the character
 * positions floor(t*N/want), t = 1, 2, ...; while fewer than want samples
 * exist, the first non-empty partitions add their last string, one each.
 * Splitters are then chosen as above.  N == 0 falls back to string-based.
 * trunc        : uint32_t[n] or NULL; string i is compared as its first
 *                trunc[i] chars (trunc[i] <= lengths[i]).
 * out_splitters: uint32_t[p-1] input indices of f_1..f_{p-1} (may be NULL if p==1)
 * out_bounds   : uint32_t[p*(p+1)]; out_bounds[i*(p+1)+j] = number of strings of
 *                run i that are <= f_j (0 for j = 0, n_i for j = p). */
sss_status sss_partition(sss_ctx* ctx, const uint8_t* chars, uint64_t n_chars,
                         const uint64_t* offsets, const uint32_t* lengths,
                         const uint32_t* trunc, const uint32_t* run_perm, uint32_t n, uint32_t p,
                         const sss_params* params, uint32_t* out_splitters, uint32_t* out_bounds);

/* Stage D -- LCP-compressed exchange and LCP-aware merge (Section 3, steps 2-3;
 * LCP compression and LCP merging of Section 2 "Algorithmic Building Blocks").
 * Merges the p sorted runs run_perm/run_lcp (partition layout) into the global
 * order: stage C picks splitters, every run piece is copied LCP-compressed into
 * its bucket (index, LCP with predecessor, chars [lcp, trunc)), and each bucket
 * is merged with LCPs.  Equal (truncated) strings keep run order.
 * trunc: as for sss_partition (NULL = full strings).  Truncation lengths must not
 * change the order (true for approx from sss_dist_prefix).
 * out_perm/out_lcp: uint32_t[n] global sorted order and full LCP array. */
sss_status sss_lcp_merge(sss_ctx* ctx, const uint8_t* chars, uint64_t n_chars,
                         const uint64_t* offsets, const uint32_t* lengths,
                         const uint32_t* trunc, const uint32_t* run_perm, const uint32_t* run_lcp,
                         uint32_t n, uint32_t p, const sss_params* params,
                         uint32_t* out_perm, uint32_t* out_lcp);

/* The whole path.  p == 1: local sort (stage A) of all strings.  p > 1: the
 * prefix-doubling merge sort (PDMS, Section 4) collapsed onto one GPU: stage A on
 * every partition, stage B, then stages C and D on the approx-truncated strings
 * (SSS_FLAG_MS: no stage B, full strings are merged).
 * out_perm, out_lcp  : uint32_t[n] global order and LCP array (required)
 * out_dist, out_approx: uint32_t[n] by input index, or NULL to skip (out_approx
 *                       is approx for p > 1 without SSS_FLAG_MS, else lengths). */
sss_status sss_sort(sss_ctx* ctx, const uint8_t* chars, uint64_t n_chars,
                    const uint64_t* offsets, const uint32_t* lengths, uint32_t n, uint32_t p,
                    const sss_params* params, uint32_t* out_perm, uint32_t* out_lcp,
                    uint32_t* out_dist, uint32_t* out_approx);

/* The whole path (as sss_sort, without dist/approx outputs) for a string set in
 * HOST memory, with the upload overlapped with stage A.  No counterpart in the
 * paper, whose input starts in the PEs' memory: here the offsets and lengths are
 * uploaded first, then the characters in one chunk per partition on a second
 * stream, and partition i's local sort (Section 3, "Initialization") starts as
 * soon as the chunk holding its strings has arrived, while later chunks are
 * still in flight.  Stages B to D follow as in sss_sort.
 * h_chars, h_offsets, h_lengths : HOST arrays (n_chars, n, n entries); pinned
 *                 (cudaHostAlloc) memory gives full copy speed
 * d_chars, d_offsets, d_lengths : caller-owned DEVICE buffers of the same sizes,
 *                 filled by the call (only the characters up to the end of the
 *                 last string are copied)
 * out_perm, out_lcp : DEVICE uint32_t[n], as for sss_sort
 * h_out_perm, h_out_lcp : HOST uint32_t[n] or NULL: copies of the outputs,
 *                 valid once the context stream has been synchronised
 * Partitions are sorted in groups of halving size (p/2, p/4, ..., 1, 1), each
 * as soon as its characters are in, with the local sort's round loop as one
 * graph launch (SSS_FLAG_GRAPH is implied).  Synchronises the stream to read the
 * partitions' character extents and, as sss_sort does, the total length.
 * SSS_FLAG_CHECKED is not supported here (SSS_ERR_UNIMPLEMENTED): validate
 * with sss_sort. */
sss_status sss_sort_host(sss_ctx* ctx, const uint8_t* h_chars, uint64_t n_chars, const uint64_t* h_offsets,
                         const uint32_t* h_lengths, uint32_t n, uint32_t p, const sss_params* params,
                         uint8_t* d_chars, uint64_t* d_offsets, uint32_t* d_lengths, uint32_t* out_perm,
                         uint32_t* out_lcp, uint32_t* h_out_perm, uint32_t* h_out_lcp);

/* Batched sorting: m independent instances, instance k being the strings
 * [first, first + n) of one shared string table of n_table strings.  All
 * instances are sorted together (stage A over all of them at once: the
 * instances are the initial segments of one radix sort), which beats one call
 * per instance by sharing every launch and synchronisation.
 * instances   : HOST array of m entries; instances must not overlap; p must be
 *               0 or 1 (SSS_ERR_UNIMPLEMENTED otherwise)
 * out_perm    : uint32_t[n_table]; out_perm[first + r] = index, relative to
 *               first, of the instance's r-th smallest string (ties by index)
 * out_lcp     : uint32_t[n_table]; the instance's LCP array (0 at r = 0)
 * out_dist    : uint32_t[n_table] or NULL; dist of table string first + i
 *               within its instance, at position first + i
 * Positions outside every instance are left with identity order and LCP 0. */
typedef struct sss_instance {
    uint64_t first;
    uint32_t n;
    uint32_t p;
} sss_instance;

sss_status sss_sort_batch(sss_ctx* ctx, const uint8_t* chars, uint64_t n_chars,
                          const uint64_t* offsets, const uint32_t* lengths, uint32_t n_table,
                          const sss_instance* instances, uint32_t m, const sss_params* params,
                          uint32_t* out_perm, uint32_t* out_lcp, uint32_t* out_dist);

/* Work memory (bytes) that sss_sort_batch needs for a table of n_table strings
 * holding m instances: the size a caller-owned workspace (sss_set_workspace)
 * must have for that call.  Pure host arithmetic; no context needed. */
size_t sss_batch_workspace_bytes(uint32_t n_table, uint32_t m, const sss_params* params);

/* ------------------------------------------------------------------------ */
/* Suffix sorting as space-efficient string sorting (the extension named in the
 * paper's Section 6, "Conclusion and Future Work": the suffixes of a text sorted
 * as strings without materialising them).  String i is the view
 * text[i .. i + min(n_text - i, max_len)) (max_len 0 = whole suffixes); the
 * characters are never copied.  The suffixes truncated to 64 characters are
 * sorted as strings by stage A (p = 1); where that leaves equal truncations,
 * prefix doubling over ranks follows: the order on the first min(2h, target)
 * characters is the order of the pairs (rank_h(i), rank_h(i + o)), o <= h,
 * sorted as 10-byte strings by stage A, until every rank is distinct or the
 * target length (max_len, else the whole suffix) is reached.  A text with
 * short repeats is done after the first sort; a text of one repeated character
 * takes log2(n / 64) rounds.  The LCPs come from the rank levels.
 * text         : DEVICE array of n_text bytes, no 0x00 byte (checked with
 *                SSS_FLAG_CHECKED); n_text < 2^32
 * out_sa       : uint32_t[n_text]; the suffix array (start positions in sorted
 *                order; with max_len, equal truncated suffixes by position)
 * out_lcp      : uint32_t[n_text]; LCP of consecutive suffixes (0 first),
 *                truncated suffixes when max_len > 0
 * Work memory: sss_suffix_workspace_bytes(n_text, params). */
size_t sss_suffix_workspace_bytes(uint64_t n_text, const sss_params* params);
sss_status sss_suffix_sort(sss_ctx* ctx, const uint8_t* text, uint64_t n_text, uint32_t max_len,
                           const sss_params* params, uint32_t* out_sa, uint32_t* out_lcp);

/* ------------------------------------------------------------------------ */
/* Allocation-free prefix doubling (stage B) for small sets.  This call has no
 * counterpart in the paper; it exists for callers that cannot allocate device
 * memory at the moment they need the result -- e.g. code running inside a host
 * framework that owns the whole device budget, or a latency-critical request
 * loop where a cudaMalloc could block or fail.  It needs no context and no
 * work memory: its state and hash table live in one fixed device array of about
 * 2.6 MB inside libsss.so, which every GPU that loads the library holds until
 * the process exits.  It calls no cudaMalloc/cudaFree.
 *
 * Computes out_approx exactly as sss_dist_prefix with run_perm = run_lcp = NULL
 * (every active string hashed every round); one CTA runs all rounds.
 *   n           : at most SSS_NOALLOC_MAX_STRINGS, else SSS_ERR_INVALID_ARG
 *                 (nothing is enqueued)
 *   chars/offsets/lengths/out_approx: device pointers, as for the other calls
 *   params      : kmin, kmax, hash_seed are used (NULL = defaults)
 *   cuda_stream : the cudaStream_t the kernel is enqueued on
 * The first call on a device (the device current at the call) looks up the
 * array's device address; make that first call before any stream capture.
 * Every call on a device shares the one array and clears the state it needs at
 * its start, so calls that may overlap on the GPU (different streams without
 * ordering) race and give undefined results; order them on one stream.  Errors
 * are returned for bad arguments and failed launches only; inputs are not
 * validated on the device. */
#define SSS_NOALLOC_MAX_STRINGS 65536u
sss_status sss_dist_prefix_noalloc(const uint8_t* chars, uint64_t n_chars, const uint64_t* offsets,
                                   const uint32_t* lengths, uint32_t n, const sss_params* params,
                                   uint32_t* out_approx, void* cuda_stream);

/* ------------------------------------------------------------------------ */
/* Instrumentation: per-kernel launch counts and (when timing is enabled) device
 * time measured with CUDA events on the context's stream around each launch. */
#define SSS_MAX_KERNELS 128

typedef struct sss_kernel_stat {
    const char* name;   /* static string */
    uint64_t launches;  /* launches since the last reset */
    double total_ms;    /* summed device time (timing enabled only) */
    uint64_t timed;     /* launches that were timed */
} sss_kernel_stat;

/* Enable (1) / disable (0) event timing of launches whose kernel name contains
 * `name_filter` (NULL or "" = all kernels). */
sss_status sss_set_timing(sss_ctx* ctx, int enable, const char* name_filter);

/* Synchronise, then copy up to `cap` entries (one per kernel that launched since
 * the last reset) into out; *count receives the number written. */
sss_status sss_kernel_stats(sss_ctx* ctx, sss_kernel_stat* out, uint32_t cap, uint32_t* count);

/* Zero all launch counts and times. */
sss_status sss_reset_stats(sss_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif /* SSS_H */
