/*
 * CPU oracle for the string sorter: TEST INFRASTRUCTURE ONLY.
 *
 * Plain, slow, obviously correct C.  Only the test suite, the package's smoke
 * check and the CPU-baseline leg of the benchmark may load it; the library's
 * product path never calls it and shares no code with it.
 *
 * Strings are (offset, length) views into one character array; lengths exclude
 * the terminator and no string contains 0x00 (the sentinel of Section 2,
 * "String Properties and Input Format").  Where a truncation array is given,
 * string i is compared as its first trunc[i] characters (trunc[i] <= lens[i]).
 *
 * Parity status: sort, LCP array, dist, doubling, sampling, splitters, bucket
 * bounds and merge are pinned by tests, and so are the 64-bit prefix-hash
 * values (oracle_prefix_key): the paper fixes no hash function, and the one
 * defined here is checked through the inverse of its finaliser against the
 * Karp-Rabin polynomial it states.
 */
#ifndef SSS_ORACLE_H
#define SSS_ORACLE_H
#include <stdint.h>
#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Three-way comparison of strings a and b (optionally truncated), unsigned bytes,
 * a proper prefix first; equal strings are ordered by index.  Returns -1, 0 or 1
 * (0 only when a == b). */
int oracle_cmp(const uint8_t* chars, const uint64_t* offs, const uint32_t* lens,
               const uint32_t* trunc, uint32_t a, uint32_t b);

/* Same comparison without the index tie-break (0 for equal strings). */
int oracle_cmp_str(const uint8_t* chars, const uint64_t* offs, const uint32_t* lens,
                   const uint32_t* trunc, uint32_t a, uint32_t b);

/* LCP of strings a and b (optionally truncated): the first differing position,
 * or the shorter length. */
uint32_t oracle_lcp_pair(const uint8_t* chars, const uint64_t* offs, const uint32_t* lens,
                         const uint32_t* trunc, uint32_t a, uint32_t b);

/* Sort the m indices in idx[] (in place) by oracle_cmp. */
void oracle_sort_idx(const uint8_t* chars, const uint64_t* offs, const uint32_t* lens,
                     const uint32_t* trunc, uint32_t* idx, uint32_t m);

/* Plain sort of all n strings: perm[r] = index of the r-th smallest string. */
void oracle_sort(const uint8_t* chars, const uint64_t* offs, const uint32_t* lens,
                 uint32_t n, uint32_t* perm);

/* LCP array of a sorted index sequence: lcp[0] = 0, lcp[r] = lcp(perm[r-1], perm[r]). */
void oracle_lcp_array(const uint8_t* chars, const uint64_t* offs, const uint32_t* lens,
                      const uint32_t* trunc, const uint32_t* perm, uint32_t m, uint32_t* lcp);

/* Exact distinguishing prefix per input index from a global sorted order:
 * dist[i] = min(len_i, 1 + max(lcp with sorted neighbours)). */
void oracle_dist(const uint32_t* lens, uint32_t n, const uint32_t* perm, const uint32_t* lcp,
                 uint32_t* dist);

/* Modular multiply in Z_P, P = 2^61 - 1 (exposed for its pin). */
uint64_t oracle_mulmod61(uint64_t a, uint64_t b);

/* SplitMix64: the first output of the sequence seeded with s (exposed for its pin). */
uint64_t oracle_splitmix64_first(uint64_t s);

/* Hash base B for a hash seed: 2 + (SplitMix64(seed) mod (P - 3)). */
uint64_t oracle_hash_base(uint64_t seed);

/* 64-bit key of the first l characters of string i (l <= its length). */
uint64_t oracle_prefix_key(const uint8_t* chars, const uint64_t* offs, const uint32_t* lens,
                           uint32_t i, uint32_t l, uint64_t seed);

/* Prefix doubling: approx[i] for every string.  rounds_out (nullable, kmax+1
 * entries) receives the number of active strings at the start of each round. */
void oracle_doubling(const uint8_t* chars, const uint64_t* offs, const uint32_t* lens,
                     uint32_t n, uint32_t kmin, uint32_t kmax, uint64_t seed,
                     uint32_t* approx, uint32_t* rounds_out);

/* Partition bounds: partition i holds input indices [floor(i*n/p), floor((i+1)*n/p)). */
uint32_t oracle_part_lo(uint32_t n, uint32_t p, uint32_t i);

/* Local sort of every partition: run_perm/run_lcp are n-long, partition i's run at
 * positions [lo_i, hi_i), lcp 0 at each partition start. */
void oracle_local_sort(const uint8_t* chars, const uint64_t* offs, const uint32_t* lens,
                       const uint32_t* trunc, uint32_t n, uint32_t p,
                       uint32_t* run_perm, uint32_t* run_lcp);

/* String-based regular sampling (v+1 samples per non-empty partition) and
 * splitter selection.  samples_out: up to p*(v+1) indices (returns the count);
 * splitters_out: p-1 entries, UINT32_MAX for "minus infinity". */
uint32_t oracle_samples(const uint32_t* run_perm, uint32_t n, uint32_t p, uint32_t v,
                        uint32_t* samples_out);
/* Character-based regular sampling (Section 3.1.2): about p*(v+1) samples taken
 * at equally spaced character positions of the runs' character arrays (trunc
 * lengths when given).  samples_out: up to p*(v+1) indices (returns the count). */
uint32_t oracle_samples_char(const uint32_t* lens, const uint32_t* trunc, const uint32_t* run_perm, uint32_t n,
                             uint32_t p, uint32_t v, uint32_t* samples_out);
void oracle_splitters(const uint8_t* chars, const uint64_t* offs, const uint32_t* lens,
                      const uint32_t* trunc, uint32_t* samples, uint32_t ns, uint32_t p,
                      uint32_t* splitters_out);

/* Bucket bounds: bounds[i*(p+1)+j] = number of strings of run i that are <= f_j
 * (j = 1..p-1), 0 for j = 0 and n_i for j = p. */
void oracle_bounds(const uint8_t* chars, const uint64_t* offs, const uint32_t* lens,
                   const uint32_t* trunc, const uint32_t* run_perm, uint32_t n, uint32_t p,
                   const uint32_t* splitters, uint32_t* bounds);

/* One row of oracle_bounds: the counts of run i (bounds + i*(p+1)). */
void oracle_bounds_row(const uint8_t* chars, const uint64_t* offs, const uint32_t* lens,
                       const uint32_t* trunc, const uint32_t* run_perm, uint32_t n, uint32_t p,
                       const uint32_t* splitters, uint32_t i, uint32_t* bounds);

/* One bucket of oracle_merge: bucket j's merged indices into out (returns how many). */
uint32_t oracle_merge_bucket(const uint8_t* chars, const uint64_t* offs, const uint32_t* lens,
                             const uint32_t* trunc, const uint32_t* run_perm, uint32_t n, uint32_t p,
                             const uint32_t* bounds, uint32_t j, uint32_t* out);

/* The whole pipeline (local sorts, doubling, string-based sampling with v,
 * splitters, bounds, merge of the approx-truncated strings) on nthreads host
 * threads: partitions, key ranges and buckets are shared out among them.  Every
 * step calls the single-threaded functions above on its share, so the outputs
 * equal theirs.  Returns 0, or -1 if a thread could not be started. */
int oracle_pdms_parallel(const uint8_t* chars, const uint64_t* offs, const uint32_t* lens, uint32_t n,
                         uint32_t p, uint32_t v, uint32_t kmin, uint32_t kmax, uint64_t seed, uint32_t nthreads,
                         uint32_t* out_perm, uint32_t* out_lcp, uint32_t* out_approx);

/* Merge: bucket j = concatenation over runs i of run_i[bounds[i][j], bounds[i][j+1]);
 * each bucket is merged by repeatedly taking the smallest head (ties: lower run);
 * buckets are emitted in order.  out_lcp is the full-string LCP array. */
void oracle_merge(const uint8_t* chars, const uint64_t* offs, const uint32_t* lens,
                  const uint32_t* trunc, const uint32_t* run_perm, uint32_t n, uint32_t p,
                  const uint32_t* bounds, uint32_t* out_perm, uint32_t* out_lcp);

/* Check a claimed sorted order: returns n if perm is sorted by oracle_cmp with
 * lcp[r] == lcp(perm[r-1], perm[r]) and lcp[0] == 0, else the first bad rank.
 * (Does not check that perm is a permutation.) */
uint32_t oracle_check_sorted(const uint8_t* chars, const uint64_t* offs, const uint32_t* lens,
                             const uint32_t* perm, const uint32_t* lcp, uint32_t n);

#ifdef __cplusplus
}
#endif
#endif
