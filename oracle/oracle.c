/*
 * CPU oracle for the string sorter: TEST INFRASTRUCTURE ONLY (see oracle.h).
 *
 * Every function is the plain definition (or the paper's procedure in the
 * paper's order) with no blocking, fusion or reordering.  Citations name the
 * paper's section / lemma / appendix the function follows.
 *
 * The paper only asks for a random hash function; this file fixes one by its
 * definition (Karp-Rabin polynomial over P = 2^61-1 with a SplitMix64
 * finaliser).  Its values are pinned by inverting the finaliser and checking
 * the polynomial, its closed forms and its linearity; everything else is pinned
 * by the tests as well.
 */
#include "oracle.h"

#include <stdlib.h>
#include <string.h>

#define ORACLE_P ((1ULL << 61) - 1)
#define ORACLE_GAMMA 0x9E3779B97F4A7C15ULL

/* ---------------------------------------------------------------------------
 * String comparison and LCP (Section 2, "String Properties and Input Format"):
 * strings end with a sentinel that is smaller than every character, so a proper
 * prefix sorts first; the LCP of s and t is the first index where they differ.
 * ------------------------------------------------------------------------- */

static uint32_t view_len(const uint32_t* lens, const uint32_t* trunc, uint32_t i) {
    return trunc ? trunc[i] : lens[i];
}

int oracle_cmp_str(const uint8_t* chars, const uint64_t* offs, const uint32_t* lens,
                   const uint32_t* trunc, uint32_t a, uint32_t b) {
    const uint8_t* sa = chars + offs[a];
    const uint8_t* sb = chars + offs[b];
    uint32_t la = view_len(lens, trunc, a), lb = view_len(lens, trunc, b);
    uint32_t m = la < lb ? la : lb;
    for (uint32_t k = 0; k < m; ++k) {
        if (sa[k] != sb[k]) return sa[k] < sb[k] ? -1 : 1;
    }
    if (la != lb) return la < lb ? -1 : 1;
    return 0;
}

int oracle_cmp(const uint8_t* chars, const uint64_t* offs, const uint32_t* lens,
               const uint32_t* trunc, uint32_t a, uint32_t b) {
    int c = oracle_cmp_str(chars, offs, lens, trunc, a, b);
    if (c != 0) return c;
    if (a == b) return 0;
    return a < b ? -1 : 1; /* equal strings: lower input index first */
}

uint32_t oracle_lcp_pair(const uint8_t* chars, const uint64_t* offs, const uint32_t* lens,
                         const uint32_t* trunc, uint32_t a, uint32_t b) {
    const uint8_t* sa = chars + offs[a];
    const uint8_t* sb = chars + offs[b];
    uint32_t la = view_len(lens, trunc, a), lb = view_len(lens, trunc, b);
    uint32_t m = la < lb ? la : lb;
    uint32_t k = 0;
    while (k < m && sa[k] == sb[k]) ++k;
    return k;
}

/* ---------------------------------------------------------------------------
 * Sorting: a plain top-down merge sort of indices under oracle_cmp.  Local
 * sorting of each PE's array is the initialization step of Section 3.
 * ------------------------------------------------------------------------- */

typedef struct {
    const uint8_t* chars;
    const uint64_t* offs;
    const uint32_t* lens;
    const uint32_t* trunc;
} str_ctx;

static void msort_rec(const str_ctx* c, uint32_t* a, uint32_t* tmp, uint32_t m) {
    if (m < 2) return;
    uint32_t h = m / 2;
    msort_rec(c, a, tmp, h);
    msort_rec(c, a + h, tmp, m - h);
    uint32_t i = 0, j = h, k = 0;
    while (i < h && j < m) {
        if (oracle_cmp(c->chars, c->offs, c->lens, c->trunc, a[j], a[i]) < 0)
            tmp[k++] = a[j++];
        else
            tmp[k++] = a[i++];
    }
    while (i < h) tmp[k++] = a[i++];
    while (j < m) tmp[k++] = a[j++];
    memcpy(a, tmp, (size_t)m * sizeof(uint32_t));
}

void oracle_sort_idx(const uint8_t* chars, const uint64_t* offs, const uint32_t* lens,
                     const uint32_t* trunc, uint32_t* idx, uint32_t m) {
    if (m < 2) return;
    str_ctx c = {chars, offs, lens, trunc};
    uint32_t* tmp = (uint32_t*)malloc((size_t)m * sizeof(uint32_t));
    msort_rec(&c, idx, tmp, m);
    free(tmp);
}

void oracle_sort(const uint8_t* chars, const uint64_t* offs, const uint32_t* lens,
                 uint32_t n, uint32_t* perm) {
    for (uint32_t i = 0; i < n; ++i) perm[i] = i;
    oracle_sort_idx(chars, offs, lens, NULL, perm, n);
}

/* LCP array (Section 2): [bot, h_1, ..., h_{n-1}] with h_r = lcp(s_{r-1}, s_r);
 * the undefined first entry is stored as 0. */
void oracle_lcp_array(const uint8_t* chars, const uint64_t* offs, const uint32_t* lens,
                      const uint32_t* trunc, const uint32_t* perm, uint32_t m, uint32_t* lcp) {
    if (m == 0) return;
    lcp[0] = 0;
    for (uint32_t r = 1; r < m; ++r) lcp[r] = oracle_lcp_pair(chars, offs, lens, trunc, perm[r - 1], perm[r]);
}

/* Distinguishing prefix (Section 2): the characters needed to rank s, i.e. one
 * more than its largest LCP with a sorted neighbour, capped at its length. */
void oracle_dist(const uint32_t* lens, uint32_t n, const uint32_t* perm, const uint32_t* lcp,
                 uint32_t* dist) {
    for (uint32_t r = 0; r < n; ++r) {
        uint32_t left = r > 0 ? lcp[r] : 0;
        uint32_t right = r + 1 < n ? lcp[r + 1] : 0;
        uint32_t m = left > right ? left : right;
        uint64_t d = (uint64_t)m + 1;
        uint32_t i = perm[r];
        dist[i] = d < lens[i] ? (uint32_t)d : lens[i];
    }
}

/* ---------------------------------------------------------------------------
 * Prefix hashing for duplicate detection (Section 4 and the appendix
 * "Distributed Duplicate Detection": prefixes are hashed with a random hash
 * function and equal hash values flag duplicates).
 *
 * Definition used here: P = 2^61 - 1, B = 2 + (SplitMix64(seed) mod (P - 3)).
 * The first l characters form big-endian 64-bit words over [8j, 8j+8), bytes at
 * or past l are zero; each word is folded as its high then its low 32-bit limb,
 * h <- (h*B + limb) mod P, from h = 0.  key = smix(h XOR (l * G)).
 * ------------------------------------------------------------------------- */

static uint64_t smix(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

uint64_t oracle_splitmix64_first(uint64_t s) { return smix(s + ORACLE_GAMMA); }

uint64_t oracle_mulmod61(uint64_t a, uint64_t b) {
    unsigned __int128 x = (unsigned __int128)a * b;
    return (uint64_t)(x % ORACLE_P);
}

static uint64_t addmod61(uint64_t a, uint64_t b) {
    unsigned __int128 x = (unsigned __int128)a + b;
    return (uint64_t)(x % ORACLE_P);
}

uint64_t oracle_hash_base(uint64_t seed) { return 2 + oracle_splitmix64_first(seed) % (ORACLE_P - 3); }

uint64_t oracle_prefix_key(const uint8_t* chars, const uint64_t* offs, const uint32_t* lens,
                           uint32_t i, uint32_t l, uint64_t seed) {
    (void)lens;
    const uint8_t* s = chars + offs[i];
    uint64_t B = oracle_hash_base(seed);
    uint64_t h = 0;
    uint32_t nw = (l + 7) / 8;
    for (uint32_t j = 0; j < nw; ++j) {
        uint64_t w = 0;
        for (uint32_t b = 0; b < 8; ++b) {
            uint32_t pos = 8 * j + b;
            uint64_t c = pos < l ? s[pos] : 0;
            w = (w << 8) | c;
        }
        h = addmod61(oracle_mulmod61(h, B), w >> 32);
        h = addmod61(oracle_mulmod61(h, B), w & 0xFFFFFFFFULL);
    }
    return smix(h ^ ((uint64_t)l * ORACLE_GAMMA));
}

static int cmp_u64(const void* x, const void* y) {
    uint64_t a = *(const uint64_t*)x, b = *(const uint64_t*)y;
    return a < b ? -1 : (a > b ? 1 : 0);
}

static uint32_t count_key(const uint64_t* sorted, uint32_t m, uint64_t key) {
    uint32_t lo = 0, hi = m; /* lower bound */
    while (lo < hi) {
        uint32_t mid = lo + (hi - lo) / 2;
        if (sorted[mid] < key) lo = mid + 1; else hi = mid;
    }
    uint32_t c = 0;
    while (lo + c < m && sorted[lo + c] == key) ++c;
    return c;
}

/* Prefix doubling (Section 4; l_init and doubling in the appendix "Distinguishing
 * Prefix Approximation via Doubling"): round k tests prefixes of length L = 2^k
 * (L_eff = min(L, len)) of the still-active strings; a string whose key occurs
 * once among the active strings has a unique L-prefix, so dist <= L_eff and it
 * retires with approx = L_eff; a string with len <= L also retires (its whole
 * string has been tested).  Strings still active after round kmax get approx = len.
 * Duplicate detection follows the appendix's sort-based route: sort the keys and
 * count equal neighbours. */
void oracle_doubling(const uint8_t* chars, const uint64_t* offs, const uint32_t* lens,
                     uint32_t n, uint32_t kmin, uint32_t kmax, uint64_t seed,
                     uint32_t* approx, uint32_t* rounds_out) {
    uint32_t* active = (uint32_t*)malloc((size_t)(n ? n : 1) * sizeof(uint32_t));
    uint64_t* key = (uint64_t*)malloc((size_t)(n ? n : 1) * sizeof(uint64_t));
    uint64_t* sorted = (uint64_t*)malloc((size_t)(n ? n : 1) * sizeof(uint64_t));
    uint32_t na = n;
    for (uint32_t i = 0; i < n; ++i) active[i] = i;
    if (rounds_out)
        for (uint32_t k = 0; k <= kmax; ++k) rounds_out[k] = 0;
    for (uint32_t k = kmin; k <= kmax && na > 0; ++k) {
        uint64_t L = 1ULL << k;
        if (rounds_out) rounds_out[k] = na;
        for (uint32_t a = 0; a < na; ++a) {
            uint32_t i = active[a];
            uint32_t le = L < lens[i] ? (uint32_t)L : lens[i];
            key[a] = oracle_prefix_key(chars, offs, lens, i, le, seed);
            sorted[a] = key[a];
        }
        qsort(sorted, na, sizeof(uint64_t), cmp_u64);
        uint32_t keep = 0;
        for (uint32_t a = 0; a < na; ++a) {
            uint32_t i = active[a];
            uint32_t le = L < lens[i] ? (uint32_t)L : lens[i];
            uint32_t c = count_key(sorted, na, key[a]);
            if (c == 1 || lens[i] <= L) {
                approx[i] = le;
            } else {
                active[keep++] = i;
            }
        }
        na = keep;
    }
    for (uint32_t a = 0; a < na; ++a) approx[active[a]] = lens[active[a]];
    free(active);
    free(key);
    free(sorted);
}

/* ---------------------------------------------------------------------------
 * Partitions (Section 2: PE i holds a contiguous subarray S_i of S).
 * ------------------------------------------------------------------------- */

uint32_t oracle_part_lo(uint32_t n, uint32_t p, uint32_t i) {
    return (uint32_t)(((uint64_t)i * n) / p);
}

void oracle_local_sort(const uint8_t* chars, const uint64_t* offs, const uint32_t* lens,
                       const uint32_t* trunc, uint32_t n, uint32_t p,
                       uint32_t* run_perm, uint32_t* run_lcp) {
    for (uint32_t i = 0; i < p; ++i) {
        uint32_t lo = oracle_part_lo(n, p, i), hi = oracle_part_lo(n, p, i + 1);
        for (uint32_t q = lo; q < hi; ++q) run_perm[q] = q;
        oracle_sort_idx(chars, offs, lens, trunc, run_perm + lo, hi - lo);
        oracle_lcp_array(chars, offs, lens, trunc, run_perm + lo, hi - lo, run_lcp + lo);
    }
}

/* String-based regular sampling (Section 3.1.1 "Local Sampling"): with equal
 * partitions every PE draws v+1 evenly spaced samples; the reading used here
 * takes local ranks ceil(t*n_i/(v+1)) - 1 for t = 1..v+1, so at most
 * omega = n_i/(v+1) strings lie between consecutive samples. */
uint32_t oracle_samples(const uint32_t* run_perm, uint32_t n, uint32_t p, uint32_t v,
                        uint32_t* samples_out) {
    uint32_t ns = 0;
    for (uint32_t i = 0; i < p; ++i) {
        uint32_t lo = oracle_part_lo(n, p, i), hi = oracle_part_lo(n, p, i + 1);
        uint64_t ni = hi - lo;
        if (ni == 0) continue;
        for (uint64_t t = 1; t <= (uint64_t)v + 1; ++t) {
            uint64_t rank = (t * ni + v) / (v + 1) - 1; /* ceil(t*ni/(v+1)) - 1 */
            samples_out[ns++] = run_perm[lo + rank];
        }
    }
    return ns;
}

/* Character-based regular sampling (Section 3.1.2; appendix "Character Based
 * Sampling").  Sampling distance w = N / (p (v+1)) with N the total number of
 * (truncated) characters of all partitions.  Partition i, whose sorted run has
 * C_i characters, draws ceil(C_i / w) - 1 samples at the character positions
 * floor(t * w), t = 1, 2, ..., of its run's character array (the run's strings
 * concatenated in sorted order); each position is moved back to the start of
 * the string holding it, i.e. the sample is that string.  If all partitions
 * together draw fewer than p (v+1) samples, the first non-empty partitions draw
 * one additional sample each, their last string, until there are p (v+1).
 * With N = 0 (no characters at all) this falls back to oracle_samples.
 * Integer arithmetic: ceil(C_i p (v+1) / N) - 1 and floor(t N / (p (v+1))).
 * samples_out: up to p*(v+1) indices (returns the count). */
uint32_t oracle_samples_char(const uint32_t* lens, const uint32_t* trunc, const uint32_t* run_perm, uint32_t n,
                             uint32_t p, uint32_t v, uint32_t* samples_out) {
    const uint64_t want = (uint64_t)p * (v + 1);
    uint64_t N = 0;
    for (uint32_t q = 0; q < n; ++q) N += trunc ? trunc[q] : lens[q];
    if (N == 0) return oracle_samples(run_perm, n, p, v, samples_out);
    uint32_t ns = 0;
    uint64_t total = 0;
    for (uint32_t i = 0; i < p; ++i) {  /* how many each partition draws */
        uint32_t lo = oracle_part_lo(n, p, i), hi = oracle_part_lo(n, p, i + 1);
        uint64_t Ci = 0;
        for (uint32_t q = lo; q < hi; ++q) Ci += trunc ? trunc[run_perm[q]] : lens[run_perm[q]];
        uint64_t cnt = (Ci * want + N - 1) / N;  /* ceil(C_i / w) */
        total += cnt ? cnt - 1 : 0;
    }
    uint64_t extra = total < want ? want - total : 0;
    for (uint32_t i = 0; i < p; ++i) {
        uint32_t lo = oracle_part_lo(n, p, i), hi = oracle_part_lo(n, p, i + 1);
        if (hi == lo) continue;
        uint64_t Ci = 0;
        for (uint32_t q = lo; q < hi; ++q) Ci += trunc ? trunc[run_perm[q]] : lens[run_perm[q]];
        uint64_t cnt = (Ci * want + N - 1) / N;
        cnt = cnt ? cnt - 1 : 0;
        for (uint64_t t = 1; t <= cnt; ++t) {
            uint64_t x = (t * N) / want;  /* character position floor(t w) in the run */
            /* the string of the run whose characters contain position x */
            uint64_t start = 0;
            for (uint32_t q = lo; q < hi; ++q) {
                uint64_t len = trunc ? trunc[run_perm[q]] : lens[run_perm[q]];
                if (x < start + len) {
                    samples_out[ns++] = run_perm[q];
                    break;
                }
                start += len;
            }
        }
        if (extra > 0) {
            samples_out[ns++] = run_perm[hi - 1];
            --extra;
        }
    }
    return ns;
}

/* Splitter computation (Section 3.1.1): sort the samples, then
 * f_j = V[j*|V|/r - 1] for 0 < j < r (here r = p).  When |V| is not a multiple of
 * p the index is floor(j*|V|/p) - 1; a negative index means f_j = minus infinity
 * (stored as UINT32_MAX). */
void oracle_splitters(const uint8_t* chars, const uint64_t* offs, const uint32_t* lens,
                      const uint32_t* trunc, uint32_t* samples, uint32_t ns, uint32_t p,
                      uint32_t* splitters_out) {
    oracle_sort_idx(chars, offs, lens, trunc, samples, ns);
    for (uint32_t j = 1; j < p; ++j) {
        int64_t k = (int64_t)(((uint64_t)j * ns) / p) - 1;
        splitters_out[j - 1] = k < 0 ? UINT32_MAX : samples[k];
    }
}

/* Buckets (Section 3, step 1): B_i^j = { s in S_i : f_j < s <= f_{j+1} } with
 * f_0 = -inf and f_p = +inf; bounds[i][j] counts the strings of run i that are
 * <= f_j (string order only, so equal strings share a bucket). */
void oracle_bounds_row(const uint8_t* chars, const uint64_t* offs, const uint32_t* lens,
                       const uint32_t* trunc, const uint32_t* run_perm, uint32_t n, uint32_t p,
                       const uint32_t* splitters, uint32_t i, uint32_t* bounds) {
    uint32_t lo = oracle_part_lo(n, p, i), hi = oracle_part_lo(n, p, i + 1);
    uint32_t* b = bounds + (size_t)i * (p + 1);
    b[0] = 0;
    b[p] = hi - lo;
    for (uint32_t j = 1; j < p; ++j) {
        uint32_t f = splitters[j - 1];
        uint32_t c = 0;
        if (f != UINT32_MAX) {
            for (uint32_t q = lo; q < hi; ++q)
                if (oracle_cmp_str(chars, offs, lens, trunc, run_perm[q], f) <= 0) ++c;
        }
        b[j] = c;
    }
}

void oracle_bounds(const uint8_t* chars, const uint64_t* offs, const uint32_t* lens,
                   const uint32_t* trunc, const uint32_t* run_perm, uint32_t n, uint32_t p,
                   const uint32_t* splitters, uint32_t* bounds) {
    for (uint32_t i = 0; i < p; ++i) oracle_bounds_row(chars, offs, lens, trunc, run_perm, n, p, splitters, i, bounds);
}

/* Merging (Section 3, step 3): each bucket receives one sorted piece from every
 * run; the pieces are merged (here by repeatedly taking the smallest head, the
 * lower run winning ties) and the buckets are concatenated in order. */
uint32_t oracle_merge_bucket(const uint8_t* chars, const uint64_t* offs, const uint32_t* lens,
                             const uint32_t* trunc, const uint32_t* run_perm, uint32_t n, uint32_t p,
                             const uint32_t* bounds, uint32_t j, uint32_t* out) {
    uint32_t* head = (uint32_t*)malloc((size_t)p * sizeof(uint32_t));
    uint32_t* end = (uint32_t*)malloc((size_t)p * sizeof(uint32_t));
    uint32_t o = 0;
    for (uint32_t i = 0; i < p; ++i) {
        uint32_t lo = oracle_part_lo(n, p, i);
        head[i] = lo + bounds[(size_t)i * (p + 1) + j];
        end[i] = lo + bounds[(size_t)i * (p + 1) + j + 1];
    }
    for (;;) {
        int best = -1;
        for (uint32_t i = 0; i < p; ++i) {
            if (head[i] >= end[i]) continue;
            if (best < 0 ||
                oracle_cmp_str(chars, offs, lens, trunc, run_perm[head[i]], run_perm[head[best]]) < 0)
                best = (int)i;
        }
        if (best < 0) break;
        out[o++] = run_perm[head[best]++];
    }
    free(head);
    free(end);
    return o;
}

void oracle_merge(const uint8_t* chars, const uint64_t* offs, const uint32_t* lens,
                  const uint32_t* trunc, const uint32_t* run_perm, uint32_t n, uint32_t p,
                  const uint32_t* bounds, uint32_t* out_perm, uint32_t* out_lcp) {
    uint32_t o = 0;
    for (uint32_t j = 0; j < p; ++j)
        o += oracle_merge_bucket(chars, offs, lens, trunc, run_perm, n, p, bounds, j, out_perm + o);
    oracle_lcp_array(chars, offs, lens, NULL, out_perm, o, out_lcp);
}

uint32_t oracle_check_sorted(const uint8_t* chars, const uint64_t* offs, const uint32_t* lens,
                             const uint32_t* perm, const uint32_t* lcp, uint32_t n) {
    if (n == 0) return 0;
    if (lcp[0] != 0) return 0;
    for (uint32_t r = 1; r < n; ++r) {
        if (oracle_cmp(chars, offs, lens, NULL, perm[r - 1], perm[r]) >= 0) return r;
        if (lcp[r] != oracle_lcp_pair(chars, offs, lens, NULL, perm[r - 1], perm[r])) return r;
    }
    return n;
}
