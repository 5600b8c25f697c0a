/*
 * The oracle's pipeline on all host cores: TEST INFRASTRUCTURE AND CPU
 * BASELINE ONLY (see oracle.h).  Nothing here defines a result: every step
 * hands a share of the work (a partition, a slice of the active strings, a
 * range of hash keys or a bucket) to one of nthreads POSIX threads, and each
 * share is computed by the single-threaded oracle functions, so the outputs
 * equal those of the plain pipeline.
 *
 * Steps (Sections 3 and 4): local sort and LCP array of every partition,
 * prefix doubling (Section 4, appendix on doubling), string-based sampling
 * (Section 3.1.1), splitters, bucket bounds (Section 3 step 1) and the merge of
 * every bucket (Section 3 step 3) on the approx-truncated strings.
 */
#include <pthread.h>
#include <stdlib.h>
#include <string.h>

#include "oracle.h"

typedef struct {
    const uint8_t* chars;
    const uint64_t* offs;
    const uint32_t* lens;
    uint32_t n, p, nthreads;
    uint64_t seed;
    /* local sort */
    uint32_t* run_perm;
    uint32_t* run_lcp;
    /* doubling round */
    const uint32_t* active;
    uint32_t na;
    uint32_t L;
    uint64_t* key;
    uint8_t* retire;
    /* bounds and merge */
    const uint32_t* approx;
    const uint32_t* splitters;
    uint32_t* bounds;
    const uint32_t* bucket_off;
    uint32_t* out_perm;
    uint32_t* out_lcp;
} par_job;

typedef struct {
    par_job* job;
    uint32_t t;
} par_arg;

static int run_threads(par_job* job, void* (*fn)(void*)) {
    uint32_t T = job->nthreads;
    pthread_t* th = (pthread_t*)malloc(sizeof(pthread_t) * T);
    par_arg* args = (par_arg*)malloc(sizeof(par_arg) * T);
    uint32_t started = 0;
    int rc = 0;
    for (uint32_t t = 0; t < T; ++t) {
        args[t].job = job;
        args[t].t = t;
        if (pthread_create(&th[t], NULL, fn, &args[t]) != 0) {
            rc = -1;
            break;
        }
        ++started;
    }
    for (uint32_t t = 0; t < started; ++t) pthread_join(th[t], NULL);
    free(th);
    free(args);
    return rc;
}

/* partition i = t, t + T, ...: sort its run and take its LCP array */
static void* local_sort_worker(void* a) {
    par_arg* pa = (par_arg*)a;
    par_job* j = pa->job;
    for (uint32_t i = pa->t; i < j->p; i += j->nthreads) {
        uint32_t lo = oracle_part_lo(j->n, j->p, i), hi = oracle_part_lo(j->n, j->p, i + 1);
        for (uint32_t q = lo; q < hi; ++q) j->run_perm[q] = q;
        oracle_sort_idx(j->chars, j->offs, j->lens, NULL, j->run_perm + lo, hi - lo);
        oracle_lcp_array(j->chars, j->offs, j->lens, NULL, j->run_perm + lo, hi - lo, j->run_lcp + lo);
    }
    return NULL;
}

/* a contiguous slice of the active strings: their keys of the L_eff-prefix */
static void* key_worker(void* a) {
    par_arg* pa = (par_arg*)a;
    par_job* j = pa->job;
    uint32_t lo = (uint32_t)(((uint64_t)pa->t * j->na) / j->nthreads);
    uint32_t hi = (uint32_t)(((uint64_t)(pa->t + 1) * j->na) / j->nthreads);
    for (uint32_t x = lo; x < hi; ++x) {
        uint32_t i = j->active[x];
        uint32_t le = j->L < j->lens[i] ? j->L : j->lens[i];
        j->key[x] = oracle_prefix_key(j->chars, j->offs, j->lens, i, le, j->seed);
    }
    return NULL;
}

static int cmp_u64p(const void* x, const void* y) {
    uint64_t a = *(const uint64_t*)x, b = *(const uint64_t*)y;
    return a < b ? -1 : (a > b ? 1 : 0);
}

/* the keys with key mod T == t: sorted, counted; a string retires when its key
 * occurs once among the active strings or its whole length has been tested */
static void* count_worker(void* a) {
    par_arg* pa = (par_arg*)a;
    par_job* j = pa->job;
    uint32_t T = j->nthreads, m = 0;
    for (uint32_t x = 0; x < j->na; ++x)
        if (j->key[x] % T == pa->t) ++m;
    uint64_t* mine = (uint64_t*)malloc(sizeof(uint64_t) * (m ? m : 1));
    m = 0;
    for (uint32_t x = 0; x < j->na; ++x)
        if (j->key[x] % T == pa->t) mine[m++] = j->key[x];
    qsort(mine, m, sizeof(uint64_t), cmp_u64p);
    for (uint32_t x = 0; x < j->na; ++x) {
        if (j->key[x] % T != pa->t) continue;
        uint64_t k = j->key[x];
        uint32_t lo = 0, hi = m; /* lower bound, then count the equal run */
        while (lo < hi) {
            uint32_t mid = lo + (hi - lo) / 2;
            if (mine[mid] < k) lo = mid + 1; else hi = mid;
        }
        uint32_t c = 0;
        while (lo + c < m && mine[lo + c] == k) ++c;
        j->retire[x] = (c == 1 || j->lens[j->active[x]] <= j->L) ? 1 : 0;
    }
    free(mine);
    return NULL;
}

static void* bounds_worker(void* a) {
    par_arg* pa = (par_arg*)a;
    par_job* j = pa->job;
    for (uint32_t i = pa->t; i < j->p; i += j->nthreads)
        oracle_bounds_row(j->chars, j->offs, j->lens, j->approx, j->run_perm, j->n, j->p, j->splitters, i,
                          j->bounds);
    return NULL;
}

static void* merge_worker(void* a) {
    par_arg* pa = (par_arg*)a;
    par_job* j = pa->job;
    for (uint32_t b = pa->t; b < j->p; b += j->nthreads)
        oracle_merge_bucket(j->chars, j->offs, j->lens, j->approx, j->run_perm, j->n, j->p, j->bounds, b,
                            j->out_perm + j->bucket_off[b]);
    return NULL;
}

/* lcp[r] = lcp(perm[r-1], perm[r]) of the full strings over a slice of ranks */
static void* lcp_worker(void* a) {
    par_arg* pa = (par_arg*)a;
    par_job* j = pa->job;
    uint32_t lo = (uint32_t)(((uint64_t)pa->t * j->n) / j->nthreads);
    uint32_t hi = (uint32_t)(((uint64_t)(pa->t + 1) * j->n) / j->nthreads);
    for (uint32_t r = lo; r < hi; ++r)
        j->out_lcp[r] = r == 0 ? 0 : oracle_lcp_pair(j->chars, j->offs, j->lens, NULL, j->out_perm[r - 1],
                                                     j->out_perm[r]);
    return NULL;
}

int oracle_pdms_parallel(const uint8_t* chars, const uint64_t* offs, const uint32_t* lens, uint32_t n,
                         uint32_t p, uint32_t v, uint32_t kmin, uint32_t kmax, uint64_t seed, uint32_t nthreads,
                         uint32_t* out_perm, uint32_t* out_lcp, uint32_t* out_approx) {
    if (nthreads == 0) nthreads = 1;
    par_job j;
    memset(&j, 0, sizeof(j));
    j.chars = chars;
    j.offs = offs;
    j.lens = lens;
    j.n = n;
    j.p = p;
    j.nthreads = nthreads;
    j.seed = seed;
    size_t nn = n ? n : 1;
    j.run_perm = (uint32_t*)malloc(nn * sizeof(uint32_t));
    j.run_lcp = (uint32_t*)malloc(nn * sizeof(uint32_t));
    uint32_t* active = (uint32_t*)malloc(nn * sizeof(uint32_t));
    j.key = (uint64_t*)malloc(nn * sizeof(uint64_t));
    j.retire = (uint8_t*)malloc(nn);
    uint32_t* smp = (uint32_t*)malloc(sizeof(uint32_t) * ((size_t)p * (v + 1) + 1));
    uint32_t* spl = (uint32_t*)malloc(sizeof(uint32_t) * (p + 1));
    j.bounds = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)p * (p + 1));
    uint32_t* boff = (uint32_t*)malloc(sizeof(uint32_t) * (p + 1));
    int rc = 0;

    /* 1. local sort of every partition */
    rc |= run_threads(&j, local_sort_worker);

    /* 2. prefix doubling, round by round over the active strings */
    uint32_t na = n;
    for (uint32_t i = 0; i < n; ++i) active[i] = i;
    for (uint32_t k = kmin; k <= kmax && na > 0 && rc == 0; ++k) {
        j.active = active;
        j.na = na;
        j.L = k >= 32 ? UINT32_MAX : (uint32_t)(1ull << k);
        rc |= run_threads(&j, key_worker);
        rc |= run_threads(&j, count_worker);
        uint32_t keep = 0;
        for (uint32_t x = 0; x < na; ++x) {
            uint32_t i = active[x];
            if (j.retire[x]) out_approx[i] = j.L < lens[i] ? j.L : lens[i];
            else active[keep++] = i;
        }
        na = keep;
    }
    for (uint32_t x = 0; x < na; ++x) out_approx[active[x]] = lens[active[x]];

    /* 3. samples and splitters (p (v+1) strings: one thread) */
    uint32_t ns = oracle_samples(j.run_perm, n, p, v, smp);
    oracle_splitters(chars, offs, lens, out_approx, smp, ns, p, spl);

    /* 4. bucket bounds per run, 5. merge per bucket, then the LCP array */
    j.approx = out_approx;
    j.splitters = spl;
    if (rc == 0) rc |= run_threads(&j, bounds_worker);
    uint32_t o = 0;
    for (uint32_t b = 0; b < p; ++b) {
        boff[b] = o;
        for (uint32_t i = 0; i < p; ++i)
            o += j.bounds[(size_t)i * (p + 1) + b + 1] - j.bounds[(size_t)i * (p + 1) + b];
    }
    boff[p] = o;
    j.bucket_off = boff;
    j.out_perm = out_perm;
    j.out_lcp = out_lcp;
    if (rc == 0) rc |= run_threads(&j, merge_worker);
    if (rc == 0) rc |= run_threads(&j, lcp_worker);

    free(j.run_perm);
    free(j.run_lcp);
    free(active);
    free(j.key);
    free(j.retire);
    free(smp);
    free(spl);
    free(j.bounds);
    free(boff);
    return rc ? -1 : 0;
}
