/*
 * cpu_engine.c -- a multi-core CPU PIR read engine in the style of the
 * paper's CPU server (Section 9.2: the CPU engine streams the database once
 * per batch of reads and is bound by the memory bus).  It is a reported
 * baseline only, timed by the benchmark beside the oracle; it is not an
 * oracle (the tests check it against oracle_read) and not part of the
 * library.  It shares no code with the oracle or the CUDA library.
 *
 * cpu_engine_read_batch: for B requests (rows of ceil(n/64) words, bit k of
 * a row selects bucket k, LSB first) the replies out[b] = XOR of the buckets
 * row b selects (Section 2, step 5).  The buckets are split into contiguous
 * ranges, one per thread (pthreads); a thread reads its range once for the
 * whole batch, 64 buckets at a time, and XORs every bucket into every
 * request's partial reply under an all-ones / all-zeros mask (every bucket
 * is touched for every request, as the server must), then the threads'
 * partial replies are XOR-combined.
 */
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    const uint64_t *table; /* n rows of row_w words */
    const uint64_t *req;   /* B rows of words64 words */
    uint64_t n, row_w, words64;
    uint32_t B;
    uint64_t k0, k1;       /* this thread's buckets */
    uint64_t *acc;         /* B x row_w partial replies */
} engine_job;

enum { ROWS_PER_BLOCK = 64 };

static void *engine_worker(void *arg) {
    engine_job *j = (engine_job *)arg;
    const uint64_t rw = j->row_w;
    memset(j->acc, 0, (size_t)j->B * rw * 8);
    for (uint64_t kb = j->k0; kb < j->k1; kb += ROWS_PER_BLOCK) {
        const uint64_t ke = kb + ROWS_PER_BLOCK < j->k1 ? kb + ROWS_PER_BLOCK : j->k1;
        /* the block of rows stays in cache while every request consumes it */
        for (uint32_t b = 0; b < j->B; b++) {
            const uint64_t *q = j->req + (uint64_t)b * j->words64;
            uint64_t *a = j->acc + (uint64_t)b * rw;
            for (uint64_t k = kb; k < ke; k++) {
                const uint64_t m = (uint64_t)0 - ((q[k >> 6] >> (k & 63)) & 1u);
                const uint64_t *r = j->table + k * rw;
                for (uint64_t w = 0; w < rw; w++) a[w] ^= r[w] & m;
            }
        }
    }
    return NULL;
}

typedef struct {
    uint64_t **accs;
    uint32_t parts;
    uint64_t w0, w1;
    uint64_t *out;
} combine_job;

static void *combine_worker(void *arg) {
    combine_job *c = (combine_job *)arg;
    for (uint64_t w = c->w0; w < c->w1; w++) {
        uint64_t v = 0;
        for (uint32_t t = 0; t < c->parts; t++) v ^= c->accs[t][w];
        c->out[w] = v;
    }
    return NULL;
}

/* Returns 0, or -1 on bad arguments / allocation failure.  row_bytes must be
 * a multiple of 8; table and out 8-byte aligned. */
int cpu_engine_read_batch(const uint8_t *table, uint64_t n, uint64_t row_bytes,
                          const uint64_t *req, uint32_t B, uint8_t *out, uint32_t threads) {
    if (!table || !req || !out || row_bytes % 8 || n == 0 || threads == 0) return -1;
    if (B == 0) return 0;
    const uint64_t rw = row_bytes / 8, words64 = (n + 63) / 64;
    if ((uint64_t)threads > n) threads = (uint32_t)n;
    engine_job *jobs = calloc(threads, sizeof(engine_job));
    pthread_t *tid = calloc(threads, sizeof(pthread_t));
    uint64_t **accs = calloc(threads, sizeof(uint64_t *));
    int rc = (jobs && tid && accs) ? 0 : -1;
    for (uint32_t t = 0; t < threads && rc == 0; t++) {
        accs[t] = aligned_alloc(64, ((size_t)B * rw * 8 + 63) / 64 * 64);
        if (!accs[t]) rc = -1;
    }
    uint32_t started = 0;
    for (uint32_t t = 0; t < threads && rc == 0; t++) {
        /* whole blocks of 64 buckets per thread */
        const uint64_t blocks = (n + ROWS_PER_BLOCK - 1) / ROWS_PER_BLOCK;
        const uint64_t b0 = blocks * t / threads, b1 = blocks * (t + 1) / threads;
        jobs[t] = (engine_job){(const uint64_t *)table, req, n, rw, words64, B,
                               b0 * ROWS_PER_BLOCK, b1 * ROWS_PER_BLOCK < n ? b1 * ROWS_PER_BLOCK : n,
                               accs[t]};
        if (pthread_create(&tid[t], NULL, engine_worker, &jobs[t]) != 0) {
            rc = -1;
            break;
        }
        started++;
    }
    for (uint32_t t = 0; t < started; t++) pthread_join(tid[t], NULL);
    if (rc == 0) {
        combine_job *cj = calloc(threads, sizeof(combine_job));
        const uint64_t total = (uint64_t)B * rw;
        if (!cj) rc = -1;
        started = 0;
        for (uint32_t t = 0; t < threads && rc == 0; t++) {
            cj[t] = (combine_job){accs, threads, total * t / threads, total * (t + 1) / threads,
                                  (uint64_t *)out};
            if (pthread_create(&tid[t], NULL, combine_worker, &cj[t]) != 0) {
                rc = -1;
                break;
            }
            started++;
        }
        for (uint32_t t = 0; t < started; t++) pthread_join(tid[t], NULL);
        free(cj);
    }
    for (uint32_t t = 0; accs && t < threads; t++) free(accs[t]);
    free(accs);
    free(tid);
    free(jobs);
    return rc;
}
