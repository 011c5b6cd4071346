/*
 * oracle.c -- plain CPU reference for Talek's server side (arxiv 2001.08250).
 *
 * TEST INFRASTRUCTURE ONLY: used by the tests, the smoke check and the
 * benchmark's CPU-baseline leg to check the CUDA library.  It is scalar,
 * single-threaded and written to be read against the paper, not to be fast.
 *
 *   oracle_read           Section 2, step 5 (server answer of Chor et al.'s IT-PIR)
 *   oracle_reconstruct    Section 2, step 6 (client XOR of the l replies)
 *   oracle_mask           Section 6, step 6 (one-time mask PRNG(p); ChaCha20
 *                         of RFC 8439 taken as the PRNG)
 *   oracle_read_batch_masked  Section 6, step 7 (masked response R XOR P)
 *   oracle_cuckoo_insert  Section 5.3 (blocked cuckoo insertion, FIFO collection)
 *   oracle_bloom_*        Section 7 (interest vectors, global interest vector,
 *                         window of deltas)
 *   oracle_rice_*         Section 7, GetUpdates: compressed deltas (Rice code
 *                         of the gaps between set bits, taken as the encoding)
 */
#include "oracle.h"

#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------ */
/* IT-PIR                                                                    */
/* ------------------------------------------------------------------------ */

static int request_bit(const uint64_t *q, uint64_t k) {
    return (int)((q[k >> 6] >> (k & 63)) & 1u);
}

void oracle_read(const uint8_t *T, uint64_t n, uint32_t d, uint32_t z,
                 const uint64_t *q, uint8_t *out) {
    uint64_t bucket = (uint64_t)d * z;
    for (uint64_t j = 0; j < bucket; j++) out[j] = 0;
    for (uint64_t k = 0; k < n; k++) {
        if (request_bit(q, k)) {
            const uint8_t *row = T + k * bucket;
            for (uint64_t j = 0; j < bucket; j++) out[j] ^= row[j];
        }
    }
}

void oracle_read_batch(const uint8_t *T, uint64_t n, uint32_t d, uint32_t z,
                       const uint64_t *R, uint32_t B, uint8_t *out) {
    uint64_t words = (n + 63) / 64;
    uint64_t bucket = (uint64_t)d * z;
    for (uint32_t b = 0; b < B; b++) oracle_read(T, n, d, z, R + b * words, out + b * bucket);
}

void oracle_reconstruct(const uint8_t *replies, uint32_t l, uint64_t bytes, uint8_t *out) {
    for (uint64_t j = 0; j < bytes; j++) out[j] = 0;
    for (uint32_t i = 0; i < l; i++)
        for (uint64_t j = 0; j < bytes; j++) out[j] ^= replies[i * bytes + j];
}

uint64_t oracle_splitmix64_next(uint64_t *state) {
    *state += 0x9E3779B97F4A7C15ULL;
    uint64_t z = *state;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* ------------------------------------------------------------------------ */
/* Serialized PIR: one-time masks                                            */
/* ------------------------------------------------------------------------ */

static uint32_t rotl32(uint32_t v, int c) { return (v << c) | (v >> (32 - c)); }

static uint32_t load_le32(const uint8_t *p) {
    return (uint32_t)p[0] | ((uint32_t)p[1] << 8) | ((uint32_t)p[2] << 16) | ((uint32_t)p[3] << 24);
}

/* RFC 8439 section 2.1: the quarter round on four words of the state. */
static void quarter_round(uint32_t *x, int a, int b, int c, int d) {
    x[a] += x[b]; x[d] ^= x[a]; x[d] = rotl32(x[d], 16);
    x[c] += x[d]; x[b] ^= x[c]; x[b] = rotl32(x[b], 12);
    x[a] += x[b]; x[d] ^= x[a]; x[d] = rotl32(x[d], 8);
    x[c] += x[d]; x[b] ^= x[c]; x[b] = rotl32(x[b], 7);
}

void oracle_chacha20_block(const uint8_t key[32], uint32_t counter, const uint8_t nonce[12],
                           uint8_t out[64]) {
    /* RFC 8439 section 2.3: state = the four words of "expand 32-byte k",
     * the key, the block counter, the nonce (all little-endian words) */
    uint32_t state[16], x[16];
    state[0] = load_le32((const uint8_t *)"expa");
    state[1] = load_le32((const uint8_t *)"nd 3");
    state[2] = load_le32((const uint8_t *)"2-by");
    state[3] = load_le32((const uint8_t *)"te k");
    for (int i = 0; i < 8; i++) state[4 + i] = load_le32(key + 4 * i);
    state[12] = counter;
    for (int i = 0; i < 3; i++) state[13 + i] = load_le32(nonce + 4 * i);
    for (int i = 0; i < 16; i++) x[i] = state[i];
    /* 20 rounds: ten times a column round then a diagonal round */
    for (int r = 0; r < 10; r++) {
        quarter_round(x, 0, 4, 8, 12);
        quarter_round(x, 1, 5, 9, 13);
        quarter_round(x, 2, 6, 10, 14);
        quarter_round(x, 3, 7, 11, 15);
        quarter_round(x, 0, 5, 10, 15);
        quarter_round(x, 1, 6, 11, 12);
        quarter_round(x, 2, 7, 8, 13);
        quarter_round(x, 3, 4, 9, 14);
    }
    /* add the input state, serialise little-endian */
    for (int i = 0; i < 16; i++) {
        uint32_t v = x[i] + state[i];
        out[4 * i + 0] = (uint8_t)(v & 0xFF);
        out[4 * i + 1] = (uint8_t)((v >> 8) & 0xFF);
        out[4 * i + 2] = (uint8_t)((v >> 16) & 0xFF);
        out[4 * i + 3] = (uint8_t)((v >> 24) & 0xFF);
    }
}

void oracle_mask(const uint8_t seed[32], uint64_t nbytes, uint8_t *out) {
    const uint8_t nonce[12] = {0};
    uint8_t block[64];
    for (uint64_t off = 0; off < nbytes; off += 64) {
        oracle_chacha20_block(seed, (uint32_t)(off / 64), nonce, block);
        for (uint64_t j = 0; j < 64 && off + j < nbytes; j++) out[off + j] = block[j];
    }
}

void oracle_read_batch_masked(const uint8_t *T, uint64_t n, uint32_t d, uint32_t z,
                              const uint64_t *R, uint32_t B, const uint8_t *seeds, uint8_t *out) {
    uint64_t words = (n + 63) / 64;
    uint64_t bucket = (uint64_t)d * z;
    uint8_t *mask = (uint8_t *)malloc(bucket ? bucket : 1);
    if (!mask) return;
    for (uint32_t b = 0; b < B; b++) {
        uint8_t *o = out + (uint64_t)b * bucket;
        oracle_read(T, n, d, z, R + (uint64_t)b * words, o);   /* R_i, step 5 */
        oracle_mask(seeds + (uint64_t)b * 32, bucket, mask);  /* P_i, step 6 */
        for (uint64_t j = 0; j < bucket; j++) o[j] ^= mask[j];  /* R_i XOR P_i, step 7 */
    }
    free(mask);
}

/* ------------------------------------------------------------------------ */
/* Blocked cuckoo table                                                      */
/* ------------------------------------------------------------------------ */

struct oracle_cuckoo {
    uint64_t n;
    uint32_t d, z;
    uint64_t capacity;
    uint32_t max_evictions;
    uint64_t rng;        /* splitmix64 state, seeded with s_cuckoo */
    uint8_t *payload;    /* n*d*z bytes; an empty slot is all zero */
    uint8_t *used;       /* n*d flags */
    uint64_t *b1, *b2;   /* candidate buckets of the item in each slot */
    uint64_t *seq;       /* first-insert sequence number of the item in each slot */
    uint64_t next_seq;
    uint64_t live;
};

oracle_cuckoo *oracle_cuckoo_create(uint64_t n, uint32_t d, uint32_t z, uint64_t capacity,
                                    uint32_t max_evictions, uint64_t seed) {
    if (n == 0 || d == 0 || z == 0) return NULL;
    oracle_cuckoo *c = (oracle_cuckoo *)calloc(1, sizeof(*c));
    if (!c) return NULL;
    uint64_t slots = n * d;
    c->n = n;
    c->d = d;
    c->z = z;
    c->capacity = capacity;
    c->max_evictions = max_evictions;
    c->rng = seed;
    c->payload = (uint8_t *)calloc(slots, z);
    c->used = (uint8_t *)calloc(slots, 1);
    c->b1 = (uint64_t *)calloc(slots, sizeof(uint64_t));
    c->b2 = (uint64_t *)calloc(slots, sizeof(uint64_t));
    c->seq = (uint64_t *)calloc(slots, sizeof(uint64_t));
    if (!c->payload || !c->used || !c->b1 || !c->b2 || !c->seq) {
        oracle_cuckoo_destroy(c);
        return NULL;
    }
    return c;
}

void oracle_cuckoo_destroy(oracle_cuckoo *c) {
    if (!c) return;
    free(c->payload);
    free(c->used);
    free(c->b1);
    free(c->b2);
    free(c->seq);
    free(c);
}

const uint8_t *oracle_cuckoo_table(const oracle_cuckoo *c) { return c->payload; }
uint64_t oracle_cuckoo_live(const oracle_cuckoo *c) { return c->live; }

int oracle_cuckoo_slot(const oracle_cuckoo *c, uint64_t slot, uint64_t *b1, uint64_t *b2,
                       uint64_t *seq) {
    if (slot >= c->n * c->d || !c->used[slot]) return 0;
    *b1 = c->b1[slot];
    *b2 = c->b2[slot];
    *seq = c->seq[slot];
    return 1;
}

/* The lowest free slot index of bucket e, or -1 if the bucket is full. */
static int64_t lowest_free(const oracle_cuckoo *c, uint64_t e) {
    for (uint32_t j = 0; j < c->d; j++)
        if (!c->used[e * c->d + j]) return (int64_t)(e * c->d + j);
    return -1;
}

/* One item in flight: what a slot holds. */
typedef struct {
    uint64_t b1, b2, seq;
    uint8_t *data; /* z bytes */
} item_t;

static void put(oracle_cuckoo *c, uint64_t slot, const item_t *it) {
    c->used[slot] = 1;
    c->b1[slot] = it->b1;
    c->b2[slot] = it->b2;
    c->seq[slot] = it->seq;
    memcpy(c->payload + slot * c->z, it->data, c->z);
}

/* Copy of everything an insertion can change, for the rollback. */
typedef struct {
    uint8_t *payload, *used;
    uint64_t *b1, *b2, *seq;
    uint64_t live;
} snapshot_t;

static int take_snapshot(const oracle_cuckoo *c, snapshot_t *s) {
    uint64_t slots = c->n * c->d;
    s->payload = (uint8_t *)malloc(slots * c->z);
    s->used = (uint8_t *)malloc(slots);
    s->b1 = (uint64_t *)malloc(slots * 8);
    s->b2 = (uint64_t *)malloc(slots * 8);
    s->seq = (uint64_t *)malloc(slots * 8);
    if (!s->payload || !s->used || !s->b1 || !s->b2 || !s->seq) return ORACLE_ENOMEM;
    memcpy(s->payload, c->payload, slots * c->z);
    memcpy(s->used, c->used, slots);
    memcpy(s->b1, c->b1, slots * 8);
    memcpy(s->b2, c->b2, slots * 8);
    memcpy(s->seq, c->seq, slots * 8);
    s->live = c->live;
    return ORACLE_OK;
}

static void restore_snapshot(oracle_cuckoo *c, const snapshot_t *s) {
    uint64_t slots = c->n * c->d;
    memcpy(c->payload, s->payload, slots * c->z);
    memcpy(c->used, s->used, slots);
    memcpy(c->b1, s->b1, slots * 8);
    memcpy(c->b2, s->b2, slots * 8);
    memcpy(c->seq, s->seq, slots * 8);
    c->live = s->live;
}

static void free_snapshot(snapshot_t *s) {
    free(s->payload);
    free(s->used);
    free(s->b1);
    free(s->b2);
    free(s->seq);
}

int oracle_cuckoo_insert(oracle_cuckoo *c, uint64_t b1, uint64_t b2, const uint8_t *msg,
                         uint32_t *evictions) {
    if (evictions) *evictions = 0;
    if (b1 >= c->n || b2 >= c->n) return ORACLE_EINVAL;
    uint64_t slots = c->n * c->d;

    uint8_t *carried = (uint8_t *)malloc(c->z);
    uint8_t *victim = (uint8_t *)malloc(c->z);
    if (!carried || !victim) {
        free(carried);
        free(victim);
        return ORACLE_ENOMEM;
    }

    /* Garbage collection only frees slots, so an eviction walk (and hence a
     * possible rollback) is needed only if both buckets are full right now. */
    int may_walk = lowest_free(c, b1) < 0 && lowest_free(c, b2) < 0;
    snapshot_t snap = {0};
    if (may_walk && take_snapshot(c, &snap) != ORACLE_OK) {
        free_snapshot(&snap);
        free(carried);
        free(victim);
        return ORACLE_ENOMEM;
    }

    /* Step 1: the server keeps `capacity` messages; delete the oldest. */
    if (c->capacity > 0 && c->live == c->capacity) {
        uint64_t oldest = slots;
        for (uint64_t s = 0; s < slots; s++)
            if (c->used[s] && (oldest == slots || c->seq[s] < c->seq[oldest])) oldest = s;
        c->used[oldest] = 0;
        memset(c->payload + oldest * c->z, 0, c->z);
        c->live--;
    }

    memcpy(carried, msg, c->z);
    item_t delta = {b1, b2, c->next_seq, carried};

    /* Step 2: spare capacity in b1, else in b2 (lowest free slot). */
    int64_t f = lowest_free(c, b1);
    if (f < 0) f = lowest_free(c, b2);
    int placed = 0;
    uint32_t moves = 0;
    if (f >= 0) {
        put(c, (uint64_t)f, &delta);
        placed = 1;
    } else {
        /* Step 3: choose beta_e from {b1, b2} with randomness from s_cuckoo. */
        uint64_t e = (oracle_splitmix64_next(&c->rng) & 1u) ? b2 : b1;
        /* Step 4: evict a random entry of beta_e, insert delta there, carry the
         * evicted entry to its alternate bucket; stop at a bucket with space. */
        for (uint32_t i = 0; i < c->max_evictions && !placed; i++) {
            uint64_t v = e * c->d + oracle_splitmix64_next(&c->rng) % c->d;
            item_t out = {c->b1[v], c->b2[v], c->seq[v], victim};
            memcpy(victim, c->payload + v * c->z, c->z);
            put(c, v, &delta);
            moves++;
            /* delta becomes the evicted entry */
            memcpy(carried, victim, c->z);
            delta.b1 = out.b1;
            delta.b2 = out.b2;
            delta.seq = out.seq;
            e = (e == delta.b1) ? delta.b2 : delta.b1;
            int64_t g = lowest_free(c, e);
            if (g >= 0) {
                put(c, (uint64_t)g, &delta);
                placed = 1;
            }
        }
    }
    free(carried);
    free(victim);

    if (!placed) {
        restore_snapshot(c, &snap);
        free_snapshot(&snap);
        if (evictions) *evictions = moves;
        return ORACLE_EFULL;
    }
    if (may_walk) free_snapshot(&snap);
    c->next_seq++;
    c->live++;
    if (evictions) *evictions = moves;
    return ORACLE_OK;
}

/* ------------------------------------------------------------------------ */
/* Bloom interest vectors                                                    */
/* ------------------------------------------------------------------------ */

struct oracle_bloom {
    uint64_t m;
    uint32_t k, window, writes_per_delta;
    uint32_t cur;   /* index of the delta receiving inserts */
    uint32_t count; /* writes summarised by the current delta */
    uint8_t *bits;  /* window deltas of m bits, one byte per bit */
};

oracle_bloom *oracle_bloom_create(uint64_t m, uint32_t k, uint32_t window,
                                  uint32_t writes_per_delta) {
    if (m == 0 || k == 0 || window == 0) return NULL;
    oracle_bloom *b = (oracle_bloom *)calloc(1, sizeof(*b));
    if (!b) return NULL;
    b->m = m;
    b->k = k;
    b->window = window;
    b->writes_per_delta = writes_per_delta;
    b->bits = (uint8_t *)calloc((size_t)window * m, 1);
    if (!b->bits) {
        free(b);
        return NULL;
    }
    return b;
}

void oracle_bloom_destroy(oracle_bloom *b) {
    if (!b) return;
    free(b->bits);
    free(b);
}

/* Before a write: once the current delta summarises writes_per_delta writes,
 * open a new delta in place of the oldest one of the window.  The window thus
 * holds the `window` most recent deltas, the newest possibly partial. */
static void begin_write(oracle_bloom *b) {
    if (b->writes_per_delta && b->count == b->writes_per_delta) {
        b->cur = (b->cur + 1) % b->window;
        memset(b->bits + (uint64_t)b->cur * b->m, 0, b->m);
        b->count = 0;
    }
}

int oracle_bloom_insert(oracle_bloom *b, const uint64_t *positions) {
    for (uint32_t i = 0; i < b->k; i++)
        if (positions[i] >= b->m) return ORACLE_EINVAL;
    begin_write(b);
    for (uint32_t i = 0; i < b->k; i++) b->bits[(uint64_t)b->cur * b->m + positions[i]] = 1;
    b->count++;
    return ORACLE_OK;
}

void oracle_bloom_or_vector(oracle_bloom *b, const uint64_t *vec) {
    begin_write(b);
    for (uint64_t p = 0; p < b->m; p++)
        if ((vec[p >> 6] >> (p & 63)) & 1u) b->bits[(uint64_t)b->cur * b->m + p] = 1;
    b->count++;
}

void oracle_bloom_get(const oracle_bloom *b, uint64_t *out_words) {
    uint64_t words = (b->m + 63) / 64;
    for (uint64_t w = 0; w < words; w++) out_words[w] = 0;
    for (uint32_t j = 0; j < b->window; j++)
        for (uint64_t p = 0; p < b->m; p++)
            if (b->bits[(uint64_t)j * b->m + p]) out_words[p >> 6] |= 1ULL << (p & 63);
}

int oracle_bloom_delta(const oracle_bloom *b, uint32_t age, uint64_t *out_words) {
    if (age == 0 || age > b->window) return ORACLE_EINVAL;
    uint32_t j = (b->cur + b->window - (age - 1)) % b->window;
    uint64_t words = (b->m + 63) / 64;
    for (uint64_t w = 0; w < words; w++) out_words[w] = 0;
    for (uint64_t p = 0; p < b->m; p++)
        if (b->bits[(uint64_t)j * b->m + p]) out_words[p >> 6] |= 1ULL << (p & 63);
    return ORACLE_OK;
}

int oracle_bloom_contains(const oracle_bloom *b, const uint64_t *positions) {
    for (uint32_t i = 0; i < b->k; i++) {
        if (positions[i] >= b->m) return 0;
        int set = 0;
        for (uint32_t j = 0; j < b->window; j++)
            if (b->bits[(uint64_t)j * b->m + positions[i]]) set = 1;
        if (!set) return 0;
    }
    return 1;
}

/* ------------------------------------------------------------------------ */
/* Compressed deltas: Golomb-Rice code of the gaps between set bits          */
/* ------------------------------------------------------------------------ */

uint32_t oracle_rice_param(uint64_t m, uint64_t count) {
    if (count == 0) return 0;
    uint64_t g = (m - count) / count;
    uint32_t k = 0;
    while (g >= 2) {   /* floor(log2 g) for g >= 1 */
        g >>= 1;
        k++;
    }
    return k;
}

static int put_bit(uint8_t *out, uint64_t cap, uint64_t pos, int bit) {
    if (pos / 8 >= cap) return 0;
    if (bit) out[pos / 8] |= (uint8_t)(1u << (pos % 8));
    return 1;
}

uint64_t oracle_rice_encode(const uint64_t *bits, uint64_t m, uint32_t k, uint8_t *out,
                            uint64_t cap, uint64_t *count) {
    uint64_t pos = 0, n = 0;
    int64_t prev = -1;
    for (uint64_t j = 0; j < cap; j++) out[j] = 0;
    for (uint64_t p = 0; p < m; p++) {
        if (!((bits[p / 64] >> (p % 64)) & 1u)) continue;
        uint64_t gap = (uint64_t)((int64_t)p - prev - 1);
        uint64_t q = gap >> k;
        for (uint64_t i = 0; i < q; i++)
            if (!put_bit(out, cap, pos++, 1)) return UINT64_MAX;
        if (!put_bit(out, cap, pos++, 0)) return UINT64_MAX;
        for (uint32_t i = 0; i < k; i++)
            if (!put_bit(out, cap, pos++, (int)((gap >> i) & 1u))) return UINT64_MAX;
        prev = (int64_t)p;
        n++;
    }
    if (count) *count = n;
    return pos;
}

int oracle_rice_decode(const uint8_t *in, uint64_t nbits, uint32_t k, uint64_t count, uint64_t m,
                       uint64_t *bits) {
    uint64_t words = (m + 63) / 64, pos = 0;
    int64_t prev = -1;
    for (uint64_t w = 0; w < words; w++) bits[w] = 0;
    for (uint64_t c = 0; c < count; c++) {
        uint64_t q = 0;
        for (;;) {
            if (pos >= nbits) return ORACLE_EINVAL;
            int b = (in[pos / 8] >> (pos % 8)) & 1;
            pos++;
            if (!b) break;
            q++;
        }
        uint64_t r = 0;
        for (uint32_t i = 0; i < k; i++) {
            if (pos >= nbits) return ORACLE_EINVAL;
            r |= (uint64_t)((in[pos / 8] >> (pos % 8)) & 1) << i;
            pos++;
        }
        uint64_t p = (uint64_t)(prev + 1) + (q << k) + r;
        if (p >= m) return ORACLE_EINVAL;
        bits[p / 64] |= 1ull << (p % 64);
        prev = (int64_t)p;
    }
    return ORACLE_OK;
}
