/*
 * oracle.h -- plain, slow CPU reference for Talek's server-side state.
 *
 * TEST INFRASTRUCTURE ONLY.  This code exists to check the CUDA library
 * against the paper.  Only the tests, the package's smoke check and the
 * benchmark's CPU-baseline leg may load it.  It shares no code, header,
 * table or constant with the CUDA library, and it never calls it.
 *
 * Naming: n = number of buckets (the paper's b), d = slots per bucket,
 * z = message bytes per slot.  A bucket is d*z contiguous bytes; the table is
 * n buckets back to back.  Request vectors are packed LSB-first in 64-bit
 * words: bit k is bit (k % 64) of word k / 64; bits at positions >= n are
 * ignored.
 */
#ifndef TALEK_ORACLE_H
#define TALEK_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ORACLE_OK 0
#define ORACLE_EINVAL (-1)
#define ORACLE_ENOMEM (-2)
#define ORACLE_EFULL (-3)

/* ---- IT-PIR (Section 2) ------------------------------------------------ */

/* Server answer, Section 2 step 5: out = XOR of every bucket T[k] whose bit
 * q[k] is 1.  out has d*z bytes. */
void oracle_read(const uint8_t *T, uint64_t n, uint32_t d, uint32_t z,
                 const uint64_t *q, uint8_t *out);

/* B independent answers; R has B rows of ceil(n/64) words, out B rows of d*z. */
void oracle_read_batch(const uint8_t *T, uint64_t n, uint32_t d, uint32_t z,
                       const uint64_t *R, uint32_t B, uint8_t *out);

/* Client reconstruction, Section 2 step 6: out = R_1 XOR ... XOR R_l. */
void oracle_reconstruct(const uint8_t *replies, uint32_t l, uint64_t bytes, uint8_t *out);

/* splitmix64 sequential generator (Steele, Lea & Flood 2014): advances *state
 * and returns the next output. */
uint64_t oracle_splitmix64_next(uint64_t *state);

/* ---- Serialized PIR (Section 6) ---------------------------------------- */

/* The ChaCha20 block function as RFC 8439 section 2.3 defines it: the 64
 * keystream bytes of block `counter` under a 32-byte key and a 12-byte nonce. */
void oracle_chacha20_block(const uint8_t key[32], uint32_t counter, const uint8_t nonce[12],
                           uint8_t out[64]);

/* One-time mask of Section 6 step 6, P = PRNG(p): the paper leaves the PRNG
 * open; here it is the ChaCha20 keystream under key p (32 bytes) with an
 * all-zero nonce, blocks 0, 1, 2, ... in order, cut to nbytes bytes. */
void oracle_mask(const uint8_t seed[32], uint64_t nbytes, uint8_t *out);

/* Masked server responses, Section 6 step 7: out[b] = oracle_read(R[b]) XOR
 * PRNG(seeds[b]); seeds has B rows of 32 bytes. */
void oracle_read_batch_masked(const uint8_t *T, uint64_t n, uint32_t d, uint32_t z,
                              const uint64_t *R, uint32_t B, const uint8_t *seeds, uint8_t *out);

/* ---- blocked cuckoo table with FIFO garbage collection (Section 5.3) --- */

typedef struct oracle_cuckoo oracle_cuckoo;

/* capacity = number of messages kept (0 = never collect); max_evictions =
 * bound on the eviction walk; seed = s_cuckoo. NULL on bad arguments. */
oracle_cuckoo *oracle_cuckoo_create(uint64_t n, uint32_t d, uint32_t z, uint64_t capacity,
                                    uint32_t max_evictions, uint64_t seed);
void oracle_cuckoo_destroy(oracle_cuckoo *c);

/* Insert one message with candidate buckets b1, b2.  Returns ORACLE_OK,
 * ORACLE_EINVAL (bucket out of range) or ORACLE_EFULL (eviction bound hit:
 * table, metadata and the collected item are restored; the random draws made
 * stay consumed).  *evictions = number of evictions made. */
int oracle_cuckoo_insert(oracle_cuckoo *c, uint64_t b1, uint64_t b2, const uint8_t *msg,
                         uint32_t *evictions);

const uint8_t *oracle_cuckoo_table(const oracle_cuckoo *c);
uint64_t oracle_cuckoo_live(const oracle_cuckoo *c);
/* Slot metadata; returns 1 if the slot holds an item (and fills b1, b2, seq). */
int oracle_cuckoo_slot(const oracle_cuckoo *c, uint64_t slot, uint64_t *b1, uint64_t *b2,
                       uint64_t *seq);

/* ---- Bloom interest vectors (Section 7) -------------------------------- */

typedef struct oracle_bloom oracle_bloom;

/* m bits, k positions per insert, a window of the `window` most recent deltas;
 * each delta summarises `writes_per_delta` writes (0 = a single delta that is
 * never replaced).  A new delta opens, in place of the oldest, at the first
 * write that finds the current one complete. */
oracle_bloom *oracle_bloom_create(uint64_t m, uint32_t k, uint32_t window,
                                  uint32_t writes_per_delta);
void oracle_bloom_destroy(oracle_bloom *b);
/* Set k positions (each < m) in the current delta. Returns ORACLE_EINVAL on a
 * position out of range (nothing changes). */
int oracle_bloom_insert(oracle_bloom *b, const uint64_t *positions);
/* OR a whole m-bit interest vector (ceil(m/64) words) into the current delta;
 * counts as one write. Bits >= m are ignored. */
void oracle_bloom_or_vector(oracle_bloom *b, const uint64_t *vec);
/* Global interest vector = OR of the deltas in the window (ceil(m/64) words). */
void oracle_bloom_get(const oracle_bloom *b, uint64_t *out_words);
/* The age-th most recent delta (age 1 = the current one, up to window), as
 * ceil(m/64) words; returns ORACLE_EINVAL for an age outside 1..window. */
int oracle_bloom_delta(const oracle_bloom *b, uint32_t age, uint64_t *out_words);
/* 1 if all k positions are set in the global interest vector. */
int oracle_bloom_contains(const oracle_bloom *b, const uint64_t *positions);

/* ---- Compressed interest-vector deltas (Section 7, GetUpdates) ---------
 * The paper sends Bloom-filter deltas compressed; the encoding taken here is
 * the Golomb-Rice code of the gaps between consecutive set bits: for set
 * bits p_0 < p_1 < ..., gap_i = p_i - p_{i-1} - 1 (p_{-1} = -1), written as
 * q = gap_i >> k one-bits, a zero bit, then the k low bits of gap_i (least
 * significant first).  The stream is packed LSB-first: stream bit j is bit
 * (j % 8) of byte j / 8. */

/* Rice parameter for `count` set bits among m: 0 if count = 0 or the mean
 * gap g = (m - count) / count (integer division) is 0, else floor(log2 g). */
uint32_t oracle_rice_param(uint64_t m, uint64_t count);

/* Encodes the set bits of an m-bit vector (ceil(m/64) words; bits >= m
 * ignored) with parameter k.  Writes ceil(nbits/8) bytes to out (cap bytes
 * available) and returns nbits, or UINT64_MAX if the stream would not fit;
 * *count = set bits encoded. */
uint64_t oracle_rice_encode(const uint64_t *bits, uint64_t m, uint32_t k, uint8_t *out,
                            uint64_t cap, uint64_t *count);

/* Decodes `count` codes of parameter k from a stream of nbits bits into an
 * m-bit vector (ceil(m/64) words, cleared first).  Returns ORACLE_OK, or
 * ORACLE_EINVAL if the stream is short or a position falls at or past m. */
int oracle_rice_decode(const uint8_t *in, uint64_t nbits, uint32_t k, uint64_t count, uint64_t m,
                       uint64_t *bits);

#ifdef __cplusplus
}
#endif
#endif
