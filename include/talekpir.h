/*
 * talekpir.h -- C ABI of libtalekpir, a GB300 (sm_103a) engine for the
 * server side of Talek's private messaging (arxiv 2001.08250).
 *
 * A server holds a blocked cuckoo hash table of n buckets, each of d slots of
 * msg_bytes bytes (Sections 4.3 and 5.3).  A PIR read (Section 2, step 5)
 * returns the XOR of every bucket whose bit is set in the client's request
 * vector; every bucket is read for every request, whatever the bits are, so
 * the server's memory accesses do not depend on the request.
 *
 * Naming: n is the number of BUCKETS (the paper calls it b; the paper's n is
 * the number of stored messages).  row_bytes = d * msg_bytes is the size of a
 * bucket and of one reply.
 *
 * Layouts (all little-endian, all contiguous):
 *   table      n rows of row_bytes; slot j of bucket k starts at byte
 *              k*row_bytes + j*msg_bytes.  An empty slot holds zero bytes.
 *   req_bits   B rows of ceil(n/64) uint64 words; bucket k is bit (k % 64) of
 *              word k / 64 of the row (LSB first).  Bits at positions >= n are
 *              ignored.
 *   out        B rows of row_bytes: row b is the reply to request row b.
 *
 * Conventions:
 *   - The caller owns every request and output buffer; the library owns the
 *     device tables.  Pointers named d_* are device pointers on the current
 *     CUDA device; all others are host pointers.
 *   - Every call returns a tpir_status, except the creators, which return NULL
 *     and leave the reason in tpir_last_error() (per thread).
 *   - On an error no output is written, except where stated.
 *   - msg_bytes must be a positive multiple of 16; d is 1..64; n >= 1.
 *   - One tpir_db is used from one host thread at a time.
 */
#ifndef TALEKPIR_H
#define TALEKPIR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    TPIR_OK = 0,
    TPIR_EINVAL = -1,    /* bad argument (size, pointer, bucket index) */
    TPIR_ENOMEM = -2,    /* device allocation failed or HBM budget exceeded */
    TPIR_EFULL = -3,     /* cuckoo eviction bound hit; table rolled back */
    TPIR_EAGAIN = -4,    /* serve queue full; try again */
    TPIR_ETIMEDOUT = -5, /* a bounded wait inside a kernel gave up */
    TPIR_ECUDA = -6,     /* a CUDA runtime call failed */
    TPIR_ESHUTDOWN = -7  /* server is shutting down */
} tpir_status;

typedef struct tpir_db tpir_db;

/* Version string of the library. */
const char *tpir_version(void);
/* Status of the last failed creator call on this thread. */
tpir_status tpir_last_error(void);
/* Human-readable name of a status code (static string). */
const char *tpir_strerror(tpir_status s);

/* ---- tables (Sections 4.3, 5.3; Fig. "Talek Variables") ------------------
 * tpir_db_create allocates an all-zero table of n buckets x d slots x
 * msg_bytes on the current device, 256-byte aligned, plus its host-side
 * cuckoo metadata.  Returns NULL on error (EINVAL, ENOMEM, ECUDA). */
tpir_db *tpir_db_create(uint64_t n, uint32_t d, uint32_t msg_bytes);
void tpir_db_destroy(tpir_db *db);

/* ---- Row shards (the scale-out Section 9.4 proposes: one server's database
 * split over several machines, each holding a portion of it) -------------
 * tpir_db_create_shard makes a db of `rows` buckets that stands for buckets
 * [row_begin, row_begin + rows) of a logical table of n_total buckets
 * (row_begin a multiple of 64, so a shard owns whole request words).  Reads
 * on a shard take FULL-length request rows (ceil(n_total/64) words, the same
 * buffer every shard reads) and return the shard's partial reply, the XOR of
 * its selected buckets; the XOR of all shards' partial replies is the reply of
 * the whole table (tpir_xor_combine is the exchange's combine step).  Masks of
 * a masked read apply to the partial, so a sharded server masks on one shard.
 * Shards are loaded with tpir_db_load / tpir_db_load_async (the shard's rows
 * of the table, e.g. a snapshot of a writer's table); the cuckoo writes
 * return TPIR_EINVAL on a shard.  NULL on error (EINVAL: shape or range). */
tpir_db *tpir_db_create_shard(uint64_t n_total, uint64_t row_begin, uint64_t rows, uint32_t d,
                              uint32_t msg_bytes);
/* n_total and row_begin of a shard (n and 0 for a whole table). */
tpir_status tpir_db_shard_info(const tpir_db *db, uint64_t *n_total, uint64_t *row_begin);
/* Balanced split of n_total buckets into `parts` shards in whole request
 * words (64 buckets): the range of shard `index`.  *rows is 0 for the shards
 * left empty when parts > ceil(n_total/64).  Pure host arithmetic. */
tpir_status tpir_shard_plan(uint64_t n_total, uint32_t parts, uint32_t index, uint64_t *row_begin,
                            uint64_t *rows);

/* Shape and state: any output pointer may be NULL.  *d_table is the device
 * address of the table; *epoch counts the writes applied so far. */
tpir_status tpir_db_info(const tpir_db *db, uint64_t *n, uint32_t *d, uint32_t *msg_bytes,
                         const void **d_table, uint64_t *epoch);

/* Blocks until every write, load and read already submitted on this db (on
 * its own stream or any other) has completed on the device. */
tpir_status tpir_db_sync(tpir_db *db);

/* Cuckoo policy (Section 5.3): keep at most `capacity` messages, collecting
 * the oldest first (0 = never collect); give up an eviction walk after
 * `max_evictions` evictions; s_cuckoo seeds the random choices (splitmix64),
 * so that replicas given the same writes in the same order agree.
 * Defaults: 0, 500, 0.  Only allowed while the table holds no item. */
tpir_status tpir_db_set_policy(tpir_db *db, uint64_t capacity, uint32_t max_evictions,
                               uint64_t s_cuckoo);

/* Bulk payload load/dump of the whole table (bytes = n*row_bytes), from/to a
 * host buffer.  Load replaces the payload and forgets all cuckoo metadata (the
 * table is then read-only content for the write path's purposes: later writes
 * treat every slot as free).  Synchronous. */
tpir_status tpir_db_load(tpir_db *db, const void *host_table, size_t bytes);
/* Asynchronous bulk load on `stream` from a device or pinned host buffer
 * (same effect on metadata as tpir_db_load). */
tpir_status tpir_db_load_async(tpir_db *db, const void *src, size_t bytes, void *stream);
tpir_status tpir_db_dump(tpir_db *db, void *host_table, size_t bytes);

/* ---- writes (Section 5.3, server steps 1-4) ------------------------------
 * Inserts msg (msg_bytes, host) with candidate buckets b1, b2 < n: collects
 * the oldest message if the table is at capacity, places the message in the
 * lowest free slot of b1, else of b2, else walks evictions from a bucket
 * chosen with s_cuckoo's randomness.  The placement is computed on the host
 * (metadata only); the slot moves and the payload write run on the device in
 * the db's stream order, after every read submitted before this call and
 * before every read submitted after it.  Returns EFULL (nothing changed; the
 * random draws stay consumed) when the walk exceeds max_evictions.
 * *evictions_out (may be NULL) = evictions made.  The move list and the
 * message travel in the launch itself when they are small (up to 384 moves
 * and 20 KiB of messages), so such a write returns as soon as it is
 * enqueued; larger ones go through a staging buffer kept with the db.  On a
 * CUDA or allocation failure the placement is taken back. */
tpir_status tpir_write(tpir_db *db, uint64_t b1, uint64_t b2, const void *msg,
                       uint32_t *evictions_out);

/* `count` writes in order, as if by `count` tpir_write calls, with one
 * host-to-device copy and one move kernel: b1, b2 (count words), msgs
 * (count x msg_bytes), all host.  status_out[i] / evictions_out[i] (may be
 * NULL) receive each write's result; the call returns TPIR_OK unless a
 * CUDA/allocation failure stopped it (then nothing was applied on the device). */
tpir_status tpir_write_batch(tpir_db *db, uint32_t count, const uint64_t *b1, const uint64_t *b2,
                             const void *msgs, tpir_status *status_out, uint32_t *evictions_out);

/* A cuckoo write that allocates no device or pinned memory.  The paper has no
 * counterpart: this entry point exists for callers that cannot allocate, such
 * as a serving thread for which a cudaMalloc (which may synchronise the whole
 * device) is an unbounded stall, or a process whose device memory is all
 * owned by another allocator under a hard budget.  Same placement rules and
 * result as tpir_write, but the message d_msg is a DEVICE buffer of msg_bytes
 * (16-byte aligned) that must stay valid until `stream` (a cudaStream_t, NULL
 * = legacy default stream) reaches this write; the slot moves run on `stream`,
 * after every read already submitted on this db and before every later read.
 * Limits: msg_bytes <= 65536 and the db's max_evictions <= 500, else
 * TPIR_EINVAL (nothing changes).  EFULL as for tpir_write.
 * The moves run after every earlier write to this db, on whatever stream it
 * ran.  On any error the placement is taken back (table and metadata
 * unchanged).  Not allowed while `stream` is being captured into a graph
 * (TPIR_EINVAL): the events that order it against the db's other work
 * cannot cross a capture boundary.
 * The moves use one temporary slot held in a 64 KiB device array that every
 * GPU loading the library keeps until exit; the first call on a device looks
 * up that array's address.  All calls share the array: calls whose moves
 * overlap on the GPU (writes to different dbs on different streams) race, so
 * order them on one stream. */
tpir_status tpir_write_noalloc(tpir_db *db, uint64_t b1, uint64_t b2, const void *d_msg,
                               uint32_t *evictions_out, void *stream);

/* ---- PIR reads (Section 2 step 5; batching as in Section 9.2) -------------
 * Synchronous: req_bits (host, B rows) in, out (host, B x row_bytes) out.
 * B = 0 is a no-op.  Sees every write made before the call. */
tpir_status tpir_read_batch(tpir_db *db, const uint64_t *req_bits, uint32_t B, void *out);

/* Synchronous, for request sets larger than one batch: B_total rows of
 * req_bits (host) in batches of `batch` (one scan launch each), replies into
 * out (host, B_total x row_bytes).  Three device slots rotate, each holding a
 * group of four batches: a group's rows are copied in two groups ahead of
 * its scans and its replies copied out after them, on a copy stream, so the
 * copies overlap the scans (with pinned host buffers; pageable ones work but
 * serialise), and the scans of a group run back to back.  Device memory for
 * the slots is allocated on first use and kept with the db.  Same replies as
 * tpir_read_batch on each batch. */
tpir_status tpir_read_batch_pipelined(tpir_db *db, const uint64_t *req_bits, uint64_t B_total,
                                      uint32_t batch, void *out);

/* Asynchronous on `stream` (a cudaStream_t; NULL = legacy default stream):
 * d_req_bits and d_out are device buffers that must stay valid until the
 * stream reaches this point.  d_out must not overlap d_req_bits or the table.
 * Ordered after all writes already made on this db. */
tpir_status tpir_read_batch_async(tpir_db *db, const uint64_t *d_req_bits, uint32_t B,
                                  void *d_out, void *stream);

/* ---- Serialized PIR (Section 6) -----------------------------------------
 * Masked reads, steps 5-7: reply b = (XOR of the buckets request b selects)
 * XOR P_b, with P_b = PRNG(seed_b) the one-time mask of the 32-byte seed the
 * client sent with the request.  The paper leaves the PRNG open; here it is
 * the ChaCha20 keystream of RFC 8439 under key seed_b with an all-zero nonce,
 * blocks 0, 1, 2, ... in order, cut to row_bytes.  seeds: B rows of 32 bytes.
 * Same kernels, ordering and error behaviour as the unmasked reads; the masks
 * are generated on the device by the kernel that initialises the replies.
 * Synchronous form: all buffers are host memory. */
tpir_status tpir_read_batch_masked(tpir_db *db, const uint64_t *req_bits, uint32_t B,
                                   const uint8_t *seeds, void *out);
/* Asynchronous form: device buffers; d_seeds 16-byte aligned (else EINVAL). */
tpir_status tpir_read_batch_masked_async(tpir_db *db, const uint64_t *d_req_bits, uint32_t B,
                                         const uint8_t *d_seeds, void *d_out, void *stream);
/* The masks alone, P_b for b < rows, nbytes each (a multiple of 16), into the
 * device buffer d_out (rows x nbytes): the client's step 9, or a leader that
 * checks a combination.  d_seeds and d_out 16-byte aligned. */
tpir_status tpir_mask_generate(const uint8_t *d_seeds, uint32_t rows, uint64_t nbytes,
                               void *d_out, void *stream);
/* The leader's combination, step 8: d_dst = XOR of `count` device buffers
 * d_srcs[0..count-1] of nbytes each (nbytes a multiple of 16, every buffer
 * 16-byte aligned; d_dst may be one of the sources; 1 <= count <= 64).
 * d_srcs itself is a host array of device pointers. */
tpir_status tpir_xor_combine(const void *const *d_srcs, uint32_t count, uint64_t nbytes,
                             void *d_dst, void *stream);

/* Force a kernel choice for tests and benchmarks: 0 = automatic (plain for
 * B <= 4, tensor-core for B >= 48 on rows of >= 256 bytes, register-tiled
 * batched otherwise), 1 = plain streaming kernel (B <= 4 per launch,
 * larger B is split into launches; TMA-staged where the row width allows),
 * 2 = batched register-tiled kernel, 3 = plain kernel with register
 * streaming only (the path used for row widths the TMA-staged one skips),
 * 4 = batched Four-Russians kernel (groups of 8 buckets, 256 combinations in
 * shared memory, one lookup per request and group), 5 = batched tensor-core
 * kernel (the GF(2) product as an exact integer product of 0/1 matrices on
 * tcgen05: packed 4-bit e2m1 operands with unit block scales, fp32
 * accumulators, reduced mod 2; batches of more than 128 requests run on
 * pairs of SMs sharing each M = 256 MMA, cta_group::2, unless a tuning plan
 * chose single CTAs; a device that cannot hold the pairs' clusters takes
 * single CTAs).  The tensor-core kernel reads a
 * bit-transposed copy of the table (each column's bits over 64 buckets in
 * one word; as large as the table), allocated and built by the first read
 * that uses it and then kept equal to the table by every write and load. */
tpir_status tpir_db_set_kernel(tpir_db *db, int kernel);

/* Autotuner of the batched read.  For this table and a batch of B requests
 * it times, on the table itself:
 *   - every admissible tile shape of the register-tiled kernel (lanes along
 *     the row, warps along requests / row / buckets, i.e. the batch tile
 *     width and the row tile width, and the rows per pipeline stage);
 *   - the tensor-core kernel's schedules (equal spans of stages per CTA, or
 *     items of whole k-chunks of 4096 .. 32768 buckets or the planned size;
 *     request words staged by TMA or loaded by the expander threads; above
 *     128 requests items on CTA pairs and on single CTAs) when rows are 256
 *     bytes or wider;
 *   - the Four-Russians kernel (B >= 32, rows of 256 bytes or more) and the
 *     plain kernel (B <= 16);
 * and keeps (a) the fastest tile shape for every later launch of the
 * register-tiled kernel with this row width and batch-size class
 * (ceil(log2 B)), and (b) the fastest kernel, with its tensor-core schedule,
 * for every later automatic choice with this row width and batch class
 * (tables of another size take the plan of the nearest table-size class,
 * ceil(log2 n)): single-table reads, many-table launches and the serve loop
 * then take the measured winner instead of the built-in batch thresholds.  reps = timed launches per candidate (0 = 3).  Allocates
 * scratch buffers for the trial requests and replies. */
typedef struct {
    uint32_t lw_log2, warps_b, warps_w, warps_k, stage_rows;
    uint32_t tile_b, tile_w;   /* requests and 32-bit words per CTA tile */
    uint32_t candidates;       /* register-tiled shapes timed */
    double us_per_launch;      /* of the chosen register-tiled shape */
    double lop3_tops;          /* B*n*row_words / time */
    uint32_t kernel;           /* fastest kernel (as in tpir_db_set_kernel) */
    uint32_t tensor_mode;      /* its tensor-core schedule: 1 spans, 2 items (on CTA pairs above
                                  128 requests), 3 items on single CTAs */
    uint32_t tensor_kc_rows;   /* items: k-chunk buckets (0: planned size) */
    uint32_t tensor_loads;     /* 1: request words loaded by threads, not TMA */
    uint32_t tensor_candidates;
    double us_lop3, us_tensor, us_m4rm, us_plain;  /* best of each kernel (0: not timed) */
} tpir_tune_result;
tpir_status tpir_autotune(tpir_db *db, uint32_t B, uint32_t reps, tpir_tune_result *out);
/* The tuned shapes and kernel choices as JSON (one plan per line), and back;
 * clear forgets them. */
tpir_status tpir_tune_save(const char *path);
tpir_status tpir_tune_load(const char *path);
tpir_status tpir_tune_clear(void);

/* Many tables in ONE persistent launch per kernel kind (the uneven-batching
 * workload): job i reads B_i rows of d_req_bits_i against db_i into d_out_i.
 * Tables may differ in n, d and msg_bytes.  Jobs of >= 48 requests on rows of
 * >= 256 bytes go to the tensor-core kernel: those of more than 128 requests
 * on tables of >= 8192 buckets share one CTA-pair launch, the rest one
 * single-CTA launch (each per request-staging mode), the others one
 * launch of the register-tiled kernel (a db forced to kernel 4 sends its jobs
 * to the Four-Russians kernel instead: one launch for jobs of up to 256
 * requests, one for larger ones; forced to 2, to the register-tiled one).  A
 * job with d_seeds (B x 32 bytes, 16-byte aligned) is masked as in
 * tpir_read_batch_masked_async; NULL = plain replies.  Up to TPIR_MAX_JOBS
 * jobs per call. */
#define TPIR_MAX_JOBS 128
typedef struct {
    tpir_db *db;
    uint32_t B;
    const uint64_t *d_req_bits;
    void *d_out;
    const uint8_t *d_seeds;
} tpir_read_job;
tpir_status tpir_read_multi_async(const tpir_read_job *jobs, uint32_t njobs, void *stream);

/* The same many-table read captured once into a CUDA graph (per kernel kind
 * one output-initialisation kernel and one persistent scan kernel), for
 * workloads that repeat the launch with the same buffers.  tpir_graph_launch orders the replay after every write
 * already made to the jobs' dbs.  The dbs and buffers must outlive the graph. */
typedef struct tpir_graph tpir_graph;
tpir_status tpir_read_multi_graph_create(const tpir_read_job *jobs, uint32_t njobs,
                                         tpir_graph **out);
tpir_status tpir_graph_launch(tpir_graph *g, void *stream);
void tpir_graph_destroy(tpir_graph *g);

/* Self-test of failure detection (no counterpart in the paper): runs one CTA
 * whose bounded wait, on a barrier nothing arrives at, gives up after
 * limit_us microseconds (1..1000000) exactly as the scan kernels' waits do;
 * returns the status word it left (TPIR_ETIMEDOUT expected), cleared, with the
 * CUDA context still usable. */
tpir_status tpir_selftest_wait_timeout(uint32_t limit_us);

/* Reads and clears the device-side status word that bounded waits inside the
 * kernels set when they give up (TPIR_OK or TPIR_ETIMEDOUT). Synchronises the
 * device. */
tpir_status tpir_device_status(void);

/* Kernel launches the library has enqueued in this process so far, of every
 * kind (reads, reply initialisation, writes, transposed-copy upkeep, interest
 * vectors, compression); the difference of two calls counts the launches
 * made between them.  Does not synchronise. */
uint64_t tpir_kernel_launches(void);

/* ---- private notifications (Section 7) ----------------------------------
 * The global interest vector of a db: m_bits bits, k positions per write, the
 * OR of the `window` most recent deltas; each delta summarises
 * writes_per_delta writes (0 = a single delta that is never replaced), and a
 * new delta opens, in place of the oldest, at the first write that finds the
 * current one complete.  Kept on the device. */
tpir_status tpir_bloom_create(tpir_db *db, uint64_t m_bits, uint32_t k, uint32_t window,
                              uint32_t writes_per_delta);
/* One write's interest vector given as its k bit positions (host, each < m). */
tpir_status tpir_bloom_insert(tpir_db *db, const uint64_t *positions);
/* `count` writes at once: positions is count x k (host). */
tpir_status tpir_bloom_insert_batch(tpir_db *db, const uint64_t *positions, uint32_t count);
/* One write's interest vector given whole (ceil(m/64) words, host); bits >= m
 * are ignored. */
tpir_status tpir_bloom_or_vector(tpir_db *db, const uint64_t *vec);
/* GetUpdates: the global interest vector, ceil(m/64) words (host). */
tpir_status tpir_bloom_get(tpir_db *db, uint64_t *out_words);

/* Compressed GetUpdates (Section 7: the servers send compressed Bloom-filter
 * deltas; the paper fixes no encoding).  The encoding is the Golomb-Rice code
 * of the gaps between set bits: for set bits p_0 < p_1 < ... and p_{-1} = -1,
 * gap_i = p_i - p_{i-1} - 1 is written as (gap_i >> k) one-bits, a zero bit,
 * then the k low bits of gap_i, least significant first; the stream is
 * packed LSB-first (stream bit j = bit j % 8 of byte j / 8).  k < 0 chooses
 * k = floor(log2 g) for the mean gap g = (m - count) / count (0 if g = 0 or
 * count = 0).  The decoder needs m, k and count.
 * tpir_bloom_get_compressed encodes, on the device, which = 0: the global
 * interest vector, or which = i >= 1: the i-th most recent delta of the window
 * (1 = the current one); writes ceil(nbits/8) bytes to the host buffer out.
 * Returns TPIR_ENOMEM (with *nbits = UINT64_MAX or the stream length) if the
 * stream does not fit cap_bytes; EINVAL for which > window. */
tpir_status tpir_bloom_get_compressed(tpir_db *db, uint32_t which, int32_t k, void *out,
                                      uint64_t cap_bytes, uint64_t *nbits, uint64_t *count,
                                      uint32_t *k_used);
/* The same encoding of any m-bit vector in device memory, on `stream`:
 * d_result (device, 3 words) receives nbits (UINT64_MAX if the stream would
 * pass cap_bytes, a multiple of 4), count and k; d_out 4-byte aligned. */
tpir_status tpir_rice_encode_async(const uint64_t *d_bits, uint64_t m, int32_t k, void *d_out,
                                   uint64_t cap_bytes, uint64_t *d_result, void *stream);

/* ---- serving: continuous batching over resident tables -------------------
 * A server thread admits reads and writes as they arrive into a FIFO per
 * table, keeps tables resident under an HBM budget, and forms launch units
 * one table at a time: the table whose oldest waiting op arrived first gets
 * all its waiting writes applied in arrival order and up to max_batch of its
 * waiting reads read in one launch after them (the kernel chosen by the
 * batch, as for tpir_read_batch_async: a table that gathered 48 or more reads
 * goes to the tensor-core kernel).  A table with no waiting read is never
 * scanned.  Up to max_inflight units are on the device at once, each table's
 * in order.  A read sees every write to its table admitted before its unit
 * was formed; its completion reports that write count (epoch). */
typedef struct tpir_server tpir_server;

typedef struct {
    uint64_t hbm_budget_bytes; /* tables + staging must fit; 0 = 64 GiB */
    uint32_t max_batch;        /* reads per table per launch (<= 1024); 0 = 256 */
    uint32_t max_inflight;     /* launch units in flight (1..16); 0 = 4 */
    uint32_t queue_capacity;   /* admitted, unfinished ops; 0 = 65536 */
    uint32_t tick_us;          /* batching window: a table's unit is formed once
                                  its oldest waiting op has waited this long
                                  or max_batch reads are waiting; 0 = at once */
} tpir_serve_config;

typedef struct {
    uint64_t tag;
    int32_t status;    /* tpir_status of the op */
    uint32_t kind;     /* 0 = read, 1 = write */
    uint32_t table_id;
    uint32_t evictions;
    uint64_t epoch;    /* writes to the table that the read saw / the write's number */
    int64_t t_arrive_ns, t_launch_ns, t_done_ns; /* CLOCK_MONOTONIC */
} tpir_completion;

typedef struct {
    uint64_t reads_done, writes_done, rejected, failed;
    uint64_t launches;
    double reads_per_s;               /* since the first admitted read */
    double p50_ms, p99_ms, max_ms;    /* read latency, arrival to completion */
    double mean_batch;                /* reads per table per launch */
    uint64_t hbm_bytes_in_use;
    uint64_t eviction_hist[8];        /* 0, 1, 2-3, 4-7, ..., >= 64 */
    uint64_t kernel_launches[6];      /* read launches by kernel (index as in
                                         tpir_db_set_kernel: 1 plain, 2 register-
                                         tiled, 4 Four-Russians, 5 tensor-core) */
} tpir_stats;

tpir_status tpir_serve_create(const tpir_serve_config *cfg, tpir_server **out);
/* Adds an all-zero table; ENOMEM if it does not fit in the budget. */
tpir_status tpir_serve_add_table(tpir_server *s, uint64_t n, uint32_t d, uint32_t msg_bytes,
                                 uint32_t *table_id);
/* The db of a table, e.g. to load its payload or set its policy before serving. */
tpir_status tpir_serve_table(tpir_server *s, uint32_t table_id, tpir_db **db);
/* Enqueue a read: req_bits (host, one row) is copied at once; out (host,
 * row_bytes) is written before the completion is reported.  t_arrive_ns = the
 * arrival time to measure latency from (0 = now).  EAGAIN if the queue is full. */
tpir_status tpir_serve_submit_read(tpir_server *s, uint32_t table_id, const uint64_t *req_bits,
                                   void *out, uint64_t tag, int64_t t_arrive_ns);
/* Enqueue a write (copied at once); bloom_positions (k words, may be NULL)
 * are OR-ed into the table's interest vector if it has one. */
tpir_status tpir_serve_submit_write(tpir_server *s, uint32_t table_id, uint64_t b1, uint64_t b2,
                                    const void *msg, const uint64_t *bloom_positions, uint64_t tag,
                                    int64_t t_arrive_ns);
/* Completed ops, oldest first; *ndone <= max. */
tpir_status tpir_serve_poll(tpir_server *s, tpir_completion *done, uint32_t max, uint32_t *ndone);
/* Blocks until every admitted op has completed. */
tpir_status tpir_serve_drain(tpir_server *s);
tpir_status tpir_serve_stats(tpir_server *s, tpir_stats *st);
tpir_status tpir_serve_reset_stats(tpir_server *s);
/* Stops admitting (later submits return ESHUTDOWN), drains, frees everything. */
tpir_status tpir_serve_destroy(tpir_server *s);

#ifdef __cplusplus
}
#endif
#endif /* TALEKPIR_H */
