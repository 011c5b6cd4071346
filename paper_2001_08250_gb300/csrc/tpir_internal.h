// Internal declarations of libtalekpir (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>

#include <atomic>
#include <cstdint>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/talekpir.h"

namespace tpir {

// ---------------------------------------------------------------------------
// Batched scan (register-tiled GF(2) product), one persistent launch over a
// list of jobs.  Each job is cut into items = (B-tile, W-tile, k-chunk).
// ---------------------------------------------------------------------------
constexpr int kConsumerWarps = 8;                    // compute warps per CTA (2 warpgroups)
constexpr int kProducerThreads = 128;                // 1 warpgroup: TMA issue + masks
constexpr int kScanThreads = kProducerThreads + 32 * kConsumerWarps;  // 384
// Register split (setmaxnreg): the CTA is launched with 384 x 168 registers;
// the producer warpgroup gives registers back, the consumers take them:
// 128 x 64 + 256 x 216 = 63488 <= 384 x 168 = 64512.  The launch is
// refused unless the kernel was compiled to exactly kScanLaunchRegs registers
// per thread.
constexpr int kScanLaunchRegs = 168;
constexpr int kProducerRegs = 64;
constexpr int kConsumerRegs = 216;
static_assert(kProducerThreads * kProducerRegs + 32 * kConsumerWarps * kConsumerRegs <=
                  kScanThreads * kScanLaunchRegs,
              "register split exceeds the launch allocation");
constexpr int kMR = 8;                               // requests per thread
constexpr int kNW = 16;                              // 32-bit words per thread
constexpr int kStages = 6;                           // smem pipeline depth
constexpr int kStageBytes = 36 * 1024;               // table tile + masks, per stage
constexpr int kScanSmem = kStages * kStageBytes + 256;

// Warp layout of a CTA tile: LW lanes along the row (W), 32/LW lanes along
// the requests; WB warps along requests, WW along W and WK along buckets
// (WB * WW * WK = 8).  Warps along buckets take alternate rows of each stage
// and XOR-reduce their partials into the output at the end.
struct Shape {
  uint8_t lw_log2;     // 2..5
  uint8_t wb;          // warps along B
  uint8_t ww;          // warps along W
  uint8_t wk;          // warps along k (buckets)
  uint8_t srows_log2;  // rows (buckets) per pipeline stage
  __host__ __device__ int lw() const { return 1 << lw_log2; }
  __host__ __device__ int bt() const { return wb * (32 / lw()) * kMR; }  // requests per tile
  __host__ __device__ int wt() const { return ww * lw() * kNW; }         // words per tile
  __host__ __device__ int srows() const { return 1 << srows_log2; }
};

struct ScanJob {
  const uint32_t* T;   // table, n rows of Wd words
  const uint64_t* R;   // request bits, B rows of words64
  uint32_t* out;       // B rows of Wd words (initialised first when split)
  const uint8_t* seeds;  // B x 32-byte mask seeds (serialized PIR), or null
  uint64_t n;
  uint32_t Wd;         // row length in 32-bit words (d*msg_bytes/4)
  uint32_t words64;    // u64 words per request row
  uint32_t B;
  Shape shape;
  uint32_t n_bt, n_wt, n_kc;
  uint32_t kc_rows;    // buckets per k-chunk (multiple of 64)
  uint32_t item_begin; // index of this job's first item in the launch
  uint32_t split;      // partial replies are XOR-reduced (n_kc > 1, wk > 1 or masked)
};

constexpr uint32_t kItemCounterSlots = 256;  // launches with distinct item counters
constexpr uint32_t kEndItem = 0xFFFFFFFFu;

struct ScanLaunch {
  uint32_t njobs;
  uint32_t total_items;
  uint32_t counter_slot;  // this launch's item counter (reset by the zero kernel)
  uint32_t dynamic;       // claim items from the counter (else CTA c takes c, c + grid, ...)
  ScanJob jobs[TPIR_MAX_JOBS];
};
static_assert(sizeof(ScanLaunch) <= 32000, "kernel parameters must stay below 32 KB");
// Assigns the next item-counter slot (rotating).
uint32_t next_counter_slot();

// Schedule of a one-table tensor-core launch: mode 0 = planned (above 128
// requests with TMA-staged rows: items on CTA pairs; else spans or items as
// the cost model finds), 1 = spans (if admissible), 2 = items of kc_rows
// buckets (0: the cost model's size; on CTA pairs above 128 requests), 3 =
// the same items on single CTAs; loads = 1: request words loaded by the
// expander threads instead of staged by TMA (room for a deeper ring of table
// stages; single CTAs).
struct GSched {
  uint32_t mode = 0;
  uint32_t kc_rows = 0;
  uint32_t loads = 0;
};
// Fills a job's tiling from its shape/k-chunking and validates smem fit.
bool finalize_job(ScanJob& j);
Shape choose_shape(uint32_t Wd, uint32_t B);
// Tuned shapes (plan.cpp): the shape the autotuner measured fastest for a
// row width and a batch-size class, if any.
bool plan_lookup(uint32_t Wd, uint32_t B, Shape* out);
// Tuned kernel choice (plan.cpp) for a row width, batch-size class and
// table-size class: the kernel and, for the tensor-core kernel, its schedule.
struct KernelPlan {
  int kernel = 0;
  GSched sched;
};
// *exact (if given): the plan was tuned for this table-size class; plans of
// another size class lend their kernel choice, not their schedule.
bool kernel_plan_lookup(uint32_t Wd, uint32_t B, uint64_t n, KernelPlan* out,
                        bool* exact = nullptr);
int scan_stage_bytes(const Shape& s);

// Launch with programmatic dependent launch (PDL) allowed: the kernel may
// start while the previous kernel of the stream runs; it must execute
// griddepcontrol.wait before touching anything that kernel writes.
// Kernel launches the library has enqueued in this process (every kind);
// tpir_kernel_launches() returns it.
inline std::atomic<uint64_t> g_kernel_launches{0};
inline void count_launches(uint64_t k = 1) { g_kernel_launches.fetch_add(k, std::memory_order_relaxed); }

template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem,
                              cudaStream_t st, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  const cudaError_t e = cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
  if (e == cudaSuccess) count_launches();
  return e;
}

// Launch helpers (scan.cu).  All return cudaError_t of the launch.
cudaError_t launch_batched(const ScanLaunch& L, int grid, cudaStream_t st);
// seeds: B x 32-byte mask seeds, or null (the replies start at zero)
cudaError_t launch_plain(const uint32_t* T, uint64_t n, uint32_t Wd, const uint64_t* R,
                         uint32_t words64, uint32_t B, uint32_t* out, const uint8_t* seeds,
                         cudaStream_t st, int ctas);
cudaError_t launch_zero_outputs(const ScanLaunch& L, cudaStream_t st);
// Initialises B replies of row_u4 16-byte words before a scan XOR-reduces into
// them: zeros, or the masks of `seeds` (PDL-chained).
cudaError_t launch_init_replies(uint4* out, uint32_t B, uint32_t row_u4, const uint8_t* seeds,
                                cudaStream_t st);
// Tensor-core batched read (gf2mma.cu): the GF(2) product as an exact integer
// product of 0/1 matrices on tcgen05 (packed e2m1 operands), reduced mod 2.
// Tt is the table's bit-transposed copy (tcopy.cu).
cudaError_t launch_gf2_mma(const uint64_t* Tt, uint64_t n, uint32_t Wd, const uint64_t* R,
                           uint32_t words64, uint32_t B, uint32_t* out, const uint8_t* seeds,
                           cudaStream_t st, const GSched* sched = nullptr);
// True if span mode is admissible for this shape (at most one k-chunk of
// stages per CTA).
bool gf2_span_ok(uint64_t n, uint32_t Wd, uint32_t B);
struct M4Request;
// Many tables in one launch of the tensor-core kernel (up to TPIR_MAX_JOBS).
cudaError_t launch_gf2_mma_multi(const M4Request* reqs, uint32_t count, cudaStream_t st);
int device_sm_count();
int plain_ctas_per_sm();
int batched_ctas_per_sm();

// State kernels (state.cu)
struct MoveOp {   // one step of a write's slot moves, executed in order
  uint64_t dst;   // slot index (bucket*d + j), or kTmpSlot
  uint64_t src;   // slot index, kTmpSlot, or payload index (kind 1)
  uint32_t kind;  // 0 copy slot->slot, 1 payload->slot, 2 zero slot
  uint32_t pad;
};
constexpr uint64_t kTmpSlot = ~0ull;
cudaError_t launch_apply_moves(uint8_t* table, uint32_t z, const MoveOp* ops, uint32_t nops,
                               const uint8_t* payloads, uint8_t* tmp, cudaStream_t st);
// A small batch of writes with its moves and new messages in the kernel
// parameters (no staging): at most OPS moves and BYTES of messages (payload
// index i = bytes i*z .. of `payload`).  Two sizes: the launch copies the whole
// parameter block, so a single write of a slot up to 4 KiB takes the small one.
template <uint32_t OPS, uint32_t BYTES>
struct ParamMovesT {
  static constexpr uint32_t kOps = OPS, kBytes = BYTES;
  uint32_t nops;
  uint32_t pad;
  MoveOp ops[OPS];
  __align__(16) uint8_t payload[BYTES];
};
using ParamMovesS = ParamMovesT<48, 4096>;
using ParamMoves = ParamMovesT<384, 20 * 1024>;
constexpr uint32_t kParamOps = ParamMoves::kOps;
constexpr uint32_t kParamBytes = ParamMoves::kBytes;
static_assert(sizeof(ParamMoves) + 64 < 32000, "kernel parameters must stay below 32 KB");
cudaError_t launch_apply_moves_param(uint8_t* table, uint32_t z, const ParamMoves& m, uint8_t* tmp,
                                     cudaStream_t st);
cudaError_t launch_apply_moves_param(uint8_t* table, uint32_t z, const ParamMovesS& m, uint8_t* tmp,
                                     cudaStream_t st);
cudaError_t launch_bloom_set(uint64_t* delta, const uint64_t* pos, uint64_t count, cudaStream_t st);
cudaError_t launch_bloom_or(uint64_t* delta, const uint64_t* vec, uint64_t m, cudaStream_t st);
cudaError_t launch_bloom_union(const uint64_t* deltas, uint32_t window, uint64_t words,
                               uint64_t* out, cudaStream_t st);

// Bit-transposed copy of a table for the tensor-core read (tcopy.cu):
// Tt[kb][c] holds bit c of the rows of buckets 64 kb .. 64 kb + 63.
constexpr uint32_t kTcopyMaxBlocks = 480;  // blocks a partial rebuild takes by value
struct TcopyBlocks {
  uint32_t count;  // 0: every block
  uint32_t pad;
  uint64_t kb[kTcopyMaxBlocks];
};
static_assert(sizeof(TcopyBlocks) + 64 < 32000, "kernel parameters must stay below 32 KB");
uint64_t tcopy_bytes(uint64_t n, uint32_t row_bytes);
int read_device_status_and_clear(int* status);
// Device address of the status word on the current device (for kernels in
// other translation units).
int* device_status_word();
// Four-Russians batched read (m4rm.cu): one table, or many in one launch.
struct M4Request {
  const uint32_t* T;
  uint64_t n;
  uint32_t Wd;
  const uint64_t* R;
  uint32_t words64;
  uint32_t B;
  uint32_t* out;
  const uint8_t* seeds;  // B x 32-byte mask seeds, or null
  const uint64_t* Tt = nullptr;  // tensor-core jobs: the bit-transposed table
  uint32_t kc_rows = 0;          // tensor-core jobs: k-chunk rows (0: planned)
  uint32_t loads = 0;            // tensor-core jobs: request words loaded by threads
};
cudaError_t launch_m4rm(const uint32_t* T, uint64_t n, uint32_t Wd, const uint64_t* R,
                        uint32_t words64, uint32_t B, uint32_t* out, const uint8_t* seeds,
                        cudaStream_t st);
// Serialized-PIR helpers (mask.cu): the masks alone, and the leader's XOR of
// several replies.
cudaError_t launch_mask_fill(uint4* out, uint32_t rows, uint32_t row_u4, const uint8_t* seeds,
                             cudaStream_t st);
constexpr uint32_t kMaxCombine = 64;
cudaError_t launch_xor_combine(const uint4* const* srcs, uint32_t count, uint64_t n4, uint4* dst,
                               cudaStream_t st);
// wide: 512-request tiles (jobs of more than 256 requests), else 256
cudaError_t launch_m4rm_multi(const M4Request* reqs, uint32_t count, bool wide, cudaStream_t st);
constexpr uint32_t kM4rmMinB = 176;  // batch from which the Four-Russians kernel beats LOP3
constexpr uint32_t kPlainMaxB = 4;    // requests per launch of the plain kernel
constexpr uint32_t kTensorMinB = 48;  // batch from which the tensor-core kernel beats LOP3 (measured)
cudaError_t launch_selftest_wait(uint64_t limit_ns, cudaStream_t st);
// Rice coding of sparse bit vectors (rice.cu).
struct RiceRequest {
  const uint64_t* bits;  // ceil(m/64) words
  uint64_t m;
  int32_t k;             // < 0: chosen from the set-bit count
  uint32_t* out;         // cap_words 32-bit words
  uint64_t cap_words;
  uint64_t* result;      // device: nbits (UINT64_MAX if past cap), count, k
};
// scratch: rice_scratch_bytes(m) of device memory, free until the stream
// passes the encode
size_t rice_scratch_bytes(uint64_t m);
cudaError_t launch_rice_encode(const RiceRequest& q, void* scratch, cudaStream_t st);

// Host cuckoo metadata (cuckoo.cpp): same placement rules as the paper's
// Section 5.3 insertion; emits the device moves of one insertion.
class CuckooMeta {
 public:
  CuckooMeta(uint64_t n, uint32_t d);
  void set_policy(uint64_t capacity, uint32_t max_evictions, uint64_t seed);
  void clear();
  uint64_t live() const { return live_; }
  // What one successful insert changed, so that a caller whose device work
  // could not be enqueued can take it back (rollback): the slots and item
  // positions it overwrote, the ring entry of the new item, and the counters
  // and generator state before it.
  struct Undo {
    std::vector<std::pair<uint64_t, uint64_t>> slots, items;
    uint64_t head = 0, live = 0, next_seq = 0, rng = 0;
    uint64_t ring_b1 = 0, ring_b2 = 0, ring_slot = 0;
  };
  // Returns TPIR_OK / TPIR_EINVAL / TPIR_EFULL; on OK appends the moves to
  // `ops` (payload index `payload_idx` for the new message) and, if `undo`
  // is given, records how to take the insert back.
  tpir_status insert(uint64_t b1, uint64_t b2, uint64_t payload_idx, std::vector<MoveOp>& ops,
                     uint32_t* evictions, Undo* undo = nullptr);
  // Takes back a successful insert (the most recent one not yet taken back):
  // the metadata, counters and generator are as if it had not been made.
  void rollback(const Undo& u);
  uint64_t capacity() const { return capacity_; }
  uint32_t max_evictions() const { return max_ev_; }
  uint64_t rng_state() const { return rng_; }
  void set_rng_state(uint64_t r) { rng_ = r; }

 private:
  static constexpr uint64_t kEmpty = ~0ull;
  uint64_t n_;
  uint32_t d_;
  uint64_t capacity_ = 0;
  uint32_t max_ev_ = 500;
  uint64_t rng_ = 0;
  std::vector<uint64_t> slot_item_;   // item seq held by each slot
  std::vector<uint64_t> item_slot_;   // ring indexed by seq % ring
  std::vector<uint64_t> item_b1_, item_b2_;
  uint64_t head_ = 0, next_seq_ = 0, live_ = 0;
  uint64_t ring_ = 0;
  uint64_t next_rand();
  int64_t lowest_free(uint64_t e) const;
  uint64_t& islot(uint64_t seq) { return item_slot_[seq % ring_]; }
};

}  // namespace tpir

// Host/device staging of one batch of writes (payloads, move list, Bloom
// positions); reusable once the stream that consumed it has passed that point.
struct tpir_write_staging {
  uint8_t* h = nullptr;  // pinned
  uint64_t h_cap = 0;
  uint8_t* d_payload = nullptr;
  uint64_t pay_cap = 0;
  tpir::MoveOp* d_ops = nullptr;
  uint64_t ops_cap = 0;
  uint64_t* d_pos = nullptr;
  uint64_t pos_cap = 0;
  cudaEvent_t done = nullptr;  // recorded after the last work that read the staging
  void release();
};

// The db object behind the opaque C handle.
struct tpir_bloom_state {
  uint64_t m = 0, words = 0;
  uint32_t k = 0, window = 1, per_delta = 0;
  uint32_t cur = 0, count = 0;
  uint64_t* d_deltas = nullptr;   // window x words
  uint64_t* d_out = nullptr;      // words
  uint32_t* d_rice = nullptr;     // compressed-stream staging (GetUpdates)
  uint64_t rice_cap = 0;          // its bytes
  uint64_t* d_rice_res = nullptr; // nbits, count, k
  void* d_rice_scratch = nullptr;  // per-block scan values
  uint64_t rice_scratch_cap = 0;
};

struct tpir_db {
  uint64_t n = 0;
  uint32_t d = 0, z = 0;
  uint32_t row_bytes = 0, Wd = 0, words64 = 0;  // words64: request row stride
  // row shard of a larger logical table: buckets [row_begin, row_begin + n)
  // of n_total (n_total = 0: a whole table); reads start req_off words into
  // each request row
  uint64_t n_total = 0, row_begin = 0;
  uint32_t req_off = 0;
  int device = 0;
  uint8_t* d_table = nullptr;
  uint64_t epoch = 0;
  int forced_kernel = 0;
  cudaStream_t stream = nullptr;        // the db's own stream (writes, sync reads)
  cudaEvent_t last_write = nullptr;     // recorded after each write
  cudaEvent_t stream_mark = nullptr;    // marks the db stream for foreign-stream writes
  std::vector<std::pair<cudaStream_t, cudaEvent_t>> read_events;  // async reads per stream
  tpir::CuckooMeta* meta = nullptr;
  // write staging of the db's own API calls
  tpir_write_staging stage;
  uint8_t* d_tmp = nullptr;             // one slot: breaks cycles of slot moves
  // sync read staging
  uint64_t* d_req = nullptr;
  uint8_t* d_out = nullptr;
  uint64_t req_cap = 0, out_cap = 0;
  // pipelined host-buffer reads: a copy stream, three slots of request and
  // reply buffers, and per slot the events copy-in done / scan done / copy-out done
  cudaStream_t copy_stream = nullptr;
  uint8_t* d_pipe = nullptr;
  uint64_t pipe_cap = 0;
  cudaEvent_t pipe_ev[9] = {nullptr};
  tpir_bloom_state bloom;
  // bit-transposed copy for the tensor-core read (allocated on first use,
  // then kept equal to the table in stream order)
  uint64_t* d_tt = nullptr;
  bool tt_valid = false;
};

namespace tpir {
// The bit-transposed copy (tcopy.cu): built if missing or stale, rebuilt after
// a bulk load (if it exists), and its blocks holding moved slots rebuilt after
// a write's moves; each enqueued on `st` after the table's own update.
cudaError_t tcopy_ensure(tpir_db* db, cudaStream_t st);
cudaError_t tcopy_after_load(tpir_db* db, cudaStream_t st);
cudaError_t tcopy_after_moves(tpir_db* db, const MoveOp* ops, size_t nops, cudaStream_t st);
tpir_status set_error(tpir_status s);
tpir_status cuda_status(cudaError_t e);
// enqueue a read of db on stream (device buffers), honoring write ordering;
// d_seeds (B x 32 bytes) masks the replies (serialized PIR), null = plain
// (*kernel_used, if given, receives the kernel chosen: 1 plain, 2 register-
// tiled, 3 plain register-streaming, 4 Four-Russians, 5 tensor-core)
// kernel_choice (0 = automatic) overrides the choice
tpir_status enqueue_read(tpir_db* db, const uint64_t* d_req, uint32_t B, void* d_out,
                         cudaStream_t st, const uint8_t* d_seeds = nullptr,
                         int* kernel_used = nullptr, int kernel_choice = 0);
// The kernel a read of B requests takes on db unless told otherwise.
int auto_kernel(const tpir_db* db, uint32_t B);
// order stream `st` after the db's last write, and record a read event
void order_after_writes(tpir_db* db, cudaStream_t st);
void note_read(tpir_db* db, cudaStream_t st);
// A batch of writes: host-side placement, device moves enqueued on `st`
// using `stg` (which must be free); records db->last_write on `st`.
tpir_status apply_writes_core(tpir_db* db, uint32_t count, const uint64_t* b1, const uint64_t* b2,
                              const uint8_t* msgs, tpir_status* st_out, uint32_t* ev_out,
                              cudaStream_t st, tpir_write_staging& stg);
// Bloom positions of `count` writes, same staging contract.
tpir_status bloom_insert_core(tpir_db* db, const uint64_t* pos, uint32_t count, cudaStream_t st,
                              tpir_write_staging& stg);
// Many jobs in one persistent launch per kernel kind (Four-Russians for large
// batches, register-tiled for the rest); no cross-stream ordering done here.
tpir_status enqueue_multi(const tpir_read_job* jobs, uint32_t njobs, cudaStream_t st);
tpir_status enqueue_multi_lop3(const tpir_read_job* jobs, uint32_t njobs, cudaStream_t st);
int multi_kernel(const tpir_read_job& q);
void order_writes_after_reads(tpir_db* db, cudaStream_t st);
bool grow_dev(void** p, uint64_t* cap, uint64_t need);
bool grow_pinned(void** p, uint64_t* cap, uint64_t need);
uint64_t db_device_bytes(uint64_t n, uint32_t d, uint32_t z);
ScanJob make_job(const tpir_db* db, const uint64_t* d_req, uint32_t B, void* d_out);
void plan_single(ScanJob& j, int grid);
int batched_grid();
}  // namespace tpir
