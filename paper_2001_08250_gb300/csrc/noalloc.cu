// A cuckoo write that allocates nothing, for callers that cannot allocate.
//
// tpir_write may grow its pinned host staging and its device staging
// (payload, move list) with cudaMallocHost / cudaMalloc, and every write
// routes the moves through a temporary slot the db allocated.  Some callers
// cannot afford that: a serving thread for which a cudaMalloc (which may
// synchronise the whole device) is an unbounded stall, or a process whose
// device memory is all owned by another allocator (a framework's caching
// pool) under a hard budget.  tpir_write_noalloc takes the message as the
// caller's device buffer, passes the ordered slot moves to the kernel by value
// (in its parameters), and uses as its temporary slot a file-scope device
// array, sized once for every device that loads the library.
#include <cstring>
#include <mutex>

#include "tpir_internal.h"

namespace tpir {
namespace {

constexpr uint32_t kNoallocMaxMsgBytes = 64 * 1024;   // largest slot the temporary holds
constexpr uint32_t kNoallocMaxEvictions = 500;        // bound on the walk length accepted
// Touched slots <= evictions + 3 (new item's slot, victims, final free slot,
// collected slot); each needs at most one copy plus one temporary hop.
constexpr uint32_t kNoallocMaxOps = 2 * (kNoallocMaxEvictions + 3) + 2;

// The scratch: one slot for breaking cycles of slot moves.  Every call shares
// it and it keeps the last call's contents (nothing in it needs to start at
// zero: a move writes the temporary before reading it).
static __device__ __align__(256) uint8_t g_noalloc_tmp[kNoallocMaxMsgBytes];

// The move list travels in the kernel parameters; the launch copies the whole
// parameter block, so walks of up to 48 moves (nearly all) take a small one.
template <uint32_t OPS>
struct NoallocMovesT {
  uint32_t count;
  uint32_t pad;
  MoveOp ops[OPS];
};
using NoallocMoves = NoallocMovesT<kNoallocMaxOps>;
using NoallocMovesS = NoallocMovesT<48>;
static_assert(sizeof(NoallocMoves) + 64 < 32000, "kernel parameters must stay below 32 KB");

template <typename NM>
__global__ void __launch_bounds__(256) apply_moves_noalloc_kernel(
    uint8_t* __restrict__ table, uint32_t z, const __grid_constant__ NM m,
    const uint8_t* __restrict__ msg, uint8_t* __restrict__ tmp) {
  const uint32_t z4 = z / 16;
  for (uint32_t i = 0; i < m.count; ++i) {
    const MoveOp op = m.ops[i];
    uint4* dst = reinterpret_cast<uint4*>(op.dst == kTmpSlot ? tmp : table + op.dst * z);
    if (op.kind == 2) {
      for (uint32_t j = threadIdx.x; j < z4; j += blockDim.x) dst[j] = make_uint4(0u, 0u, 0u, 0u);
    } else {
      const uint8_t* s8 = op.kind == 1 ? msg : (op.src == kTmpSlot ? tmp : table + op.src * z);
      const uint4* src = reinterpret_cast<const uint4*>(s8);
      for (uint32_t j = threadIdx.x; j < z4; j += blockDim.x) dst[j] = src[j];
    }
    __syncthreads();  // the next move may read what this one wrote
  }
}

// Device address of g_noalloc_tmp on the current device, looked up once per
// device (the host-side name of the array is only a stand-in).
tpir_status noalloc_scratch(void** out) {
  static std::mutex mu;
  static void* addr[64] = {nullptr};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return TPIR_ECUDA;
  std::lock_guard<std::mutex> g(mu);
  if (!addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_tmp) != cudaSuccess || !p) return TPIR_ECUDA;
    addr[dev] = p;
  }
  *out = addr[dev];
  return TPIR_OK;
}

}  // namespace
}  // namespace tpir

using namespace tpir;

extern "C" tpir_status tpir_write_noalloc(tpir_db* db, uint64_t b1, uint64_t b2, const void* d_msg,
                                          uint32_t* evictions_out, void* stream) {
  if (evictions_out) *evictions_out = 0;
  if (!db || !d_msg || (reinterpret_cast<uintptr_t>(d_msg) & 15)) return TPIR_EINVAL;
  if (db->n_total) return TPIR_EINVAL;  // shards hold snapshots: no cuckoo writes
  if (db->z > kNoallocMaxMsgBytes) return TPIR_EINVAL;                   // slot too large
  if (db->meta->max_evictions() > kNoallocMaxEvictions) return TPIR_EINVAL;
  if (b1 >= db->n || b2 >= db->n) return TPIR_EINVAL;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  // the events that order this write against the db's other work cannot be
  // used across a capture boundary: refuse a stream being captured
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cap) != cudaSuccess) return TPIR_ECUDA;
  if (cap != cudaStreamCaptureStatusNone) return TPIR_EINVAL;
  void* tmp = nullptr;
  tpir_status s = noalloc_scratch(&tmp);
  if (s != TPIR_OK) return s;

  std::vector<MoveOp> ops;
  uint32_t ev = 0;
  CuckooMeta::Undo undo;
  s = db->meta->insert(b1, b2, 0, ops, &ev, &undo);
  if (s != TPIR_OK) {  // EFULL: metadata rolled back, nothing to move
    if (evictions_out) *evictions_out = ev;
    return s;
  }
  if (ops.size() > kNoallocMaxOps) {  // cannot happen within the bounds above
    db->meta->rollback(undo);
    return TPIR_EINVAL;
  }

  // after every read already submitted on this db (its own stream included)
  // and after every earlier write to it, whichever stream that ran on
  order_writes_after_reads(db, st);
  cudaError_t e = cudaEventRecord(db->stream_mark, db->stream);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(st, db->stream_mark, 0);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(st, db->last_write, 0);
  if (e == cudaSuccess) {
    const uint8_t* msg = static_cast<const uint8_t*>(d_msg);
    if (ops.size() <= 48) {
      NoallocMovesS m;
      m.count = static_cast<uint32_t>(ops.size());
      m.pad = 0;
      std::memcpy(m.ops, ops.data(), ops.size() * sizeof(MoveOp));
      apply_moves_noalloc_kernel<NoallocMovesS><<<1, 256, 0, st>>>(db->d_table, db->z, m, msg,
                                                                   static_cast<uint8_t*>(tmp));
      count_launches();
    } else {
      NoallocMoves m;
      m.count = static_cast<uint32_t>(ops.size());
      m.pad = 0;
      std::memcpy(m.ops, ops.data(), ops.size() * sizeof(MoveOp));
      apply_moves_noalloc_kernel<NoallocMoves><<<1, 256, 0, st>>>(db->d_table, db->z, m, msg,
                                                                  static_cast<uint8_t*>(tmp));
      count_launches();
    }
    e = cudaGetLastError();
  }
  // the tensor-core read's transposed copy (if the db has one) follows the
  // moves; it allocates nothing
  if (e == cudaSuccess) e = tcopy_after_moves(db, ops.data(), ops.size(), st);
  if (e == cudaSuccess) e = cudaEventRecord(db->last_write, st);
  if (e != cudaSuccess) {
    // the host placement is taken back: the table and its metadata agree
    db->meta->rollback(undo);
    return cuda_status(e);
  }
  if (evictions_out) *evictions_out = ev;
  db->epoch += 1;
  return TPIR_OK;
}
