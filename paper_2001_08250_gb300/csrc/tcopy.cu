// Bit-transposed copy of a table for the tensor-core read.
//
// The tensor-core kernel multiplies the request bits by the table bits with
// packed 4-bit operands, which the tensor cores accept only K-major: for each
// table column (bit c of a row), its bits over consecutive buckets must be
// contiguous.  The row-major table (a bucket's row contiguous) is therefore
// kept a second time, bit-transposed in 64-bucket blocks:
//
//   Tt[kb][c]  (uint64)  bit i = bit c of the row of bucket 64 kb + i
//                        (bit c of a row: bit c % 8 of byte c / 8, LSB first);
//                        buckets past n are zero.
//
// The copy is built in full on first use and after a bulk load, and block by
// block after the slot moves of a write (only the 64-bucket blocks holding a
// moved slot), in the same stream order as the table itself, so it always
// matches the table for every later read.
#include <algorithm>
#include <vector>

#include "tpir_internal.h"

namespace tpir {
namespace {

// One work item: block kb (64 buckets) x 8 words (256 columns) of the row.
// Warp w takes word w: lane l holds word w of buckets 64 kb + l and
// 64 kb + 32 + l, and 32 ballots give the word's 32 columns over the 64
// buckets; lane j keeps column 32 w + j and stores it (32 lanes x 8 bytes,
// contiguous).
__global__ void __launch_bounds__(256) tcopy_kernel(const uint32_t* __restrict__ T, uint64_t n,
                                                    uint32_t Wd, uint64_t* __restrict__ Tt,
                                                    uint64_t nblocks, const __grid_constant__ TcopyBlocks bl) {
  const uint32_t warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t chunks = (Wd + 7) / 8;
  const uint64_t items = (bl.count ? bl.count : nblocks) * chunks;
  const uint64_t row_bits = static_cast<uint64_t>(Wd) * 32;
  for (uint64_t it = blockIdx.x; it < items; it += gridDim.x) {
    const uint64_t kb = bl.count ? bl.kb[it / chunks] : it / chunks;
    const uint32_t w = static_cast<uint32_t>(it % chunks) * 8 + warp;
    if (w >= Wd) continue;  // uniform over the warp
    const uint64_t r0 = 64 * kb + lane, r1 = r0 + 32;
    const uint32_t x0 = r0 < n ? __ldg(T + r0 * Wd + w) : 0u;
    const uint32_t x1 = r1 < n ? __ldg(T + r1 * Wd + w) : 0u;
    uint64_t mine = 0;
#pragma unroll
    for (uint32_t j = 0; j < 32; ++j) {
      const uint32_t lo = __ballot_sync(0xFFFFFFFFu, (x0 >> j) & 1u);
      const uint32_t hi = __ballot_sync(0xFFFFFFFFu, (x1 >> j) & 1u);
      if (lane == j) mine = static_cast<uint64_t>(lo) | (static_cast<uint64_t>(hi) << 32);
    }
    Tt[kb * row_bits + static_cast<uint64_t>(w) * 32 + lane] = mine;
  }
}

cudaError_t launch_tcopy(const tpir_db* db, const TcopyBlocks& bl, cudaStream_t st) {
  const uint64_t nblocks = (db->n + 63) / 64;
  const uint64_t items = (bl.count ? bl.count : nblocks) * ((db->Wd + 7) / 8);
  if (items == 0) return cudaSuccess;
  const uint64_t grid = std::min<uint64_t>(items, static_cast<uint64_t>(device_sm_count()) * 8);
  tcopy_kernel<<<static_cast<uint32_t>(grid), 256, 0, st>>>(
      reinterpret_cast<const uint32_t*>(db->d_table), db->n, db->Wd, db->d_tt, nblocks, bl);
  count_launches();
  return cudaGetLastError();
}

}  // namespace

uint64_t tcopy_bytes(uint64_t n, uint32_t row_bytes) { return (n + 63) / 64 * 64 * row_bytes; }

cudaError_t tcopy_ensure(tpir_db* db, cudaStream_t st) {
  if (db->tt_valid) return cudaSuccess;
  if (!db->d_tt) {
    cudaError_t e = cudaMalloc(reinterpret_cast<void**>(&db->d_tt), tcopy_bytes(db->n, db->row_bytes));
    if (e != cudaSuccess) {
      db->d_tt = nullptr;
      return e;
    }
  }
  TcopyBlocks all{};
  const cudaError_t e = launch_tcopy(db, all, st);
  if (e == cudaSuccess) db->tt_valid = true;
  return e;
}

cudaError_t tcopy_after_load(tpir_db* db, cudaStream_t st) {
  if (!db->d_tt) return cudaSuccess;  // built on first use
  db->tt_valid = false;
  return tcopy_ensure(db, st);
}

cudaError_t tcopy_after_moves(tpir_db* db, const MoveOp* ops, size_t nops, cudaStream_t st) {
  if (!db->d_tt || !db->tt_valid || nops == 0) return cudaSuccess;
  TcopyBlocks bl{};
  std::vector<uint64_t> kbs;
  kbs.reserve(nops);
  for (size_t i = 0; i < nops; ++i)
    if (ops[i].dst != kTmpSlot) kbs.push_back(ops[i].dst / db->d / 64);
  std::sort(kbs.begin(), kbs.end());
  kbs.erase(std::unique(kbs.begin(), kbs.end()), kbs.end());
  if (kbs.size() > kTcopyMaxBlocks) return launch_tcopy(db, bl, st);  // rebuild it all
  bl.count = static_cast<uint32_t>(kbs.size());
  std::copy(kbs.begin(), kbs.end(), bl.kb);
  return launch_tcopy(db, bl, st);
}

}  // namespace tpir
