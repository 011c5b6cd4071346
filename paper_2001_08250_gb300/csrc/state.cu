// Server-state kernels for sm_103a.
//
//  apply_moves_kernel  the device half of a cuckoo write (Section 5.3): the
//                      host computes where every touched item ends up and
//                      emits an ordered list of slot copies (with a one-slot
//                      temporary to break cycles), payload writes and slot
//                      clears (FIFO collection); one CTA runs them in order.
//  bloom_*_kernel      Section 7: OR a write's interest vector (k positions or
//                      a whole vector) into the current delta, and form the
//                      global interest vector as the OR of the window's deltas.
#include "tpir_internal.h"

namespace tpir {
namespace {

__global__ void __launch_bounds__(256) apply_moves_kernel(uint8_t* __restrict__ table, uint32_t z,
                                                          const MoveOp* __restrict__ ops,
                                                          uint32_t nops,
                                                          const uint8_t* __restrict__ payloads,
                                                          uint8_t* __restrict__ tmp) {
  const uint32_t z4 = z / 16;  // uint4 per slot
  for (uint32_t i = 0; i < nops; ++i) {
    const MoveOp op = ops[i];
    uint4* dst = reinterpret_cast<uint4*>(op.dst == kTmpSlot ? tmp : table + op.dst * z);
    if (op.kind == 2) {
      for (uint32_t j = threadIdx.x; j < z4; j += blockDim.x) dst[j] = make_uint4(0u, 0u, 0u, 0u);
    } else {
      const uint8_t* s8 = op.kind == 1 ? payloads + op.src * z
                                       : (op.src == kTmpSlot ? tmp : table + op.src * z);
      const uint4* src = reinterpret_cast<const uint4*>(s8);
      for (uint32_t j = threadIdx.x; j < z4; j += blockDim.x) dst[j] = src[j];
    }
    __syncthreads();  // the next op may read what this one wrote
  }
}

// The same moves for a small batch of writes, with the move list and the new
// messages passed by value in the kernel parameters: no staging buffer, no
// copy before the launch, so a single write costs one launch.
template <typename PM>
__global__ void __launch_bounds__(256) apply_moves_param_kernel(uint8_t* __restrict__ table,
                                                                uint32_t z,
                                                                const __grid_constant__ PM m,
                                                                uint8_t* __restrict__ tmp) {
  const uint32_t z4 = z / 16;
  for (uint32_t i = 0; i < m.nops; ++i) {
    const MoveOp op = m.ops[i];
    uint4* dst = reinterpret_cast<uint4*>(op.dst == kTmpSlot ? tmp : table + op.dst * z);
    if (op.kind == 2) {
      for (uint32_t j = threadIdx.x; j < z4; j += blockDim.x) dst[j] = make_uint4(0u, 0u, 0u, 0u);
    } else if (op.kind == 1) {
      const uint4* src = reinterpret_cast<const uint4*>(m.payload + op.src * z);
      for (uint32_t j = threadIdx.x; j < z4; j += blockDim.x) dst[j] = src[j];
    } else {
      const uint4* src = reinterpret_cast<const uint4*>(op.src == kTmpSlot ? tmp : table + op.src * z);
      for (uint32_t j = threadIdx.x; j < z4; j += blockDim.x) dst[j] = src[j];
    }
    __syncthreads();  // the next op may read what this one wrote
  }
}

__global__ void bloom_set_kernel(uint64_t* __restrict__ delta, const uint64_t* __restrict__ pos,
                                 uint64_t count) {
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < count;
       i += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t p = pos[i];
    atomicOr(reinterpret_cast<unsigned long long*>(delta + (p >> 6)), 1ull << (p & 63));
  }
}

__global__ void bloom_or_kernel(uint64_t* __restrict__ delta, const uint64_t* __restrict__ vec,
                                uint64_t m) {
  const uint64_t words = (m + 63) / 64;
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < words;
       i += (uint64_t)gridDim.x * blockDim.x) {
    uint64_t v = vec[i];
    if (i == words - 1 && (m & 63)) v &= (1ull << (m & 63)) - 1;
    delta[i] |= v;
  }
}

__global__ void bloom_union_kernel(const uint64_t* __restrict__ deltas, uint32_t window,
                                   uint64_t words, uint64_t* __restrict__ out) {
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < words;
       i += (uint64_t)gridDim.x * blockDim.x) {
    uint64_t v = 0;
    for (uint32_t j = 0; j < window; ++j) v |= deltas[j * words + i];
    out[i] = v;
  }
}

}  // namespace

cudaError_t launch_apply_moves(uint8_t* table, uint32_t z, const MoveOp* ops, uint32_t nops,
                               const uint8_t* payloads, uint8_t* tmp, cudaStream_t st) {
  if (nops == 0) return cudaSuccess;
  apply_moves_kernel<<<1, 256, 0, st>>>(table, z, ops, nops, payloads, tmp);
  count_launches();
  return cudaGetLastError();
}

cudaError_t launch_apply_moves_param(uint8_t* table, uint32_t z, const ParamMoves& m, uint8_t* tmp,
                                     cudaStream_t st) {
  if (m.nops == 0) return cudaSuccess;
  apply_moves_param_kernel<ParamMoves><<<1, 256, 0, st>>>(table, z, m, tmp);
  count_launches();
  return cudaGetLastError();
}

cudaError_t launch_apply_moves_param(uint8_t* table, uint32_t z, const ParamMovesS& m, uint8_t* tmp,
                                     cudaStream_t st) {
  if (m.nops == 0) return cudaSuccess;
  apply_moves_param_kernel<ParamMovesS><<<1, 256, 0, st>>>(table, z, m, tmp);
  count_launches();
  return cudaGetLastError();
}

cudaError_t launch_bloom_set(uint64_t* delta, const uint64_t* pos, uint64_t count,
                             cudaStream_t st) {
  if (count == 0) return cudaSuccess;
  const uint64_t blocks = (count + 255) / 256;
  bloom_set_kernel<<<static_cast<uint32_t>(blocks < 1024 ? blocks : 1024), 256, 0, st>>>(delta, pos,
                                                                                        count);
  count_launches();
  return cudaGetLastError();
}

cudaError_t launch_bloom_or(uint64_t* delta, const uint64_t* vec, uint64_t m, cudaStream_t st) {
  const uint64_t words = (m + 63) / 64;
  const uint64_t blocks = (words + 255) / 256;
  bloom_or_kernel<<<static_cast<uint32_t>(blocks < 1024 ? blocks : 1024), 256, 0, st>>>(delta, vec,
                                                                                       m);
  count_launches();
  return cudaGetLastError();
}

cudaError_t launch_bloom_union(const uint64_t* deltas, uint32_t window, uint64_t words,
                               uint64_t* out, cudaStream_t st) {
  const uint64_t blocks = (words + 255) / 256;
  bloom_union_kernel<<<static_cast<uint32_t>(blocks < 1024 ? blocks : 1024), 256, 0, st>>>(
      deltas, window, words, out);
  count_launches();
  return cudaGetLastError();
}

}  // namespace tpir
