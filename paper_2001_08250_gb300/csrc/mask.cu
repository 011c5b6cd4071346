// Serialized PIR (Section 6) helpers around the masked reads: the one-time
// masks alone (step 9, or a leader checking a combination) and the leader's
// XOR of the servers' masked replies (step 8).  The masked reads themselves
// run through the scan kernels (db.cpp), whose reply-initialisation kernels
// write the masks.
#include <algorithm>

#include "chacha.cuh"
#include "tpir_internal.h"

namespace tpir {
namespace {

// Both kernels are launched with PDL: they let the next kernel of the stream
// start at once, and wait for the previous one before touching memory.
__global__ void mask_fill_kernel(uint4* __restrict__ out, uint32_t rows, uint32_t row_u4,
                                 const uint8_t* __restrict__ seeds) {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  asm volatile("griddepcontrol.wait;" ::: "memory");
  init_replies(out, rows, row_u4, seeds, blockIdx.x * (uint64_t)blockDim.x + threadIdx.x,
               (uint64_t)gridDim.x * blockDim.x);
}

struct CombineSrcs {
  const uint4* p[kMaxCombine];
  uint32_t count;
};

// dst[i] = XOR over the sources of src[i]; each element is read and written
// by one thread only, so dst may be one of the sources.
__global__ void __launch_bounds__(256) xor_combine_kernel(const __grid_constant__ CombineSrcs S,
                                                          uint64_t n4, uint4* dst) {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  asm volatile("griddepcontrol.wait;" ::: "memory");
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n4;
       i += (uint64_t)gridDim.x * blockDim.x) {
    uint4 a = S.p[0][i];
    for (uint32_t k = 1; k < S.count; ++k) {
      const uint4 b = S.p[k][i];
      a.x ^= b.x;
      a.y ^= b.y;
      a.z ^= b.z;
      a.w ^= b.w;
    }
    dst[i] = a;
  }
}

}  // namespace

cudaError_t launch_mask_fill(uint4* out, uint32_t rows, uint32_t row_u4, const uint8_t* seeds,
                             cudaStream_t st) {
  const uint64_t blocks = static_cast<uint64_t>(rows) * ((row_u4 + 3) / 4);
  if (blocks == 0) return cudaSuccess;
  const uint32_t grid = static_cast<uint32_t>(
      std::min<uint64_t>((blocks + 255) / 256, static_cast<uint64_t>(device_sm_count()) * 8));
  return launch_pdl(mask_fill_kernel, dim3(grid), dim3(256), 0, st, out, rows, row_u4, seeds);
}

cudaError_t launch_xor_combine(const uint4* const* srcs, uint32_t count, uint64_t n4, uint4* dst,
                               cudaStream_t st) {
  if (n4 == 0) return cudaSuccess;
  if (count == 0 || count > kMaxCombine) return cudaErrorInvalidValue;
  CombineSrcs S{};
  for (uint32_t k = 0; k < count; ++k) S.p[k] = srcs[k];
  S.count = count;
  const uint32_t grid = static_cast<uint32_t>(
      std::min<uint64_t>((n4 + 255) / 256, static_cast<uint64_t>(device_sm_count()) * 8));
  return launch_pdl(xor_combine_kernel, dim3(grid), dim3(256), 0, st, S, n4, dst);
}

}  // namespace tpir

using namespace tpir;

extern "C" tpir_status tpir_mask_generate(const uint8_t* d_seeds, uint32_t rows, uint64_t nbytes,
                                          void* d_out, void* stream) {
  if (rows == 0 || nbytes == 0) return TPIR_OK;
  if (!d_seeds || !d_out || (nbytes & 15) || nbytes / 16 > 0xFFFFFFFFull ||
      (reinterpret_cast<uintptr_t>(d_seeds) & 15) || (reinterpret_cast<uintptr_t>(d_out) & 15))
    return set_error(TPIR_EINVAL);
  return cuda_status(launch_mask_fill(static_cast<uint4*>(d_out), rows,
                                      static_cast<uint32_t>(nbytes / 16), d_seeds,
                                      static_cast<cudaStream_t>(stream)));
}

extern "C" tpir_status tpir_xor_combine(const void* const* d_srcs, uint32_t count, uint64_t nbytes,
                                        void* d_dst, void* stream) {
  if (!d_srcs || !d_dst || count == 0 || count > kMaxCombine || (nbytes & 15) ||
      (reinterpret_cast<uintptr_t>(d_dst) & 15))
    return set_error(TPIR_EINVAL);
  const uint4* srcs[kMaxCombine];
  for (uint32_t k = 0; k < count; ++k) {
    if (!d_srcs[k] || (reinterpret_cast<uintptr_t>(d_srcs[k]) & 15)) return set_error(TPIR_EINVAL);
    srcs[k] = static_cast<const uint4*>(d_srcs[k]);
  }
  return cuda_status(launch_xor_combine(srcs, count, nbytes / 16, static_cast<uint4*>(d_dst),
                                        static_cast<cudaStream_t>(stream)));
}
