// Issue rate of the block-scaled 4-bit MMA the tensor-core read is built on
// (compiled and run by tests/test_gpu_mma_rates.py): back-to-back
// tcgen05.mma kind::mxf4 (e2m1 x e2m1, UE8M0 scales 1.0), K = 64, N = 224,
// operands in shared memory, on every SM:
//  - single:  cta_group::1, M = 128, one CTA per SM;
//  - pair:    cta_group::2, M = 256 over a cluster of two CTAs, each holding
//             128 rows of A and 112 rows of B.
// Prints cycles per MMA at 2070 MHz and the 0/1 multiply-add rate; every
// wait is bounded and a timeout is reported, not waited out.
#include <cstdint>
#include <cstdio>
#include <cuda_runtime.h>

#define CK(x)                                                                        \
  do {                                                                               \
    cudaError_t e_ = (x);                                                            \
    if (e_ != cudaSuccess) {                                                         \
      printf("CUDA %s at %d: %s\n", #x, __LINE__, cudaGetErrorString(e_));           \
      return 1;                                                                      \
    }                                                                                \
  } while (0)

constexpr int kN = 224;

__device__ __forceinline__ uint32_t saddr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ uint64_t gtimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// K-major operand without swizzle: 8-row x 16-byte core matrices, 128 bytes
// apart along K, 256 bytes apart along M / N (rows of 32 bytes = K 64)
__device__ __forceinline__ uint64_t desc(uint32_t addr) {
  return static_cast<uint64_t>((addr >> 4) & 0x3FFFu) | (static_cast<uint64_t>(128 >> 4) << 16) |
         (static_cast<uint64_t>(256 >> 4) << 32) | (1ull << 46);
}
__device__ __forceinline__ void cluster_sync() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" :::
                   "memory");
}

// PAIR = 0: cta_group::1, M = 128; PAIR = 1: cta_group::2, M = 256 (clusters of 2)
template <int PAIR>
__global__ void __launch_bounds__(128, 1) mma_rate(int iters, int* status) {
  __shared__ __align__(1024) uint8_t sA[128 * 32];
  __shared__ __align__(1024) uint8_t sB[kN * 32];
  __shared__ __align__(8) uint64_t bar;
  __shared__ uint32_t s_tmem;
  const uint32_t tid = threadIdx.x, warp = tid >> 5;
  uint32_t rank = 0;
  if (PAIR) asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(rank));
  for (int i = tid; i < 128 * 32; i += 128) sA[i] = (i * 7) & 1 ? 0x22 : 0x20;
  for (int i = tid; i < kN * 32; i += 128) sB[i] = (i * 5) & 2 ? 0x02 : 0x22;
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(saddr(&bar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    if (PAIR) {
      asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(
                       saddr(&s_tmem))
                   : "memory");
      asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
    } else {
      asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(
                       saddr(&s_tmem))
                   : "memory");
      asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = s_tmem;
  {  // scale factors 1.0 in columns 448..511 of this CTA's 128 lanes
    const uint32_t one = 0x7F7F7F7Fu;
    for (int c = 448; c < 512; c += 8)
      asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1,%1,%1,%1,%1,%1,%1,%1};" ::"r"(
                       tmem + ((warp * 32u) << 16) + c),
                   "r"(one)
                   : "memory");
    asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (PAIR) cluster_sync();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (tid == 0 && rank == 0) {
    const uint64_t ad = desc(saddr(sA)), bd = desc(saddr(sB));
    const uint32_t m = PAIR ? 256u : 128u;
    const uint32_t idesc = (1u << 7) | (1u << 10) | (static_cast<uint32_t>(kN >> 3) << 17) | (1u << 23) |
                           ((m >> 4) << 24);
    const uint32_t sfa = tmem + 448, sfb = tmem + 480;
    for (int i = 0; i < iters; ++i) {
      const uint32_t acc = i > 0 ? 1u : 0u;
      if (PAIR)
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %6, 0;\n\t"
            "tcgen05.mma.cta_group::2.kind::mxf4.block_scale.scale_vec::2X [%0], %1, %2, %3, [%4], [%5], p;\n\t}" ::"r"(
                tmem),
            "l"(ad), "l"(bd), "r"(idesc), "r"(sfa), "r"(sfb), "r"(acc)
            : "memory");
      else
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %6, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::mxf4.block_scale.scale_vec::2X [%0], %1, %2, %3, [%4], [%5], p;\n\t}" ::"r"(
                tmem),
            "l"(ad), "l"(bd), "r"(idesc), "r"(sfa), "r"(sfb), "r"(acc)
            : "memory");
    }
    if (PAIR)
      asm volatile(
          "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %1;" ::"r"(
              saddr(&bar)),
          "h"(static_cast<uint16_t>(3))
          : "memory");
    else
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                       saddr(&bar))
                   : "memory");
  }
  __syncwarp();
  const uint64_t t0 = gtimer();
  for (;;) {  // bounded wait for the MMAs
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(saddr(&bar))
        : "memory");
    if (done) break;
    if (gtimer() - t0 > 2000000000ull) {
      atomicExch(status, 1);
      break;
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (PAIR) cluster_sync();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (warp == 0) {
    if (PAIR)
      asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, 512;" ::"r"(tmem) : "memory");
    else
      asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tmem) : "memory");
  }
}

template <int PAIR>
int run(const char* name, int sms, int* dst) {
  const int grid = PAIR ? (sms / 2) * 2 : sms, iters = 20000;
  // 150 KiB of unused dynamic shared memory: one CTA per SM
  CK(cudaFuncSetAttribute(mma_rate<PAIR>, cudaFuncAttributeMaxDynamicSharedMemorySize, 150 * 1024));
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(128);
  cfg.dynamicSmemBytes = 150 * 1024;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = PAIR ? 2 : 1;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  CK(cudaLaunchKernelEx(&cfg, mma_rate<PAIR>, iters, dst));
  CK(cudaEventRecord(e0));
  CK(cudaLaunchKernelEx(&cfg, mma_rate<PAIR>, iters, dst));
  CK(cudaEventRecord(e1));
  CK(cudaEventSynchronize(e1));
  float ms;
  CK(cudaEventElapsedTime(&ms, e0, e1));
  int st;
  CK(cudaMemcpy(&st, dst, 4, cudaMemcpyDeviceToHost));
  // multiply-adds per SM per MMA: 128 x 224 x 64 in both forms
  const double flops = 2.0 * grid * static_cast<double>(iters) * 128.0 * kN * 64.0;
  printf("%s: %.3f ms, %.1f cycles per MMA at 2070 MHz, %.2f PFLOP/s of 0/1 MACs, status %d\n", name, ms,
         ms * 1e-3 * 2.07e9 / iters, flops / (ms * 1e-3) / 1e15, st);
  return st;
}

int main() {
  int sms = 0;
  CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, 0));
  int* dst;
  CK(cudaMalloc(&dst, 4));
  CK(cudaMemset(dst, 0, 4));
  int rc = run<0>("single M=128", sms, dst);
  rc |= run<1>("pair M=256", sms, dst);
  CK(cudaGetLastError());
  return rc;
}
