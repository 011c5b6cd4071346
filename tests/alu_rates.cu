// Throughput measurement behind two design decisions of the read kernels
// (compiled and run by tests/test_gpu_alu_rates.py):
//  - the integer roofline of the batched read: how many LOP3 (acc = (a & b) ^ acc,
//    the conditional-XOR of one 32-bit word) an SM retires per clock;
//  - whether the 1-bit AND-POPC form of the GF(2) product can beat it: the
//    throughput of mma.sync.aligned.m16n8k256 b1 and.popc on this part.
#include <cstdio>
#include <cstdint>
#include <cuda_runtime.h>

__global__ void lop3_kernel(const uint32_t* in, uint32_t* out, int iters) {
  uint32_t a = in[threadIdx.x & 31], b = in[(threadIdx.x + 7) & 31];
  uint32_t acc[32];
#pragma unroll
  for (int i = 0; i < 32; ++i) acc[i] = in[i] ^ threadIdx.x;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < 32; ++i)
      asm volatile("lop3.b32 %0, %1, %2, %0, 0x6A;" : "+r"(acc[i]) : "r"(a), "r"(b));
    a += 1;  // keep the inputs live (1 extra op per 32)
  }
  uint32_t s = 0;
#pragma unroll
  for (int i = 0; i < 32; ++i) s ^= acc[i];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void b1mma_kernel(const uint32_t* in, uint32_t* out, int iters) {
  uint32_t a0 = in[threadIdx.x & 31], a1 = in[(threadIdx.x + 1) & 31], a2 = in[(threadIdx.x + 2) & 31], a3 = in[(threadIdx.x + 3) & 31];
  uint32_t b0 = in[(threadIdx.x + 4) & 31], b1 = in[(threadIdx.x + 5) & 31];
  int c[8][4];
#pragma unroll
  for (int k = 0; k < 8; ++k)
#pragma unroll
    for (int i = 0; i < 4; ++i) c[k][i] = 0;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int k = 0; k < 8; ++k)
      asm volatile(
          "mma.sync.aligned.m16n8k256.row.col.s32.b1.b1.s32.and.popc {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};"
          : "+r"(c[k][0]), "+r"(c[k][1]), "+r"(c[k][2]), "+r"(c[k][3])
          : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
  }
  int s = 0;
#pragma unroll
  for (int k = 0; k < 8; ++k)
#pragma unroll
    for (int i = 0; i < 4; ++i) s ^= c[k][i];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

int main() {
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, 0);
  int clk = 0;
  cudaDeviceGetAttribute(&clk, cudaDevAttrClockRate, 0);
  const int blocks = sms * 4, threads = 256;
  uint32_t *in, *out;
  cudaMalloc(&in, 32 * 4);
  cudaMemset(in, 0x5A, 32 * 4);
  cudaMalloc(&out, blocks * threads * 4);
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  for (int rep = 0; rep < 3; ++rep) {
    const int iters = 4096;
    lop3_kernel<<<blocks, threads>>>(in, out, iters);
    cudaEventRecord(e0);
    lop3_kernel<<<blocks, threads>>>(in, out, iters);
    cudaEventRecord(e1);
    cudaEventSynchronize(e1);
    float ms;
    cudaEventElapsedTime(&ms, e0, e1);
    double ops = (double)blocks * threads * iters * 32;
    printf("lop3: %.3f ms, %.3f Tops/s, %.1f ops/clk/SM at %d MHz attr clock\n", ms, ops / ms / 1e9,
           ops / (ms * 1e-3) / sms / (clk * 1e3), clk / 1000);
  }
  for (int rep = 0; rep < 3; ++rep) {
    const int iters = 512;
    b1mma_kernel<<<blocks, threads>>>(in, out, iters);
    cudaEventRecord(e0);
    b1mma_kernel<<<blocks, threads>>>(in, out, iters);
    cudaEventRecord(e1);
    cudaEventSynchronize(e1);
    float ms;
    cudaEventElapsedTime(&ms, e0, e1);
    double mmas = (double)blocks * (threads / 32) * iters * 8;
    double bitmacs = mmas * 16 * 8 * 256;
    printf("b1mma: %.3f ms, %.1f T bit-MAC/s, %.0f bit-MAC/clk/SM\n", ms, bitmacs / ms / 1e9,
           bitmacs / (ms * 1e-3) / sms / (clk * 1e3));
  }
  cudaError_t e = cudaGetLastError();
  printf("status: %s\n", cudaGetErrorString(e));
  return e == cudaSuccess ? 0 : 1;
}
