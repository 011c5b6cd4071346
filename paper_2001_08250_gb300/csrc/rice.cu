// Compressed interest-vector deltas for GetUpdates (Section 7): the server
// sends its window of Bloom-filter deltas compressed.  The paper names no
// encoding; the library writes the Golomb-Rice code of the gaps between set
// bits: for set bits p_0 < p_1 < ..., gap_i = p_i - p_{i-1} - 1 (p_{-1} = -1)
// is written as (gap_i >> k) one-bits, a zero bit, then the k low bits of
// gap_i, least significant first; the stream is packed LSB-first (stream bit
// j = bit j % 8 of byte j / 8).  k defaults to floor(log2 g) for the mean gap
// g = (m - count) / count (0 when g = 0 or there are no set bits).
//
// Four kernels, each over blocks of 1024 words (one per thread): count the set
// bits (and zero the stream), which fixes k; per block, the first and last
// set bit and the code bits of its set bits after the first (those depend
// only on positions inside the block: a block max-scan of each word's last
// set bit gives the set bit before each word's first one); one CTA scans the
// blocks for the set bit before each block and each block's first stream
// bit; per block, every thread writes its codes with atomicOr.  A stream that
// would pass the buffer's end is reported (nbits = UINT64_MAX) and nothing is
// written past the end.
#include <cstdint>

#include "tpir_internal.h"

namespace tpir {
namespace {

constexpr int kRThreads = 1024;

struct RiceJob {
  const uint64_t* bits;
  uint64_t m;
  int32_t k;           // < 0: choose from the set-bit count
  uint32_t* out;       // cap_words 32-bit words
  uint64_t cap_words;
  uint64_t* result;    // nbits (or UINT64_MAX), count, k
};

__device__ __forceinline__ uint64_t r_word(const RiceJob& J, uint64_t w) {
  const uint64_t W = (J.m + 63) / 64;
  if (w >= W) return 0;
  uint64_t x = J.bits[w];
  const uint64_t rem = J.m - w * 64;
  if (rem < 64) x &= (1ull << rem) - 1;  // bits at or past m are ignored
  return x;
}

__device__ __forceinline__ void r_or(const RiceJob& J, uint64_t word, uint32_t v) {
  if (v && word < J.cap_words) atomicOr(J.out + word, v);
}

// stream bits [a, a + q) set to one
__device__ void r_ones(const RiceJob& J, uint64_t a, uint64_t q) {
  while (q) {
    const uint32_t off = static_cast<uint32_t>(a & 31);
    const uint32_t n = q < 32u - off ? static_cast<uint32_t>(q) : 32u - off;
    const uint32_t mask = (n == 32 ? 0xFFFFFFFFu : ((1u << n) - 1u)) << off;
    r_or(J, a >> 5, mask);
    a += n;
    q -= n;
  }
}

// the k low bits of v at stream bits [a, a + k)
__device__ void r_bits(const RiceJob& J, uint64_t a, uint64_t v, uint32_t k) {
  while (k) {
    const uint32_t off = static_cast<uint32_t>(a & 31);
    const uint32_t n = k < 32u - off ? k : 32u - off;
    const uint32_t piece = static_cast<uint32_t>(v & ((n == 32) ? 0xFFFFFFFFull : ((1ull << n) - 1)));
    r_or(J, a >> 5, piece << off);
    a += n;
    v >>= n;
    k -= n;
  }
}

template <typename T, typename Op>
__device__ __forceinline__ T r_block_scan(T x, T identity, Op op, T* warp_tot, T* block_total) {
  // inclusive scan within the warp, then across the warps' totals
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  T v = x;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const T y = __shfl_up_sync(0xFFFFFFFFu, v, d);
    if (lane >= d) v = op(v, y);
  }
  if (lane == 31) warp_tot[warp] = v;
  __syncthreads();
  if (warp == 0) {
    T t = lane < kRThreads / 32 ? warp_tot[lane] : identity;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const T y = __shfl_up_sync(0xFFFFFFFFu, t, d);
      if (lane >= d) t = op(t, y);
    }
    warp_tot[lane] = t;  // inclusive totals of warps 0..lane
  }
  __syncthreads();
  const T before = warp == 0 ? identity : warp_tot[warp - 1];
  const T incl = op(before, v);
  const T excl_in_warp = __shfl_up_sync(0xFFFFFFFFu, incl, 1);
  const T excl = lane == 0 ? before : excl_in_warp;
  if (block_total) *block_total = warp_tot[kRThreads / 32 - 1];
  __syncthreads();
  return excl;
}

// Per-block values of the scan: first and last set bit of the block (-1 if
// none), code bits of the block's set bits after its first, then (from the
// scan) the set bit before the block and the block's first stream bit.
struct RiceBlock {
  long long first, last;
  unsigned long long inner;
  long long prev;
  unsigned long long off;
};

__device__ __forceinline__ uint32_t r_param(const RiceJob& J, uint64_t count) {
  if (J.k >= 0) return static_cast<uint32_t>(J.k);
  if (!count) return 0;
  const uint64_t g = (J.m - count) / count;
  return g ? 63u - static_cast<uint32_t>(__clzll(static_cast<long long>(g))) : 0u;
}

// 1: the stream zeroed, set bits counted (result[1] zeroed by the host)
__global__ void __launch_bounds__(kRThreads) rice_count_kernel(const RiceJob J) {
  const uint64_t W = (J.m + 63) / 64;
  const uint64_t w = blockIdx.x * (uint64_t)kRThreads + threadIdx.x;
  for (uint64_t i = w; i < J.cap_words; i += (uint64_t)gridDim.x * kRThreads) J.out[i] = 0u;
  unsigned long long c = w < W ? __popcll(r_word(J, w)) : 0ull;
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) c += __shfl_down_sync(0xFFFFFFFFu, c, d);
  if ((threadIdx.x & 31) == 0 && c) atomicAdd(reinterpret_cast<unsigned long long*>(J.result + 1), c);
}

// 2: per block (kRThreads words): first / last set bit, inner code bits
__global__ void __launch_bounds__(kRThreads) rice_block_kernel(const RiceJob J, RiceBlock* blocks) {
  __shared__ long long s_max[32];
  __shared__ unsigned long long s_sum[32];
  const uint32_t k = r_param(J, J.result[1]);
  const uint64_t w = blockIdx.x * (uint64_t)kRThreads + threadIdx.x;
  const uint64_t x = r_word(J, w);
  const long long last = x ? static_cast<long long>(w * 64 + 63 - __clzll(static_cast<long long>(x))) : -1;
  const long long first_here = x ? static_cast<long long>(w * 64 + __ffsll(static_cast<long long>(x)) - 1) : -1;
  long long block_last;
  const long long prev = r_block_scan<long long>(
      last, -1LL, [](long long a, long long b) { return a > b ? a : b; }, s_max, &block_last);
  // the block's first set bit opens the first word with bits; its code needs
  // the set bit before the block and is left to the scan
  unsigned long long len = 0;
  long long p0 = prev;
  uint64_t y = x;
  while (y) {
    const long long p = static_cast<long long>(w * 64 + __ffsll(static_cast<long long>(y)) - 1);
    if (p0 >= 0) len += ((static_cast<uint64_t>(p - p0 - 1)) >> k) + 1 + k;
    p0 = p;
    y &= y - 1;
  }
  unsigned long long inner;
  r_block_scan<unsigned long long>(len, 0ull, [](unsigned long long a, unsigned long long b) { return a + b; },
                                   s_sum, &inner);
  // the first set bit of the block: the word with bits whose prev is -1
  __shared__ long long s_first;
  if (threadIdx.x == 0) s_first = -1;
  __syncthreads();
  if (x && prev < 0) s_first = first_here;
  __syncthreads();
  if (threadIdx.x == 0) blocks[blockIdx.x] = RiceBlock{s_first, block_last, inner, -1, 0};
}

// 3: one CTA scans the blocks: the set bit before each block, its offset
__global__ void __launch_bounds__(kRThreads) rice_scan_kernel(const RiceJob J, RiceBlock* blocks,
                                                              uint32_t nblocks) {
  __shared__ long long s_max[32];
  __shared__ unsigned long long s_sum[32];
  const uint32_t k = r_param(J, J.result[1]);
  long long carry_prev = -1;
  unsigned long long carry_off = 0;
  for (uint32_t base = 0; base < nblocks; base += kRThreads) {
    const uint32_t b = base + threadIdx.x;
    const RiceBlock blk = b < nblocks ? blocks[b] : RiceBlock{-1, -1, 0, -1, 0};
    long long chunk_last;
    long long prev = r_block_scan<long long>(
        blk.last, -1LL, [](long long a, long long c) { return a > c ? a : c; }, s_max, &chunk_last);
    if (carry_prev > prev) prev = carry_prev;
    unsigned long long len = blk.inner;
    if (blk.first >= 0) len += ((static_cast<uint64_t>(blk.first - prev - 1)) >> k) + 1 + k;
    unsigned long long chunk_len;
    const unsigned long long off =
        carry_off + r_block_scan<unsigned long long>(len, 0ull,
                                                     [](unsigned long long a, unsigned long long c) { return a + c; },
                                                     s_sum, &chunk_len);
    if (b < nblocks) {
      blocks[b].prev = prev;
      blocks[b].off = off;
    }
    if (chunk_last > carry_prev) carry_prev = chunk_last;
    carry_off += chunk_len;
  }
  if (threadIdx.x == 0) {
    J.result[0] = carry_off <= J.cap_words * 32 ? carry_off : ~0ull;
    J.result[2] = k;
  }
}

// 4: per block, the codes at the block's offset
__global__ void __launch_bounds__(kRThreads) rice_write_kernel(const RiceJob J, const RiceBlock* blocks) {
  __shared__ long long s_max[32];
  __shared__ unsigned long long s_sum[32];
  const uint32_t k = r_param(J, J.result[1]);
  const RiceBlock blk = blocks[blockIdx.x];
  const uint64_t w = blockIdx.x * (uint64_t)kRThreads + threadIdx.x;
  const uint64_t x = r_word(J, w);
  const long long last = x ? static_cast<long long>(w * 64 + 63 - __clzll(static_cast<long long>(x))) : -1;
  long long block_last;
  long long prev = r_block_scan<long long>(
      last, -1LL, [](long long a, long long b) { return a > b ? a : b; }, s_max, &block_last);
  if (blk.prev > prev) prev = blk.prev;
  unsigned long long len = 0;
  {
    long long p0 = prev;
    uint64_t y = x;
    while (y) {
      const long long p = static_cast<long long>(w * 64 + __ffsll(static_cast<long long>(y)) - 1);
      len += ((static_cast<uint64_t>(p - p0 - 1)) >> k) + 1 + k;
      p0 = p;
      y &= y - 1;
    }
  }
  unsigned long long total;
  const unsigned long long off =
      blk.off + r_block_scan<unsigned long long>(len, 0ull,
                                                 [](unsigned long long a, unsigned long long b) { return a + b; },
                                                 s_sum, &total);
  long long p0 = prev;
  uint64_t y = x, a = off;
  while (y) {
    const long long p = static_cast<long long>(w * 64 + __ffsll(static_cast<long long>(y)) - 1);
    const uint64_t gap = static_cast<uint64_t>(p - p0 - 1);
    const uint64_t q = gap >> k;
    r_ones(J, a, q);
    a += q + 1;  // the zero bit stays zero
    if (k) r_bits(J, a, gap, k);
    a += k;
    p0 = p;
    y &= y - 1;
  }
}

}  // namespace

size_t rice_scratch_bytes(uint64_t m) {
  const uint64_t W = (m + 63) / 64;
  return ((W + kRThreads - 1) / kRThreads) * sizeof(RiceBlock);
}

cudaError_t launch_rice_encode(const RiceRequest& q, void* scratch, cudaStream_t st) {
  const uint64_t W = (q.m + 63) / 64;
  const uint64_t nb = (W + kRThreads - 1) / kRThreads;
  if (nb == 0 || nb > 0x7FFFFFFFull) return cudaErrorInvalidValue;
  const RiceJob J{q.bits, q.m, q.k, q.out, q.cap_words, q.result};
  RiceBlock* blocks = static_cast<RiceBlock*>(scratch);
  cudaError_t e = cudaMemsetAsync(q.result, 0, 3 * sizeof(uint64_t), st);
  if (e != cudaSuccess) return e;
  rice_count_kernel<<<static_cast<uint32_t>(nb), kRThreads, 0, st>>>(J);
  rice_block_kernel<<<static_cast<uint32_t>(nb), kRThreads, 0, st>>>(J, blocks);
  rice_scan_kernel<<<1, kRThreads, 0, st>>>(J, blocks, static_cast<uint32_t>(nb));
  rice_write_kernel<<<static_cast<uint32_t>(nb), kRThreads, 0, st>>>(J, blocks);
  count_launches(4);
  return cudaGetLastError();
}

}  // namespace tpir
