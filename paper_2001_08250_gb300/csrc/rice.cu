// Compressed interest-vector deltas for GetUpdates (Section 7): the server
// sends its window of Bloom-filter deltas compressed.  The paper names no
// encoding; the library writes the Golomb-Rice code of the gaps between set
// bits: for set bits p_0 < p_1 < ..., gap_i = p_i - p_{i-1} - 1 (p_{-1} = -1)
// is written as (gap_i >> k) one-bits, a zero bit, then the k low bits of
// gap_i, least significant first; the stream is packed LSB-first (stream bit
// j = bit j % 8 of byte j / 8).  k defaults to floor(log2 g) for the mean gap
// g = (m - count) / count (0 when g = 0 or there are no set bits).
//
// One CTA encodes one vector (a grid encodes several, e.g. a window of
// deltas).  Words are taken 1024 at a time, one per thread: a block max-scan
// of the last set bit of each word gives every word the position of the set
// bit before its first one (carried across chunks), a block sum-scan of the
// words' code lengths gives each word's bit offset, and each thread writes
// its codes with atomicOr into the stream, which the CTA zeroes first.  A
// stream that would pass the buffer's end is reported (nbits = UINT64_MAX)
// and nothing is written past the end.
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

struct RiceLaunch {
  RiceJob jobs[kRiceMaxJobs];
};

__global__ void __launch_bounds__(kRThreads) rice_encode_kernel(const __grid_constant__ RiceLaunch L) {
  __shared__ long long s_max[32];
  __shared__ unsigned long long s_sum[32];
  __shared__ unsigned long long s_cnt;
  const RiceJob& J = L.jobs[blockIdx.x];
  const uint64_t W = (J.m + 63) / 64;
  for (uint64_t i = threadIdx.x; i < J.cap_words; i += kRThreads) J.out[i] = 0u;
  // pass 0: number of set bits, and k
  unsigned long long c = 0;
  for (uint64_t w = threadIdx.x; w < W; w += kRThreads) c += __popcll(r_word(J, w));
  if (threadIdx.x == 0) s_cnt = 0;
  __syncthreads();
  atomicAdd(&s_cnt, c);
  __syncthreads();
  const uint64_t count = s_cnt;
  uint32_t k = 0;
  if (J.k >= 0) {
    k = static_cast<uint32_t>(J.k);
  } else if (count) {
    const uint64_t g = (J.m - count) / count;
    k = g ? 63u - static_cast<uint32_t>(__clzll(static_cast<long long>(g))) : 0u;
  }
  __threadfence_block();
  __syncthreads();
  // pass 1: chunks of kRThreads words
  long long carry_prev = -1;
  unsigned long long carry_off = 0;
  for (uint64_t base = 0; base < W; base += kRThreads) {
    const uint64_t w = base + threadIdx.x;
    const uint64_t x = r_word(J, w);
    const long long last = x ? static_cast<long long>(w * 64 + 63 - __clzll(static_cast<long long>(x))) : -1;
    long long chunk_max;
    long long prev = r_block_scan<long long>(last, -1LL, [](long long a, long long b) { return a > b ? a : b; },
                                             s_max, &chunk_max);
    if (carry_prev > prev) prev = carry_prev;
    // code length of this word's set bits
    unsigned long long len = 0;
    {
      long long p0 = prev;
      uint64_t y = x;
      while (y) {
        const long long p = static_cast<long long>(w * 64 + __ffsll(static_cast<long long>(y)) - 1);
        const uint64_t gap = static_cast<uint64_t>(p - p0 - 1);
        len += (gap >> k) + 1 + k;
        p0 = p;
        y &= y - 1;
      }
    }
    unsigned long long chunk_len;
    const unsigned long long off =
        carry_off + r_block_scan<unsigned long long>(len, 0ull,
                                                     [](unsigned long long a, unsigned long long b) { return a + b; },
                                                     s_sum, &chunk_len);
    // codes
    {
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
    if (chunk_max > carry_prev) carry_prev = chunk_max;
    carry_off += chunk_len;
  }
  if (threadIdx.x == 0) {
    J.result[0] = carry_off <= J.cap_words * 32 ? carry_off : ~0ull;
    J.result[1] = count;
    J.result[2] = k;
  }
}

}  // namespace

cudaError_t launch_rice_encode(const RiceRequest* reqs, uint32_t count, cudaStream_t st) {
  if (count == 0) return cudaSuccess;
  if (count > kRiceMaxJobs) return cudaErrorInvalidValue;
  RiceLaunch L{};
  for (uint32_t i = 0; i < count; ++i)
    L.jobs[i] = RiceJob{reqs[i].bits, reqs[i].m, reqs[i].k, reqs[i].out, reqs[i].cap_words,
                        reqs[i].result};
  rice_encode_kernel<<<count, kRThreads, 0, st>>>(L);
  return cudaGetLastError();
}

}  // namespace tpir
