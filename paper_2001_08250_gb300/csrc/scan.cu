// PIR read kernels for sm_103a: the server answer of Section 2 (step 5),
//   out[b][j] = XOR over buckets k with bit(R[b], k) = 1 of T[k][j],
// computed for every bucket and every request with no data-dependent skip:
// each bucket is loaded and combined under an all-ones / all-zeros mask.
//
//  plain_scan_kernel    B <= 4 requests per launch.  HBM-bound stream of the
//                       whole table with 128-bit non-allocating loads, split
//                       over CTAs by bucket ranges (split-K); partial replies
//                       are XOR-reduced into the zeroed output with red.xor.
//  batched_scan_kernel  B requests share one pass over the table (the GF(2)
//                       product Out = R (x) T).  Persistent, warp-specialised:
//                       one producer warp streams table tiles into a shared
//                       memory ring with cp.async.bulk + mbarriers and expands
//                       request bits into 32-bit masks; eight consumer warps
//                       hold an 8-request x 16-word register tile each and do
//                       one LOP3 (acc ^= mask & word) per request-word pair.
//                       Items are (job, B-tile, W-tile, k-chunk), so the same
//                       launch serves one table or many uneven tables.
#include "tpir_internal.h"

namespace tpir {

// Device-side status word: set to TPIR_ETIMEDOUT by a bounded wait that gave up.
__device__ int g_status;

namespace {

constexpr uint64_t kWaitLimitNs = 4000000000ull;  // 4 s: far above any legitimate wait

__device__ __forceinline__ uint64_t globaltimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
               : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.expect_tx.relaxed.cta.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile(
      "{\n\t.reg .b64 st;\n\t"
      "mbarrier.arrive.release.cta.shared::cta.b64 st, [%0];\n\t}" ::"r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.acquire.cta.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Waits for the phase of `parity` to complete.  Gives up (returns false) after
// kWaitLimitNs or when another warp of the CTA has given up already.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, volatile int* abort_flag) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = globaltimer();
  while (!mbar_try_wait(bar, parity)) {
    if (*abort_flag) return false;
    if (globaltimer() - t0 > kWaitLimitNs) {
      *abort_flag = 1;
      atomicExch(&g_status, (int)TPIR_ETIMEDOUT);
      return false;
    }
  }
  return true;
}

// 1-D bulk copy global -> this CTA's shared memory, completing on `bar`.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes,
                                         uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ uint4 ld_stream(const uint4* p) {
  uint4 v;
  asm volatile("ld.global.nc.L1::no_allocate.L2::256B.v4.u32 {%0,%1,%2,%3}, [%4];"
               : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
               : "l"(p));
  return v;
}

__device__ __forceinline__ void red_xor64(uint32_t* p, uint32_t lo, uint32_t hi) {
  const uint64_t v = (static_cast<uint64_t>(hi) << 32) | lo;
  asm volatile("red.relaxed.gpu.global.xor.b64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ uint32_t bit_mask(uint64_t w, uint32_t pos) {
  return 0u - static_cast<uint32_t>((w >> pos) & 1u);
}

// ---------------------------------------------------------------------------
// Plain streaming kernel
// ---------------------------------------------------------------------------
// grid.y = column slices of <= 256 uint4 (4 KiB) of a row, grid.x = bucket
// ranges of rows_per_cta.  A slice narrower than 256 uint4 is covered by
// 256/Us rows at once; those partials are folded in shared memory.
template <int NB, int UNR>
__global__ void __launch_bounds__(256) plain_scan_kernel(const uint4* __restrict__ T, uint64_t n,
                                                         uint32_t U,
                                                         const uint64_t* __restrict__ R,
                                                         uint32_t words64, uint32_t B,
                                                         uint4* __restrict__ out,
                                                         uint64_t rows_per_cta) {
  __shared__ uint4 fold[NB * 256];
  const uint32_t c0 = blockIdx.y * 256u;
  const uint32_t Us = min(256u, U - c0);
  const uint32_t rpi = 256u / Us;
  const uint32_t t = threadIdx.x;
  const bool active = t < rpi * Us;
  const uint32_t roff = t / Us;
  const uint32_t cl = t - roff * Us;
  const uint64_t k0 = static_cast<uint64_t>(blockIdx.x) * rows_per_cta;
  const uint64_t k1 = min(n, k0 + rows_per_cta);

  uint4 acc[NB];
#pragma unroll
  for (int b = 0; b < NB; ++b) acc[b] = make_uint4(0u, 0u, 0u, 0u);

  if (active && k0 < k1) {
    const uint4* base = T + c0 + cl;
    uint64_t k = k0 + roff;
    const uint64_t step = rpi;
    for (; k + (UNR - 1) * step < k1; k += UNR * step) {
      uint4 v[UNR];
#pragma unroll
      for (int u = 0; u < UNR; ++u) v[u] = ld_stream(base + (k + u * step) * U);
#pragma unroll
      for (int u = 0; u < UNR; ++u) {
        const uint64_t kk = k + u * step;
#pragma unroll
        for (int b = 0; b < NB; ++b) {
          if (b < (int)B) {
            const uint32_t m = bit_mask(__ldg(R + b * (uint64_t)words64 + (kk >> 6)), kk & 63);
            acc[b].x ^= v[u].x & m;
            acc[b].y ^= v[u].y & m;
            acc[b].z ^= v[u].z & m;
            acc[b].w ^= v[u].w & m;
          }
        }
      }
    }
    for (; k < k1; k += step) {
      const uint4 v = ld_stream(base + k * U);
#pragma unroll
      for (int b = 0; b < NB; ++b) {
        if (b < (int)B) {
          const uint32_t m = bit_mask(__ldg(R + b * (uint64_t)words64 + (k >> 6)), k & 63);
          acc[b].x ^= v.x & m;
          acc[b].y ^= v.y & m;
          acc[b].z ^= v.z & m;
          acc[b].w ^= v.w & m;
        }
      }
    }
  }
  if (rpi > 1) {
#pragma unroll
    for (int b = 0; b < NB; ++b) fold[b * 256 + t] = acc[b];
    __syncthreads();
    if (t < Us) {
#pragma unroll
      for (int b = 0; b < NB; ++b) {
        uint4 s = make_uint4(0u, 0u, 0u, 0u);
        for (uint32_t r = 0; r < rpi; ++r) {
          const uint4 p = fold[b * 256 + r * Us + t];
          s.x ^= p.x;
          s.y ^= p.y;
          s.z ^= p.z;
          s.w ^= p.w;
        }
        acc[b] = s;
      }
    }
  }
  if (t < Us && k0 < k1) {
#pragma unroll
    for (int b = 0; b < NB; ++b) {
      if (b < (int)B) {
        uint32_t* o = reinterpret_cast<uint32_t*>(out + static_cast<uint64_t>(b) * U + c0 + t);
        red_xor64(o, acc[b].x, acc[b].y);
        red_xor64(o + 2, acc[b].z, acc[b].w);
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Batched persistent kernel
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t find_job(const ScanLaunch& L, uint32_t item) {
  uint32_t lo = 0, hi = L.njobs - 1;
  while (lo < hi) {
    const uint32_t mid = (lo + hi + 1) >> 1;
    if (L.jobs[mid].item_begin <= item)
      lo = mid;
    else
      hi = mid - 1;
  }
  return lo;
}

struct Item {
  uint32_t job, bt, wt;
  uint64_t k0, k1;
};

__device__ __forceinline__ Item decode_item(const ScanLaunch& L, uint32_t item) {
  Item it;
  it.job = find_job(L, item);
  const ScanJob& J = L.jobs[it.job];
  uint32_t local = item - J.item_begin;
  it.bt = local % J.n_bt;
  local /= J.n_bt;
  it.wt = local % J.n_wt;
  const uint32_t kc = local / J.n_wt;
  it.k0 = static_cast<uint64_t>(kc) * J.kc_rows;
  it.k1 = min(J.n, it.k0 + J.kc_rows);
  return it;
}

__global__ void __launch_bounds__(kScanThreads, 1)
    batched_scan_kernel(const __grid_constant__ ScanLaunch L) {
  extern __shared__ __align__(128) uint8_t smem_raw[];
  uint64_t* full = reinterpret_cast<uint64_t*>(smem_raw);
  uint64_t* empty = full + kStages;
  uint8_t* stages = smem_raw + 256;
  __shared__ int s_abort;

  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(&full[s], 32);
      mbar_init(&empty[s], kConsumerWarps);
    }
    s_abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  volatile int* abort_flag = &s_abort;

  uint32_t iter = 0;  // pipeline stage counter, identical in producer and consumers

  if (warp == kConsumerWarps) {
    // ---------------- producer warp ----------------
    bool ok = true;
    for (uint32_t item = blockIdx.x; ok && item < L.total_items; item += gridDim.x) {
      const Item it = decode_item(L, item);
      const ScanJob& J = L.jobs[it.job];
      const uint32_t bt_ = J.shape.bt(), wt_ = J.shape.wt(), sr = J.shape.srows();
      const uint32_t w0 = it.wt * wt_;
      const uint32_t wcount = min(wt_, J.Wd - w0);
      const uint32_t b0 = it.bt * bt_;
      for (uint64_t ks = it.k0; ks < it.k1; ks += sr, ++iter) {
        const uint32_t s = iter % kStages;
        const uint32_t ph = (iter / kStages) & 1u;
        if (!mbar_wait(&empty[s], ph ^ 1u, abort_flag)) {
          ok = false;
          break;
        }
        uint32_t* tsm = reinterpret_cast<uint32_t*>(stages + s * kStageBytes);
        uint32_t* msm = tsm + sr * wt_;
        const uint32_t rows = static_cast<uint32_t>(it.k1 - ks < sr ? it.k1 - ks : sr);
        if (lane == 0) mbar_expect_tx(&full[s], rows * wcount * 4u);
        __syncwarp();
        for (uint32_t r = lane; r < rows; r += 32)
          bulk_g2s(tsm + r * wt_, J.T + (ks + r) * J.Wd + w0, wcount * 4u, &full[s]);
        // request bits -> 32-bit masks, zero for rows past the chunk and for
        // request slots past B
        const uint32_t sh = static_cast<uint32_t>(ks & 63);
        for (uint32_t b = lane; b < bt_; b += 32) {
          uint64_t wbits = 0;
          if (b0 + b < J.B) wbits = __ldg(J.R + static_cast<uint64_t>(b0 + b) * J.words64 + (ks >> 6));
          wbits >>= sh;
          for (uint32_t r = 0; r < sr; ++r)
            msm[r * bt_ + b] = (r < rows) ? bit_mask(wbits, r) : 0u;
        }
        mbar_arrive(&full[s]);
      }
    }
    if (*abort_flag && lane == 0) {
      // give the copies already issued a bounded chance to land before exit
      const uint32_t first = iter > kStages ? iter - kStages : 0;
      for (uint32_t x = first; x < iter; ++x) {
        const uint64_t t0 = globaltimer();
        while (!mbar_try_wait(&full[x % kStages], (x / kStages) & 1u) &&
               globaltimer() - t0 < kWaitLimitNs) {
        }
      }
    }
    return;
  }

  // ---------------- consumer warps ----------------
  const int cw = warp;
  for (uint32_t item = blockIdx.x; item < L.total_items; item += gridDim.x) {
    const Item it = decode_item(L, item);
    const ScanJob& J = L.jobs[it.job];
    const uint32_t lw_log2 = J.shape.lw_log2;
    const uint32_t lw = 1u << lw_log2;
    const uint32_t ww = J.shape.ww, wbw = J.shape.wb * ww, wk = J.shape.wk;
    const uint32_t bt_ = J.shape.bt(), wt_ = J.shape.wt(), sr = J.shape.srows();
    const uint32_t wk_idx = cw / wbw, rem = cw % wbw;
    const uint32_t wb_idx = rem / ww, ww_idx = rem % ww;
    const uint32_t lwi = lane & (lw - 1), lbi = lane >> lw_log2;
    const uint32_t rq0 = (wb_idx * (32u >> lw_log2) + lbi) * kMR;
    const uint32_t wbase = ww_idx * (lw * kNW) + lwi * 4u;
    const uint32_t seg = lw * 4u;

    uint32_t acc[kMR][kNW];
#pragma unroll
    for (int i = 0; i < kMR; ++i)
#pragma unroll
      for (int q = 0; q < kNW; ++q) acc[i][q] = 0u;

    bool ok = true;
    for (uint64_t ks = it.k0; ks < it.k1; ks += sr, ++iter) {
      const uint32_t s = iter % kStages;
      const uint32_t ph = (iter / kStages) & 1u;
      if (!mbar_wait(&full[s], ph, abort_flag)) {
        ok = false;
        break;
      }
      const uint32_t* tsm = reinterpret_cast<const uint32_t*>(stages + s * kStageBytes);
      const uint32_t* msm = tsm + sr * wt_;
      const uint32_t rows = static_cast<uint32_t>(it.k1 - ks < sr ? it.k1 - ks : sr);
      for (uint32_t r = wk_idx; r < rows; r += wk) {
        const uint4 m0 = *reinterpret_cast<const uint4*>(msm + r * bt_ + rq0);
        const uint4 m1 = *reinterpret_cast<const uint4*>(msm + r * bt_ + rq0 + 4);
        uint4 tv[4];
#pragma unroll
        for (int j = 0; j < 4; ++j)
          tv[j] = *reinterpret_cast<const uint4*>(tsm + r * wt_ + wbase + j * seg);
        const uint32_t m[kMR] = {m0.x, m0.y, m0.z, m0.w, m1.x, m1.y, m1.z, m1.w};
        const uint32_t w[kNW] = {tv[0].x, tv[0].y, tv[0].z, tv[0].w, tv[1].x, tv[1].y,
                                 tv[1].z, tv[1].w, tv[2].x, tv[2].y, tv[2].z, tv[2].w,
                                 tv[3].x, tv[3].y, tv[3].z, tv[3].w};
#pragma unroll
        for (int i = 0; i < kMR; ++i)
#pragma unroll
          for (int q = 0; q < kNW; ++q) acc[i][q] ^= m[i] & w[q];
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(&empty[s]);
    }
    if (!ok) return;

    // epilogue: store (single k-chunk) or XOR-reduce (split over k-chunks)
    const bool split = J.split != 0;
    const uint32_t b0 = it.bt * bt_ + rq0;
    const uint32_t w0 = it.wt * wt_ + wbase;
#pragma unroll
    for (int i = 0; i < kMR; ++i) {
      const uint32_t b = b0 + i;
      if (b >= J.B) continue;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const uint32_t wd = w0 + j * seg;
        if (wd >= J.Wd) continue;
        uint32_t* o = J.out + static_cast<uint64_t>(b) * J.Wd + wd;
        if (split) {
          red_xor64(o, acc[i][4 * j], acc[i][4 * j + 1]);
          red_xor64(o + 2, acc[i][4 * j + 2], acc[i][4 * j + 3]);
        } else {
          *reinterpret_cast<uint4*>(o) =
              make_uint4(acc[i][4 * j], acc[i][4 * j + 1], acc[i][4 * j + 2], acc[i][4 * j + 3]);
        }
      }
    }
  }
}

// Zeroes the outputs of the jobs that are split over k-chunks (their CTAs
// XOR-reduce into the output).  grid.y = job.
__global__ void zero_outputs_kernel(const __grid_constant__ ScanLaunch L) {
  const ScanJob& J = L.jobs[blockIdx.y];
  if (!J.split) return;
  const uint64_t n4 = static_cast<uint64_t>(J.B) * J.Wd / 4;
  uint4* o = reinterpret_cast<uint4*>(J.out);
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n4;
       i += (uint64_t)gridDim.x * blockDim.x)
    o[i] = make_uint4(0u, 0u, 0u, 0u);
}

}  // namespace

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
int device_sm_count() {
  static int cached[64] = {0};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) return 1;
  if (!cached[dev]) {
    int v = 0;
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
    cached[dev] = v > 0 ? v : 1;
  }
  return cached[dev];
}

int plain_ctas_per_sm() {
  static int cached = 0;
  if (!cached) {
    int v = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, plain_scan_kernel<4, 8>, 256, 0);
    cached = v > 0 ? v : 1;
  }
  return cached;
}

int batched_ctas_per_sm() {
  static int cached = 0;
  if (!cached) {
    cudaFuncSetAttribute(batched_scan_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         kScanSmem);
    int v = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, batched_scan_kernel, kScanThreads,
                                                  kScanSmem);
    cached = v > 0 ? v : 1;
  }
  return cached;
}

int scan_stage_bytes(const Shape& s) { return s.srows() * (s.wt() + s.bt()) * 4; }

static uint32_t pow2_ceil(uint32_t x) {
  uint32_t p = 1;
  while (p < x) p <<= 1;
  return p;
}

Shape choose_shape(uint32_t Wd, uint32_t B) {
  Shape s{};
  // widest warp span (LW lanes x 16 words) that does not exceed the row
  int lw_log2 = 5;
  while (lw_log2 > 2 && (1u << lw_log2) * kNW > Wd) --lw_log2;
  s.lw_log2 = static_cast<uint8_t>(lw_log2);
  const uint32_t lw = 1u << lw_log2;
  const uint32_t warp_b = (32 / lw) * kMR;  // requests per warp
  const uint32_t warp_w = lw * kNW;         // words per warp
  // warps along B as the batch fills them, then along W as the row allows,
  // the rest along k
  uint32_t wb = pow2_ceil((B + warp_b - 1) / warp_b);
  if (wb > 8) wb = 8;
  if (wb < 1) wb = 1;
  uint32_t ww = pow2_ceil((Wd + warp_w - 1) / warp_w);
  if (ww > 8 / wb) ww = 8 / wb;
  const uint32_t wk = 8 / (wb * ww);
  s.wb = static_cast<uint8_t>(wb);
  s.ww = static_cast<uint8_t>(ww);
  s.wk = static_cast<uint8_t>(wk);
  int sr_log2 = 5;
  while (sr_log2 > 0) {
    s.srows_log2 = static_cast<uint8_t>(sr_log2);
    if (scan_stage_bytes(s) <= kStageBytes) break;
    --sr_log2;
  }
  s.srows_log2 = static_cast<uint8_t>(sr_log2);
  return s;
}

bool finalize_job(ScanJob& j) {
  const Shape& s = j.shape;
  if (scan_stage_bytes(s) > kStageBytes) return false;
  if (s.wb * s.ww * s.wk != kConsumerWarps) return false;
  if (j.kc_rows == 0 || (j.kc_rows % s.srows()) != 0) return false;
  j.n_bt = (j.B + s.bt() - 1) / s.bt();
  j.n_wt = (j.Wd + s.wt() - 1) / s.wt();
  j.n_kc = static_cast<uint32_t>((j.n + j.kc_rows - 1) / j.kc_rows);
  j.split = (j.n_kc > 1 || s.wk > 1) ? 1u : 0u;
  return true;
}

cudaError_t launch_batched(const ScanLaunch& L, int grid, cudaStream_t st) {
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(batched_scan_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, kScanSmem);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  if (L.total_items == 0) return cudaSuccess;
  batched_scan_kernel<<<grid, kScanThreads, kScanSmem, st>>>(L);
  return cudaGetLastError();
}

cudaError_t launch_zero_outputs(const ScanLaunch& L, cudaStream_t st) {
  bool any = false;
  for (uint32_t i = 0; i < L.njobs; ++i) any |= L.jobs[i].split != 0;
  if (!any) return cudaSuccess;
  dim3 grid(64, L.njobs);
  zero_outputs_kernel<<<grid, 256, 0, st>>>(L);
  return cudaGetLastError();
}

cudaError_t launch_plain(const uint32_t* T, uint64_t n, uint32_t Wd, const uint64_t* R,
                         uint32_t words64, uint32_t B, uint32_t* out, cudaStream_t st, int ctas) {
  if (B == 0) return cudaSuccess;
  const uint32_t U = Wd / 4;
  cudaError_t e = cudaMemsetAsync(out, 0, static_cast<size_t>(B) * Wd * 4, st);
  if (e != cudaSuccess) return e;
  const uint32_t slices = (U + 255) / 256;
  if (ctas <= 0) ctas = device_sm_count() * plain_ctas_per_sm();
  uint64_t chunks = static_cast<uint64_t>(ctas) / slices;
  if (chunks < 1) chunks = 1;
  if (chunks > n) chunks = n;
  const uint64_t rows_per_cta = (n + chunks - 1) / chunks;
  chunks = (n + rows_per_cta - 1) / rows_per_cta;
  dim3 grid(static_cast<uint32_t>(chunks), slices);
  const uint4* T4 = reinterpret_cast<const uint4*>(T);
  uint4* o4 = reinterpret_cast<uint4*>(out);
  if (B == 1)
    plain_scan_kernel<1, 8><<<grid, 256, 0, st>>>(T4, n, U, R, words64, B, o4, rows_per_cta);
  else if (B == 2)
    plain_scan_kernel<2, 8><<<grid, 256, 0, st>>>(T4, n, U, R, words64, B, o4, rows_per_cta);
  else
    plain_scan_kernel<4, 8><<<grid, 256, 0, st>>>(T4, n, U, R, words64, B, o4, rows_per_cta);
  return cudaGetLastError();
}

int read_device_status_and_clear(int* status) {
  int v = 0;
  cudaError_t e = cudaMemcpyFromSymbol(&v, g_status, sizeof(int));
  if (e != cudaSuccess) return -1;
  const int zero = 0;
  cudaMemcpyToSymbol(g_status, &zero, sizeof(int));
  *status = v;
  return 0;
}

}  // namespace tpir
