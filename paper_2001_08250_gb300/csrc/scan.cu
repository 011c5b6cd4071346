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
#include <atomic>
#include <algorithm>

#include "chacha.cuh"
#include "tpir_internal.h"

namespace tpir {

// Device-side status word: set to TPIR_ETIMEDOUT by a bounded wait that gave up.
__device__ int g_status;

// Item counters of the batched kernel's dynamic schedule, one per launch in a
// rotation of kItemCounterSlots: the zero kernel that precedes a launch resets
// its slot, the launch's CTAs claim items from it.
__device__ uint32_t g_item_counter[kItemCounterSlots];

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
// limit_ns or when another warp of the CTA has given up already; giving up
// sets the CTA's abort flag and the device status word.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, volatile int* abort_flag,
                                          uint64_t limit_ns = kWaitLimitNs) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = globaltimer();
  while (!mbar_try_wait(bar, parity)) {
    if (*abort_flag) return false;
    if (globaltimer() - t0 > limit_ns) {
      *abort_flag = 1;
      atomicExch(&g_status, (int)TPIR_ETIMEDOUT);
      return false;
    }
  }
  return true;
}

// Like mbar_wait, with a short sleep between polls: for waiters that run
// ahead of the pipeline and should leave issue slots to the compute warps.
__device__ __forceinline__ bool mbar_wait_backoff(uint64_t* bar, uint32_t parity,
                                                  volatile int* abort_flag) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = globaltimer();
  while (!mbar_try_wait(bar, parity)) {
    if (*abort_flag) return false;
    if (globaltimer() - t0 > kWaitLimitNs) {
      *abort_flag = 1;
      atomicExch(&g_status, (int)TPIR_ETIMEDOUT);
      return false;
    }
    __nanosleep(64);
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

// Programmatic dependent launch: let the next kernel of the stream start its
// launch now / wait until the previous kernel of the stream has completed and
// its memory is visible.  Both are no-ops without a programmatic dependency.
__device__ __forceinline__ void pdl_launch_dependents() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// ---------------------------------------------------------------------------
// Plain streaming kernel
// ---------------------------------------------------------------------------
// grid.y = column slices of <= kPlainSlice uint4 (512 B) of a row, grid.x =
// bucket ranges of rows_per_cta.  The 256 threads cover 256/Us rows of the
// slice at once (one warp per 512 B row segment); their partials are folded in
// shared memory, so each output word receives one red.xor per bucket range.
constexpr uint32_t kPlainSlice = 32;  // uint4 per column slice

template <int NB, int UNR>
__global__ void __launch_bounds__(256) plain_scan_kernel(const uint4* __restrict__ T, uint64_t n,
                                                         uint32_t U,
                                                         const uint64_t* __restrict__ R,
                                                         uint32_t words64, uint32_t B,
                                                         uint4* __restrict__ out,
                                                         uint64_t rows_per_cta) {
  __shared__ uint4 fold[NB * 256];
  pdl_launch_dependents();
  const uint32_t c0 = blockIdx.y * kPlainSlice;
  const uint32_t Us = min(kPlainSlice, U - c0);
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
    const uint64_t step = rpi;
    // UNR rows in flight per thread; rows past the range are neither loaded
    // nor combined (they belong to another CTA or lie beyond the table)
    for (uint64_t k = k0 + roff; k < k1; k += UNR * step) {
      uint4 v[UNR];
#pragma unroll
      for (int u = 0; u < UNR; ++u) {
        const uint64_t kk = k + u * step;
        v[u] = kk < k1 ? ld_stream(base + kk * U) : make_uint4(0u, 0u, 0u, 0u);
      }
#pragma unroll
      for (int u = 0; u < UNR; ++u) {
        const uint64_t kk = k + u * step;
        if (kk >= k1) break;
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
  // the reply was zeroed by the previous kernel of the stream
  pdl_wait();
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
// Plain TMA streaming kernel
// ---------------------------------------------------------------------------
// One CTA per SM streams a contiguous bucket range through a ring of
// kPlainStages shared-memory stages, each filled by ONE 1-D bulk copy of whole
// rows (up to kPlainStageBytes), so ~192 KiB per SM are in flight whatever the
// register pressure.  Eight consumer warps XOR the staged rows: with U <= 256
// uint4 per row (U dividing 256), thread t owns column t % U of every
// (256/U)-th row; with U = 256*CPT it owns columns t, t+256, ... of every row.
// Partials of threads sharing a column are folded in shared memory and the
// CTA's reply is XOR-reduced into the zeroed output with red.xor.
constexpr int kPlainStages = 6;
constexpr int kPlainStageBytes = 32 * 1024;
constexpr int kPlainThreads = 32 * 9;  // 8 consumer warps + 1 producer warp
constexpr int kPlainTmaSmem = kPlainStages * kPlainStageBytes + 128;

template <int NB, int CPT>
__global__ void __launch_bounds__(kPlainThreads, 1)
    plain_tma_kernel(const uint4* __restrict__ T, uint64_t n, uint32_t U,
                     const uint64_t* __restrict__ R, uint32_t words64, uint32_t B,
                     uint4* __restrict__ out, uint64_t rows_per_cta) {
  extern __shared__ __align__(128) uint8_t smem_raw[];
  uint64_t* full = reinterpret_cast<uint64_t*>(smem_raw);
  uint64_t* empty = full + kPlainStages;
  uint4* stages = reinterpret_cast<uint4*>(smem_raw + 128);
  __shared__ int s_abort;
  constexpr int NC = CPT > 0 ? CPT : 1;  // accumulators per request

  pdl_launch_dependents();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint64_t k0 = static_cast<uint64_t>(blockIdx.x) * rows_per_cta;
  const uint64_t k1 = min(n, k0 + rows_per_cta);
  const uint32_t stage_rows = max(1u, static_cast<uint32_t>(kPlainStageBytes / (U * 16u)));
  if (threadIdx.x == 0) {
    for (int s = 0; s < kPlainStages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 8);
    }
    s_abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  volatile int* abort_flag = &s_abort;

  if (warp == 8) {
    // ---- producer: one bulk copy per stage
    uint32_t iter = 0;
    if (lane == 0) {
      for (uint64_t ks = k0; ks < k1; ks += stage_rows, ++iter) {
        const uint32_t s = iter % kPlainStages, ph = (iter / kPlainStages) & 1u;
        if (!mbar_wait_backoff(&empty[s], ph ^ 1u, abort_flag)) break;
        const uint32_t rows = static_cast<uint32_t>(k1 - ks < stage_rows ? k1 - ks : stage_rows);
        const uint32_t bytes = rows * U * 16u;
        mbar_expect_tx(&full[s], bytes);
        bulk_g2s(stages + static_cast<uint64_t>(s) * (kPlainStageBytes / 16), T + ks * U, bytes,
                 &full[s]);
        mbar_arrive(&full[s]);
      }
      if (*abort_flag) {
        const uint32_t first = iter > kPlainStages ? iter - kPlainStages : 0;
        for (uint32_t x = first; x < iter; ++x) {
          const uint64_t t0 = globaltimer();
          while (!mbar_try_wait(&full[x % kPlainStages], (x / kPlainStages) & 1u) &&
                 globaltimer() - t0 < kWaitLimitNs) {
          }
        }
      }
    }
    return;
  }

  // ---- consumers
  const uint32_t t = threadIdx.x;  // 0..255
  const uint32_t rpi = CPT > 0 ? 1u : 256u / U;
  const uint32_t roff = CPT > 0 ? 0u : t / U;
  const uint32_t col = CPT > 0 ? t : t % U;
  uint4 acc[NB][NC];
#pragma unroll
  for (int b = 0; b < NB; ++b)
#pragma unroll
    for (int c = 0; c < NC; ++c) acc[b][c] = make_uint4(0u, 0u, 0u, 0u);

  uint32_t iter = 0;
  bool ok = true;
  for (uint64_t ks = k0; ks < k1; ks += stage_rows, ++iter) {
    const uint32_t s = iter % kPlainStages, ph = (iter / kPlainStages) & 1u;
    if (!mbar_wait(&full[s], ph, abort_flag)) {
      ok = false;
      break;
    }
    const uint4* st = stages + static_cast<uint64_t>(s) * (kPlainStageBytes / 16);
    const uint32_t rows = static_cast<uint32_t>(k1 - ks < stage_rows ? k1 - ks : stage_rows);
    for (uint32_t r = roff; r < rows; r += rpi) {
      const uint64_t k = ks + r;
      uint32_t m[NB];
#pragma unroll
      for (int b = 0; b < NB; ++b)
        m[b] = b < (int)B ? bit_mask(__ldg(R + b * (uint64_t)words64 + (k >> 6)), k & 63) : 0u;
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        const uint4 v = st[r * U + col + c * 256u];
#pragma unroll
        for (int b = 0; b < NB; ++b) {
          acc[b][c].x ^= v.x & m[b];
          acc[b][c].y ^= v.y & m[b];
          acc[b][c].z ^= v.z & m[b];
          acc[b][c].w ^= v.w & m[b];
        }
      }
    }
    __syncwarp();
    if (lane == 0) mbar_arrive(&empty[s]);
  }
  // (after a give-up every consumer still passes the fold barriers below, so
  // none waits for a peer that left; only the reduction is skipped)

  // fold the partials of threads that share a column (U < 256), then reduce
  if (CPT == 0 && rpi > 1) {
    // the ring is idle now: reuse stage 0's first 256*NB uint4 as fold space
    asm volatile("bar.sync 2, 256;" ::: "memory");
    uint4* fold = stages;
#pragma unroll
    for (int b = 0; b < NB; ++b) fold[b * 256 + t] = acc[b][0];
    asm volatile("bar.sync 2, 256;" ::: "memory");
    if (t < U) {
#pragma unroll
      for (int b = 0; b < NB; ++b) {
        uint4 x = make_uint4(0u, 0u, 0u, 0u);
        for (uint32_t r = 0; r < rpi; ++r) {
          const uint4 p = fold[b * 256 + r * U + t];
          x.x ^= p.x;
          x.y ^= p.y;
          x.z ^= p.z;
          x.w ^= p.w;
        }
        acc[b][0] = x;
      }
    }
  }
  pdl_wait();
  if (ok && !*abort_flag && k0 < k1 && (CPT > 0 || t < U)) {
#pragma unroll
    for (int b = 0; b < NB; ++b) {
      if (b >= (int)B) continue;
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        uint32_t* o = reinterpret_cast<uint32_t*>(out + static_cast<uint64_t>(b) * U + col + c * 256u);
        red_xor64(o, acc[b][c].x, acc[b][c].y);
        red_xor64(o + 2, acc[b][c].z, acc[b][c].w);
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

__device__ __forceinline__ void xor_row(uint32_t (&acc)[kMR][kNW], const uint4& m0, const uint4& m1,
                                        const uint4& t0, const uint4& t1, const uint4& t2,
                                        const uint4& t3) {
  const uint32_t m[kMR] = {m0.x, m0.y, m0.z, m0.w, m1.x, m1.y, m1.z, m1.w};
  const uint32_t w[kNW] = {t0.x, t0.y, t0.z, t0.w, t1.x, t1.y, t1.z, t1.w,
                           t2.x, t2.y, t2.z, t2.w, t3.x, t3.y, t3.z, t3.w};
#pragma unroll
  for (int i = 0; i < kMR; ++i)
#pragma unroll
    for (int q = 0; q < kNW; ++q) acc[i][q] ^= m[i] & w[q];
}

__device__ __forceinline__ uint4 lds4a(uint32_t addr) {
  uint4 v;
  asm volatile("ld.shared.v4.u32 {%0,%1,%2,%3}, [%4];"
               : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
               : "r"(addr));
  return v;
}

// One consumer warp's `nr` rows of a stage (rows first, first + wk, ...),
// addressed by 32-bit shared-memory byte offsets.  The masks and table words
// of the next row are loaded while the current row's 128 LOP3s run (measured
// faster on GB300 than two-rows-per-iteration or ping-pong operand sets).
// LW_LOG2 fixes the lane layout so that a thread's four 16-byte segments sit
// at immediate offsets.
template <int LW_LOG2>
__device__ __forceinline__ void consume_rows(uint32_t (&acc)[kMR][kNW], uint32_t ma, uint32_t ta,
                                             uint32_t nr, uint32_t mstep, uint32_t tstep) {
  constexpr uint32_t SEG = (1u << LW_LOG2) * 16u;
  if (nr == 0) return;
  uint4 m0 = lds4a(ma), m1 = lds4a(ma + 16);
  uint4 t0 = lds4a(ta), t1 = lds4a(ta + SEG), t2 = lds4a(ta + 2 * SEG), t3 = lds4a(ta + 3 * SEG);
  for (;;) {
    if (--nr) {
      ma += mstep;
      ta += tstep;
      const uint4 n0 = lds4a(ma), n1 = lds4a(ma + 16);
      const uint4 u0 = lds4a(ta), u1 = lds4a(ta + SEG), u2 = lds4a(ta + 2 * SEG), u3 = lds4a(ta + 3 * SEG);
      xor_row(acc, m0, m1, t0, t1, t2, t3);
      m0 = n0; m1 = n1; t0 = u0; t1 = u1; t2 = u2; t3 = u3;
    } else {
      xor_row(acc, m0, m1, t0, t1, t2, t3);
      break;
    }
  }
}

// One consumer warp's share of one item: wait for each stage, XOR its rows,
// release the stage, then store (single k-chunk) or XOR-reduce (split) the
// 8-request x 16-word register tile.  Returns false if a wait gave up.
template <int LW_LOG2>
__device__ __forceinline__ bool consume_item(const ScanJob& J, const Item& it, uint32_t cw,
                                             uint32_t lane, uint64_t* full, uint64_t* empty,
                                             uint8_t* stages, volatile int* abort_flag,
                                             uint32_t& iter) {
  constexpr uint32_t LW = 1u << LW_LOG2;
  const uint32_t ww = J.shape.ww, wbw = J.shape.wb * ww, wk = J.shape.wk;
  const uint32_t bt_ = J.shape.bt(), wt_ = J.shape.wt(), sr = J.shape.srows();
  const uint32_t wk_idx = cw / wbw, rem = cw % wbw;
  const uint32_t wb_idx = rem / ww, ww_idx = rem % ww;
  const uint32_t lwi = lane & (LW - 1), lbi = lane >> LW_LOG2;
  const uint32_t rq0 = (wb_idx * (32u >> LW_LOG2) + lbi) * kMR;
  const uint32_t wbase = ww_idx * (LW * kNW) + lwi * 4u;

  uint32_t acc[kMR][kNW];
#pragma unroll
  for (int i = 0; i < kMR; ++i)
#pragma unroll
    for (int q = 0; q < kNW; ++q) acc[i][q] = 0u;

  const uint32_t moff = (wk_idx * bt_ + rq0) * 4u, toff = (wk_idx * wt_ + wbase) * 4u;
  const uint32_t mstep = wk * bt_ * 4u, tstep = wk * wt_ * 4u;
  const uint32_t stage0 = smem_u32(stages);
  for (uint64_t ks = it.k0; ks < it.k1; ks += sr, ++iter) {
    const uint32_t s = iter % kStages;
    const uint32_t ph = (iter / kStages) & 1u;
    if (!mbar_wait(&full[s], ph, abort_flag)) return false;
    const uint32_t rows = static_cast<uint32_t>(it.k1 - ks < sr ? it.k1 - ks : sr);
    const uint32_t nr = rows > wk_idx ? (rows - wk_idx + wk - 1) / wk : 0u;
    const uint32_t tbase = stage0 + s * kStageBytes;
    consume_rows<LW_LOG2>(acc, tbase + sr * wt_ * 4u + moff, tbase + toff, nr, mstep, tstep);
    __syncwarp();
    if (lane == 0) mbar_arrive(&empty[s]);
  }

  // outputs are zeroed / released by the previous kernel of the stream
  pdl_wait();
  const bool split = J.split != 0;
  const uint32_t b0 = it.bt * bt_ + rq0;
  const uint32_t w0 = it.wt * wt_ + wbase;
#pragma unroll
  for (int i = 0; i < kMR; ++i) {
    const uint32_t b = b0 + i;
    if (b >= J.B) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const uint32_t wd = w0 + j * LW * 4u;
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
  return true;
}

__global__ void __launch_bounds__(kScanThreads, 1)
    batched_scan_kernel(const __grid_constant__ ScanLaunch L) {
  extern __shared__ __align__(128) uint8_t smem_raw[];
  uint64_t* full = reinterpret_cast<uint64_t*>(smem_raw);
  uint64_t* empty = full + kStages;
  uint64_t* claim_full = empty + kStages;
  uint64_t* claim_empty = claim_full + 1;
  uint8_t* stages = smem_raw + 256;
  __shared__ int s_abort;
  __shared__ uint32_t s_claim;
  __shared__ uint32_t s_hdr[kStages];

  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  pdl_launch_dependents();
  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(&full[s], kProducerThreads);
      mbar_init(&empty[s], kConsumerWarps);
    }
    mbar_init(claim_full, 1);
    mbar_init(claim_empty, kProducerThreads);
    s_abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  volatile int* abort_flag = &s_abort;

  uint32_t iter = 0;  // pipeline stage counter, identical in producer and consumers

  if (threadIdx.x < kProducerThreads) {
    // ---------------- producer warpgroup ----------------
    // Thread 0 claims items (listed by descending cost) from the launch's
    // counter and publishes each claim through claim_full; every producer
    // thread acknowledges it on claim_empty before thread 0 may post the next
    // one (so no waiter can miss a phase).  Warp 0 issues the bulk copies;
    // all 128 threads expand request bits.  The claimed item id rides in the
    // header of its first stage; once the items run out an END header
    // releases the consumers.
    asm volatile("setmaxnreg.dec.sync.aligned.u32 %0;" ::"n"(kProducerRegs));
    const uint32_t ptid = threadIdx.x;
    uint32_t* counter = &g_item_counter[L.counter_slot];
    bool ok = true;
    for (uint32_t r = 0; ok; ++r) {
      uint32_t item;
      if (L.dynamic) {
        if (ptid == 0) {
          bool go = true;
          if (r == 0)
            pdl_wait();  // the previous kernel reset the counter
          else
            go = mbar_wait(claim_empty, (r - 1) & 1u, abort_flag);
          if (go) {
            s_claim = atomicAdd(counter, 1u);
            mbar_arrive(claim_full);
          }
        }
        if (!mbar_wait(claim_full, r & 1u, abort_flag)) break;
        item = *reinterpret_cast<volatile uint32_t*>(&s_claim);
        mbar_arrive(claim_empty);
      } else {
        item = blockIdx.x + r * gridDim.x;  // items of one job cost the same
      }
      if (item >= L.total_items) {
        const uint32_t s = iter % kStages, ph = (iter / kStages) & 1u;
        if (mbar_wait(&empty[s], ph ^ 1u, abort_flag)) {
          if (ptid == 0) s_hdr[s] = kEndItem;
          mbar_arrive(&full[s]);
        }
        ++iter;
        break;
      }
      const Item it = decode_item(L, item);
      const ScanJob& J = L.jobs[it.job];
      const uint32_t bt_ = J.shape.bt(), wt_ = J.shape.wt(), sr = J.shape.srows();
      const uint32_t w0 = it.wt * wt_;
      const uint32_t wcount = min(wt_, J.Wd - w0);
      const uint32_t b0 = it.bt * bt_;
      // a tile spanning whole rows is contiguous in global and shared memory
      const bool whole_rows = (wt_ == J.Wd);
      // each thread's request words (b = ptid + 128 c, c < 4; a B-tile holds at
      // most 512 requests): one 64-bit word
      // covers 64 buckets, i.e. several stages, so it is loaded once per word
      uint64_t wcache[4] = {0, 0, 0, 0};
      uint64_t widx = ~0ull;
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
        if (ptid == 0 && ks == it.k0) s_hdr[s] = item;
        if (warp == 0) {
          if (lane == 0) mbar_expect_tx(&full[s], rows * wcount * 4u);
          __syncwarp();
          if (whole_rows) {
            if (lane == 0) bulk_g2s(tsm, J.T + ks * J.Wd, rows * wcount * 4u, &full[s]);
          } else {
            for (uint32_t q = lane; q < rows; q += 32)
              bulk_g2s(tsm + q * wt_, J.T + (ks + q) * J.Wd + w0, wcount * 4u, &full[s]);
          }
        }
        // request bits -> 32-bit masks, zero for rows past the chunk and for
        // request slots past B
        if ((ks >> 6) != widx) {
          widx = ks >> 6;
#pragma unroll
          for (uint32_t c = 0; c < 4; ++c) {
            const uint32_t b = ptid + c * kProducerThreads;
            wcache[c] = (b < bt_ && b0 + b < J.B)
                            ? __ldg(J.R + static_cast<uint64_t>(b0 + b) * J.words64 + widx)
                            : 0ull;
          }
        }
        const uint32_t sh = static_cast<uint32_t>(ks & 63);
#pragma unroll
        for (uint32_t c = 0; c < 4; ++c) {
          const uint32_t b = ptid + c * kProducerThreads;
          if (b < bt_) {
            const uint64_t wbits = wcache[c] >> sh;
            for (uint32_t q = 0; q < sr; ++q)
              msm[q * bt_ + b] = (q < rows) ? bit_mask(wbits, q) : 0u;
          }
        }
        mbar_arrive(&full[s]);
      }
    }
    if (*abort_flag && ptid == 0) {
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

  // ---------------- consumer warpgroups ----------------
  asm volatile("setmaxnreg.inc.sync.aligned.u32 %0;" ::"n"(kConsumerRegs));
  const uint32_t cw = static_cast<uint32_t>(warp - kProducerThreads / 32);
  for (;;) {
    // the header of the next item's first stage names the item (or END)
    const uint32_t s = iter % kStages, ph = (iter / kStages) & 1u;
    if (!mbar_wait(&full[s], ph, abort_flag)) return;
    const uint32_t item = *reinterpret_cast<volatile uint32_t*>(&s_hdr[s]);
    if (item == kEndItem) return;
    const Item it = decode_item(L, item);
    const ScanJob& J = L.jobs[it.job];
    bool ok;
    switch (J.shape.lw_log2) {
      case 5: ok = consume_item<5>(J, it, cw, lane, full, empty, stages, abort_flag, iter); break;
      case 4: ok = consume_item<4>(J, it, cw, lane, full, empty, stages, abort_flag, iter); break;
      case 3: ok = consume_item<3>(J, it, cw, lane, full, empty, stages, abort_flag, iter); break;
      default: ok = consume_item<2>(J, it, cw, lane, full, empty, stages, abort_flag, iter); break;
    }
    if (!ok) return;
  }
}

// Initialises B replies before a scan XOR-reduces into them: zeros, or the
// one-time masks of a serialized-PIR read.  It lets the scan launch at once
// (the scan only waits for it before its reduction) but waits itself for the
// previous kernel, which may still be reducing into a buffer the caller reuses.
__global__ void init_replies_kernel(uint4* __restrict__ out, uint32_t B, uint32_t row_u4,
                                    const uint8_t* __restrict__ seeds) {
  pdl_launch_dependents();
  pdl_wait();
  init_replies(out, B, row_u4, seeds, blockIdx.x * (uint64_t)blockDim.x + threadIdx.x,
               (uint64_t)gridDim.x * blockDim.x);
}

// Resets the launch's item counter and initialises the outputs of the jobs
// whose partial replies are XOR-reduced (zeros, or the masks of a masked
// job).  grid.y = job.
__global__ void zero_outputs_kernel(const __grid_constant__ ScanLaunch L) {
  pdl_launch_dependents();
  pdl_wait();
  if (blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0) g_item_counter[L.counter_slot] = 0u;
  const ScanJob& J = L.jobs[blockIdx.y];
  if (!J.split) return;
  init_replies(reinterpret_cast<uint4*>(J.out), J.B, J.Wd / 4, J.seeds,
               blockIdx.x * (uint64_t)blockDim.x + threadIdx.x, (uint64_t)gridDim.x * blockDim.x);
}

// Self-test of the bounded wait: one CTA waits on an mbarrier that nothing
// ever arrives at, with a short limit, exactly as the scan kernels wait on
// their pipelines; the wait gives up, sets the status word and the kernel
// returns, leaving the context usable.
__global__ void selftest_wait_kernel(uint64_t limit_ns) {
  __shared__ uint64_t bar;
  __shared__ int abort_flag;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  mbar_wait(&bar, 0u, &abort_flag, limit_ns);
}

}  // namespace

cudaError_t launch_selftest_wait(uint64_t limit_ns, cudaStream_t st) {
  selftest_wait_kernel<<<1, 32, 0, st>>>(limit_ns);
  count_launches();
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
int device_sm_count() {
  // per device, computed once (a race only repeats the query)
  static std::atomic<int> cached[64] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) return 1;
  int c = cached[dev].load(std::memory_order_acquire);
  if (!c) {
    int v = 0;
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
    c = v > 0 ? v : 1;
    cached[dev].store(c, std::memory_order_release);
  }
  return c;
}

template <int NB>
static int plain_occupancy() {
  static std::atomic<int> cached{0};  // computed once (a race only repeats the query)
  int c = cached.load(std::memory_order_acquire);
  if (!c) {
    int v = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, plain_scan_kernel<NB, 8>, 256, 0);
    c = v > 0 ? v : 1;
    cached.store(c, std::memory_order_release);
  }
  return c;
}

int plain_ctas_per_sm() { return plain_occupancy<1>(); }


int batched_ctas_per_sm() {
  static std::atomic<int> cached{0};  // computed once (a race only repeats the query)
  int c = cached.load(std::memory_order_acquire);
  if (!c) {
    cudaFuncSetAttribute(batched_scan_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         kScanSmem);
    int v = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, batched_scan_kernel, kScanThreads,
                                                  kScanSmem);
    c = v > 0 ? v : 1;
    cached.store(c, std::memory_order_release);
  }
  return c;
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
  j.split = (j.n_kc > 1 || s.wk > 1 || j.seeds) ? 1u : 0u;
  return true;
}

cudaError_t launch_batched(const ScanLaunch& L, int grid, cudaStream_t st) {
  static std::atomic<bool> attr_set{false};  // idempotent set-up: a race only repeats it
  if (!attr_set.load(std::memory_order_acquire)) {
    // the setmaxnreg split is only safe with the register count it was sized for
    cudaFuncAttributes fa{};
    cudaError_t e = cudaFuncGetAttributes(&fa, batched_scan_kernel);
    if (e != cudaSuccess) return e;
    if (fa.numRegs != kScanLaunchRegs) return cudaErrorInvalidConfiguration;
    e = cudaFuncSetAttribute(batched_scan_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             kScanSmem);
    if (e != cudaSuccess) return e;
    attr_set.store(true, std::memory_order_release);
  }
  if (L.total_items == 0) return cudaSuccess;
  return launch_pdl(batched_scan_kernel, dim3(grid), dim3(kScanThreads), kScanSmem, st, L);
}

cudaError_t launch_zero_outputs(const ScanLaunch& L, cudaStream_t st) {
  bool any = false;
  for (uint32_t i = 0; i < L.njobs; ++i) any |= L.jobs[i].split != 0;
  return launch_pdl(zero_outputs_kernel, dim3(any ? 64 : 1, L.njobs), dim3(256), 0, st, L);
}

template <int NB, int CPT>
static cudaError_t launch_plain_tma_t(const uint4* T4, uint64_t n, uint32_t U, const uint64_t* R,
                                      uint32_t words64, uint32_t B, uint4* o4, cudaStream_t st) {
  static std::atomic<bool> attr_set{false};  // idempotent set-up: a race only repeats it
  if (!attr_set.load(std::memory_order_acquire)) {
    cudaError_t e = cudaFuncSetAttribute(plain_tma_kernel<NB, CPT>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, kPlainTmaSmem);
    if (e != cudaSuccess) return e;
    attr_set.store(true, std::memory_order_release);
  }
  uint64_t ctas = std::min<uint64_t>(device_sm_count(), n);
  const uint64_t rows_per_cta = (n + ctas - 1) / ctas;
  ctas = (n + rows_per_cta - 1) / rows_per_cta;
  return launch_pdl(plain_tma_kernel<NB, CPT>, dim3(static_cast<uint32_t>(ctas)),
                    dim3(kPlainThreads), kPlainTmaSmem, st, T4, n, U, R, words64, B, o4,
                    rows_per_cta);
}

template <int NB, int CMAX>
static cudaError_t launch_plain_tma(const uint4* T4, uint64_t n, uint32_t U, const uint64_t* R,
                                    uint32_t words64, uint32_t B, uint4* o4, cudaStream_t st) {
  if (U <= 256) return launch_plain_tma_t<NB, 0>(T4, n, U, R, words64, B, o4, st);
  switch (U / 256) {
    case 1: return launch_plain_tma_t<NB, 1>(T4, n, U, R, words64, B, o4, st);
    case 2: return launch_plain_tma_t<NB, 2>(T4, n, U, R, words64, B, o4, st);
    case 4: return launch_plain_tma_t<NB, 4>(T4, n, U, R, words64, B, o4, st);
    default: return launch_plain_tma_t<NB, CMAX>(T4, n, U, R, words64, B, o4, st);
  }
}

// Rows the TMA kernel handles: U dividing 256, or U = 256 * {1,2,4,8}; the
// 4-request variant stops at 4 column groups (its accumulators must stay in
// registers).
static bool plain_tma_ok(uint32_t U, int nb) {
  if (U <= 256) return (256 % U) == 0;
  const uint32_t c = U / 256;
  const uint32_t cmax = nb == 4 ? 4 : 8;
  return (U % 256) == 0 && (c == 1 || c == 2 || c == 4 || c == 8) && c <= cmax;
}

cudaError_t launch_init_replies(uint4* out, uint32_t B, uint32_t row_u4, const uint8_t* seeds,
                                cudaStream_t st) {
  // one thread per 16-byte word (zeros) or per 64-byte keystream block (masks)
  const uint64_t work = seeds ? static_cast<uint64_t>(B) * ((row_u4 + 3) / 4)
                              : static_cast<uint64_t>(B) * row_u4;
  if (work == 0) return cudaSuccess;
  return launch_pdl(init_replies_kernel,
                    dim3(static_cast<uint32_t>(std::min<uint64_t>((work + 255) / 256, 1024))),
                    dim3(256), 0, st, out, B, row_u4, seeds);
}

cudaError_t launch_plain(const uint32_t* T, uint64_t n, uint32_t Wd, const uint64_t* R,
                         uint32_t words64, uint32_t B, uint32_t* out, const uint8_t* seeds,
                         cudaStream_t st, int ctas) {
  if (B == 0) return cudaSuccess;
  const uint32_t U = Wd / 4;
  uint4* o4 = reinterpret_cast<uint4*>(out);
  cudaError_t e = launch_init_replies(o4, B, U, seeds, st);
  if (e != cudaSuccess) return e;
  const int nb = B == 1 ? 1 : (B == 2 ? 2 : 4);
  const uint4* T4 = reinterpret_cast<const uint4*>(T);
  if (ctas == 0 && plain_tma_ok(U, nb)) {
    if (nb == 1) return launch_plain_tma<1, 8>(T4, n, U, R, words64, B, o4, st);
    if (nb == 2) return launch_plain_tma<2, 8>(T4, n, U, R, words64, B, o4, st);
    return launch_plain_tma<4, 4>(T4, n, U, R, words64, B, o4, st);
  }
  // register-streaming kernel for other row widths (ctas < 0 forces it)
  const uint32_t slices = (U + kPlainSlice - 1) / kPlainSlice;
  if (ctas <= 0)
    ctas = device_sm_count() *
           (nb == 1 ? plain_occupancy<1>() : nb == 2 ? plain_occupancy<2>() : plain_occupancy<4>());
  uint64_t chunks = static_cast<uint64_t>(ctas) / slices;
  if (chunks < 1) chunks = 1;
  if (chunks > n) chunks = n;
  const uint64_t rows_per_cta = (n + chunks - 1) / chunks;
  chunks = (n + rows_per_cta - 1) / rows_per_cta;
  dim3 grid(static_cast<uint32_t>(chunks), slices);
  if (nb == 1)
    return launch_pdl(plain_scan_kernel<1, 8>, grid, dim3(256), 0, st, T4, n, U, R, words64, B, o4, rows_per_cta);
  if (nb == 2)
    return launch_pdl(plain_scan_kernel<2, 8>, grid, dim3(256), 0, st, T4, n, U, R, words64, B, o4, rows_per_cta);
  return launch_pdl(plain_scan_kernel<4, 8>, grid, dim3(256), 0, st, T4, n, U, R, words64, B, o4, rows_per_cta);
}

int* device_status_word() {
  // per device, looked up once (a race only repeats the lookup)
  static std::atomic<int*> addr[64] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
  int* a = addr[dev].load(std::memory_order_acquire);
  if (!a) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_status) != cudaSuccess) return nullptr;
    a = static_cast<int*>(p);
    addr[dev].store(a, std::memory_order_release);
  }
  return a;
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
