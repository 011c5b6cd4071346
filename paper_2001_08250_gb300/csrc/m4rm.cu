// Four-Russians ("method of four Russians", M4RM) form of the batched read.
//
// The server answer of Section 2 (step 5) for B requests is the GF(2)
// product Out = R (x) T.  Cut the buckets into groups of 8.  For one group and
// one 64-word column tile, the 256 XOR combinations of its 8 row segments are
// built once in shared memory (Gray-code order: one XOR per combination); a
// request then adds the whole group with ONE lookup C[v] (v = its 8 request
// bits for the group) and ONE XOR per word, where the register-tiled kernel
// spends 8 LOP3s.  Every row is still read and combined for every request:
// the combinations are built whatever the bits are, and every request looks
// up every group.
//
// Persistent CTA per SM, three warpgroups:
//   producer (setmaxnreg 56): warp 0 streams 64-row x 256-byte table tiles into
//     a 4-stage mbarrier ring with cp.async.bulk; all 128 threads write the
//     requests' 8-bit group indices (one byte per request and group);
//   two consumer warpgroups (setmaxnreg 224): per group, every thread builds
//     16 combinations x 16 bytes of the table into a double-buffered 2 x 64 KiB
//     combination table, the warps meet on a bounded mbarrier, then every
//     thread adds MR requests x 16 bytes by lookup.  Lanes run along the row,
//     so both the stores and the lookups of a warp are bank-conflict free.
// Items are (job, B-tile, W-tile, k-chunk) over one or many tables, claimed
// dynamically from a per-launch counter; split k-chunks XOR-reduce into the
// output zeroed by a PDL-chained kernel.
#include <algorithm>
#include <atomic>
#include <vector>

#include "chacha.cuh"
#include "tpir_internal.h"

namespace tpir {
namespace {

constexpr int kWT = 64;            // words per column tile (256 B of each row)
constexpr int kSR = 64;            // rows per stage (one 64-bit request word)
constexpr int kGroups = kSR / 8;   // groups per stage
constexpr int kM4Stages = 4;
constexpr int kTileBytes = kSR * kWT * 4;             // 16 KiB
constexpr int kM4Threads = 384;
constexpr int kM4ProducerThreads = 128;
constexpr int kCombBytes = 256 * kWT * 4;             // 64 KiB per buffer
constexpr uint64_t kM4WaitLimitNs = 4000000000ull;

constexpr uint32_t kM4MaxJobs = TPIR_MAX_JOBS;
constexpr uint32_t kM4CounterSlots = 256;
constexpr uint32_t kM4End = 0xFFFFFFFFu;

struct M4Job {
  const uint32_t* T;
  const uint64_t* R;
  uint32_t* out;
  const uint8_t* seeds;  // B x 32-byte mask seeds, or null
  uint64_t n;
  uint32_t Wd, words64, B;
  uint32_t n_bt, n_wt, n_kc;
  uint32_t kc_rows;  // multiple of 64
  uint32_t split;
  uint32_t item_begin;
  uint32_t pad;
};

// The launch's job table is a kernel parameter sized by NJ: one job for a
// single-table read (small parameters), kM4MaxJobs for many tables.
template <int NJ>
struct M4Launch {
  uint32_t njobs, total_items, counter_slot;
  uint32_t dynamic;  // informational: launches with NJ > 1 claim items from the counter
  M4Job jobs[NJ];
};

// Item counters of the dynamic schedule (one per launch, rotating), reset by
// the zero kernel that precedes each launch.
__device__ uint32_t g_m4_counter[kM4CounterSlots];

struct M4Item {
  uint32_t job, bt, wt;
  uint64_t k0, k1;
};

template <int NJ>
__device__ __forceinline__ M4Item m4_decode(const M4Launch<NJ>& L, uint32_t item) {
  uint32_t lo = 0, hi = L.njobs - 1;
  while (lo < hi) {
    const uint32_t mid = (lo + hi + 1) >> 1;
    if (L.jobs[mid].item_begin <= item)
      lo = mid;
    else
      hi = mid - 1;
  }
  const M4Job& J = L.jobs[lo];
  M4Item it;
  it.job = lo;
  uint32_t local = item - J.item_begin;
  it.bt = local % J.n_bt;
  local /= J.n_bt;
  it.wt = local % J.n_wt;
  it.k0 = static_cast<uint64_t>(local / J.n_wt) * J.kc_rows;
  it.k1 = min(J.n, it.k0 + J.kc_rows);
  return it;
}

// stage = tile + one byte per request (16 * MR per B-tile) and group
template <int MR>
struct M4Layout {
  static constexpr int kStage = kTileBytes + kGroups * 16 * MR;
  static constexpr int kSmem = 256 + kM4Stages * kStage + 2 * kCombBytes;
};

__device__ __forceinline__ uint64_t gtimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ uint32_t s_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void b_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(s_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void b_expect(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.expect_tx.relaxed.cta.shared::cta.b64 [%0], %1;" ::"r"(s_u32(bar)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void b_arrive(uint64_t* bar) {
  asm volatile(
      "{\n\t.reg .b64 st;\n\tmbarrier.arrive.release.cta.shared::cta.b64 st, [%0];\n\t}" ::"r"(
          s_u32(bar))
      : "memory");
}
__device__ __forceinline__ bool b_try(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.acquire.cta.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(s_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait: false after the limit or once another warp has given up.
__device__ __forceinline__ bool b_wait(uint64_t* bar, uint32_t parity, volatile int* abort_flag,
                                       int* status) {
  if (b_try(bar, parity)) return true;
  const uint64_t t0 = gtimer();
  while (!b_try(bar, parity)) {
    if (*abort_flag) return false;
    if (gtimer() - t0 > kM4WaitLimitNs) {
      *abort_flag = 1;
      atomicExch(status, static_cast<int>(TPIR_ETIMEDOUT));
      return false;
    }
  }
  return true;
}
__device__ __forceinline__ void bulk(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          s_u32(dst)),
      "l"(src), "r"(bytes), "r"(s_u32(bar))
      : "memory");
}
__device__ __forceinline__ uint4 ld128(uint32_t a) {
  uint4 v;
  asm volatile("ld.shared.v4.u32 {%0,%1,%2,%3}, [%4];"
               : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
               : "r"(a));
  return v;
}
__device__ __forceinline__ void st128(uint32_t a, const uint4& v) {
  asm volatile("st.shared.v4.u32 [%0], {%1,%2,%3,%4};" ::"r"(a), "r"(v.x), "r"(v.y), "r"(v.z),
               "r"(v.w)
               : "memory");
}
__device__ __forceinline__ void x4(uint4& a, const uint4& b) {
  a.x ^= b.x;
  a.y ^= b.y;
  a.z ^= b.z;
  a.w ^= b.w;
}
__device__ __forceinline__ void red64(uint32_t* p, uint32_t lo, uint32_t hi) {
  const uint64_t v = (static_cast<uint64_t>(hi) << 32) | lo;
  asm volatile("red.relaxed.gpu.global.xor.b64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

template <int MR, int NJ>
__global__ void __launch_bounds__(kM4Threads, 1)
    m4rm_scan_kernel(const __grid_constant__ M4Launch<NJ> L, int* status) {
  constexpr int BT = 16 * MR;  // requests per B-tile (8 warps x 2 halves x MR)
  constexpr int SB = M4Layout<MR>::kStage;
  extern __shared__ __align__(128) uint8_t smem[];
  uint64_t* full = reinterpret_cast<uint64_t*>(smem);
  uint64_t* empty = full + kM4Stages;
  uint64_t* grp = empty + kM4Stages;  // consumer warps meet here once per group
  uint64_t* claim_full = grp + 1;
  uint64_t* claim_empty = claim_full + 1;
  uint8_t* stages = smem + 256;
  uint8_t* comb = stages + kM4Stages * SB;
  __shared__ int s_abort;
  __shared__ uint32_t s_claim;
  __shared__ uint32_t s_hdr[kM4Stages];

  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < kM4Stages; ++s) {
      b_init(&full[s], kM4ProducerThreads);
      b_init(&empty[s], 8);
    }
    b_init(grp, 8);
    b_init(claim_full, 1);
    b_init(claim_empty, kM4ProducerThreads);
    s_abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  volatile int* abort_flag = &s_abort;
  uint32_t iter = 0;

  if (threadIdx.x < kM4ProducerThreads) {
    // ---------------- producer warpgroup ----------------
    asm volatile("setmaxnreg.dec.sync.aligned.u32 56;");
    // Thread 0 claims items (jobs listed by descending cost) from the
    // launch's counter and passes each claim to the warpgroup (claim_full),
    // which acknowledges it (claim_empty) before the next claim is posted.
    // The item id rides in the header of its first stage; an END header
    // releases the consumers.
    const uint32_t ptid = threadIdx.x;
    uint32_t* counter = &g_m4_counter[L.counter_slot];
    bool ok = true;
    for (uint32_t r = 0; ok; ++r) {
      uint32_t item;
      if constexpr (NJ > 1) {
        if (ptid == 0) {
          bool go = true;
          if (r == 0)
            asm volatile("griddepcontrol.wait;" ::: "memory");  // counter reset
          else
            go = b_wait(claim_empty, (r - 1) & 1u, abort_flag, status);
          if (go) {
            s_claim = atomicAdd(counter, 1u);
            b_arrive(claim_full);
          }
        }
        if (!b_wait(claim_full, r & 1u, abort_flag, status)) break;
        item = *reinterpret_cast<volatile uint32_t*>(&s_claim);
        b_arrive(claim_empty);
      } else {
        item = blockIdx.x + r * gridDim.x;  // one job: items cost the same
      }
      if (item >= L.total_items) {
        if constexpr (NJ > 1) {
          const uint32_t s = iter % kM4Stages, ph = (iter / kM4Stages) & 1u;
          if (b_wait(&empty[s], ph ^ 1u, abort_flag, status)) {
            if (ptid == 0) s_hdr[s] = kM4End;
            b_arrive(&full[s]);
          }
          ++iter;
        }
        break;
      }
      const M4Item it = m4_decode(L, item);
      const M4Job& J = L.jobs[it.job];
      const uint64_t k0 = it.k0, k1 = it.k1;
      const uint32_t w0 = it.wt * kWT;
      const uint32_t wcount = min(static_cast<uint32_t>(kWT), J.Wd - w0);
      const uint32_t b0 = it.bt * BT;
      for (uint64_t ks = k0; ks < k1; ks += kSR, ++iter) {
        const uint32_t s = iter % kM4Stages, ph = (iter / kM4Stages) & 1u;
        if (!b_wait(&empty[s], ph ^ 1u, abort_flag, status)) {
          ok = false;
          break;
        }
        uint8_t* st = stages + s * SB;
        uint8_t* bytes = st + kTileBytes;
        const uint32_t rows = static_cast<uint32_t>(k1 - ks < kSR ? k1 - ks : kSR);
        if constexpr (NJ > 1) {
          if (ptid == 0 && ks == k0) s_hdr[s] = item;
        }
        if (warp == 0) {
          if (lane == 0) b_expect(&full[s], rows * wcount * 4u);
          __syncwarp();
          for (uint32_t r2 = lane; r2 < rows; r2 += 32)
            bulk(st + r2 * (kWT * 4), J.T + (ks + r2) * J.Wd + w0, wcount * 4u, &full[s]);
        }
        // each request's 64 bits for the stage -> 8 group indices (bytes);
        // bits of rows past the chunk and requests past B are zero
        const uint64_t valid = rows >= 64 ? ~0ull : ((1ull << rows) - 1ull);
        for (uint32_t b = ptid; b < static_cast<uint32_t>(BT); b += kM4ProducerThreads) {
          uint64_t w = 0;
          if (b0 + b < J.B) w = __ldg(J.R + static_cast<uint64_t>(b0 + b) * J.words64 + (ks >> 6));
          w &= valid;
#pragma unroll
          for (int g = 0; g < kGroups; ++g) bytes[g * BT + b] = static_cast<uint8_t>(w >> (8 * g));
        }
        b_arrive(&full[s]);
      }
    }
    if (*abort_flag && ptid == 0) {
      const uint32_t first = iter > kM4Stages ? iter - kM4Stages : 0;
      for (uint32_t x = first; x < iter; ++x) {
        const uint64_t t0 = gtimer();
        while (!b_try(&full[x % kM4Stages], (x / kM4Stages) & 1u) &&
               gtimer() - t0 < kM4WaitLimitNs) {
        }
      }
    }
    return;
  }

  // ---------------- consumer warpgroups ----------------
  asm volatile("setmaxnreg.inc.sync.aligned.u32 224;");
  const uint32_t t = threadIdx.x - kM4ProducerThreads;  // 0..255
  const uint32_t cw = t >> 5;
  // build role: 16-byte column chunk c, combinations e*16 .. e*16+15
  const uint32_t bc = t & 15, be = t >> 4;
  // lookup role: chunk lc of requests rq0 .. rq0+MR-1
  const uint32_t lc = lane & 15;
  const uint32_t rq0 = (cw * 2 + (lane >> 4)) * MR;
  const uint32_t comb0 = s_u32(comb);
  uint32_t gidx = 0;  // groups processed: parity of the group barrier, comb buffer
  for (uint32_t r = 0;; ++r) {
    uint32_t item;
    if constexpr (NJ > 1) {
      // the header of the next item's first stage names the item (or END)
      const uint32_t s = iter % kM4Stages, ph = (iter / kM4Stages) & 1u;
      if (!b_wait(&full[s], ph, abort_flag, status)) return;
      item = *reinterpret_cast<volatile uint32_t*>(&s_hdr[s]);
      if (item == kM4End) return;
    } else {
      item = blockIdx.x + r * gridDim.x;
      if (item >= L.total_items) return;
    }
    const M4Item it = m4_decode(L, item);
    const M4Job& J = L.jobs[it.job];
    const uint32_t bt = it.bt, wt = it.wt;
    const uint64_t k0 = it.k0, k1 = it.k1;
    uint4 acc[MR];
#pragma unroll
    for (int i = 0; i < MR; ++i) acc[i] = make_uint4(0u, 0u, 0u, 0u);

    for (uint64_t ks = k0; ks < k1; ks += kSR, ++iter) {
      const uint32_t s = iter % kM4Stages, ph = (iter / kM4Stages) & 1u;
      if (!b_wait(&full[s], ph, abort_flag, status)) return;
      const uint32_t st = s_u32(stages + s * SB);
      const uint32_t bytes = st + kTileBytes;
      const uint32_t rows = static_cast<uint32_t>(k1 - ks < kSR ? k1 - ks : kSR);
      const uint32_t ngroups = (rows + 7) / 8;
      for (uint32_t g = 0; g < ngroups; ++g, ++gidx) {
        const uint32_t cb = comb0 + (gidx & 1u) * kCombBytes;
        // ---- build: combinations be*16 + j of the group's 8 row segments
        {
          uint4 r8[8];
#pragma unroll
          for (int i = 0; i < 8; ++i) r8[i] = ld128(st + (g * 8 + i) * (kWT * 4) + bc * 16);
          uint4 cur = make_uint4(0u, 0u, 0u, 0u);
#pragma unroll
          for (int i = 4; i < 8; ++i) {
            const uint32_t m = 0u - ((be >> (i - 4)) & 1u);
            cur.x ^= r8[i].x & m;
            cur.y ^= r8[i].y & m;
            cur.z ^= r8[i].z & m;
            cur.w ^= r8[i].w & m;
          }
          const uint32_t sa = cb + be * 16 * (kWT * 4) + bc * 16;
          st128(sa, cur);  // gray(0) = 0
#pragma unroll
          for (int j = 1; j < 16; ++j) {
            // Gray code: step j flips bit ctz(j)
            const int flip = (j & 1) ? 0 : (j & 2) ? 1 : (j & 4) ? 2 : 3;
            x4(cur, r8[flip]);
            st128(sa + static_cast<uint32_t>(j ^ (j >> 1)) * (kWT * 4), cur);
          }
        }
        __syncwarp();
        if (lane == 0) b_arrive(grp);
        if (!b_wait(grp, gidx & 1u, abort_flag, status)) return;
        // ---- lookups: one 16-byte load and XOR per request and group
        {
          const uint32_t ba = bytes + g * BT + rq0;
#pragma unroll
          for (int q = 0; q < MR / 16; ++q) {
            const uint4 v = ld128(ba + q * 16);
            const uint32_t vw[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
            for (int k = 0; k < 16; ++k) {
              // byte k of the 16 -> (index << 8) = the combination's offset
              const uint32_t off = __byte_perm(vw[k >> 2], 0u, 0x4404u | ((k & 3) << 4));
              x4(acc[q * 16 + k], ld128(cb + off + lc * 16));
            }
          }
        }
      }
      __syncwarp();
      if (lane == 0) b_arrive(&empty[s]);
    }

    // epilogue (outputs zeroed / released by the previous kernel of the stream)
    asm volatile("griddepcontrol.wait;" ::: "memory");
    const uint32_t wd = wt * kWT + lc * 4;
    if (wd < J.Wd) {
#pragma unroll
      for (int i = 0; i < MR; ++i) {
        const uint32_t b = bt * BT + rq0 + i;
        if (b >= J.B) continue;
        uint32_t* o = J.out + static_cast<uint64_t>(b) * J.Wd + wd;
        if (J.split) {
          red64(o, acc[i].x, acc[i].y);
          red64(o + 2, acc[i].z, acc[i].w);
        } else {
          *reinterpret_cast<uint4*>(o) = acc[i];
        }
      }
    }
  }
}

// Resets the launch's item counter and initialises the outputs of its split
// jobs (zeros, or the masks of masked jobs).
// grid.y = job.
template <int NJ>
__global__ void m4_zero_kernel(const __grid_constant__ M4Launch<NJ> L) {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  asm volatile("griddepcontrol.wait;" ::: "memory");
  if (blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0) g_m4_counter[L.counter_slot] = 0u;
  const M4Job& J = L.jobs[blockIdx.y];
  if (!J.split) return;
  init_replies(reinterpret_cast<uint4*>(J.out), J.B, J.Wd / 4, J.seeds,
               blockIdx.x * (uint64_t)blockDim.x + threadIdx.x, (uint64_t)gridDim.x * blockDim.x);
}


uint32_t m4_next_slot() {
  static std::atomic<uint32_t> next{0};
  return next.fetch_add(1, std::memory_order_relaxed) % kM4CounterSlots;
}

template <int MR, int NJ>
cudaError_t m4_prepare() {
  static std::atomic<bool> ready{false};  // idempotent set-up: a race only repeats it
  if (ready.load(std::memory_order_acquire)) return cudaSuccess;
  // the setmaxnreg split (128 x 56 + 256 x 224) assumes 168 registers at launch
  cudaFuncAttributes fa{};
  cudaError_t e = cudaFuncGetAttributes(&fa, m4rm_scan_kernel<MR, NJ>);
  if (e != cudaSuccess) return e;
  if (fa.numRegs != kScanLaunchRegs) return cudaErrorInvalidConfiguration;
  e = cudaFuncSetAttribute(m4rm_scan_kernel<MR, NJ>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           M4Layout<MR>::kSmem);
  if (e != cudaSuccess) return e;
  ready.store(true, std::memory_order_release);
  return cudaSuccess;
}

template <int MR, int NJ>
cudaError_t m4_launch_all(M4Launch<NJ>& L, cudaStream_t st) {
  cudaError_t e = m4_prepare<MR, NJ>();
  if (e != cudaSuccess) return e;
  L.counter_slot = m4_next_slot();
  bool any = false;
  for (uint32_t i = 0; i < L.njobs; ++i) any |= L.jobs[i].split != 0;
  if (any || L.dynamic)
    e = launch_pdl(m4_zero_kernel<NJ>, dim3(any ? 64 : 1, L.njobs), dim3(256), 0, st, L);
  if (e != cudaSuccess) return e;
  const uint32_t grid = std::min<uint32_t>(L.total_items, device_sm_count());
  return launch_pdl(m4rm_scan_kernel<MR, NJ>, dim3(grid), dim3(kM4Threads), M4Layout<MR>::kSmem,
                   st, L, device_status_word());
}

// k-chunk of one job (multiple of 64 rows) minimising rounds x rows on the grid
uint32_t m4_plan_single(uint64_t n, uint64_t tiles, int grid) {
  const uint64_t max_kc = std::max<uint64_t>(1, (n + kSR - 1) / kSR);
  const uint64_t hi = std::min<uint64_t>(max_kc, static_cast<uint64_t>(grid) * 4 / tiles + 2);
  double best = 1e300;
  uint64_t best_rows = kSR;
  for (uint64_t nkc = 1; nkc <= hi; ++nkc) {
    uint64_t rows = (n + nkc - 1) / nkc;
    rows = (rows + kSR - 1) / kSR * kSR;
    const uint64_t items = tiles * ((n + rows - 1) / rows);
    const uint64_t rounds = (items + grid - 1) / grid;
    const double cost = static_cast<double>(rounds) * (static_cast<double>(rows) + 64.0) +
                        1e-6 * static_cast<double>(items);
    if (cost < best) {
      best = cost;
      best_rows = rows;
    }
  }
  return static_cast<uint32_t>(std::min<uint64_t>(best_rows, 0xFFFFFFC0ull));
}

M4Job m4_job(const uint32_t* T, uint64_t n, uint32_t Wd, const uint64_t* R, uint32_t words64,
             uint32_t B, uint32_t* out, const uint8_t* seeds, uint32_t bt) {
  M4Job j{};
  j.T = T;
  j.R = R;
  j.out = out;
  j.seeds = seeds;
  j.n = n;
  j.Wd = Wd;
  j.words64 = words64;
  j.B = B;
  j.n_bt = (B + bt - 1) / bt;
  j.n_wt = (Wd + kWT - 1) / kWT;
  return j;
}

}  // namespace

cudaError_t launch_m4rm(const uint32_t* T, uint64_t n, uint32_t Wd, const uint64_t* R,
                        uint32_t words64, uint32_t B, uint32_t* out, const uint8_t* seeds,
                        cudaStream_t st) {
  if (B == 0) return cudaSuccess;
  if (!device_status_word()) return cudaErrorInvalidSymbol;
  const bool wide = B > 256;
  M4Launch<1> L;
  L.njobs = 1;
  M4Job j = m4_job(T, n, Wd, R, words64, B, out, seeds, wide ? 512u : 256u);
  j.kc_rows = m4_plan_single(n, static_cast<uint64_t>(j.n_bt) * j.n_wt, device_sm_count());
  j.n_kc = static_cast<uint32_t>((n + j.kc_rows - 1) / j.kc_rows);
  j.split = (j.n_kc > 1 || seeds) ? 1u : 0u;  // masks: reduce onto the masked replies
  j.item_begin = 0;
  L.jobs[0] = j;
  L.total_items = j.n_bt * j.n_wt * j.n_kc;
  L.dynamic = 0;  // items of one job cost the same: static assignment, no counter
  return wide ? m4_launch_all<32, 1>(L, st) : m4_launch_all<16, 1>(L, st);
}

cudaError_t launch_m4rm_multi(const M4Request* reqs, uint32_t count, bool wide, cudaStream_t st) {
  if (count == 0) return cudaSuccess;
  if (count > kM4MaxJobs) return cudaErrorInvalidValue;
  if (!device_status_word()) return cudaErrorInvalidSymbol;
  const int grid = device_sm_count();
  // items of about equal cost: per 64-row chunk of one request x 64-word tile
  // the work is the same for every job, so chunks are sized on the total
  std::vector<M4Job> js;
  double total_rows = 0;
  for (uint32_t i = 0; i < count; ++i) {
    const M4Request& q = reqs[i];
    M4Job j = m4_job(q.T, q.n, q.Wd, q.R, q.words64, q.B, q.out, q.seeds, wide ? 512u : 256u);
    total_rows += static_cast<double>(j.n_bt) * j.n_wt * static_cast<double>(q.n);
    js.push_back(j);
  }
  uint64_t target = static_cast<uint64_t>(total_rows / (static_cast<double>(grid) * 8.0));
  target = std::max<uint64_t>(kSR, (target + kSR - 1) / kSR * kSR);
  std::vector<double> cost(js.size());
  for (size_t i = 0; i < js.size(); ++i) {
    M4Job& j = js[i];
    j.kc_rows = static_cast<uint32_t>(std::min<uint64_t>(target, (j.n + kSR - 1) / kSR * kSR));
    j.n_kc = static_cast<uint32_t>((j.n + j.kc_rows - 1) / j.kc_rows);
    j.split = (j.n_kc > 1 || j.seeds) ? 1u : 0u;
    cost[i] = static_cast<double>(std::min<uint64_t>(j.kc_rows, j.n));
  }
  std::vector<size_t> order(js.size());
  for (size_t i = 0; i < order.size(); ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](size_t a, size_t b) { return cost[a] > cost[b]; });
  M4Launch<kM4MaxJobs> L;
  L.njobs = 0;
  uint32_t items = 0;
  for (size_t oi : order) {
    M4Job j = js[oi];
    j.item_begin = items;
    items += j.n_bt * j.n_wt * j.n_kc;
    L.jobs[L.njobs++] = j;
  }
  L.total_items = items;
  L.dynamic = 1;
  return wide ? m4_launch_all<32, kM4MaxJobs>(L, st) : m4_launch_all<16, kM4MaxJobs>(L, st);
}

}  // namespace tpir
