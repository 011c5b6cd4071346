// Autotuner of the batched read.
//
// For a table's row width and a batch size, every admissible tile shape of
// the register-tiled kernel (lanes along the row LW, warps along requests /
// row / buckets, rows per pipeline stage) is timed on the table itself with
// CUDA events; the fastest is cached under (row width, batch-size class) and
// used by every later launch of that kernel.  Then the other kernels are
// timed on the same batch -- the tensor-core kernel under each schedule
// (spans, items of several k-chunk sizes), the Four-Russians kernel, the
// plain kernel -- and the fastest kernel with its schedule is cached under
// (row width, batch-size class, table-size class): the automatic choice of
// single-table reads, many-table launches and the serve loop follows it
// instead of the built-in batch thresholds.  Both caches can be saved to and
// loaded from a small JSON file.
#include <cstdio>
#include <iterator>
#include <map>
#include <mutex>
#include <tuple>
#include <utility>
#include <vector>

#include "tpir_internal.h"

namespace tpir {
namespace {

std::mutex g_plan_mu;
std::map<std::pair<uint32_t, uint32_t>, Shape> g_plans;
std::map<std::tuple<uint32_t, uint32_t, uint32_t>, KernelPlan> g_kplans;

uint32_t bclass(uint32_t B) {
  uint32_t c = 0;
  while ((1u << c) < B) ++c;
  return c;  // ceil(log2 B)
}
uint32_t nclass(uint64_t n) {
  uint32_t c = 0;
  while ((1ull << c) < n) ++c;
  return c;  // ceil(log2 n)
}

// All shapes the kernel accepts for this row width and batch size, without
// tiles that would mostly pad (B-tile over twice the batch, W-tile over twice
// the row).
std::vector<Shape> candidates(uint32_t Wd, uint32_t B) {
  std::vector<Shape> out;
  for (int lw = 2; lw <= 5; ++lw) {
    if (lw > 2 && (1u << lw) * kNW > Wd) continue;
    for (int wb = 1; wb <= 8; wb *= 2)
      for (int ww = 1; ww * wb <= 8; ww *= 2) {
        const int wk = 8 / (wb * ww);
        Shape s{};
        s.lw_log2 = static_cast<uint8_t>(lw);
        s.wb = static_cast<uint8_t>(wb);
        s.ww = static_cast<uint8_t>(ww);
        s.wk = static_cast<uint8_t>(wk);
        if (static_cast<uint32_t>(s.bt()) > 2 * std::max<uint32_t>(B, 8)) continue;
        if (static_cast<uint32_t>(s.wt()) > 2 * std::max<uint32_t>(Wd, 64)) continue;
        for (int sr = 5; sr >= 0; --sr) {
          s.srows_log2 = static_cast<uint8_t>(sr);
          if (scan_stage_bytes(s) <= kStageBytes && (1 << sr) >= wk) {
            out.push_back(s);
            break;
          }
        }
      }
  }
  return out;
}

}  // namespace

bool plan_lookup(uint32_t Wd, uint32_t B, Shape* out) {
  std::lock_guard<std::mutex> g(g_plan_mu);
  auto it = g_plans.find({Wd, bclass(B)});
  if (it == g_plans.end()) return false;
  *out = it->second;
  return true;
}

// The plan of the same row width and batch class whose table-size class is
// nearest (exact first; a tie takes the smaller tables' plan).
bool kernel_plan_lookup(uint32_t Wd, uint32_t B, uint64_t n, KernelPlan* out, bool* exact) {
  std::lock_guard<std::mutex> g(g_plan_mu);
  if (g_kplans.empty()) return false;
  const uint32_t bc = bclass(B), nc = nclass(n);
  auto hi = g_kplans.lower_bound(std::make_tuple(Wd, bc, nc));
  auto best = g_kplans.end();
  uint32_t dist = ~0u;
  if (hi != g_kplans.end() && std::get<0>(hi->first) == Wd && std::get<1>(hi->first) == bc) {
    best = hi;
    dist = std::get<2>(hi->first) - nc;
  }
  if (hi != g_kplans.begin()) {
    auto lo = std::prev(hi);
    if (std::get<0>(lo->first) == Wd && std::get<1>(lo->first) == bc &&
        nc - std::get<2>(lo->first) <= dist)
      best = lo;
  }
  if (best == g_kplans.end()) return false;
  *out = best->second;
  if (exact) *exact = std::get<2>(best->first) == nc;
  return true;
}

}  // namespace tpir

using namespace tpir;

extern "C" {

tpir_status tpir_autotune(tpir_db* db, uint32_t B, uint32_t reps, tpir_tune_result* out) {
  if (!db || B == 0 || B > (1u << 20) || !out) return TPIR_EINVAL;
  if (reps == 0) reps = 3;
  const uint64_t rb = static_cast<uint64_t>(B) * db->words64 * 8;
  const uint64_t ob = static_cast<uint64_t>(B) * db->row_bytes;
  uint64_t* d_req = nullptr;
  uint8_t* d_out = nullptr;
  cudaStream_t st = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaMalloc(reinterpret_cast<void**>(&d_req), rb);
  if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(&d_out), ob);
  // the kernels' work does not depend on the bits: any content times the same
  if (e == cudaSuccess) e = cudaMemset(d_req, 0x5A, rb);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  const std::vector<Shape> cand = candidates(db->Wd, B);
  const int grid = batched_grid();
  double best = 1e300;
  Shape best_s{};
  uint32_t tried = 0;
  if (e == cudaSuccess) order_after_writes(db, st);
  for (const Shape& s : cand) {
    if (e != cudaSuccess) break;
    ScanLaunch L;
    L.njobs = 1;
    ScanJob j = make_job(db, d_req, B, d_out);
    j.shape = s;
    plan_single(j, grid);
    j.item_begin = 0;
    if (!finalize_job(j)) continue;
    L.jobs[0] = j;
    L.total_items = j.n_bt * j.n_wt * j.n_kc;
    L.dynamic = 0;
    auto run = [&]() {
      L.counter_slot = next_counter_slot();
      cudaError_t x = launch_zero_outputs(L, st);
      if (x == cudaSuccess)
        x = launch_batched(L, static_cast<int>(std::min<uint64_t>(L.total_items, grid)), st);
      return x;
    };
    e = run();  // warm-up
    if (e == cudaSuccess) e = cudaEventRecord(e0, st);
    for (uint32_t r = 0; r < reps && e == cudaSuccess; ++r) e = run();
    if (e == cudaSuccess) e = cudaEventRecord(e1, st);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e != cudaSuccess) break;
    ++tried;
    const double us = 1e3 * ms / reps;
    if (us < best) {
      best = us;
      best_s = s;
    }
  }
  // the other kernels on the same batch: us per launch of each candidate
  auto time_it = [&](auto&& launch) -> double {
    if (e != cudaSuccess) return 0.0;
    e = launch();  // warm-up (and, for the tensor-core kernel, the transposed copy)
    if (e == cudaSuccess) e = cudaEventRecord(e0, st);
    for (uint32_t r = 0; r < reps && e == cudaSuccess; ++r) e = launch();
    if (e == cudaSuccess) e = cudaEventRecord(e1, st);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    return e == cudaSuccess ? 1e3 * ms / reps : 0.0;
  };
  KernelPlan best_k;
  best_k.kernel = 2;
  double best_k_us = best;
  double us_tensor = 0.0, us_m4rm = 0.0, us_plain = 0.0;
  uint32_t tensor_tried = 0;
  if (e == cudaSuccess && db->Wd >= 64) {
    std::vector<GSched> scheds;
    for (uint32_t loads : {0u, 1u}) {
      if (gf2_span_ok(db->n, db->Wd, B)) scheds.push_back(GSched{1, 0, loads});
      scheds.push_back(GSched{2, 0, loads});
      for (uint32_t kc : {4096u, 8192u, 16384u, 32768u})
        if (kc < (db->n + 255) / 256 * 256) scheds.push_back(GSched{2, kc, loads});
    }
    if (B > 128) {  // items on CTA pairs (mode 2 above) against items on single CTAs
      scheds.push_back(GSched{3, 0, 0});
      for (uint32_t kc : {4096u, 8192u, 16384u, 32768u})
        if (kc < (db->n + 255) / 256 * 256) scheds.push_back(GSched{3, kc, 0});
    }
    for (const GSched& sc : scheds) {
      const double us = time_it([&]() {
        cudaError_t x = tcopy_ensure(db, st);
        if (x == cudaSuccess)
          x = launch_gf2_mma(db->d_tt, db->n, db->Wd, d_req, db->words64, B,
                             reinterpret_cast<uint32_t*>(d_out), nullptr, st, &sc);
        return x;
      });
      if (e != cudaSuccess) break;
      ++tensor_tried;
      if (us_tensor == 0.0 || us < us_tensor) us_tensor = us;
      if (us < best_k_us) {
        best_k_us = us;
        best_k.kernel = 5;
        best_k.sched = sc;
      }
    }
  }
  if (e == cudaSuccess && db->Wd >= 64 && B >= 32) {
    us_m4rm = time_it([&]() {
      return launch_m4rm(reinterpret_cast<const uint32_t*>(db->d_table), db->n, db->Wd, d_req,
                         db->words64, B, reinterpret_cast<uint32_t*>(d_out), nullptr, st);
    });
    if (e == cudaSuccess && us_m4rm < best_k_us) {
      best_k_us = us_m4rm;
      best_k.kernel = 4;
      best_k.sched = GSched{};
    }
  }
  if (e == cudaSuccess && B <= 16) {
    us_plain = time_it([&]() {
      cudaError_t x = cudaSuccess;
      for (uint32_t b0 = 0; b0 < B && x == cudaSuccess; b0 += kPlainMaxB)
        x = launch_plain(reinterpret_cast<const uint32_t*>(db->d_table), db->n, db->Wd,
                         d_req + static_cast<uint64_t>(b0) * db->words64, db->words64,
                         std::min(kPlainMaxB, B - b0),
                         reinterpret_cast<uint32_t*>(d_out + static_cast<uint64_t>(b0) * db->row_bytes),
                         nullptr, st, 0);
      return x;
    });
    if (e == cudaSuccess && us_plain < best_k_us) {
      best_k_us = us_plain;
      best_k.kernel = 1;
      best_k.sched = GSched{};
    }
  }
  if (st) cudaStreamSynchronize(st);
  cudaFree(d_req);
  cudaFree(d_out);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (st) cudaStreamDestroy(st);
  if (e != cudaSuccess) return cuda_status(e);
  if (!tried) return TPIR_EINVAL;
  {
    std::lock_guard<std::mutex> g(g_plan_mu);
    g_plans[{db->Wd, bclass(B)}] = best_s;
    g_kplans[std::make_tuple(db->Wd, bclass(B), nclass(db->n))] = best_k;
  }
  out->kernel = static_cast<uint32_t>(best_k.kernel);
  out->tensor_mode = best_k.kernel == 5 ? best_k.sched.mode : 0u;
  out->tensor_kc_rows = best_k.kernel == 5 ? best_k.sched.kc_rows : 0u;
  out->tensor_loads = best_k.kernel == 5 ? best_k.sched.loads : 0u;
  out->tensor_candidates = tensor_tried;
  out->us_lop3 = best;
  out->us_tensor = us_tensor;
  out->us_m4rm = us_m4rm;
  out->us_plain = us_plain;
  out->lw_log2 = best_s.lw_log2;
  out->warps_b = best_s.wb;
  out->warps_w = best_s.ww;
  out->warps_k = best_s.wk;
  out->stage_rows = best_s.srows();
  out->tile_b = best_s.bt();
  out->tile_w = best_s.wt();
  out->candidates = tried;
  out->us_per_launch = best;
  out->lop3_tops = static_cast<double>(B) * db->n * db->Wd / (best * 1e-6) / 1e12;
  return TPIR_OK;
}

tpir_status tpir_tune_clear(void) {
  std::lock_guard<std::mutex> g(g_plan_mu);
  g_plans.clear();
  g_kplans.clear();
  return TPIR_OK;
}

tpir_status tpir_tune_save(const char* path) {
  if (!path) return TPIR_EINVAL;
  FILE* f = std::fopen(path, "w");
  if (!f) return TPIR_EINVAL;
  std::lock_guard<std::mutex> g(g_plan_mu);
  std::fprintf(f, "{\"plans\": [\n");
  size_t i = 0;
  for (const auto& kv : g_plans) {
    const Shape& s = kv.second;
    std::fprintf(f,
                 "{\"row_words\": %u, \"batch_class\": %u, \"lw_log2\": %u, \"warps_b\": %u, "
                 "\"warps_w\": %u, \"warps_k\": %u, \"stage_rows_log2\": %u}%s\n",
                 kv.first.first, kv.first.second, s.lw_log2, s.wb, s.ww, s.wk, s.srows_log2,
                 (++i < g_plans.size() || !g_kplans.empty()) ? "," : "");
  }
  size_t k = 0;
  for (const auto& kv : g_kplans) {
    const KernelPlan& p = kv.second;
    std::fprintf(f,
                 "{\"row_words\": %u, \"batch_class\": %u, \"n_class\": %u, \"kernel\": %d, "
                 "\"tensor_mode\": %u, \"tensor_kc_rows\": %u, \"tensor_loads\": %u}%s\n",
                 std::get<0>(kv.first), std::get<1>(kv.first), std::get<2>(kv.first), p.kernel,
                 p.sched.mode, p.sched.kc_rows, p.sched.loads, ++k < g_kplans.size() ? "," : "");
  }
  std::fprintf(f, "]}\n");
  std::fclose(f);
  return TPIR_OK;
}

tpir_status tpir_tune_load(const char* path) {
  if (!path) return TPIR_EINVAL;
  FILE* f = std::fopen(path, "r");
  if (!f) return TPIR_EINVAL;
  char line[512];
  std::map<std::pair<uint32_t, uint32_t>, Shape> plans;
  std::map<std::tuple<uint32_t, uint32_t, uint32_t>, KernelPlan> kplans;
  tpir_status rc = TPIR_OK;
  while (std::fgets(line, sizeof line, f)) {
    unsigned wd, bc, lw, wb, ww, wk, sr;
    unsigned nc, tm, kc, tl;
    int kern;
    if (std::sscanf(line,
                    " {\"row_words\": %u, \"batch_class\": %u, \"n_class\": %u, \"kernel\": %d, "
                    "\"tensor_mode\": %u, \"tensor_kc_rows\": %u, \"tensor_loads\": %u",
                    &wd, &bc, &nc, &kern, &tm, &kc, &tl) == 7) {
      // accept only choices the library can run
      if (!(kern == 1 || kern == 2 || kern == 4 || kern == 5) || tm > 3 || wd == 0 || (wd % 4) != 0 ||
          (kern >= 4 && wd < 64) || kc > 32768 || (kc % 256) != 0 || tl > 1) {
        rc = TPIR_EINVAL;
        continue;
      }
      KernelPlan p;
      p.kernel = kern;
      p.sched.mode = tm;
      p.sched.kc_rows = kc;
      p.sched.loads = tl;
      kplans[std::make_tuple(wd, bc, nc)] = p;
      continue;
    }
    if (std::sscanf(line,
                    " {\"row_words\": %u, \"batch_class\": %u, \"lw_log2\": %u, \"warps_b\": %u, "
                    "\"warps_w\": %u, \"warps_k\": %u, \"stage_rows_log2\": %u",
                    &wd, &bc, &lw, &wb, &ww, &wk, &sr) != 7)
      continue;
    Shape s{};
    s.lw_log2 = static_cast<uint8_t>(lw);
    s.wb = static_cast<uint8_t>(wb);
    s.ww = static_cast<uint8_t>(ww);
    s.wk = static_cast<uint8_t>(wk);
    s.srows_log2 = static_cast<uint8_t>(sr);
    // accept only shapes the kernel can run
    if (lw < 2 || lw > 5 || wb * ww * wk != static_cast<unsigned>(kConsumerWarps) || sr > 5 ||
        scan_stage_bytes(s) > kStageBytes || wd == 0 || (wd % 4) != 0) {
      rc = TPIR_EINVAL;
      continue;
    }
    plans[{wd, bc}] = s;
  }
  std::fclose(f);
  std::lock_guard<std::mutex> g(g_plan_mu);
  for (const auto& kv : plans) g_plans[kv.first] = kv.second;
  for (const auto& kv : kplans) g_kplans[kv.first] = kv.second;
  return rc;
}

}  // extern "C"
