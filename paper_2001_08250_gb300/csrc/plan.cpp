// Autotuner of the batched read's tile shape.
//
// For a table's row width and a batch size, every admissible tile shape of
// the batched kernel (lanes along the row LW, warps along requests / row /
// buckets, rows per pipeline stage) is timed on the table itself with CUDA
// events; the fastest is cached under (row width, batch-size class) and used
// by every later launch planned for that class -- single-table reads, the
// many-table launch and the serve loop.  The cache can be saved to and loaded
// from a small JSON file.
#include <cstdio>
#include <map>
#include <mutex>
#include <utility>
#include <vector>

#include "tpir_internal.h"

namespace tpir {
namespace {

std::mutex g_plan_mu;
std::map<std::pair<uint32_t, uint32_t>, Shape> g_plans;

uint32_t bclass(uint32_t B) {
  uint32_t c = 0;
  while ((1u << c) < B) ++c;
  return c;  // ceil(log2 B)
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
  }
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
                 ++i < g_plans.size() ? "," : "");
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
  tpir_status rc = TPIR_OK;
  while (std::fgets(line, sizeof line, f)) {
    unsigned wd, bc, lw, wb, ww, wk, sr;
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
  return rc;
}

}  // extern "C"
