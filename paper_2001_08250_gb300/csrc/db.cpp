// C ABI of libtalekpir: tables, PIR reads, cuckoo writes, interest vectors.
// Every step of a read or write runs in this library's kernels; the host code
// here validates arguments, plans launches, moves buffers and keeps the
// cuckoo metadata.
#include <algorithm>
#include <atomic>
#include <cstring>
#include <new>

#include "tpir_internal.h"

namespace {
thread_local tpir_status g_last = TPIR_OK;
}  // namespace

namespace tpir {

tpir_status set_error(tpir_status s) {
  g_last = s;
  return s;
}

tpir_status cuda_status(cudaError_t e) {
  if (e == cudaSuccess) return TPIR_OK;
  if (e == cudaErrorMemoryAllocation) return TPIR_ENOMEM;
  return TPIR_ECUDA;
}

uint64_t db_device_bytes(uint64_t n, uint32_t d, uint32_t z) {
  return n * static_cast<uint64_t>(d) * z;
}

bool grow_dev(void** p, uint64_t* cap, uint64_t need) {
  if (*cap >= need) return true;
  uint64_t c = std::max<uint64_t>(need, *cap * 2);
  if (*p) cudaFree(*p);
  *p = nullptr;
  *cap = 0;
  if (cudaMalloc(p, c) != cudaSuccess) {
    *p = nullptr;
    return false;
  }
  *cap = c;
  return true;
}

bool grow_pinned(void** p, uint64_t* cap, uint64_t need) {
  if (*cap >= need) return true;
  uint64_t c = std::max<uint64_t>(need, *cap * 2);
  if (*p) cudaFreeHost(*p);
  *p = nullptr;
  *cap = 0;
  if (cudaMallocHost(p, c) != cudaSuccess) {
    *p = nullptr;
    return false;
  }
  *cap = c;
  return true;
}

void order_after_writes(tpir_db* db, cudaStream_t st) {
  if (db->epoch > 0 || db->last_write) cudaStreamWaitEvent(st, db->last_write, 0);
}

void note_read(tpir_db* db, cudaStream_t st) {
  if (st == db->stream) return;  // same stream: ordered already
  for (auto& pr : db->read_events) {
    if (pr.first == st) {
      cudaEventRecord(pr.second, st);
      return;
    }
  }
  cudaEvent_t ev;
  if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) return;
  cudaEventRecord(ev, st);
  db->read_events.emplace_back(st, ev);
}

// Writes go on `st` after every read already submitted on other streams.
void order_writes_after_reads(tpir_db* db, cudaStream_t st) {
  for (auto& pr : db->read_events)
    if (pr.first != st) cudaStreamWaitEvent(st, pr.second, 0);
}

// ---- launch planning -------------------------------------------------------

// Per-row cost of one item of a job, in SM clocks: the larger of its LOP3
// work (64 per SM per clock) and its table bytes (HBM share per SM).
static double row_cost(const ScanJob& j) {
  const Shape& s = j.shape;
  const double alu = static_cast<double>(s.bt()) * s.wt() / 64.0;
  const double mem = static_cast<double>(std::min<uint32_t>(s.wt(), j.Wd)) * 4.0 / 24.0;
  return std::max(alu, mem) + 8.0;
}

// Chooses kc_rows for one job so that items fill `grid` CTAs with the least
// makespan (rounds of items x rows per item).
void plan_single(ScanJob& j, int grid) {
  const uint32_t sr = j.shape.srows();
  const uint64_t tiles = static_cast<uint64_t>((j.B + j.shape.bt() - 1) / j.shape.bt()) *
                         ((j.Wd + j.shape.wt() - 1) / j.shape.wt());
  const uint64_t max_kc = std::max<uint64_t>(1, (j.n + sr - 1) / sr);
  const uint64_t hi = std::min<uint64_t>(max_kc, static_cast<uint64_t>(grid) * 4 / std::max<uint64_t>(1, tiles) + 2);
  double best = 1e300;
  uint32_t best_rows = 0;
  for (uint64_t nkc = 1; nkc <= hi; ++nkc) {
    uint64_t rows = (j.n + nkc - 1) / nkc;
    rows = (rows + sr - 1) / sr * sr;
    const uint64_t items = tiles * ((j.n + rows - 1) / rows);
    const uint64_t rounds = (items + grid - 1) / grid;
    const double cost = static_cast<double>(rounds) * (static_cast<double>(rows) + 32.0) +
                        1e-6 * static_cast<double>(items);
    if (cost < best) {
      best = cost;
      best_rows = static_cast<uint32_t>(std::min<uint64_t>(rows, 0xFFFFFFF0ull));
    }
  }
  j.kc_rows = best_rows;
}

ScanJob make_job(const tpir_db* db, const uint64_t* d_req, uint32_t B, void* d_out) {
  ScanJob j{};
  j.T = reinterpret_cast<const uint32_t*>(db->d_table);
  j.R = d_req;
  j.out = reinterpret_cast<uint32_t*>(d_out);
  j.n = db->n;
  j.Wd = db->Wd;
  j.words64 = db->words64;
  j.B = B;
  if (!plan_lookup(db->Wd, B, &j.shape)) j.shape = choose_shape(db->Wd, B);
  return j;
}

int batched_grid() { return device_sm_count() * batched_ctas_per_sm(); }

uint32_t next_counter_slot() {
  static std::atomic<uint32_t> next{0};
  return next.fetch_add(1, std::memory_order_relaxed) % kItemCounterSlots;
}

int auto_kernel(const tpir_db* db, uint32_t B) {
  if (db->forced_kernel) return db->forced_kernel;
  KernelPlan kp;
  if (kernel_plan_lookup(db->Wd, B, db->n, &kp)) return kp.kernel;  // measured winner
  // plain stream for a few requests; the tensor-core kernel once its
  // 128-request M-tiles are well filled (measured crossover with the
  // register-tiled kernel on GB300); the register-tiled kernel in between
  if (B <= kPlainMaxB) return 1;
  if (B >= kTensorMinB && db->Wd >= 64) return 5;
  return 2;
}

tpir_status enqueue_read(tpir_db* db, const uint64_t* d_req, uint32_t B, void* d_out,
                         cudaStream_t st, const uint8_t* d_seeds, int* kernel_used,
                         int kernel_choice) {
  if (B == 0) return TPIR_OK;
  d_req += db->req_off;  // a row shard reads its own words of each request row
  order_after_writes(db, st);
  const int kernel = kernel_choice ? kernel_choice : auto_kernel(db, B);
  if (kernel_used) *kernel_used = kernel;
  cudaError_t e = cudaSuccess;
  if (kernel == 1 || kernel == 3) {
    const uint32_t* T = reinterpret_cast<const uint32_t*>(db->d_table);
    for (uint32_t b0 = 0; b0 < B && e == cudaSuccess; b0 += kPlainMaxB) {
      const uint32_t nb = std::min(kPlainMaxB, B - b0);
      e = launch_plain(T, db->n, db->Wd, d_req + static_cast<uint64_t>(b0) * db->words64,
                       db->words64, nb,
                       reinterpret_cast<uint32_t*>(static_cast<uint8_t*>(d_out) +
                                                   static_cast<uint64_t>(b0) * db->row_bytes),
                       d_seeds ? d_seeds + static_cast<uint64_t>(b0) * 32 : nullptr, st,
                       kernel == 3 ? -1 : 0);
    }
  } else if (kernel == 5) {
    KernelPlan kp;
    bool exact = false;
    const bool planned = kernel_plan_lookup(db->Wd, B, db->n, &kp, &exact) && kp.kernel == 5 && exact;
    e = tcopy_ensure(db, st);
    if (e == cudaSuccess)
      e = launch_gf2_mma(db->d_tt, db->n, db->Wd, d_req, db->words64, B,
                         reinterpret_cast<uint32_t*>(d_out), d_seeds, st,
                         planned ? &kp.sched : nullptr);
  } else if (kernel == 4) {
    e = launch_m4rm(reinterpret_cast<const uint32_t*>(db->d_table), db->n, db->Wd, d_req,
                    db->words64, B, reinterpret_cast<uint32_t*>(d_out), d_seeds, st);
  } else {
    ScanLaunch L;
    L.njobs = 1;
    ScanJob j = make_job(db, d_req, B, d_out);
    j.seeds = d_seeds;
    const int grid = batched_grid();
    plan_single(j, grid);
    j.item_begin = 0;
    if (!finalize_job(j)) return TPIR_EINVAL;
    L.jobs[0] = j;
    L.total_items = j.n_bt * j.n_wt * j.n_kc;
    L.counter_slot = next_counter_slot();
    L.dynamic = 0;
    e = launch_zero_outputs(L, st);
    if (e == cudaSuccess)
      e = launch_batched(L, static_cast<int>(std::min<uint64_t>(L.total_items, grid)), st);
  }
  if (e != cudaSuccess) return cuda_status(e);
  note_read(db, st);
  return TPIR_OK;
}

tpir_status apply_writes_core(tpir_db* db, uint32_t count, const uint64_t* b1, const uint64_t* b2,
                              const uint8_t* msgs, tpir_status* st_out, uint32_t* ev_out,
                              cudaStream_t st, tpir_write_staging& stg) {
  if (count == 0) return TPIR_OK;
  std::vector<MoveOp> ops;
  ops.reserve(count * 2);
  const uint64_t z = db->z;
  // every successful insert is recorded so that the whole call can be taken
  // back if its device work cannot be enqueued: then nothing has changed,
  // not even the random draws of eviction walks that failed with EFULL
  std::vector<CuckooMeta::Undo> undos;
  undos.reserve(count);
  std::vector<tpir_status> sts(count);
  std::vector<uint32_t> evs(count);
  const uint64_t rng0 = db->meta->rng_state();
  uint32_t ok = 0;
  for (uint32_t i = 0; i < count; ++i) {
    CuckooMeta::Undo u;
    sts[i] = db->meta->insert(b1[i], b2[i], i, ops, &evs[i], &u);
    if (sts[i] == TPIR_OK) {
      ++ok;
      undos.push_back(std::move(u));
    }
  }
  auto take_back = [&]() {
    for (auto it = undos.rbegin(); it != undos.rend(); ++it) db->meta->rollback(*it);
    db->meta->set_rng_state(rng0);
  };
  if (!ops.empty()) {
    const uint64_t pay_bytes = count * z;
    cudaError_t e = cudaSuccess;
    if (ops.size() <= ParamMovesS::kOps && pay_bytes <= ParamMovesS::kBytes) {
      // a single write of a slot up to 4 KiB: moves and message by value in a
      // small parameter block, one launch, no staging to wait for
      thread_local ParamMovesS m;
      m.nops = static_cast<uint32_t>(ops.size());
      m.pad = 0;
      std::memcpy(m.ops, ops.data(), ops.size() * sizeof(MoveOp));
      std::memcpy(m.payload, msgs, pay_bytes);
      e = launch_apply_moves_param(db->d_table, db->z, m, db->d_tmp, st);
      if (e == cudaSuccess) e = tcopy_after_moves(db, ops.data(), ops.size(), st);
    } else if (ops.size() <= kParamOps && pay_bytes <= kParamBytes) {
      // small batch: the same with the larger parameter block
      thread_local ParamMoves m;
      m.nops = static_cast<uint32_t>(ops.size());
      m.pad = 0;
      std::memcpy(m.ops, ops.data(), ops.size() * sizeof(MoveOp));
      std::memcpy(m.payload, msgs, pay_bytes);
      e = launch_apply_moves_param(db->d_table, db->z, m, db->d_tmp, st);
      if (e == cudaSuccess) e = tcopy_after_moves(db, ops.data(), ops.size(), st);
    } else {
      const uint64_t ops_bytes = ops.size() * sizeof(MoveOp);
      if (!grow_pinned(reinterpret_cast<void**>(&stg.h), &stg.h_cap, pay_bytes + ops_bytes) ||
          !grow_dev(reinterpret_cast<void**>(&stg.d_payload), &stg.pay_cap, pay_bytes) ||
          !grow_dev(reinterpret_cast<void**>(&stg.d_ops), &stg.ops_cap, ops_bytes) ||
          (!stg.done && cudaEventCreateWithFlags(&stg.done, cudaEventDisableTiming) != cudaSuccess)) {
        take_back();
        return TPIR_ENOMEM;
      }
      std::memcpy(stg.h, msgs, pay_bytes);
      std::memcpy(stg.h + pay_bytes, ops.data(), ops_bytes);
      e = cudaMemcpyAsync(stg.d_payload, stg.h, pay_bytes, cudaMemcpyHostToDevice, st);
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(stg.d_ops, stg.h + pay_bytes, ops_bytes, cudaMemcpyHostToDevice, st);
      if (e == cudaSuccess)
        e = launch_apply_moves(db->d_table, db->z, stg.d_ops, static_cast<uint32_t>(ops.size()),
                               stg.d_payload, db->d_tmp, st);
      if (e == cudaSuccess) e = cudaEventRecord(stg.done, st);
      if (e == cudaSuccess) e = tcopy_after_moves(db, ops.data(), ops.size(), st);
    }
    if (e == cudaSuccess) e = cudaEventRecord(db->last_write, st);
    if (e != cudaSuccess) {
      take_back();
      return cuda_status(e);
    }
  }
  if (st_out) std::copy(sts.begin(), sts.end(), st_out);
  if (ev_out) std::copy(evs.begin(), evs.end(), ev_out);
  db->epoch += ok;
  return TPIR_OK;
}

// Positions of `count` writes (k each) into the current delta, opening new
// deltas (in place of the oldest) whenever the current one is complete.
tpir_status bloom_insert_core(tpir_db* db, const uint64_t* pos, uint32_t count, cudaStream_t st,
                              tpir_write_staging& stg) {
  tpir_bloom_state& bl = db->bloom;
  if (!bl.d_deltas) return TPIR_EINVAL;
  for (uint64_t i = 0; i < static_cast<uint64_t>(count) * bl.k; ++i)
    if (pos[i] >= bl.m) return TPIR_EINVAL;
  const uint64_t bytes = static_cast<uint64_t>(count) * bl.k * 8;
  if (!grow_pinned(reinterpret_cast<void**>(&stg.h), &stg.h_cap, bytes) ||
      !grow_dev(reinterpret_cast<void**>(&stg.d_pos), &stg.pos_cap, bytes) ||
      (!stg.done && cudaEventCreateWithFlags(&stg.done, cudaEventDisableTiming) != cudaSuccess))
    return TPIR_ENOMEM;
  std::memcpy(stg.h, pos, bytes);
  cudaError_t e = cudaMemcpyAsync(stg.d_pos, stg.h, bytes, cudaMemcpyHostToDevice, st);
  uint32_t i = 0;
  while (e == cudaSuccess && i < count) {
    if (bl.per_delta && bl.count == bl.per_delta) {
      bl.cur = (bl.cur + 1) % bl.window;
      bl.count = 0;
      e = cudaMemsetAsync(bl.d_deltas + static_cast<uint64_t>(bl.cur) * bl.words, 0,
                          bl.words * 8, st);
      if (e != cudaSuccess) break;
    }
    uint32_t seg = count - i;
    if (bl.per_delta) seg = std::min(seg, bl.per_delta - bl.count);
    e = launch_bloom_set(bl.d_deltas + static_cast<uint64_t>(bl.cur) * bl.words,
                         stg.d_pos + static_cast<uint64_t>(i) * bl.k,
                         static_cast<uint64_t>(seg) * bl.k, st);
    bl.count += seg;
    i += seg;
  }
  if (e == cudaSuccess) e = cudaEventRecord(stg.done, st);
  if (e == cudaSuccess) e = cudaEventRecord(db->last_write, st);
  return cuda_status(e);
}

// The kernel a job of a many-table launch takes: 4 Four-Russians (forced),
// 5 tensor-core (forced, or 48 or more requests on rows of 256 bytes or
// more), else 2 register-tiled.
int multi_kernel(const tpir_read_job& q) {
  const int forced = q.db->forced_kernel;
  if (forced == 4 && q.db->Wd >= 64) return 4;
  if (forced == 5) return 5;
  if (forced == 0) {
    KernelPlan kp;
    if (kernel_plan_lookup(q.db->Wd, q.B, q.db->n, &kp)) {
      if (kp.kernel == 5 || (kp.kernel == 4 && q.db->Wd >= 64)) return kp.kernel;
      return 2;  // the plain kernel's jobs run in the register-tiled launch
    }
    if (q.B >= kTensorMinB && q.db->Wd >= 64) return 5;
  }
  return 2;
}

tpir_status enqueue_multi(const tpir_read_job* jobs, uint32_t njobs, cudaStream_t st) {
  // large batches on rows of >= 256 bytes: one launch of the tensor-core
  // kernel (a db forced to the Four-Russians kernel: its launches, 512-request
  // tiles above 256 requests, else 256); the rest, and dbs forced to it: one
  // persistent launch of the register-tiled kernel
  std::vector<M4Request> tc, m4, m4w;
  std::vector<tpir_read_job> lop3;
  for (uint32_t i = 0; i < njobs; ++i) {
    const tpir_read_job& q = jobs[i];
    if (!q.db || (q.B && (!q.d_req_bits || !q.d_out))) return TPIR_EINVAL;
    if (q.B == 0) continue;
    if ((reinterpret_cast<uintptr_t>(q.d_out) & 15) || (reinterpret_cast<uintptr_t>(q.d_req_bits) & 7) ||
        (reinterpret_cast<uintptr_t>(q.d_seeds) & 15))
      return TPIR_EINVAL;
    const M4Request r{reinterpret_cast<const uint32_t*>(q.db->d_table), q.db->n, q.db->Wd,
                      q.d_req_bits + q.db->req_off, q.db->words64, q.B,
                      reinterpret_cast<uint32_t*>(q.d_out),
                      static_cast<const uint8_t*>(q.d_seeds)};
    const int kind = multi_kernel(q);
    if (kind == 4) {
      (q.B > 256 ? m4w : m4).push_back(r);
    } else if (kind == 5) {
      const cudaError_t e = tcopy_ensure(q.db, st);
      if (e != cudaSuccess) return cuda_status(e);
      M4Request t = r;
      t.Tt = q.db->d_tt;
      KernelPlan kp;
      bool exact = false;
      if (kernel_plan_lookup(q.db->Wd, q.B, q.db->n, &kp, &exact) && kp.kernel == 5 && exact) {
        if (kp.sched.mode == 2) t.kc_rows = kp.sched.kc_rows;
        t.loads = kp.sched.loads;
      }
      tc.push_back(t);
    } else {
      lop3.push_back(q);
    }
  }
  tpir_status s = enqueue_multi_lop3(lop3.data(), static_cast<uint32_t>(lop3.size()), st);
  if (s == TPIR_OK && !tc.empty())
    s = cuda_status(launch_gf2_mma_multi(tc.data(), static_cast<uint32_t>(tc.size()), st));
  if (s == TPIR_OK && !m4w.empty())
    s = cuda_status(launch_m4rm_multi(m4w.data(), static_cast<uint32_t>(m4w.size()), true, st));
  if (s == TPIR_OK && !m4.empty())
    s = cuda_status(launch_m4rm_multi(m4.data(), static_cast<uint32_t>(m4.size()), false, st));
  return s;
}

tpir_status enqueue_multi_lop3(const tpir_read_job* jobs, uint32_t njobs, cudaStream_t st) {
  if (njobs == 0) return TPIR_OK;
  ScanLaunch L;
  L.njobs = 0;
  const int grid = batched_grid();
  // shapes first, then k-chunks sized so that items cost about the same
  std::vector<ScanJob> js;
  double total = 0.0;
  for (uint32_t i = 0; i < njobs; ++i) {
    const tpir_read_job& q = jobs[i];
    if (!q.db || (q.B && (!q.d_req_bits || !q.d_out))) return TPIR_EINVAL;
    if (q.B == 0) continue;
    if ((reinterpret_cast<uintptr_t>(q.d_out) & 15) || (reinterpret_cast<uintptr_t>(q.d_req_bits) & 7) ||
        (reinterpret_cast<uintptr_t>(q.d_seeds) & 15))
      return TPIR_EINVAL;
    ScanJob j = make_job(q.db, q.d_req_bits + q.db->req_off, q.B, q.d_out);
    j.seeds = static_cast<const uint8_t*>(q.d_seeds);
    const double tiles = static_cast<double>((j.B + j.shape.bt() - 1) / j.shape.bt()) *
                         ((j.Wd + j.shape.wt() - 1) / j.shape.wt());
    total += tiles * static_cast<double>(j.n) * row_cost(j);
    js.push_back(j);
  }
  if (js.empty()) return TPIR_OK;
  // ~8 items per CTA of about equal cost; jobs listed by descending item cost,
  // the order in which the kernel's CTAs claim them
  const double target = total / (static_cast<double>(grid) * 8.0);
  std::vector<double> item_cost(js.size());
  for (size_t i = 0; i < js.size(); ++i) {
    ScanJob& j = js[i];
    const uint32_t sr = j.shape.srows();
    const double rc = row_cost(j);
    uint64_t rows = static_cast<uint64_t>(target / rc);
    rows = std::max<uint64_t>(sr, (rows + sr - 1) / sr * sr);
    const uint64_t nmax = (j.n + sr - 1) / sr * sr;
    j.kc_rows = static_cast<uint32_t>(std::min<uint64_t>(rows, std::min<uint64_t>(nmax, 0xFFFFFFF0ull)));
    if (!finalize_job(j)) return TPIR_EINVAL;
    item_cost[i] = static_cast<double>(std::min<uint64_t>(j.kc_rows, j.n)) * rc;
  }
  std::vector<size_t> order(js.size());
  for (size_t i = 0; i < order.size(); ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(),
                   [&](size_t a, size_t b) { return item_cost[a] > item_cost[b]; });
  uint32_t items = 0;
  for (size_t oi : order) {
    ScanJob j = js[oi];
    j.item_begin = items;
    items += j.n_bt * j.n_wt * j.n_kc;
    L.jobs[L.njobs++] = j;
  }
  L.total_items = items;
  L.counter_slot = next_counter_slot();
  L.dynamic = 1;
  cudaError_t e = launch_zero_outputs(L, st);
  if (e == cudaSuccess) e = launch_batched(L, static_cast<int>(std::min<uint32_t>(items, grid)), st);
  return cuda_status(e);
}

void tpir_write_staging_release(tpir_write_staging& s) {
  if (s.h) cudaFreeHost(s.h);
  cudaFree(s.d_payload);
  cudaFree(s.d_ops);
  cudaFree(s.d_pos);
  if (s.done) cudaEventDestroy(s.done);
  s = tpir_write_staging();
}

}  // namespace tpir

using namespace tpir;

void tpir_write_staging::release() { tpir::tpir_write_staging_release(*this); }

// ============================================================================
// C ABI
// ============================================================================
extern "C" {

const char* tpir_version(void) { return "libtalekpir 0.1 (sm_103a)"; }

tpir_status tpir_last_error(void) { return g_last; }

const char* tpir_strerror(tpir_status s) {
  switch (s) {
    case TPIR_OK: return "ok";
    case TPIR_EINVAL: return "invalid argument";
    case TPIR_ENOMEM: return "out of device memory or HBM budget";
    case TPIR_EFULL: return "cuckoo table full: eviction bound hit";
    case TPIR_EAGAIN: return "queue full, try again";
    case TPIR_ETIMEDOUT: return "bounded device wait timed out";
    case TPIR_ECUDA: return "CUDA runtime error";
    case TPIR_ESHUTDOWN: return "server shut down";
  }
  return "unknown status";
}

tpir_db* tpir_db_create(uint64_t n, uint32_t d, uint32_t msg_bytes) {
  if (n == 0 || d == 0 || d > 64 || msg_bytes == 0 || (msg_bytes % 16) != 0 ||
      static_cast<uint64_t>(d) * msg_bytes > (1ull << 30) || n > (1ull << 40)) {
    set_error(TPIR_EINVAL);
    return nullptr;
  }
  tpir_db* db = new (std::nothrow) tpir_db();
  if (!db) {
    set_error(TPIR_ENOMEM);
    return nullptr;
  }
  db->n = n;
  db->d = d;
  db->z = msg_bytes;
  db->row_bytes = d * msg_bytes;
  db->Wd = db->row_bytes / 4;
  db->words64 = static_cast<uint32_t>((n + 63) / 64);
  cudaGetDevice(&db->device);
  cudaError_t e = cudaMalloc(reinterpret_cast<void**>(&db->d_table), n * db->row_bytes);
  if (e == cudaSuccess) e = cudaMemset(db->d_table, 0, n * db->row_bytes);
  if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(&db->d_tmp), msg_bytes);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&db->stream, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&db->last_write, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&db->stream_mark, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventRecord(db->last_write, db->stream);
  if (e != cudaSuccess) {
    set_error(cuda_status(e));
    tpir_db_destroy(db);
    return nullptr;
  }
  db->meta = new (std::nothrow) CuckooMeta(n, d);
  if (!db->meta) {
    set_error(TPIR_ENOMEM);
    tpir_db_destroy(db);
    return nullptr;
  }
  db->meta->set_policy(0, 500, 0);
  return db;
}

tpir_db* tpir_db_create_shard(uint64_t n_total, uint64_t row_begin, uint64_t rows, uint32_t d,
                              uint32_t msg_bytes) {
  if (n_total == 0 || rows == 0 || (row_begin % 64) != 0 || row_begin >= n_total ||
      rows > n_total - row_begin || (n_total + 63) / 64 > 0xFFFFFFFFull) {
    set_error(TPIR_EINVAL);
    return nullptr;
  }
  tpir_db* db = tpir_db_create(rows, d, msg_bytes);
  if (!db) return nullptr;
  db->n_total = n_total;
  db->row_begin = row_begin;
  db->words64 = static_cast<uint32_t>((n_total + 63) / 64);
  db->req_off = static_cast<uint32_t>(row_begin / 64);
  return db;
}

tpir_status tpir_db_shard_info(const tpir_db* db, uint64_t* n_total, uint64_t* row_begin) {
  if (!db) return TPIR_EINVAL;
  if (n_total) *n_total = db->n_total ? db->n_total : db->n;
  if (row_begin) *row_begin = db->row_begin;
  return TPIR_OK;
}

tpir_status tpir_shard_plan(uint64_t n_total, uint32_t parts, uint32_t index, uint64_t* row_begin,
                            uint64_t* rows) {
  if (n_total == 0 || parts == 0 || index >= parts || !row_begin || !rows) return TPIR_EINVAL;
  // whole 64-bucket request words, split as evenly as possible
  const uint64_t words = (n_total + 63) / 64;
  const uint64_t w0 = words * index / parts, w1 = words * (index + 1) / parts;
  *row_begin = std::min(n_total, w0 * 64);
  *rows = std::min(n_total, w1 * 64) - *row_begin;
  return TPIR_OK;
}

void tpir_db_destroy(tpir_db* db) {
  if (!db) return;
  if (db->stream) cudaStreamSynchronize(db->stream);
  for (auto& pr : db->read_events) {
    cudaEventSynchronize(pr.second);
    cudaEventDestroy(pr.second);
  }
  cudaFree(db->d_table);
  db->stage.release();
  cudaFree(db->d_tmp);
  cudaFree(db->d_tt);
  cudaFree(db->d_req);
  cudaFree(db->d_out);
  cudaFree(db->bloom.d_deltas);
  cudaFree(db->bloom.d_out);
  cudaFree(db->bloom.d_rice);
  cudaFree(db->bloom.d_rice_res);
  cudaFree(db->bloom.d_rice_scratch);
  if (db->copy_stream) cudaStreamSynchronize(db->copy_stream);
  cudaFree(db->d_pipe);
  for (cudaEvent_t ev : db->pipe_ev)
    if (ev) cudaEventDestroy(ev);
  if (db->copy_stream) cudaStreamDestroy(db->copy_stream);
  if (db->last_write) cudaEventDestroy(db->last_write);
  if (db->stream_mark) cudaEventDestroy(db->stream_mark);
  if (db->stream) cudaStreamDestroy(db->stream);
  delete db->meta;
  delete db;
}

tpir_status tpir_db_info(const tpir_db* db, uint64_t* n, uint32_t* d, uint32_t* msg_bytes,
                         const void** d_table, uint64_t* epoch) {
  if (!db) return TPIR_EINVAL;
  if (n) *n = db->n;
  if (d) *d = db->d;
  if (msg_bytes) *msg_bytes = db->z;
  if (d_table) *d_table = db->d_table;
  if (epoch) *epoch = db->epoch;
  return TPIR_OK;
}

tpir_status tpir_db_sync(tpir_db* db) {
  if (!db) return TPIR_EINVAL;
  cudaError_t e = cudaEventSynchronize(db->last_write);
  for (auto& pr : db->read_events)
    if (e == cudaSuccess) e = cudaEventSynchronize(pr.second);
  if (e == cudaSuccess) e = cudaStreamSynchronize(db->stream);
  return cuda_status(e);
}

tpir_status tpir_db_set_policy(tpir_db* db, uint64_t capacity, uint32_t max_evictions,
                               uint64_t s_cuckoo) {
  if (!db) return TPIR_EINVAL;
  if (db->meta->live() != 0) return TPIR_EINVAL;
  db->meta->set_policy(capacity, max_evictions, s_cuckoo);
  return TPIR_OK;
}

tpir_status tpir_db_set_kernel(tpir_db* db, int kernel) {
  if (!db || kernel < 0 || kernel > 5) return TPIR_EINVAL;
  db->forced_kernel = kernel;
  return TPIR_OK;
}

tpir_status tpir_db_load(tpir_db* db, const void* host_table, size_t bytes) {
  if (!db || !host_table || bytes != db->n * db->row_bytes) return TPIR_EINVAL;
  cudaError_t e = cudaEventSynchronize(db->last_write);
  if (e != cudaSuccess) return cuda_status(e);
  order_writes_after_reads(db, db->stream);
  e = cudaMemcpyAsync(db->d_table, host_table, bytes, cudaMemcpyHostToDevice, db->stream);
  if (e == cudaSuccess) e = tcopy_after_load(db, db->stream);
  if (e == cudaSuccess) e = cudaEventRecord(db->last_write, db->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(db->stream);
  if (e != cudaSuccess) return cuda_status(e);
  db->meta->clear();
  return TPIR_OK;
}

tpir_status tpir_db_load_async(tpir_db* db, const void* src, size_t bytes, void* stream) {
  if (!db || !src || bytes != db->n * db->row_bytes) return TPIR_EINVAL;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  order_writes_after_reads(db, st);
  cudaError_t e = cudaEventRecord(db->stream_mark, db->stream);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(st, db->stream_mark, 0);
  if (e == cudaSuccess) e = cudaMemcpyAsync(db->d_table, src, bytes, cudaMemcpyDefault, st);
  if (e == cudaSuccess) e = tcopy_after_load(db, st);
  if (e == cudaSuccess) e = cudaEventRecord(db->last_write, st);
  if (e != cudaSuccess) return cuda_status(e);
  db->meta->clear();
  return TPIR_OK;
}

tpir_status tpir_db_dump(tpir_db* db, void* host_table, size_t bytes) {
  if (!db || !host_table || bytes != db->n * db->row_bytes) return TPIR_EINVAL;
  order_writes_after_reads(db, db->stream);
  cudaError_t e =
      cudaMemcpyAsync(host_table, db->d_table, bytes, cudaMemcpyDeviceToHost, db->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(db->stream);
  return cuda_status(e);
}

tpir_status tpir_write(tpir_db* db, uint64_t b1, uint64_t b2, const void* msg,
                       uint32_t* evictions_out) {
  if (evictions_out) *evictions_out = 0;
  if (!db || !msg) return TPIR_EINVAL;
  tpir_status s = TPIR_OK;
  uint32_t ev = 0;
  tpir_status r = tpir_write_batch(db, 1, &b1, &b2, msg, &s, &ev);
  if (evictions_out) *evictions_out = ev;
  return r != TPIR_OK ? r : s;
}

tpir_status tpir_write_batch(tpir_db* db, uint32_t count, const uint64_t* b1, const uint64_t* b2,
                             const void* msgs, tpir_status* status_out, uint32_t* evictions_out) {
  if (!db || (count && (!b1 || !b2 || !msgs))) return TPIR_EINVAL;
  if (db->n_total) return TPIR_EINVAL;  // shards hold snapshots: no cuckoo writes
  if (count == 0) return TPIR_OK;
  // the staging of the previous call that used it must have been consumed
  // (small batches pass their moves in the kernel parameters and use none)
  if (db->stage.done) {
    cudaError_t e = cudaEventSynchronize(db->stage.done);
    if (e != cudaSuccess) return cuda_status(e);
  }
  order_writes_after_reads(db, db->stream);
  return apply_writes_core(db, count, b1, b2, static_cast<const uint8_t*>(msgs), status_out,
                           evictions_out, db->stream, db->stage);
}

// Synchronous read through the db's own staging; seeds (host, B x 32 bytes)
// masks the replies, null = plain.
static tpir_status read_batch_sync(tpir_db* db, const uint64_t* req_bits, uint32_t B,
                                   const uint8_t* seeds, void* out) {
  if (!db) return TPIR_EINVAL;
  if (B == 0) return TPIR_OK;
  if (!req_bits || !out) return TPIR_EINVAL;
  const uint64_t rb = static_cast<uint64_t>(B) * db->words64 * 8;
  const uint64_t ob = static_cast<uint64_t>(B) * db->row_bytes;
  // the seeds follow the request rows in the same staging buffer, 16-byte aligned
  const uint64_t ra = (rb + 15) / 16 * 16;
  const uint64_t sb = seeds ? static_cast<uint64_t>(B) * 32 : 0;
  if (!grow_dev(reinterpret_cast<void**>(&db->d_req), &db->req_cap, ra + sb) ||
      !grow_dev(reinterpret_cast<void**>(&db->d_out), &db->out_cap, ob))
    return TPIR_ENOMEM;
  uint8_t* d_seeds = seeds ? reinterpret_cast<uint8_t*>(db->d_req) + ra : nullptr;
  cudaError_t e = cudaMemcpyAsync(db->d_req, req_bits, rb, cudaMemcpyHostToDevice, db->stream);
  if (e == cudaSuccess && seeds)
    e = cudaMemcpyAsync(d_seeds, seeds, sb, cudaMemcpyHostToDevice, db->stream);
  if (e != cudaSuccess) return cuda_status(e);
  tpir_status s = enqueue_read(db, db->d_req, B, db->d_out, db->stream, d_seeds);
  if (s != TPIR_OK) return s;
  e = cudaMemcpyAsync(out, db->d_out, ob, cudaMemcpyDeviceToHost, db->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(db->stream);
  if (e != cudaSuccess) return cuda_status(e);
  int st = 0;
  if (read_device_status_and_clear(&st) != 0) return TPIR_ECUDA;
  return st ? static_cast<tpir_status>(st) : TPIR_OK;
}

tpir_status tpir_read_batch_pipelined(tpir_db* db, const uint64_t* req_bits, uint64_t B_total,
                                      uint32_t batch, void* out) {
  if (!db) return TPIR_EINVAL;
  if (B_total == 0) return TPIR_OK;
  if (!req_bits || !out || batch == 0) return TPIR_EINVAL;
  // Three device slots rotate, each holding a group of kGroup batches: the
  // group's request rows are copied in two groups ahead of its scans and its
  // replies copied out after them, on a copy stream.  The scans of a group
  // follow one another with no stream operation between them, so each one's
  // ramp-up overlaps the previous one's tail (programmatic dependent launch);
  // only a group's first scan waits on the copy events.
  constexpr int kSlots = 3;
  constexpr uint64_t kGroup = 4;
  const uint64_t gb = kGroup * batch;  // request rows per group
  const uint64_t rb = gb * db->words64 * 8;
  const uint64_t ob = gb * db->row_bytes;
  const uint64_t ra = (rb + 255) / 256 * 256, oa = (ob + 255) / 256 * 256;
  if (!grow_dev(reinterpret_cast<void**>(&db->d_pipe), &db->pipe_cap, kSlots * (ra + oa)))
    return TPIR_ENOMEM;
  cudaError_t e = cudaSuccess;
  if (!db->copy_stream) e = cudaStreamCreateWithFlags(&db->copy_stream, cudaStreamNonBlocking);
  for (int i = 0; e == cudaSuccess && i < 3 * kSlots; ++i)
    if (!db->pipe_ev[i]) e = cudaEventCreateWithFlags(&db->pipe_ev[i], cudaEventDisableTiming);
  if (e != cudaSuccess) return cuda_status(e);
  cudaStream_t cp = db->copy_stream, cs = db->stream;
  cudaEvent_t* in_done = db->pipe_ev;              // request rows copied in
  cudaEvent_t* scan_done = db->pipe_ev + kSlots;   // scans of the slot done
  cudaEvent_t* out_done = db->pipe_ev + 2 * kSlots;  // replies copied out
  const uint64_t ngroup = (B_total + gb - 1) / gb;
  auto req_of = [&](uint64_t i) { return reinterpret_cast<uint64_t*>(db->d_pipe + (i % kSlots) * (ra + oa)); };
  auto out_of = [&](uint64_t i) { return db->d_pipe + (i % kSlots) * (ra + oa) + ra; };
  auto rows = [&](uint64_t i) { return std::min<uint64_t>(gb, B_total - i * gb); };
  // copy-in of group i: into its slot, once the scans that last read the slot are done
  auto copy_in = [&](uint64_t i) -> cudaError_t {
    cudaError_t r = cudaSuccess;
    if (i >= kSlots) r = cudaStreamWaitEvent(cp, scan_done[i % kSlots], 0);
    if (r == cudaSuccess)
      r = cudaMemcpyAsync(req_of(i), req_bits + i * gb * db->words64, rows(i) * db->words64 * 8,
                          cudaMemcpyHostToDevice, cp);
    if (r == cudaSuccess) r = cudaEventRecord(in_done[i % kSlots], cp);
    return r;
  };
  for (uint64_t i = 0; e == cudaSuccess && i < std::min<uint64_t>(2, ngroup); ++i) e = copy_in(i);
  for (uint64_t i = 0; e == cudaSuccess && i < ngroup; ++i) {
    const int s = static_cast<int>(i % kSlots);
    e = cudaStreamWaitEvent(cs, in_done[s], 0);
    if (e == cudaSuccess && i >= kSlots) e = cudaStreamWaitEvent(cs, out_done[s], 0);
    if (e != cudaSuccess) break;
    for (uint64_t b0 = 0; b0 < rows(i); b0 += batch) {
      const uint32_t nb = static_cast<uint32_t>(std::min<uint64_t>(batch, rows(i) - b0));
      const tpir_status st = enqueue_read(db, req_of(i) + b0 * db->words64, nb,
                                         out_of(i) + b0 * db->row_bytes, cs);
      if (st != TPIR_OK) {
        cudaStreamSynchronize(cp);
        cudaStreamSynchronize(cs);
        return st;
      }
    }
    e = cudaEventRecord(scan_done[s], cs);
    if (e == cudaSuccess && i + 2 < ngroup) e = copy_in(i + 2);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(cp, scan_done[s], 0);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(static_cast<uint8_t*>(out) + i * gb * db->row_bytes, out_of(i),
                          rows(i) * db->row_bytes, cudaMemcpyDeviceToHost, cp);
    if (e == cudaSuccess) e = cudaEventRecord(out_done[s], cp);
  }
  const cudaError_t e2 = cudaStreamSynchronize(cp);
  if (e == cudaSuccess) e = e2;
  if (e != cudaSuccess) return cuda_status(e);
  int st = 0;
  if (read_device_status_and_clear(&st) != 0) return TPIR_ECUDA;
  return st ? static_cast<tpir_status>(st) : TPIR_OK;
}

tpir_status tpir_read_batch(tpir_db* db, const uint64_t* req_bits, uint32_t B, void* out) {
  return read_batch_sync(db, req_bits, B, nullptr, out);
}

tpir_status tpir_read_batch_masked(tpir_db* db, const uint64_t* req_bits, uint32_t B,
                                   const uint8_t* seeds, void* out) {
  if (B && !seeds) return TPIR_EINVAL;
  return read_batch_sync(db, req_bits, B, seeds, out);
}

tpir_status tpir_read_batch_async(tpir_db* db, const uint64_t* d_req_bits, uint32_t B,
                                  void* d_out, void* stream) {
  if (!db) return TPIR_EINVAL;
  if (B == 0) return TPIR_OK;
  if (!d_req_bits || !d_out) return TPIR_EINVAL;
  if ((reinterpret_cast<uintptr_t>(d_out) & 15) || (reinterpret_cast<uintptr_t>(d_req_bits) & 7))
    return TPIR_EINVAL;
  return enqueue_read(db, d_req_bits, B, d_out, static_cast<cudaStream_t>(stream));
}

tpir_status tpir_read_batch_masked_async(tpir_db* db, const uint64_t* d_req_bits, uint32_t B,
                                         const uint8_t* d_seeds, void* d_out, void* stream) {
  if (!db) return TPIR_EINVAL;
  if (B == 0) return TPIR_OK;
  if (!d_req_bits || !d_out || !d_seeds) return TPIR_EINVAL;
  if ((reinterpret_cast<uintptr_t>(d_out) & 15) || (reinterpret_cast<uintptr_t>(d_req_bits) & 7) ||
      (reinterpret_cast<uintptr_t>(d_seeds) & 15))
    return TPIR_EINVAL;
  return enqueue_read(db, d_req_bits, B, d_out, static_cast<cudaStream_t>(stream), d_seeds);
}

tpir_status tpir_read_multi_async(const tpir_read_job* jobs, uint32_t njobs, void* stream) {
  if (njobs == 0) return TPIR_OK;
  if (!jobs || njobs > TPIR_MAX_JOBS) return TPIR_EINVAL;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  for (uint32_t i = 0; i < njobs; ++i)
    if (!jobs[i].db) return TPIR_EINVAL;
  for (uint32_t i = 0; i < njobs; ++i)
    if (jobs[i].B) order_after_writes(jobs[i].db, st);
  tpir_status s = enqueue_multi(jobs, njobs, st);
  if (s != TPIR_OK) return s;
  for (uint32_t i = 0; i < njobs; ++i)
    if (jobs[i].B) note_read(jobs[i].db, st);
  return TPIR_OK;
}

struct tpir_graph {
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  std::vector<tpir_db*> dbs;
};

tpir_status tpir_read_multi_graph_create(const tpir_read_job* jobs, uint32_t njobs,
                                         tpir_graph** out) {
  if (!out || !jobs || njobs == 0 || njobs > TPIR_MAX_JOBS) return TPIR_EINVAL;
  *out = nullptr;
  for (uint32_t i = 0; i < njobs; ++i)
    if (!jobs[i].db) return TPIR_EINVAL;
  tpir_graph* g = new (std::nothrow) tpir_graph();
  if (!g) return TPIR_ENOMEM;
  (void)batched_grid();  // one-time kernel attributes, outside the capture
  // the tensor-core jobs' transposed copies exist before the capture (their
  // allocation and first build cannot be captured); later writes and loads
  // keep them current in stream order
  for (uint32_t i = 0; i < njobs; ++i) {
    if (!jobs[i].B || multi_kernel(jobs[i]) != 5) continue;
    tpir_db* db = jobs[i].db;
    order_writes_after_reads(db, db->stream);
    cudaError_t e = cudaStreamWaitEvent(db->stream, db->last_write, 0);
    if (e == cudaSuccess) e = tcopy_ensure(db, db->stream);
    if (e == cudaSuccess) e = cudaEventRecord(db->last_write, db->stream);
    if (e != cudaSuccess) {
      delete g;
      return cuda_status(e);
    }
  }
  cudaStream_t st = nullptr;
  cudaError_t e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
  tpir_status s = TPIR_OK;
  if (e == cudaSuccess) {
    s = enqueue_multi(jobs, njobs, st);
    cudaError_t e2 = cudaStreamEndCapture(st, &g->graph);
    if (s == TPIR_OK && e2 != cudaSuccess) e = e2;
  }
  if (e == cudaSuccess && s == TPIR_OK) e = cudaGraphInstantiate(&g->exec, g->graph, 0);
  if (st) cudaStreamDestroy(st);
  if (e != cudaSuccess || s != TPIR_OK) {
    tpir_graph_destroy(g);
    return s != TPIR_OK ? s : cuda_status(e);
  }
  for (uint32_t i = 0; i < njobs; ++i)
    if (jobs[i].B) g->dbs.push_back(jobs[i].db);
  *out = g;
  return TPIR_OK;
}

tpir_status tpir_graph_launch(tpir_graph* g, void* stream) {
  if (!g || !g->exec) return TPIR_EINVAL;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  for (tpir_db* db : g->dbs) order_after_writes(db, st);
  cudaError_t e = cudaGraphLaunch(g->exec, st);
  if (e != cudaSuccess) return cuda_status(e);
  for (tpir_db* db : g->dbs) note_read(db, st);
  return TPIR_OK;
}

void tpir_graph_destroy(tpir_graph* g) {
  if (!g) return;
  if (g->exec) cudaGraphExecDestroy(g->exec);
  if (g->graph) cudaGraphDestroy(g->graph);
  delete g;
}

tpir_status tpir_selftest_wait_timeout(uint32_t limit_us) {
  if (limit_us == 0 || limit_us > 1000000) return TPIR_EINVAL;
  cudaError_t e = launch_selftest_wait(static_cast<uint64_t>(limit_us) * 1000ull, nullptr);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return cuda_status(e);
  int st = 0;
  if (read_device_status_and_clear(&st) != 0) return TPIR_ECUDA;
  return st ? static_cast<tpir_status>(st) : TPIR_OK;
}

tpir_status tpir_device_status(void) {
  cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return cuda_status(e);
  int st = 0;
  if (read_device_status_and_clear(&st) != 0) return TPIR_ECUDA;
  return st ? static_cast<tpir_status>(st) : TPIR_OK;
}

uint64_t tpir_kernel_launches(void) { return g_kernel_launches.load(std::memory_order_relaxed); }

// ---- Bloom -----------------------------------------------------------------
tpir_status tpir_bloom_create(tpir_db* db, uint64_t m_bits, uint32_t k, uint32_t window,
                              uint32_t writes_per_delta) {
  if (!db || m_bits == 0 || k == 0 || window == 0 || m_bits > (1ull << 36)) return TPIR_EINVAL;
  tpir_bloom_state& bl = db->bloom;
  cudaFree(bl.d_deltas);
  cudaFree(bl.d_out);
  bl.d_deltas = nullptr;
  bl.d_out = nullptr;
  bl.m = m_bits;
  bl.words = (m_bits + 63) / 64;
  bl.k = k;
  bl.window = window;
  bl.per_delta = writes_per_delta;
  bl.cur = 0;
  bl.count = 0;
  cudaError_t e = cudaMalloc(reinterpret_cast<void**>(&bl.d_deltas), bl.words * 8 * window);
  if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(&bl.d_out), bl.words * 8);
  if (e == cudaSuccess) e = cudaMemsetAsync(bl.d_deltas, 0, bl.words * 8 * window, db->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(db->stream);
  if (e != cudaSuccess) {
    cudaFree(bl.d_deltas);
    cudaFree(bl.d_out);
    bl.d_deltas = nullptr;
    bl.d_out = nullptr;
    return cuda_status(e);
  }
  return TPIR_OK;
}

tpir_status tpir_bloom_insert(tpir_db* db, const uint64_t* positions) {
  return tpir_bloom_insert_batch(db, positions, 1);
}

tpir_status tpir_bloom_insert_batch(tpir_db* db, const uint64_t* positions, uint32_t count) {
  if (!db || (count && !positions)) return TPIR_EINVAL;
  if (count == 0) return TPIR_OK;
  cudaError_t e = cudaEventSynchronize(db->last_write);
  if (e != cudaSuccess) return cuda_status(e);
  order_writes_after_reads(db, db->stream);
  return bloom_insert_core(db, positions, count, db->stream, db->stage);
}

tpir_status tpir_bloom_or_vector(tpir_db* db, const uint64_t* vec) {
  if (!db || !vec || !db->bloom.d_deltas) return TPIR_EINVAL;
  tpir_bloom_state& bl = db->bloom;
  cudaError_t e = cudaEventSynchronize(db->last_write);
  if (e != cudaSuccess) return cuda_status(e);
  const uint64_t bytes = bl.words * 8;
  if (!grow_pinned(reinterpret_cast<void**>(&db->stage.h), &db->stage.h_cap, bytes) ||
      !grow_dev(reinterpret_cast<void**>(&db->stage.d_pos), &db->stage.pos_cap, bytes))
    return TPIR_ENOMEM;
  std::memcpy(db->stage.h, vec, bytes);
  order_writes_after_reads(db, db->stream);
  if (bl.per_delta && bl.count == bl.per_delta) {
    bl.cur = (bl.cur + 1) % bl.window;
    bl.count = 0;
    e = cudaMemsetAsync(bl.d_deltas + static_cast<uint64_t>(bl.cur) * bl.words, 0, bytes,
                        db->stream);
  }
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(db->stage.d_pos, db->stage.h, bytes, cudaMemcpyHostToDevice, db->stream);
  if (e == cudaSuccess)
    e = launch_bloom_or(bl.d_deltas + static_cast<uint64_t>(bl.cur) * bl.words, db->stage.d_pos,
                        bl.m, db->stream);
  if (e == cudaSuccess) e = cudaEventRecord(db->last_write, db->stream);
  if (e != cudaSuccess) return cuda_status(e);
  bl.count += 1;
  return TPIR_OK;
}

tpir_status tpir_bloom_get_compressed(tpir_db* db, uint32_t which, int32_t k, void* out,
                                      uint64_t cap_bytes, uint64_t* nbits, uint64_t* count,
                                      uint32_t* k_used) {
  if (nbits) *nbits = 0;
  if (!db || !out || !db->bloom.d_deltas || which > db->bloom.window || k > 63) return TPIR_EINVAL;
  tpir_bloom_state& bl = db->bloom;
  const uint64_t cap = (cap_bytes + 3) / 4 * 4;
  if (!grow_dev(reinterpret_cast<void**>(&bl.d_rice), &bl.rice_cap, cap)) return TPIR_ENOMEM;
  if (!bl.d_rice_res && cudaMalloc(reinterpret_cast<void**>(&bl.d_rice_res), 3 * 8) != cudaSuccess)
    return TPIR_ENOMEM;
  // 0: the global interest vector; i >= 1: the i-th most recent delta
  const uint64_t* vec = bl.d_out;
  cudaError_t e = cudaSuccess;
  if (which == 0)
    e = launch_bloom_union(bl.d_deltas, bl.window, bl.words, bl.d_out, db->stream);
  else
    vec = bl.d_deltas + static_cast<uint64_t>((bl.cur + bl.window - (which - 1)) % bl.window) * bl.words;
  const RiceRequest rq{vec, bl.m, k, bl.d_rice, cap / 4, bl.d_rice_res};
  if (!grow_dev(reinterpret_cast<void**>(&bl.d_rice_scratch), &bl.rice_scratch_cap,
                rice_scratch_bytes(bl.m)))
    return TPIR_ENOMEM;
  if (e == cudaSuccess) e = launch_rice_encode(rq, bl.d_rice_scratch, db->stream);
  uint64_t res[3] = {0, 0, 0};
  if (e == cudaSuccess) e = cudaMemcpyAsync(res, bl.d_rice_res, sizeof(res), cudaMemcpyDeviceToHost, db->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(db->stream);
  if (e != cudaSuccess) return cuda_status(e);
  if (count) *count = res[1];
  if (k_used) *k_used = static_cast<uint32_t>(res[2]);
  if (nbits) *nbits = res[0];
  if (res[0] == ~0ull || (res[0] + 7) / 8 > cap_bytes) return TPIR_ENOMEM;  // stream past cap
  if (res[0]) e = cudaMemcpy(out, bl.d_rice, (res[0] + 7) / 8, cudaMemcpyDeviceToHost);
  return cuda_status(e);
}

tpir_status tpir_rice_encode_async(const uint64_t* d_bits, uint64_t m, int32_t k, void* d_out,
                                   uint64_t cap_bytes, uint64_t* d_result, void* stream) {
  if (!d_bits || !d_out || !d_result || m == 0 || k > 63 || (cap_bytes & 3) ||
      (reinterpret_cast<uintptr_t>(d_out) & 3) || (reinterpret_cast<uintptr_t>(d_bits) & 7) ||
      (reinterpret_cast<uintptr_t>(d_result) & 7))
    return TPIR_EINVAL;
  const RiceRequest rq{d_bits, m, k, static_cast<uint32_t*>(d_out), cap_bytes / 4, d_result};
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  // scratch from the stream-ordered allocator: calls on other streams do not share it
  void* scratch = nullptr;
  cudaError_t e = cudaMallocAsync(&scratch, rice_scratch_bytes(m), st);
  if (e == cudaSuccess) e = launch_rice_encode(rq, scratch, st);
  if (scratch) {
    const cudaError_t f = cudaFreeAsync(scratch, st);
    if (e == cudaSuccess) e = f;
  }
  return cuda_status(e);
}

tpir_status tpir_bloom_get(tpir_db* db, uint64_t* out_words) {
  if (!db || !out_words || !db->bloom.d_deltas) return TPIR_EINVAL;
  tpir_bloom_state& bl = db->bloom;
  cudaError_t e = launch_bloom_union(bl.d_deltas, bl.window, bl.words, bl.d_out, db->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(out_words, bl.d_out, bl.words * 8, cudaMemcpyDeviceToHost, db->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(db->stream);
  return cuda_status(e);
}

}  // extern "C"
