// Continuous-batching server over device-resident tables.
//
// The leader of Section 6 sequences writes and forwards batches of reads; the
// paper's prototype batches reads before the GPU and notes that reads may be
// reordered freely while writes must apply in sequence order (Section 9.2).
// This server does that on one GPU:
//   - submit_* admit ops into a FIFO (bounded: EAGAIN when full);
//   - a worker thread forms a launch whenever a pipeline slot is free: it
//     scans the FIFO in arrival order, applies each table's writes (host
//     placement + device moves) and collects up to max_batch reads per table;
//     the collected reads run after the writes of that launch (stream
//     order): tables with a few reads stream through the plain kernel, all
//     others share ONE persistent launch of the batched scan kernel;
//   - up to max_inflight launches are queued on the device at once, with their
//     request/reply copies on a copy stream overlapping the running kernels,
//     so reads that arrive while others are on the GPU join the next launch;
//   - a read sees every write to its table applied before its launch; its
//     completion reports that write count (epoch).
// Tables are admitted against an HBM budget (tables + launch staging).
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <new>
#include <thread>
#include <unordered_map>

#include "tpir_internal.h"

namespace {

using namespace tpir;

// Tables with at most this many reads in a launch use the plain kernel.
constexpr uint32_t kServePlainMaxB = 4;

int64_t now_ns() {
  return std::chrono::duration_cast<std::chrono::nanoseconds>(
             std::chrono::steady_clock::now().time_since_epoch())
      .count();
}

struct Op {
  uint32_t kind;  // 0 read, 1 write
  uint32_t table;
  uint64_t tag;
  int64_t t_arrive;
  void* out = nullptr;              // read: host reply buffer
  std::vector<uint64_t> req;        // read: request row
  uint64_t b1 = 0, b2 = 0;          // write
  std::vector<uint8_t> msg;         // write
  std::vector<uint64_t> bloom;      // write: k positions (may be empty)
};

struct ReadRec {
  uint64_t tag;
  uint32_t table;
  int64_t t_arrive;
  void* out;
  uint64_t out_off;  // byte offset of the reply in the slot's reply staging
  uint32_t bytes;
  uint64_t epoch;
};

struct WriteRec {
  uint64_t tag;
  uint32_t table;
  int64_t t_arrive;
  tpir_status status;
  uint32_t evictions;
  uint64_t epoch;
};

struct Slot {
  cudaEvent_t h2d_done = nullptr, kern_done = nullptr, done = nullptr;
  uint64_t* h_req = nullptr;
  uint64_t h_req_cap = 0;
  uint64_t* d_req = nullptr;
  uint64_t d_req_cap = 0;
  uint8_t* h_out = nullptr;
  uint64_t h_out_cap = 0;
  uint8_t* d_out = nullptr;
  uint64_t d_out_cap = 0;
  std::vector<ReadRec> reads;
  std::vector<WriteRec> writes;
  std::vector<tpir_write_staging> wstage;  // one per table written in this launch
  std::vector<tpir_write_staging> bstage;  // Bloom positions, one per table
  int64_t t_launch = 0;
};

struct Table {
  tpir_db* db = nullptr;
  uint64_t bytes = 0;
};

}  // namespace

struct tpir_server {
  tpir_serve_config cfg{};
  int device = 0;
  std::vector<Table> tables;
  uint64_t hbm_tables = 0;
  uint64_t staging_reserve = 0;
  cudaStream_t compute = nullptr, copy = nullptr;

  std::mutex mu;
  std::condition_variable cv_work, cv_idle;
  std::deque<Op> queue;
  uint64_t unfinished = 0;  // admitted and not yet completed
  bool stop = false;

  std::vector<Slot> slots;
  std::deque<int> inflight;  // slot indices, oldest first
  std::vector<int> free_slots;

  std::mutex cmu;
  std::deque<tpir_completion> done;
  // stats
  std::vector<double> lat_ms;
  uint64_t reads_done = 0, writes_done = 0, rejected = 0, failed = 0, launches = 0;
  uint64_t batch_tables = 0, batch_reads = 0;
  int64_t t_first = 0, t_last = 0;
  uint64_t ev_hist[8] = {0};

  std::thread worker;
};

namespace {

uint64_t slot_staging_bytes(const tpir_serve_config& c) {
  // request + reply staging a launch may grow to (bounded per slot)
  return 256ull << 20;
}

int hist_bucket(uint32_t ev) {
  if (ev == 0) return 0;
  int b = 1;
  uint32_t lim = 2;
  while (b < 7 && ev >= lim) {
    ++b;
    lim <<= 1;
  }
  return b;
}

void retire(tpir_server* s, int si) {
  Slot& sl = s->slots[si];
  const int64_t t = now_ns();
  std::vector<tpir_completion> cs;
  cs.reserve(sl.reads.size() + sl.writes.size());
  for (const WriteRec& w : sl.writes) {
    tpir_completion c{};
    c.tag = w.tag;
    c.status = w.status;
    c.kind = 1;
    c.table_id = w.table;
    c.evictions = w.evictions;
    c.epoch = w.epoch;
    c.t_arrive_ns = w.t_arrive;
    c.t_launch_ns = sl.t_launch;
    c.t_done_ns = t;
    cs.push_back(c);
  }
  for (const ReadRec& r : sl.reads) {
    std::memcpy(r.out, sl.h_out + r.out_off, r.bytes);
    tpir_completion c{};
    c.tag = r.tag;
    c.status = TPIR_OK;
    c.kind = 0;
    c.table_id = r.table;
    c.epoch = r.epoch;
    c.t_arrive_ns = r.t_arrive;
    c.t_launch_ns = sl.t_launch;
    c.t_done_ns = t;
    cs.push_back(c);
  }
  {
    std::lock_guard<std::mutex> g(s->cmu);
    for (const auto& c : cs) {
      s->done.push_back(c);
      if (c.kind == 0) {
        s->reads_done++;
        s->lat_ms.push_back((c.t_done_ns - c.t_arrive_ns) * 1e-6);
        if (!s->t_first || c.t_arrive_ns < s->t_first) s->t_first = c.t_arrive_ns;
        s->t_last = std::max(s->t_last, c.t_done_ns);
      } else {
        s->writes_done++;
        if (c.status != TPIR_OK) s->failed++;
        s->ev_hist[hist_bucket(c.evictions)]++;
      }
    }
  }
  sl.reads.clear();
  sl.writes.clear();
  {
    std::lock_guard<std::mutex> g(s->mu);
    s->unfinished -= cs.size();
    if (s->unfinished == 0) s->cv_idle.notify_all();
  }
}

// Forms one launch from the FIFO into slot `si`; returns false if nothing was
// admitted into it.
bool form_launch(tpir_server* s, int si) {
  Slot& sl = s->slots[si];
  std::vector<Op> taken_writes;
  std::unordered_map<uint32_t, std::vector<Op>> reads_by_table;
  std::vector<uint32_t> table_order;
  {
    std::lock_guard<std::mutex> g(s->mu);
    if (s->queue.empty()) return false;
    std::unordered_map<uint32_t, uint32_t> count;
    std::deque<Op> keep;
    uint32_t njobs = 0;
    while (!s->queue.empty()) {
      Op op = std::move(s->queue.front());
      s->queue.pop_front();
      if (op.kind == 1) {
        taken_writes.push_back(std::move(op));
        continue;
      }
      auto it = count.find(op.table);
      const bool new_table = it == count.end();
      if ((new_table && njobs >= TPIR_MAX_JOBS) ||
          (!new_table && it->second >= s->cfg.max_batch)) {
        keep.push_back(std::move(op));
        continue;
      }
      if (new_table) {
        count[op.table] = 1;
        ++njobs;
        table_order.push_back(op.table);
      } else {
        it->second++;
      }
      reads_by_table[op.table].push_back(std::move(op));
    }
    s->queue.swap(keep);
  }
  sl.t_launch = now_ns();

  // ---- writes, per table in arrival order, on the compute stream
  std::unordered_map<uint32_t, std::vector<size_t>> wtab;
  std::vector<uint32_t> worder;
  for (size_t i = 0; i < taken_writes.size(); ++i) {
    const uint32_t t = taken_writes[i].table;
    if (!wtab.count(t)) worder.push_back(t);
    wtab[t].push_back(i);
  }
  if (sl.wstage.size() < worder.size()) sl.wstage.resize(worder.size());
  if (sl.bstage.size() < worder.size()) sl.bstage.resize(worder.size());
  for (size_t wi = 0; wi < worder.size(); ++wi) {
    const uint32_t t = worder[wi];
    tpir_db* db = s->tables[t].db;
    const auto& idx = wtab[t];
    std::vector<uint64_t> b1(idx.size()), b2(idx.size()), pos;
    std::vector<uint8_t> msgs(idx.size() * db->z);
    uint32_t with_bloom = 0;
    for (size_t j = 0; j < idx.size(); ++j) {
      const Op& op = taken_writes[idx[j]];
      b1[j] = op.b1;
      b2[j] = op.b2;
      std::memcpy(msgs.data() + j * db->z, op.msg.data(), db->z);
    }
    std::vector<tpir_status> st(idx.size(), TPIR_OK);
    std::vector<uint32_t> ev(idx.size(), 0);
    const uint64_t epoch0 = db->epoch;
    tpir_status r = apply_writes_core(db, static_cast<uint32_t>(idx.size()), b1.data(), b2.data(),
                                      msgs.data(), st.data(), ev.data(), s->compute, sl.wstage[wi]);
    uint64_t e = epoch0;
    for (size_t j = 0; j < idx.size(); ++j) {
      const Op& op = taken_writes[idx[j]];
      const tpir_status sj = (r != TPIR_OK) ? r : st[j];
      if (sj == TPIR_OK) ++e;
      sl.writes.push_back(WriteRec{op.tag, t, op.t_arrive, sj, ev[j], e});
      if (sj == TPIR_OK && db->bloom.d_deltas && op.bloom.size() == db->bloom.k) {
        pos.insert(pos.end(), op.bloom.begin(), op.bloom.end());
        ++with_bloom;
      }
    }
    if (with_bloom) bloom_insert_core(db, pos.data(), with_bloom, s->compute, sl.bstage[wi]);
  }

  // ---- reads: pack requests and reply offsets per table
  uint64_t req_words = 0, out_bytes = 0;
  for (uint32_t t : table_order) {
    tpir_db* db = s->tables[t].db;
    const uint64_t B = reads_by_table[t].size();
    req_words += B * db->words64;
    out_bytes += (B * db->row_bytes + 255) / 256 * 256;
  }
  if (!table_order.empty()) {
    if (!grow_pinned(reinterpret_cast<void**>(&sl.h_req), &sl.h_req_cap, req_words * 8) ||
        !grow_dev(reinterpret_cast<void**>(&sl.d_req), &sl.d_req_cap, req_words * 8) ||
        !grow_pinned(reinterpret_cast<void**>(&sl.h_out), &sl.h_out_cap, out_bytes) ||
        !grow_dev(reinterpret_cast<void**>(&sl.d_out), &sl.d_out_cap, out_bytes)) {
      // cannot stage: fail these reads
      for (uint32_t t : table_order)
        for (const Op& op : reads_by_table[t]) {
          tpir_completion c{};
          c.tag = op.tag;
          c.status = TPIR_ENOMEM;
          c.table_id = t;
          c.t_arrive_ns = op.t_arrive;
          c.t_done_ns = now_ns();
          std::lock_guard<std::mutex> g(s->cmu);
          s->done.push_back(c);
          s->failed++;
        }
      table_order.clear();
    }
  }
  std::vector<tpir_read_job> jobs;
  uint64_t wo = 0, oo = 0;
  for (uint32_t t : table_order) {
    tpir_db* db = s->tables[t].db;
    auto& ops = reads_by_table[t];
    const uint32_t B = static_cast<uint32_t>(ops.size());
    for (uint32_t b = 0; b < B; ++b) {
      std::memcpy(sl.h_req + wo + static_cast<uint64_t>(b) * db->words64, ops[b].req.data(),
                  db->words64 * 8);
      sl.reads.push_back(ReadRec{ops[b].tag, t, ops[b].t_arrive, ops[b].out,
                                 oo + static_cast<uint64_t>(b) * db->row_bytes, db->row_bytes,
                                 db->epoch});
    }
    jobs.push_back(tpir_read_job{db, B, sl.d_req + wo, sl.d_out + oo});
    wo += static_cast<uint64_t>(B) * db->words64;
    oo += (static_cast<uint64_t>(B) * db->row_bytes + 255) / 256 * 256;
  }
  if (!jobs.empty()) {
    cudaMemcpyAsync(sl.d_req, sl.h_req, req_words * 8, cudaMemcpyHostToDevice, s->copy);
    cudaEventRecord(sl.h2d_done, s->copy);
    cudaStreamWaitEvent(s->compute, sl.h2d_done, 0);
    // tables with a few reads are HBM-bound: stream each with the plain
    // kernel (back-to-back launches overlap); the rest share one persistent
    // launch of the batched kernel
    std::vector<tpir_read_job> batched;
    for (const tpir_read_job& j : jobs) {
      if (j.B <= kServePlainMaxB)
        enqueue_read(j.db, j.d_req_bits, j.B, j.d_out, s->compute);
      else
        batched.push_back(j);
    }
    if (!batched.empty())
      enqueue_multi(batched.data(), static_cast<uint32_t>(batched.size()), s->compute);
    cudaEventRecord(sl.kern_done, s->compute);
    cudaStreamWaitEvent(s->copy, sl.kern_done, 0);
    cudaMemcpyAsync(sl.h_out, sl.d_out, out_bytes, cudaMemcpyDeviceToHost, s->copy);
    cudaEventRecord(sl.done, s->copy);
    std::lock_guard<std::mutex> g(s->cmu);
    s->launches++;
    s->batch_tables += jobs.size();
    s->batch_reads += sl.reads.size();
  } else {
    // writes only: completion follows the compute stream
    cudaEventRecord(sl.done, s->compute);
  }
  return true;
}

void worker_main(tpir_server* s) {
  cudaSetDevice(s->device);
  for (;;) {
    // retire finished launches, oldest first
    while (!s->inflight.empty()) {
      const int si = s->inflight.front();
      if (cudaEventQuery(s->slots[si].done) != cudaSuccess) break;
      s->inflight.pop_front();
      retire(s, si);
      s->free_slots.push_back(si);
    }
    bool pending;
    {
      std::lock_guard<std::mutex> g(s->mu);
      pending = !s->queue.empty();
      if (s->stop && !pending && s->inflight.empty()) break;
    }
    if (pending && !s->free_slots.empty()) {
      const int si = s->free_slots.back();
      s->free_slots.pop_back();
      if (form_launch(s, si))
        s->inflight.push_back(si);
      else
        s->free_slots.push_back(si);
      continue;
    }
    if (!s->inflight.empty()) {
      // a launch is running: poll its completion without burning a core
      std::this_thread::sleep_for(std::chrono::microseconds(20));
      continue;
    }
    std::unique_lock<std::mutex> lk(s->mu);
    s->cv_work.wait_for(lk, std::chrono::microseconds(s->cfg.tick_us),
                        [&] { return s->stop || !s->queue.empty(); });
  }
}

}  // namespace

extern "C" {

tpir_status tpir_serve_create(const tpir_serve_config* cfg, tpir_server** out) {
  if (!out) return TPIR_EINVAL;
  *out = nullptr;
  tpir_server* s = new (std::nothrow) tpir_server();
  if (!s) return TPIR_ENOMEM;
  if (cfg) s->cfg = *cfg;
  if (!s->cfg.hbm_budget_bytes) s->cfg.hbm_budget_bytes = 64ull << 30;
  if (!s->cfg.max_batch) s->cfg.max_batch = 256;
  if (!s->cfg.max_inflight) s->cfg.max_inflight = 2;
  if (!s->cfg.queue_capacity) s->cfg.queue_capacity = 65536;
  if (!s->cfg.tick_us) s->cfg.tick_us = 200;
  if (s->cfg.max_batch > 1024 || s->cfg.max_inflight > 8) {
    delete s;
    return TPIR_EINVAL;
  }
  cudaGetDevice(&s->device);
  s->staging_reserve = s->cfg.max_inflight * slot_staging_bytes(s->cfg);
  if (s->staging_reserve >= s->cfg.hbm_budget_bytes) {
    delete s;
    return TPIR_ENOMEM;
  }
  cudaError_t e = cudaStreamCreateWithFlags(&s->compute, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->copy, cudaStreamNonBlocking);
  s->slots.resize(s->cfg.max_inflight);
  for (uint32_t i = 0; i < s->cfg.max_inflight && e == cudaSuccess; ++i) {
    Slot& sl = s->slots[i];
    e = cudaEventCreateWithFlags(&sl.h2d_done, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&sl.kern_done, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming);
    s->free_slots.push_back(static_cast<int>(i));
  }
  if (e != cudaSuccess) {
    tpir_serve_destroy(s);
    return cuda_status(e);
  }
  s->worker = std::thread(worker_main, s);
  *out = s;
  return TPIR_OK;
}

tpir_status tpir_serve_add_table(tpir_server* s, uint64_t n, uint32_t d, uint32_t msg_bytes,
                                 uint32_t* table_id) {
  if (!s || !table_id) return TPIR_EINVAL;
  const uint64_t bytes = n * static_cast<uint64_t>(d) * msg_bytes;
  std::lock_guard<std::mutex> g(s->mu);
  if (s->stop) return TPIR_ESHUTDOWN;
  if (s->hbm_tables + bytes + s->staging_reserve > s->cfg.hbm_budget_bytes) return TPIR_ENOMEM;
  tpir_db* db = tpir_db_create(n, d, msg_bytes);
  if (!db) return tpir_last_error();
  s->tables.push_back(Table{db, bytes});
  s->hbm_tables += bytes;
  *table_id = static_cast<uint32_t>(s->tables.size() - 1);
  return TPIR_OK;
}

tpir_status tpir_serve_table(tpir_server* s, uint32_t table_id, tpir_db** db) {
  if (!s || !db) return TPIR_EINVAL;
  std::lock_guard<std::mutex> g(s->mu);
  if (table_id >= s->tables.size()) return TPIR_EINVAL;
  *db = s->tables[table_id].db;
  return TPIR_OK;
}

static tpir_status admit(tpir_server* s, Op&& op) {
  std::lock_guard<std::mutex> g(s->mu);
  if (s->stop) return TPIR_ESHUTDOWN;
  if (s->unfinished >= s->cfg.queue_capacity) {
    std::lock_guard<std::mutex> g2(s->cmu);
    s->rejected++;
    return TPIR_EAGAIN;
  }
  s->unfinished++;
  s->queue.push_back(std::move(op));
  s->cv_work.notify_one();
  return TPIR_OK;
}

tpir_status tpir_serve_submit_read(tpir_server* s, uint32_t table_id, const uint64_t* req_bits,
                                   void* out, uint64_t tag, int64_t t_arrive_ns) {
  if (!s || !req_bits || !out) return TPIR_EINVAL;
  tpir_db* db;
  {
    std::lock_guard<std::mutex> g(s->mu);
    if (table_id >= s->tables.size()) return TPIR_EINVAL;
    db = s->tables[table_id].db;
  }
  Op op;
  op.kind = 0;
  op.table = table_id;
  op.tag = tag;
  op.t_arrive = t_arrive_ns ? t_arrive_ns : now_ns();
  op.out = out;
  op.req.assign(req_bits, req_bits + db->words64);
  return admit(s, std::move(op));
}

tpir_status tpir_serve_submit_write(tpir_server* s, uint32_t table_id, uint64_t b1, uint64_t b2,
                                    const void* msg, const uint64_t* bloom_positions, uint64_t tag,
                                    int64_t t_arrive_ns) {
  if (!s || !msg) return TPIR_EINVAL;
  tpir_db* db;
  {
    std::lock_guard<std::mutex> g(s->mu);
    if (table_id >= s->tables.size()) return TPIR_EINVAL;
    db = s->tables[table_id].db;
  }
  if (b1 >= db->n || b2 >= db->n) return TPIR_EINVAL;
  Op op;
  op.kind = 1;
  op.table = table_id;
  op.tag = tag;
  op.t_arrive = t_arrive_ns ? t_arrive_ns : now_ns();
  op.b1 = b1;
  op.b2 = b2;
  const uint8_t* m = static_cast<const uint8_t*>(msg);
  op.msg.assign(m, m + db->z);
  if (bloom_positions && db->bloom.k) {
    for (uint32_t i = 0; i < db->bloom.k; ++i)
      if (bloom_positions[i] >= db->bloom.m) return TPIR_EINVAL;
    op.bloom.assign(bloom_positions, bloom_positions + db->bloom.k);
  }
  return admit(s, std::move(op));
}

tpir_status tpir_serve_poll(tpir_server* s, tpir_completion* done, uint32_t max, uint32_t* ndone) {
  if (!s || !ndone || (max && !done)) return TPIR_EINVAL;
  std::lock_guard<std::mutex> g(s->cmu);
  uint32_t n = 0;
  while (n < max && !s->done.empty()) {
    done[n++] = s->done.front();
    s->done.pop_front();
  }
  *ndone = n;
  return TPIR_OK;
}

tpir_status tpir_serve_drain(tpir_server* s) {
  if (!s) return TPIR_EINVAL;
  std::unique_lock<std::mutex> lk(s->mu);
  s->cv_idle.wait(lk, [&] { return s->unfinished == 0; });
  return TPIR_OK;
}

tpir_status tpir_serve_stats(tpir_server* s, tpir_stats* st) {
  if (!s || !st) return TPIR_EINVAL;
  std::memset(st, 0, sizeof(*st));
  std::vector<double> lat;
  {
    std::lock_guard<std::mutex> g(s->cmu);
    st->reads_done = s->reads_done;
    st->writes_done = s->writes_done;
    st->rejected = s->rejected;
    st->failed = s->failed;
    st->launches = s->launches;
    st->mean_batch = s->batch_tables ? static_cast<double>(s->batch_reads) / s->batch_tables : 0.0;
    if (s->t_last > s->t_first)
      st->reads_per_s = s->reads_done / ((s->t_last - s->t_first) * 1e-9);
    for (int i = 0; i < 8; ++i) st->eviction_hist[i] = s->ev_hist[i];
    lat = s->lat_ms;
  }
  if (!lat.empty()) {
    std::sort(lat.begin(), lat.end());
    auto pct = [&](double p) {
      size_t i = static_cast<size_t>(p * (lat.size() - 1) + 0.5);
      return lat[std::min(i, lat.size() - 1)];
    };
    st->p50_ms = pct(0.50);
    st->p99_ms = pct(0.99);
    st->max_ms = lat.back();
  }
  {
    std::lock_guard<std::mutex> g(s->mu);
    st->hbm_bytes_in_use = s->hbm_tables;
  }
  for (const Slot& sl : s->slots) st->hbm_bytes_in_use += sl.d_req_cap + sl.d_out_cap;
  return TPIR_OK;
}

tpir_status tpir_serve_reset_stats(tpir_server* s) {
  if (!s) return TPIR_EINVAL;
  std::lock_guard<std::mutex> g(s->cmu);
  s->lat_ms.clear();
  s->reads_done = s->writes_done = s->rejected = s->failed = s->launches = 0;
  s->batch_tables = s->batch_reads = 0;
  s->t_first = s->t_last = 0;
  for (auto& h : s->ev_hist) h = 0;
  return TPIR_OK;
}

tpir_status tpir_serve_destroy(tpir_server* s) {
  if (!s) return TPIR_EINVAL;
  {
    std::lock_guard<std::mutex> g(s->mu);
    s->stop = true;
    s->cv_work.notify_all();
  }
  if (s->worker.joinable()) s->worker.join();
  if (s->compute) cudaStreamSynchronize(s->compute);
  if (s->copy) cudaStreamSynchronize(s->copy);
  for (Slot& sl : s->slots) {
    if (sl.h_req) cudaFreeHost(sl.h_req);
    if (sl.h_out) cudaFreeHost(sl.h_out);
    cudaFree(sl.d_req);
    cudaFree(sl.d_out);
    for (auto& w : sl.wstage) w.release();
    for (auto& w : sl.bstage) w.release();
    if (sl.h2d_done) cudaEventDestroy(sl.h2d_done);
    if (sl.kern_done) cudaEventDestroy(sl.kern_done);
    if (sl.done) cudaEventDestroy(sl.done);
  }
  for (Table& t : s->tables) tpir_db_destroy(t.db);
  if (s->compute) cudaStreamDestroy(s->compute);
  if (s->copy) cudaStreamDestroy(s->copy);
  delete s;
  return TPIR_OK;
}

}  // extern "C"
