// Continuous-batching server over device-resident tables.
//
// The leader of Section 6 sequences writes and forwards batches of reads; the
// paper's prototype batches reads before the GPU and notes that reads may be
// reordered freely while writes must apply in sequence order (Section 9.2).
// This server does that on one GPU, one table at a time:
//   - submit_* admit ops into the FIFO of their table (bounded in total:
//     EAGAIN when full);
//   - a worker thread forms a launch unit whenever a pipeline slot is free:
//     it picks the table whose oldest waiting op arrived first, applies all of
//     that table's waiting writes in arrival order (host placement + device
//     moves) and takes up to max_batch of its waiting reads, which run after
//     those writes; the read kernel is chosen by the batch (plain stream for a
//     few reads, the register-tiled kernel, the tensor-core kernel from 48
//     reads on wide rows), so a table that collected a burst of reads is read
//     once for all of them;
//   - a unit never scans a table it has no reads for: a read waits for its own
//     table's next unit, not for a pass over every resident table;
//   - up to max_inflight units are queued on the device at once, each table's
//     units in order on one of a few streams (request and reply copies on the
//     same stream), so reads that arrive while others are on the GPU join the
//     next unit of their table;
//   - a read sees every write to its table admitted before its unit was
//     formed; its completion reports that write count (epoch).
// Tables are admitted against an HBM budget (tables + per-slot staging).
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

constexpr uint32_t kServeStreams = 4;       // each table's units run in order on one of these
constexpr uint64_t kSlotStaging = 256ull << 20;  // request + reply staging a slot may grow to

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
  int64_t t_arrive;
  void* out;
  uint64_t out_off;  // byte offset of the reply in the slot's reply staging
  uint64_t epoch;
};

struct WriteRec {
  uint64_t tag;
  int64_t t_arrive;
  tpir_status status;
  uint32_t evictions;
  uint64_t epoch;
};

struct Slot {
  cudaEvent_t done = nullptr;
  uint64_t* h_req = nullptr;
  uint64_t h_req_cap = 0;
  uint64_t* d_req = nullptr;
  uint64_t d_req_cap = 0;
  uint8_t* h_out = nullptr;
  uint64_t h_out_cap = 0;
  uint8_t* d_out = nullptr;
  uint64_t d_out_cap = 0;
  uint32_t table = 0;
  uint32_t row_bytes = 0;
  std::vector<ReadRec> reads;
  std::vector<WriteRec> writes;
  tpir_write_staging wstage;  // write batches too large for the kernel parameters
  tpir_write_staging bstage;  // Bloom positions
  int64_t t_launch = 0;
};

struct Table {
  tpir_db* db = nullptr;
  uint64_t bytes = 0;
  std::deque<Op> ops;  // admitted, not yet in a unit (arrival order)
  uint64_t nreads = 0; // reads among them
};

}  // namespace

struct tpir_server {
  tpir_serve_config cfg{};
  int device = 0;
  std::deque<Table> tables;  // stable addresses while tables are added
  uint64_t hbm_tables = 0;
  uint64_t hbm_tcopies = 0;  // bit-transposed copies made for tensor-core reads
  uint64_t staging_reserve = 0;
  cudaStream_t streams[kServeStreams] = {nullptr};

  std::mutex mu;
  std::condition_variable cv_work, cv_idle;
  uint64_t queued = 0;      // ops waiting in the tables' FIFOs
  uint64_t unfinished = 0;  // admitted and not yet completed
  bool stop = false;

  std::vector<Slot> slots;
  std::vector<int> inflight;  // slot indices
  std::vector<int> free_slots;

  std::mutex cmu;
  std::deque<tpir_completion> done;
  // stats
  std::vector<double> lat_ms;
  uint64_t reads_done = 0, writes_done = 0, rejected = 0, failed = 0, launches = 0;
  uint64_t batch_tables = 0, batch_reads = 0;
  uint64_t kernel_launches[6] = {0};
  int64_t t_first = 0, t_last = 0;
  uint64_t ev_hist[8] = {0};

  std::thread worker;
};

namespace {

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
    c.table_id = sl.table;
    c.evictions = w.evictions;
    c.epoch = w.epoch;
    c.t_arrive_ns = w.t_arrive;
    c.t_launch_ns = sl.t_launch;
    c.t_done_ns = t;
    cs.push_back(c);
  }
  for (const ReadRec& r : sl.reads) {
    std::memcpy(r.out, sl.h_out + r.out_off, sl.row_bytes);
    tpir_completion c{};
    c.tag = r.tag;
    c.status = TPIR_OK;
    c.kind = 0;
    c.table_id = sl.table;
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

void fail_reads(tpir_server* s, uint32_t t, const std::vector<Op>& reads, tpir_status why) {
  std::lock_guard<std::mutex> g(s->cmu);
  for (const Op& op : reads) {
    tpir_completion c{};
    c.tag = op.tag;
    c.status = why;
    c.table_id = t;
    c.t_arrive_ns = op.t_arrive;
    c.t_done_ns = now_ns();
    s->done.push_back(c);
    s->failed++;
  }
}

// Forms one launch unit into slot `si`: among the tables whose ops are ready
// (the oldest has waited the batching window, tick_us, or max_batch reads are
// waiting), the one whose oldest waiting op arrived first; all its waiting
// writes and up to max_batch of its reads.  Returns false if no table is
// ready; *next_ready_ns then tells when the earliest one will be (0: none).
bool form_unit(tpir_server* s, int si, int64_t* next_ready_ns) {
  Slot& sl = s->slots[si];
  std::vector<Op> writes, reads;
  uint32_t t = 0;
  Table* tab = nullptr;
  *next_ready_ns = 0;
  {
    std::lock_guard<std::mutex> g(s->mu);
    if (s->queued == 0) return false;
    const int64_t now = now_ns(), window = static_cast<int64_t>(s->cfg.tick_us) * 1000;
    int64_t oldest = INT64_MAX, soonest = INT64_MAX;
    bool found = false;
    for (uint32_t i = 0; i < s->tables.size(); ++i) {
      const Table& x = s->tables[i];
      if (x.ops.empty()) continue;
      const int64_t ta = x.ops.front().t_arrive;
      if (s->stop || now - ta >= window || x.nreads >= s->cfg.max_batch) {
        if (ta < oldest) {
          oldest = ta;
          t = i;
          found = true;
        }
      } else {
        soonest = std::min(soonest, ta + window);
      }
    }
    if (!found) {
      *next_ready_ns = soonest == INT64_MAX ? 0 : soonest;
      return false;
    }
    tab = &s->tables[t];
    std::deque<Op> keep;
    while (!tab->ops.empty()) {
      Op op = std::move(tab->ops.front());
      tab->ops.pop_front();
      if (op.kind == 1)
        writes.push_back(std::move(op));
      else if (reads.size() < s->cfg.max_batch)
        reads.push_back(std::move(op));
      else
        keep.push_back(std::move(op));
    }
    tab->ops.swap(keep);
    tab->nreads -= reads.size();
    s->queued -= writes.size() + reads.size();
  }
  tpir_db* db = tab->db;
  cudaStream_t st = s->streams[t % kServeStreams];
  sl.table = t;
  sl.row_bytes = db->row_bytes;
  sl.t_launch = now_ns();

  // ---- writes, in arrival order
  if (!writes.empty()) {
    const size_t nw = writes.size();
    std::vector<uint64_t> b1(nw), b2(nw), pos;
    std::vector<uint8_t> msgs(nw * db->z);
    for (size_t j = 0; j < nw; ++j) {
      b1[j] = writes[j].b1;
      b2[j] = writes[j].b2;
      std::memcpy(msgs.data() + j * db->z, writes[j].msg.data(), db->z);
    }
    std::vector<tpir_status> stv(nw, TPIR_OK);
    std::vector<uint32_t> ev(nw, 0);
    const uint64_t epoch0 = db->epoch;
    order_writes_after_reads(db, st);
    const tpir_status r = apply_writes_core(db, static_cast<uint32_t>(nw), b1.data(), b2.data(),
                                            msgs.data(), stv.data(), ev.data(), st, sl.wstage);
    uint64_t e = epoch0;
    uint32_t with_bloom = 0;
    for (size_t j = 0; j < nw; ++j) {
      const Op& op = writes[j];
      const tpir_status sj = (r != TPIR_OK) ? r : stv[j];
      if (sj == TPIR_OK) ++e;
      sl.writes.push_back(WriteRec{op.tag, op.t_arrive, sj, r != TPIR_OK ? 0u : ev[j], e});
      if (sj == TPIR_OK && db->bloom.d_deltas && op.bloom.size() == db->bloom.k) {
        pos.insert(pos.end(), op.bloom.begin(), op.bloom.end());
        ++with_bloom;
      }
    }
    if (with_bloom) bloom_insert_core(db, pos.data(), with_bloom, st, sl.bstage);
  }

  // ---- reads: one launch for all of them, after the writes
  if (!reads.empty()) {
    const uint32_t B = static_cast<uint32_t>(reads.size());
    const uint64_t req_bytes = static_cast<uint64_t>(B) * db->words64 * 8;
    const uint64_t out_bytes = static_cast<uint64_t>(B) * db->row_bytes;
    if (!grow_pinned(reinterpret_cast<void**>(&sl.h_req), &sl.h_req_cap, req_bytes) ||
        !grow_dev(reinterpret_cast<void**>(&sl.d_req), &sl.d_req_cap, req_bytes) ||
        !grow_pinned(reinterpret_cast<void**>(&sl.h_out), &sl.h_out_cap, out_bytes) ||
        !grow_dev(reinterpret_cast<void**>(&sl.d_out), &sl.d_out_cap, out_bytes)) {
      fail_reads(s, t, reads, TPIR_ENOMEM);
      std::lock_guard<std::mutex> g(s->mu);
      s->unfinished -= reads.size();
      reads.clear();
    }
    for (uint32_t b = 0; b < reads.size(); ++b) {
      std::memcpy(sl.h_req + static_cast<uint64_t>(b) * db->words64, reads[b].req.data(),
                  db->words64 * 8);
      sl.reads.push_back(ReadRec{reads[b].tag, reads[b].t_arrive, reads[b].out,
                                 static_cast<uint64_t>(b) * db->row_bytes, db->epoch});
    }
    if (!reads.empty()) {
      // the tensor-core kernel reads a bit-transposed copy of the table (as
      // large as the table), made on first use: only if it fits the budget
      int choice = 0;
      if (auto_kernel(db, B) == 5 && !db->d_tt) {
        const uint64_t tt = tcopy_bytes(db->n, db->row_bytes);
        std::lock_guard<std::mutex> g(s->mu);
        if (s->hbm_tables + s->hbm_tcopies + tt + s->staging_reserve <= s->cfg.hbm_budget_bytes)
          s->hbm_tcopies += tt;
        else
          choice = 2;
      }
      int kernel = 0;
      cudaMemcpyAsync(sl.d_req, sl.h_req, req_bytes, cudaMemcpyHostToDevice, st);
      const tpir_status r = enqueue_read(db, sl.d_req, B, sl.d_out, st, nullptr, &kernel, choice);
      cudaMemcpyAsync(sl.h_out, sl.d_out, out_bytes, cudaMemcpyDeviceToHost, st);
      std::lock_guard<std::mutex> g(s->cmu);
      s->launches++;
      s->batch_tables++;
      s->batch_reads += B;
      if (r == TPIR_OK && kernel > 0 && kernel < 6) s->kernel_launches[kernel]++;
    }
  }
  cudaEventRecord(sl.done, st);
  return true;
}

void worker_main(tpir_server* s) {
  cudaSetDevice(s->device);
  for (;;) {
    // retire finished units (units of different tables may finish in any order)
    for (size_t i = 0; i < s->inflight.size();) {
      const int si = s->inflight[i];
      if (cudaEventQuery(s->slots[si].done) == cudaSuccess) {
        retire(s, si);
        s->free_slots.push_back(si);
        s->inflight.erase(s->inflight.begin() + static_cast<long>(i));
      } else {
        ++i;
      }
    }
    bool pending;
    {
      std::lock_guard<std::mutex> g(s->mu);
      pending = s->queued > 0;
      if (s->stop && !pending && s->inflight.empty()) break;
    }
    int64_t next_ready = 0;
    if (pending && !s->free_slots.empty()) {
      const int si = s->free_slots.back();
      s->free_slots.pop_back();
      if (form_unit(s, si, &next_ready)) {
        s->inflight.push_back(si);
        continue;
      }
      s->free_slots.push_back(si);
    }
    if (!s->inflight.empty()) {
      // units are running: poll their completion without burning a core
      std::this_thread::sleep_for(std::chrono::microseconds(10));
      continue;
    }
    // idle: sleep until an op arrives, the earliest waiting table's batching
    // window ends, or the server stops
    std::unique_lock<std::mutex> lk(s->mu);
    const int64_t wait_ns = next_ready ? std::max<int64_t>(next_ready - now_ns(), 1000) : 1000000;
    const uint64_t q0 = s->queued;
    s->cv_work.wait_for(lk, std::chrono::nanoseconds(wait_ns),
                        [&] { return s->stop || s->queued != q0; });
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
  if (!s->cfg.max_inflight) s->cfg.max_inflight = 4;
  if (!s->cfg.queue_capacity) s->cfg.queue_capacity = 65536;
  if (s->cfg.max_batch > 1024 || s->cfg.max_inflight > 16) {
    delete s;
    return TPIR_EINVAL;
  }
  cudaGetDevice(&s->device);
  s->staging_reserve = s->cfg.max_inflight * kSlotStaging;
  if (s->staging_reserve >= s->cfg.hbm_budget_bytes) {
    delete s;
    return TPIR_ENOMEM;
  }
  cudaError_t e = cudaSuccess;
  for (uint32_t i = 0; i < kServeStreams && e == cudaSuccess; ++i)
    e = cudaStreamCreateWithFlags(&s->streams[i], cudaStreamNonBlocking);
  s->slots.resize(s->cfg.max_inflight);
  for (uint32_t i = 0; i < s->cfg.max_inflight && e == cudaSuccess; ++i) {
    e = cudaEventCreateWithFlags(&s->slots[i].done, cudaEventDisableTiming);
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
  if (s->hbm_tables + s->hbm_tcopies + bytes + s->staging_reserve > s->cfg.hbm_budget_bytes)
    return TPIR_ENOMEM;
  tpir_db* db = tpir_db_create(n, d, msg_bytes);
  if (!db) return tpir_last_error();
  s->tables.emplace_back();
  s->tables.back().db = db;
  s->tables.back().bytes = bytes;
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
  s->queued++;
  Table& t = s->tables[op.table];
  if (op.kind == 0) t.nreads++;
  t.ops.push_back(std::move(op));
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
    for (int i = 0; i < 6; ++i) st->kernel_launches[i] = s->kernel_launches[i];
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
    st->hbm_bytes_in_use = s->hbm_tables + s->hbm_tcopies;
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
  for (auto& k : s->kernel_launches) k = 0;
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
  for (cudaStream_t st : s->streams)
    if (st) cudaStreamSynchronize(st);
  for (Slot& sl : s->slots) {
    if (sl.h_req) cudaFreeHost(sl.h_req);
    if (sl.h_out) cudaFreeHost(sl.h_out);
    cudaFree(sl.d_req);
    cudaFree(sl.d_out);
    sl.wstage.release();
    sl.bstage.release();
    if (sl.done) cudaEventDestroy(sl.done);
  }
  for (Table& t : s->tables) tpir_db_destroy(t.db);
  for (cudaStream_t st : s->streams)
    if (st) cudaStreamDestroy(st);
  delete s;
  return TPIR_OK;
}

}  // extern "C"
