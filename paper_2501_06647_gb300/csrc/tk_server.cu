// Serving runtime: continuous batching of interleaved range queries and
// stream appends over one tree (host side, one worker thread).
//
// Requests take effect in ticket (arrival) order: a query sees every append
// submitted before it and none submitted after it (Section 3: a stream update
// extends the tensor that later queries range over).  The worker scans the
// queue in order.  An append is issued at once, in stream order, behind the
// batches already running: it never waits for them.  A query joins the batch
// being formed together with the T it was submitted at; the batch is answered
// after the appends scanned before it, each query against its own T (nodes
// that were complete at that T are still stored unchanged, see TkEpoch).  A
// query that reaches into the open block of its T needs that block's current
// decomposition, so the scan stops at the next append and the batch launches
// first.  Batches are bounded by a query count and an output budget (the
// device memory a batch may hold); two batch slots alternate, so the next
// batch is enqueued while the current one runs.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <unordered_set>
#include <vector>

#include "tk_internal.h"

int tk_query_batch_device(tk_tree* t, int n, const int64_t* d_ranges, const int64_t* d_offsets,
                          const int32_t* ranks, void* d_out, tk_query_info* d_info, const int64_t* d_tq,
                          bool need_tail);
cudaStream_t tk_tree_stream(const tk_tree* t);

namespace {

using Clock = std::chrono::steady_clock;

enum { REQ_QUERY = 0, REQ_APPEND = 1 };

struct Req {
  uint64_t ticket = 0;
  int kind = REQ_QUERY;
  int64_t ts = 0, te = 0;
  int32_t ranks[TK_MAX_MODES] = {};
  bool has_ranks = false;
  void* out = nullptr;
  tk_query_info* info = nullptr;
  std::vector<char> slice;
  int64_t elems = 0;  // packed output elements of a query
  Clock::time_point submitted;
};

constexpr int kRing = 16;  // staging slots of appended slices

struct Slot {
  void* d_out = nullptr;
  int64_t* d_meta = nullptr;        // ranges (2n), offsets (n+1), then each query's T (n)
  tk_query_info* d_info = nullptr;
  void* h_out = nullptr;            // pinned
  int64_t* h_meta = nullptr;        // pinned
  tk_query_info* h_info = nullptr;  // pinned
  cudaEvent_t done = nullptr;
  std::vector<Req*> reqs;
  bool busy = false;
};

}  // namespace

struct tk_server {
  tk_tree* t = nullptr;
  tk_config tcfg{};
  tk_server_config cfg{};
  cudaStream_t stream = nullptr;
  size_t es = 4;
  int64_t slice_elems = 0;
  Slot slots[2];
  std::deque<int> busy_fifo;  // slot indices in launch order (worker thread only)
  int64_t T_applied = 0;      // T after the appends issued so far (worker thread only)
  // appended slices go host -> pinned ring -> device ring -> the tree's open block
  void* h_ring = nullptr;
  void* d_ring = nullptr;
  cudaEvent_t ring_ev[kRing] = {};
  int ring_next = 0;

  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<Req*> pending;
  std::unordered_map<uint64_t, int> finished;  // ticket -> status, until collected
  std::unordered_set<uint64_t> inflight;       // submitted, not finished
  uint64_t next_ticket = 1;
  int64_t T_submitted = 0;
  bool stop = false;
  std::thread worker;

  // statistics (guarded by mu)
  std::vector<double> lat_ms;
  int64_t q_done = 0, a_done = 0, batches = 0, batched_queries = 0;
  Clock::time_point first_submit, last_done;
  bool any_submit = false;
};

namespace {

int64_t out_elems_for(const tk_server* s, int64_t L, const int32_t* ranks) {
  const int p = s->tcfg.p;
  int64_t c = 1;
  for (int n = 0; n < p; ++n) c *= ranks[n];
  c += L * ranks[0];
  for (int n = 1; n < p; ++n) c += s->tcfg.dims[n] * ranks[n];
  return c;
}

void finish_locked(tk_server* s, Req* r, int status, Clock::time_point now) {
  s->finished[r->ticket] = status;
  s->inflight.erase(r->ticket);
  if (r->kind == REQ_QUERY) {
    s->lat_ms.push_back(std::chrono::duration<double, std::milli>(now - r->submitted).count());
    ++s->q_done;
  } else {
    ++s->a_done;
  }
  s->last_done = now;
  delete r;
}

// Wait for the slot's batch and hand its outputs to the callers.
void complete_slot(tk_server* s, Slot& sl) {
  const cudaError_t e = cudaEventSynchronize(sl.done);
  const auto now = Clock::now();
  const size_t n = sl.reqs.size();
  std::lock_guard<std::mutex> lk(s->mu);
  for (size_t i = 0; i < n; ++i) {
    Req* r = sl.reqs[i];
    int status = e == cudaSuccess ? TK_OK : TK_ERR_CUDA;
    if (status == TK_OK) {
      const int64_t off = sl.h_meta[2 * n + i];
      std::memcpy(r->out, (char*)sl.h_out + off * s->es, (size_t)r->elems * s->es);
      const tk_query_info& inf = sl.h_info[i];
      if (r->info) *r->info = inf;
      if (inf.iters < 0) status = TK_ERR_WORKSPACE;
    }
    finish_locked(s, r, status, now);
  }
  sl.reqs.clear();
  sl.busy = false;
  s->cv_done.notify_all();
}

// Launch a batch of queries in a free slot (asynchronous).  tq[i] is the T
// query i is answered at; need_tail: some query reaches into the open block.
void launch(tk_server* s, Slot& sl, std::vector<Req*>& batch, const std::vector<int64_t>& tq, bool need_tail) {
  const int n = (int)batch.size();
  int64_t* rng = sl.h_meta;
  int64_t* offs = sl.h_meta + 2 * n;
  int64_t* hq = sl.h_meta + 3 * n + 1;
  offs[0] = 0;
  for (int i = 0; i < n; ++i) {
    rng[2 * i] = batch[i]->ts;
    rng[2 * i + 1] = batch[i]->te;
    offs[i + 1] = offs[i] + batch[i]->elems;
    hq[i] = tq[i];
  }
  // every query of a batch has the same requested ranks (see the batching rule)
  const int32_t* ranks = batch[0]->has_ranks ? batch[0]->ranks : nullptr;
  int rc = cudaMemcpyAsync(sl.d_meta, sl.h_meta, sizeof(int64_t) * (4 * (size_t)n + 1), cudaMemcpyHostToDevice,
                           s->stream) == cudaSuccess ? TK_OK : TK_ERR_CUDA;
  if (rc == TK_OK)
    rc = tk_query_batch_device(s->t, n, sl.d_meta, sl.d_meta + 2 * n, ranks, sl.d_out, sl.d_info,
                               sl.d_meta + 3 * n + 1, need_tail);
  if (rc == TK_OK)
    rc = cudaMemcpyAsync(sl.h_out, sl.d_out, (size_t)offs[n] * s->es, cudaMemcpyDeviceToHost, s->stream) ==
                 cudaSuccess ? TK_OK : TK_ERR_CUDA;
  if (rc == TK_OK)
    rc = cudaMemcpyAsync(sl.h_info, sl.d_info, sizeof(tk_query_info) * (size_t)n, cudaMemcpyDeviceToHost,
                         s->stream) == cudaSuccess ? TK_OK : TK_ERR_CUDA;
  if (rc == TK_OK) rc = cudaEventRecord(sl.done, s->stream) == cudaSuccess ? TK_OK : TK_ERR_CUDA;
  std::lock_guard<std::mutex> lk(s->mu);
  if (rc != TK_OK) {
    const auto now = Clock::now();
    for (Req* r : batch) finish_locked(s, r, rc, now);
    s->cv_done.notify_all();
    return;
  }
  sl.reqs = batch;
  sl.busy = true;
  ++s->batches;
  s->batched_queries += n;
}

// Issue one append on the tree's stream, behind the work already enqueued.
// Its ticket completes once the append is issued: every later query sees it.
void issue_append(tk_server* s, Req* a) {
  const size_t bytes = (size_t)s->slice_elems * s->es;
  const int k = s->ring_next;
  s->ring_next = (k + 1) % kRing;
  char* h = (char*)s->h_ring + (size_t)k * bytes;
  char* d = (char*)s->d_ring + (size_t)k * bytes;
  // the host slot is free once its previous copy has run
  int rc = cudaEventSynchronize(s->ring_ev[k]) == cudaSuccess ? TK_OK : TK_ERR_CUDA;
  if (rc == TK_OK) {
    std::memcpy(h, a->slice.data(), bytes);
    rc = cudaMemcpyAsync(d, h, bytes, cudaMemcpyHostToDevice, s->stream) == cudaSuccess ? TK_OK : TK_ERR_CUDA;
  }
  if (rc == TK_OK) rc = cudaEventRecord(s->ring_ev[k], s->stream) == cudaSuccess ? TK_OK : TK_ERR_CUDA;
  if (rc == TK_OK) rc = tk_stream_append(s->t, d, TK_IO_DEVICE);
  if (rc == TK_OK) s->T_applied += 1;
  std::lock_guard<std::mutex> lk(s->mu);
  finish_locked(s, a, rc, Clock::now());
  s->cv_done.notify_all();
}

bool same_ranks(const Req* a, const Req* b) {
  if (a->has_ranks != b->has_ranks) return false;
  return !a->has_ranks || std::memcmp(a->ranks, b->ranks, sizeof(a->ranks)) == 0;
}

void run(tk_server* s) {
  cudaSetDevice(s->tcfg.device);
  const int64_t B = s->tcfg.leaf_slices;
  while (true) {
    std::vector<Req*> apps, batch;
    std::vector<int64_t> tq;
    bool need_tail = false;
    int free_idx = -1;
    {
      std::unique_lock<std::mutex> lk(s->mu);
      const bool any_busy = !s->busy_fifo.empty();
      if (s->pending.empty() && !any_busy) {
        if (s->stop) break;
        s->cv_work.wait(lk, [&] { return s->stop || !s->pending.empty(); });
        continue;
      }
      if (!s->slots[0].busy) free_idx = 0;
      else if (!s->slots[1].busy) free_idx = 1;
      // scan the queue in ticket order (see the header comment)
      int64_t T = s->T_applied;
      int64_t elems = 0;
      while (!s->pending.empty()) {
        Req* r = s->pending.front();
        if (r->kind == REQ_APPEND) {
          if (need_tail) break;
          apps.push_back(r);
          s->pending.pop_front();
          ++T;
          continue;
        }
        if (free_idx < 0 || (int)batch.size() >= s->cfg.max_batch) break;
        if (!batch.empty() && (!same_ranks(r, batch[0]) || elems + r->elems > s->cfg.max_batch_out_elems)) break;
        elems += r->elems;
        if (T % B != 0 && r->te > T / B * B) need_tail = true;
        batch.push_back(r);
        tq.push_back(T);
        s->pending.pop_front();
      }
    }
    for (Req* a : apps) issue_append(s, a);
    if (!batch.empty()) {
      launch(s, s->slots[free_idx], batch, tq, need_tail);
      if (s->slots[free_idx].busy) s->busy_fifo.push_back(free_idx);
      continue;
    }
    if (!apps.empty() || s->busy_fifo.empty()) continue;
    Slot& oldest = s->slots[s->busy_fifo.front()];
    if (free_idx >= 0 && cudaEventQuery(oldest.done) == cudaErrorNotReady) {
      // A slot is free and the oldest batch still runs: with nothing queued,
      // wait briefly for arrivals so that they can be enqueued behind it.
      std::unique_lock<std::mutex> lk(s->mu);
      if (s->pending.empty() && !s->stop) {
        s->cv_work.wait_for(lk, std::chrono::microseconds(50));
        continue;
      }
    }
    complete_slot(s, oldest);
    s->busy_fifo.pop_front();
  }
}

void free_ring(tk_server* s) {
  if (s->h_ring) cudaFreeHost(s->h_ring);
  if (s->d_ring) cudaFree(s->d_ring);
  for (int k = 0; k < kRing; ++k)
    if (s->ring_ev[k]) cudaEventDestroy(s->ring_ev[k]);
  s->h_ring = s->d_ring = nullptr;
  for (int k = 0; k < kRing; ++k) s->ring_ev[k] = nullptr;
}

void free_slot(Slot& sl) {
  if (sl.d_out) cudaFree(sl.d_out);
  if (sl.d_meta) cudaFree(sl.d_meta);
  if (sl.d_info) cudaFree(sl.d_info);
  if (sl.h_out) cudaFreeHost(sl.h_out);
  if (sl.h_meta) cudaFreeHost(sl.h_meta);
  if (sl.h_info) cudaFreeHost(sl.h_info);
  if (sl.done) cudaEventDestroy(sl.done);
  sl = Slot{};
}

}  // namespace

extern "C" {

int tk_server_create(tk_tree* t, const tk_server_config* cfg, tk_server** out) {
  if (!t || !out) return TK_ERR_ARG;
  *out = nullptr;
  tk_server_config c{};
  c.max_batch = 1024;
  c.max_batch_out_elems = (int64_t)16 << 20;
  if (cfg) {
    if (cfg->max_batch > 0) c.max_batch = cfg->max_batch;
    if (cfg->max_batch_out_elems > 0) c.max_batch_out_elems = cfg->max_batch_out_elems;
  }
  tk_server* s = new (std::nothrow) tk_server();
  if (!s) return TK_ERR_NOMEM;
  s->t = t;
  s->cfg = c;
  tk_tree_get_config(t, &s->tcfg);
  s->stream = tk_tree_stream(t);
  s->es = s->tcfg.dtype == TK_F64 ? 8 : 4;
  s->T_submitted = tk_timespan(t);
  s->T_applied = s->T_submitted;
  s->slice_elems = 1;
  for (int n = 1; n < s->tcfg.p; ++n) s->slice_elems *= s->tcfg.dims[n];
  cudaSetDevice(s->tcfg.device);
  bool ok = true;
  for (Slot& sl : s->slots) {
    const size_t nb = (size_t)c.max_batch;
    ok = ok && cudaMalloc(&sl.d_out, (size_t)c.max_batch_out_elems * s->es) == cudaSuccess;
    ok = ok && cudaMalloc((void**)&sl.d_meta, sizeof(int64_t) * (4 * nb + 1)) == cudaSuccess;
    ok = ok && cudaMalloc((void**)&sl.d_info, sizeof(tk_query_info) * nb) == cudaSuccess;
    ok = ok && cudaMallocHost(&sl.h_out, (size_t)c.max_batch_out_elems * s->es) == cudaSuccess;
    ok = ok && cudaMallocHost((void**)&sl.h_meta, sizeof(int64_t) * (4 * nb + 1)) == cudaSuccess;
    ok = ok && cudaMallocHost((void**)&sl.h_info, sizeof(tk_query_info) * nb) == cudaSuccess;
    ok = ok && cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming) == cudaSuccess;
  }
  const size_t ring_bytes = (size_t)kRing * s->slice_elems * s->es;
  ok = ok && cudaMallocHost(&s->h_ring, ring_bytes) == cudaSuccess;
  ok = ok && cudaMalloc(&s->d_ring, ring_bytes) == cudaSuccess;
  for (int k = 0; k < kRing; ++k)
    ok = ok && cudaEventCreateWithFlags(&s->ring_ev[k], cudaEventDisableTiming) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    for (Slot& sl : s->slots) free_slot(sl);
    free_ring(s);
    delete s;
    return TK_ERR_NOMEM;
  }
  s->worker = std::thread(run, s);
  *out = s;
  return TK_OK;
}

int tk_server_submit_query(tk_server* s, int64_t t_s, int64_t t_e, const int32_t* ranks, void* out_host,
                           tk_query_info* info_host, uint64_t* ticket) {
  if (!s || !out_host) return TK_ERR_ARG;
  Req* r = new (std::nothrow) Req();
  if (!r) return TK_ERR_NOMEM;
  r->kind = REQ_QUERY;
  r->ts = t_s;
  r->te = t_e;
  if (ranks) {
    r->has_ranks = true;
    for (int n = 0; n < s->tcfg.p; ++n) {
      if (ranks[n] < 1 || ranks[n] > s->tcfg.ranks[n]) {
        delete r;
        return TK_ERR_RANK;
      }
      r->ranks[n] = ranks[n];
    }
  }
  r->out = out_host;
  r->info = info_host;
  r->elems = out_elems_for(s, t_e - t_s, ranks ? r->ranks : s->tcfg.ranks);
  if (r->elems > s->cfg.max_batch_out_elems) {
    delete r;
    return TK_ERR_TOO_BIG;
  }
  std::lock_guard<std::mutex> lk(s->mu);
  if (!(t_s >= 0 && t_s < t_e && t_e <= s->T_submitted)) {
    delete r;
    return TK_ERR_RANGE;
  }
  r->ticket = s->next_ticket++;
  r->submitted = Clock::now();
  if (!s->any_submit) {
    s->any_submit = true;
    s->first_submit = r->submitted;
  }
  if (ticket) *ticket = r->ticket;
  s->inflight.insert(r->ticket);
  s->pending.push_back(r);
  s->cv_work.notify_one();
  return TK_OK;
}

int tk_server_submit_append(tk_server* s, const void* slice_host, uint64_t* ticket) {
  if (!s || !slice_host) return TK_ERR_ARG;
  Req* r = new (std::nothrow) Req();
  if (!r) return TK_ERR_NOMEM;
  r->kind = REQ_APPEND;
  r->slice.assign((const char*)slice_host, (const char*)slice_host + s->slice_elems * s->es);
  std::lock_guard<std::mutex> lk(s->mu);
  r->ticket = s->next_ticket++;
  r->submitted = Clock::now();
  if (!s->any_submit) {
    s->any_submit = true;
    s->first_submit = r->submitted;
  }
  s->T_submitted += 1;
  if (ticket) *ticket = r->ticket;
  s->inflight.insert(r->ticket);
  s->pending.push_back(r);
  s->cv_work.notify_one();
  return TK_OK;
}

int tk_server_wait(tk_server* s, uint64_t ticket, double timeout_s) {
  if (!s) return TK_ERR_ARG;
  std::unique_lock<std::mutex> lk(s->mu);
  if (!s->finished.count(ticket) && !s->inflight.count(ticket)) return TK_ERR_ARG;  // unknown or collected
  const auto pred = [&] { return s->finished.count(ticket) != 0; };
  if (timeout_s < 0) s->cv_done.wait(lk, pred);
  else if (!s->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), pred)) return TK_ERR_TIMEOUT;
  const int st = s->finished[ticket];
  s->finished.erase(ticket);
  return st;
}

int tk_server_drain(tk_server* s, double timeout_s) {
  if (!s) return TK_ERR_ARG;
  std::unique_lock<std::mutex> lk(s->mu);
  const auto pred = [&] { return s->pending.empty() && s->q_done + s->a_done + 1 == (int64_t)s->next_ticket; };
  if (timeout_s < 0) s->cv_done.wait(lk, pred);
  else if (!s->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), pred)) return TK_ERR_TIMEOUT;
  return TK_OK;
}

int tk_server_get_stats(tk_server* s, tk_server_stats* out) {
  if (!s || !out) return TK_ERR_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  std::memset(out, 0, sizeof(*out));
  out->queries_done = s->q_done;
  out->appends_done = s->a_done;
  out->batches = s->batches;
  out->mean_batch = s->batches ? (double)s->batched_queries / (double)s->batches : 0.0;
  std::vector<double> v = s->lat_ms;
  if (!v.empty()) {
    std::sort(v.begin(), v.end());
    out->latency_p50_ms = v[v.size() / 2];
    out->latency_p99_ms = v[std::min(v.size() - 1, (size_t)(0.99 * (double)v.size()))];
    out->latency_max_ms = v.back();
  }
  if (s->any_submit && (s->q_done + s->a_done) > 0)
    out->elapsed_s = std::chrono::duration<double>(s->last_done - s->first_submit).count();
  return TK_OK;
}

void tk_server_destroy(tk_server* s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->cv_work.notify_all();
  if (s->worker.joinable()) s->worker.join();
  cudaSetDevice(s->tcfg.device);
  cudaStreamSynchronize(s->stream);
  for (Slot& sl : s->slots) free_slot(sl);
  free_ring(s);
  for (Req* r : s->pending) delete r;
  delete s;
}

}  // extern "C"
