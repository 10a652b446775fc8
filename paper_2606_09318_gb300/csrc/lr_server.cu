// lr_server.cu -- continuous-batching request loop of liblr.so.
//
// Requests (one successor array each, host or device memory) are admitted in
// arrival order while their device footprint fits the memory budget.  Each
// of n_streams worker threads owns one CUDA stream: whenever it is idle it
// takes every admitted request that is waiting (up to max_batch requests /
// max_batch_elems elements, same dtypes), ranks them as one forest in a single
// launch sequence that reads and writes each request's own buffers through
// pointer tables, and completes them individually.  Requests that arrive
// while batches run join the next batch of whichever stream frees up first,
// so work from different batches overlaps on the device.  If a batch reports
// a data error, its requests are re-ranked one by one so every request gets
// its own status.
//
// A request of at least alone_min_n elements is a batch of its own: it gains
// nothing from batching, the single-list path takes the size-dependent
// choices the batched form does not (tile-local contraction of Section 2.3,
// the level-0 form), and smaller requests do not wait for it in a batch.
// Every batch of one request is ranked through the single-list path, as
// lr_rank_ex would rank it; in plain mode every batch holds one request.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "lr.h"
#include "lr_engine.h"

namespace {

using Clock = std::chrono::steady_clock;

struct Req {
  uint64_t ticket = 0;
  lr_request r;
  size_t footprint = 0;
  lr_result res;
  bool done = false;
  void *dsucc = nullptr, *dw = nullptr, *drank = nullptr;
};

size_t wbytes(lr_dtype t) { return t == LR_I32 ? 4 : (t == LR_I64 ? 8 : 0); }

// Requests of at least this many elements are ranked alone (single-list
// path: contraction, the log form).  Smaller ones that wait together are
// one batch, chased in element order with its records prefetched into L2,
// which beats ranking requests of up to a few million elements alone on
// concurrent streams, where their footprints add up in L2.
constexpr int64_t kAloneMinDefault = (int64_t)1 << 23;

// Device bytes a request holds while it is resident: its own buffers when
// the server copies them, plus an estimate of its share of the ranking
// workspace (records, bitmap, reduced levels).
size_t footprint(const lr_request &r) {
  const size_t n = (size_t)r.n;
  const size_t io = r.on_device ? 0 : (4 + wbytes(r.wtype) + wbytes(r.rtype)) * n;
  const size_t ws = (r.wtype == LR_NONE ? 8 : 16) * n + n / 8 + n / 2 + (1u << 16);
  return io + ws;
}

}  // namespace

struct lr_server {
  lr_server_config cfg;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<Req *> pending;
  std::unordered_map<uint64_t, Req *> reqs;
  uint64_t next_ticket = 1;
  size_t resident = 0, peak = 0;
  bool stop = false;
  std::vector<std::thread> workers;
  Clock::time_point t0;
  std::vector<double> lat;
  int64_t completed = 0, elements = 0, batches = 0, ranked_alone = 0;
  double first_submit = -1, last_done = 0;

  double now_ms() const {
    return std::chrono::duration<double, std::milli>(Clock::now() - t0).count();
  }
  void worker(int idx);
};

void lr_server::worker(int idx) {
  cudaSetDevice(cfg.device);
  cudaStream_t s;
  if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) return;
  const int maxb = std::max(1, cfg.max_batch);
  // pointer tables: offsets[k+1], sptr[k], wptr[k], rptr[k]
  const size_t tbytes = 8 * (size_t)(maxb + 1) + 3 * 8 * (size_t)maxb;
  char *htab = nullptr, *dtab = nullptr;
  if (cudaMallocHost((void **)&htab, tbytes) != cudaSuccess || cudaMalloc((void **)&dtab, tbytes) != cudaSuccess) {
    return;
  }
  int64_t *hoff = (int64_t *)htab;
  void **hs = (void **)(htab + 8 * (size_t)(maxb + 1));
  void **hw = hs + maxb;
  void **hr = hw + maxb;
  int64_t *doff = (int64_t *)dtab;
  void **ds = (void **)(dtab + 8 * (size_t)(maxb + 1));
  void **dw = ds + maxb;
  void **dr = dw + maxb;
  uint64_t seed = 0x5e71e + (uint64_t)idx;
  const int64_t alone_min = cfg.alone_min_n == 0 ? kAloneMinDefault : cfg.alone_min_n;

  // the request's arrays on the device: the caller's, or the staged copies
  auto dsucc_of = [](Req *q) { return q->r.on_device ? q->r.succ : (const uint32_t *)q->dsucc; };
  auto dw_of = [](Req *q) { return q->r.on_device ? q->r.weight : (const void *)q->dw; };
  auto drank_of = [](Req *q) { return q->r.on_device ? q->r.rank : q->drank; };

  // offsets and pointer tables of b, uploaded on s; returns the element total
  auto fill_tables = [&](std::vector<Req *> &b) -> int64_t {
    const int k = (int)b.size();
    int64_t tot = 0;
    for (int j = 0; j < k; ++j) {
      hoff[j] = tot;
      tot += b[j]->r.n;
      hs[j] = (void *)dsucc_of(b[j]);
      hw[j] = (void *)dw_of(b[j]);
      hr[j] = drank_of(b[j]);
    }
    hoff[k] = tot;
    cudaMemcpyAsync(doff, hoff, 8 * (size_t)(k + 1), cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(ds, hs, 8 * (size_t)k, cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(dw, hw, 8 * (size_t)k, cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(dr, hr, 8 * (size_t)k, cudaMemcpyHostToDevice, s);
    return tot;
  };

  auto run_tables = [&](std::vector<Req *> &b) -> lr_status {
    const int k = (int)b.size();
    const int64_t tot = fill_tables(b);
    if (tot == 0) return LR_OK;
    return lr::run_ptr_batch(doff, k, tot, (const uint32_t *const *)ds, (const void *const *)dw,
                             (void *const *)dr, (int)b[0]->r.wtype, b[0]->r.rtype == LR_I32 ? 4 : 8,
                             seed++, s);
  };

  // one request through the single-list path (waits for its status)
  auto run_alone = [&](Req *q) -> lr_status {
    return lr::run_single(dsucc_of(q), dw_of(q), (int)q->r.wtype, drank_of(q), q->r.rtype == LR_I32 ? 4 : 8,
                          q->r.n, seed++, s);
  };

  for (;;) {
    std::vector<Req *> batch;
    {
      std::unique_lock<std::mutex> g(mu);
      cv_work.wait(g, [&] {
        return stop || (!pending.empty() && resident + pending.front()->footprint <= cfg.budget_bytes);
      });
      if (stop) break;
      int64_t elems = 0;
      const double t = now_ms();
      while (!pending.empty() && (int)batch.size() < maxb) {
        Req *q = pending.front();
        const bool own = cfg.plain || (alone_min >= 0 && q->r.n >= alone_min);
        if (!batch.empty()) {
          if (own) break;   // a large request starts a batch of its own
          if (q->r.wtype != batch[0]->r.wtype || q->r.rtype != batch[0]->r.rtype) break;
          if (elems + q->r.n > cfg.max_batch_elems) break;
        }
        if (resident + q->footprint > cfg.budget_bytes) break;
        pending.pop_front();
        resident += q->footprint;
        peak = std::max(peak, resident);
        q->res.t_admit_ms = t;
        batch.push_back(q);
        elems += q->r.n;
        if (own) break;
      }
    }
    if (batch.empty()) continue;
    // stage host requests into device buffers (stream-ordered pool allocations)
    lr_status stage = LR_OK;
    for (Req *q : batch) {
      if (q->r.on_device || q->r.n == 0) continue;
      const size_t n = (size_t)q->r.n;
      if (cudaMallocAsync(&q->dsucc, 4 * n, s) != cudaSuccess ||
          cudaMallocAsync(&q->drank, wbytes(q->r.rtype) * n, s) != cudaSuccess ||
          (q->r.wtype != LR_NONE && cudaMallocAsync(&q->dw, wbytes(q->r.wtype) * n, s) != cudaSuccess)) {
        cudaGetLastError();
        stage = LR_ERR_OUT_OF_MEMORY;
        break;
      }
      cudaMemcpyAsync(q->dsucc, q->r.succ, 4 * n, cudaMemcpyHostToDevice, s);
      if (q->dw) cudaMemcpyAsync(q->dw, q->r.weight, wbytes(q->r.wtype) * n, cudaMemcpyHostToDevice, s);
    }
    const double tl = now_ms();
    for (Req *q : batch) q->res.t_launch_ms = tl;
    const bool alone = batch.size() == 1;
    if (stage == LR_OK) {
      if (alone) {
        batch[0]->res.status = run_alone(batch[0]);
      } else {
        lr_status st = run_tables(batch);
        if (st == LR_OK) {
          for (Req *q : batch) q->res.status = st;
        } else {
          for (Req *q : batch) q->res.status = run_alone(q);   // attribute the error
        }
      }
      for (Req *q : batch)
        if (!q->r.on_device && q->r.n > 0 && q->res.status == LR_OK)
          cudaMemcpyAsync(q->r.rank, q->drank, wbytes(q->r.rtype) * (size_t)q->r.n, cudaMemcpyDeviceToHost, s);
    } else {
      for (Req *q : batch) q->res.status = stage;
    }
    for (Req *q : batch) {
      if (q->dsucc) cudaFreeAsync(q->dsucc, s);
      if (q->dw) cudaFreeAsync(q->dw, s);
      if (q->drank) cudaFreeAsync(q->drank, s);
      q->dsucc = q->dw = q->drank = nullptr;
    }
    if (cudaStreamSynchronize(s) != cudaSuccess)
      for (Req *q : batch) if (q->res.status == LR_OK) q->res.status = LR_ERR_CUDA;
    {
      std::lock_guard<std::mutex> g(mu);
      const double t = now_ms();
      for (Req *q : batch) {
        resident -= q->footprint;
        q->res.t_done_ms = t;
        q->done = true;
        lat.push_back(t - q->res.t_submit_ms);
        completed += 1;
        elements += q->r.n;
      }
      last_done = t;
      batches += 1;
      ranked_alone += alone ? 1 : 0;
    }
    cv_done.notify_all();
    cv_work.notify_all();
  }
  cudaStreamSynchronize(s);
  cudaFree(dtab);
  cudaFreeHost(htab);
  cudaStreamDestroy(s);
}

extern "C" {

void lr_server_config_default(lr_server_config *c) {
  if (!c) return;
  memset(c, 0, sizeof(*c));
  c->budget_bytes = (size_t)40e9;
  c->n_streams = 4;
  c->max_batch = 256;
  c->max_batch_elems = (int64_t)1 << 28;
  c->device = 0;
  c->plain = 0;
  c->alone_min_n = 0;
}

lr_status lr_server_create(const lr_server_config *cfg, lr_server **out) {
  if (!out) return LR_ERR_INVALID_ARGUMENT;
  *out = nullptr;
  lr_server_config c;
  lr_server_config_default(&c);
  if (cfg) c = *cfg;
  if (c.n_streams <= 0 || c.n_streams > 64 || c.max_batch <= 0 || c.budget_bytes == 0)
    return LR_ERR_INVALID_ARGUMENT;
  if (c.max_batch_elems <= 0 || c.max_batch_elems > LR_MAX_N) c.max_batch_elems = LR_MAX_N;
  if (cudaSetDevice(c.device) != cudaSuccess) return LR_ERR_CUDA;
  // keep freed request buffers in the pool (up to the budget) for reuse
  cudaMemPool_t pool;
  if (cudaDeviceGetDefaultMemPool(&pool, c.device) == cudaSuccess) {
    uint64_t thr = c.budget_bytes;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
  }
  lr_server *s = new lr_server();
  s->cfg = c;
  s->t0 = Clock::now();
  for (int i = 0; i < c.n_streams; ++i) s->workers.emplace_back(&lr_server::worker, s, i);
  *out = s;
  return LR_OK;
}

lr_status lr_server_submit(lr_server *s, const lr_request *req, uint64_t *ticket) {
  if (!s || !req || !ticket) return LR_ERR_INVALID_ARGUMENT;
  if (req->n < 0 || req->n > LR_MAX_N) return LR_ERR_INVALID_ARGUMENT;
  if (req->n > 0 && (!req->succ || !req->rank)) return LR_ERR_INVALID_ARGUMENT;
  if (req->rtype != LR_I32 && req->rtype != LR_I64) return LR_ERR_INVALID_ARGUMENT;
  if ((req->wtype == LR_NONE) != (req->weight == nullptr) && req->n > 0) return LR_ERR_INVALID_ARGUMENT;
  if (req->wtype != LR_NONE && req->wtype != LR_I32 && req->wtype != LR_I64) return LR_ERR_INVALID_ARGUMENT;
  const size_t fp = footprint(*req);
  if (fp > s->cfg.budget_bytes) return LR_ERR_BUDGET;
  Req *q = new Req();
  q->r = *req;
  q->footprint = fp;
  memset(&q->res, 0, sizeof(q->res));
  {
    std::lock_guard<std::mutex> g(s->mu);
    if (s->stop) { delete q; return LR_ERR_CANCELLED; }
    q->ticket = s->next_ticket++;
    q->res.t_submit_ms = s->now_ms();
    if (s->first_submit < 0) s->first_submit = q->res.t_submit_ms;
    s->reqs[q->ticket] = q;
    if (req->n == 0) {
      q->res.status = LR_OK;
      q->res.t_admit_ms = q->res.t_launch_ms = q->res.t_done_ms = q->res.t_submit_ms;
      q->done = true;
    } else {
      s->pending.push_back(q);
    }
    *ticket = q->ticket;
  }
  s->cv_work.notify_one();
  s->cv_done.notify_all();
  return LR_OK;
}

lr_status lr_server_wait(lr_server *s, uint64_t ticket, int64_t timeout_ms, lr_result *res) {
  if (!s) return LR_ERR_INVALID_ARGUMENT;
  std::unique_lock<std::mutex> g(s->mu);
  auto it = s->reqs.find(ticket);
  if (it == s->reqs.end()) return LR_ERR_NOT_FOUND;
  Req *q = it->second;
  auto ready = [&] { return q->done; };
  if (timeout_ms < 0) s->cv_done.wait(g, ready);
  else if (!s->cv_done.wait_for(g, std::chrono::milliseconds(timeout_ms), ready)) return LR_ERR_TIMEOUT;
  if (res) *res = q->res;
  lr_status st = q->res.status;
  s->reqs.erase(it);
  delete q;
  return st;
}

lr_status lr_server_stats_get(lr_server *s, lr_server_stats *out) {
  if (!s || !out) return LR_ERR_INVALID_ARGUMENT;
  std::lock_guard<std::mutex> g(s->mu);
  memset(out, 0, sizeof(*out));
  out->completed = s->completed;
  out->elements = s->elements;
  out->batches = s->batches;
  out->peak_resident_bytes = s->peak;
  out->ranked_alone = s->ranked_alone;
  if (!s->lat.empty()) {
    std::vector<double> v = s->lat;
    std::sort(v.begin(), v.end());
    auto pct = [&](double p) { return v[std::min(v.size() - 1, (size_t)(p * (v.size() - 1) + 0.5))]; };
    out->p50_ms = pct(0.50);
    out->p99_ms = pct(0.99);
    double sum = 0;
    for (double x : v) sum += x;
    out->mean_ms = sum / v.size();
  }
  const double span = s->last_done - std::max(0.0, s->first_submit);
  out->elements_per_s = span > 0 ? s->elements / (span * 1e-3) : 0.0;
  return LR_OK;
}

void lr_server_destroy(lr_server *s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> g(s->mu);
    s->stop = true;
    for (Req *q : s->pending) {
      q->res.status = LR_ERR_CANCELLED;
      q->done = true;
    }
    s->pending.clear();
  }
  s->cv_work.notify_all();
  s->cv_done.notify_all();
  for (auto &t : s->workers) t.join();
  for (auto &kv : s->reqs) delete kv.second;
  delete s;
}

}  // extern "C"
