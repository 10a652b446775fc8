// lr_pipeline.cu -- host-buffer pipeline (lr_pipeline_* of the C ABI).
//
// Ranking a host-resident list costs one copy in, the ranking, and one copy
// out; on GB300 the copies of a 2^28-element list take about half as long as
// its ranking.  A pipeline hides them behind the rankings of the
// neighbouring submissions:
//
//   up      stream: copy-in of submission j into slot q = j % depth
//   comp[s] stream: ranking of submission j, s = j % ncomp
//   down    stream: copy-out of submission j
//
// with events per slot:
//   in_ready[q]  copy-in of j done            -> ranking of j may start
//   ranked[q]    ranking of j done            -> copy-out of j may start;
//                                                copy-in of j + depth may overwrite the inputs
//   out_free[q]  copy-out of j done           -> ranking of j + depth may overwrite the ranks
//
// With depth >= 3 two rankings run at once on two streams (ncomp = 2): one
// list's chase, bound by the random-access rate, overlaps the other's
// streaming and partition passes, bound by the SMs, and two 2^28-element
// rankings finish in 0.89 of the time of one after the other.  With depth 2
// rankings run one after another (there is no third slot to copy into while
// two rankings hold theirs).  After every ranking a host function on its
// stream reads the status word the engine copied into that stream's pinned
// context memory and records a failure with its submission index.
#include <atomic>
#include <cstring>
#include <cuda_runtime.h>

#include "lr.h"
#include "lr_engine.h"

namespace {

constexpr int kMaxDepth = 4;

size_t round_up(size_t x) { return (x + 255) & ~(size_t)255; }

lr_status cuda_status(cudaError_t e) {
  if (e == cudaSuccess) return LR_OK;
  cudaGetLastError();
  return e == cudaErrorMemoryAllocation ? LR_ERR_OUT_OF_MEMORY : LR_ERR_CUDA;
}

}  // namespace

constexpr int kMaxComp = 2;

struct lr_pipeline;
struct CompLane {                         // one ranking stream and what belongs to it
  lr_pipeline *p = nullptr;
  int index = 0;                          // s
  cudaStream_t stream = nullptr;
  lr::Ctx *ctx = nullptr;                 // engine context of `stream`
  void *ws = nullptr;                     // engine workspace (with a list bound)
  std::atomic<int64_t> completed{0};      // rankings on this stream since the last wait
};

struct lr_pipeline {
  int device = 0;
  lr_opts opts;
  int64_t max_n = 0;
  int depth = 2;
  int ncomp = 1;
  size_t wbytes = 0, rbytes = 0;          // per element
  size_t off_w = 0, off_r = 0, slot_bytes = 0;
  char *slots = nullptr;
  size_t ws_bytes = 0;
  cudaStream_t up = nullptr, down = nullptr;
  CompLane comp[kMaxComp];
  cudaEvent_t in_ready[kMaxDepth] = {}, ranked[kMaxDepth] = {}, out_free[kMaxDepth] = {};
  int64_t total = 0;                      // submissions ever (slot selection)
  int64_t since_wait = 0;                 // submissions since the last wait (stream selection)
  std::atomic<int64_t> first_fail{-1};    // lowest failing index since the last wait
  std::atomic<uint32_t> fail_bits{0};
};

// Runs on the driver's callback thread, in the order of its stream, after
// each ranking on it.  Submission k (counted from the last wait) ranks on
// stream k % ncomp, so the i-th ranking a stream completes is submission
// i * ncomp + s.
static void CUDART_CB pipeline_ranked(void *arg) {
  CompLane *c = static_cast<CompLane *>(arg);
  lr_pipeline *p = c->p;
  const uint32_t bits = c->ctx->host_words[0];
  c->ctx->host_words[0] = 0;
  const int64_t idx = c->completed.fetch_add(1) * p->ncomp + c->index;
  if (bits != 0) {
    int64_t cur = p->first_fail.load();
    while ((cur < 0 || idx < cur) && !p->first_fail.compare_exchange_weak(cur, idx)) {
    }
    if (p->first_fail.load() == idx) p->fail_bits.store(bits);
  }
}

static void pipeline_free(lr_pipeline *p) {
  if (p->up) cudaStreamSynchronize(p->up);
  for (int s = 0; s < kMaxComp; ++s) {
    if (!p->comp[s].stream) continue;
    lr::release_ctx(p->comp[s].stream);
    cudaStreamSynchronize(p->comp[s].stream);
  }
  if (p->down) cudaStreamSynchronize(p->down);
  for (int q = 0; q < kMaxDepth; ++q) {
    if (p->in_ready[q]) cudaEventDestroy(p->in_ready[q]);
    if (p->ranked[q]) cudaEventDestroy(p->ranked[q]);
    if (p->out_free[q]) cudaEventDestroy(p->out_free[q]);
  }
  if (p->up) cudaStreamDestroy(p->up);
  for (int s = 0; s < kMaxComp; ++s) {
    if (p->comp[s].stream) cudaStreamDestroy(p->comp[s].stream);
    if (p->comp[s].ws) cudaFree(p->comp[s].ws);
  }
  if (p->down) cudaStreamDestroy(p->down);
  if (p->slots) cudaFree(p->slots);
  delete p;
}

extern "C" lr_status lr_pipeline_create(int64_t max_n, const lr_opts *opts, int32_t depth,
                                        lr_pipeline **out) {
  if (!out) return LR_ERR_INVALID_ARGUMENT;
  *out = nullptr;
  if (max_n <= 0 || max_n > LR_MAX_N) return LR_ERR_INVALID_ARGUMENT;
  if (depth == 0) depth = 2;
  if (depth < 2 || depth > kMaxDepth) return LR_ERR_INVALID_ARGUMENT;
  lr_opts o;
  if (opts) o = *opts;
  else lr_opts_default(&o);
  if (o.workspace != nullptr || o.max_lists < 0) return LR_ERR_INVALID_ARGUMENT;
  if (o.wtype != LR_NONE && o.wtype != LR_I32 && o.wtype != LR_I64) return LR_ERR_INVALID_ARGUMENT;
  if (o.rtype != LR_I32 && o.rtype != LR_I64) return LR_ERR_INVALID_ARGUMENT;
  if (o.rtype == LR_I32 && max_n >= ((int64_t)1 << 31)) return LR_ERR_INVALID_ARGUMENT;
  lr_status st = lr::setup_device_once();
  if (st != LR_OK) return st;

  lr_pipeline *p = new lr_pipeline();
  cudaGetDevice(&p->device);
  o.sync = 0;
  o.n_total = 0;
  p->opts = o;
  p->max_n = max_n;
  p->depth = depth;
  p->ncomp = depth >= 3 ? 2 : 1;
  p->wbytes = o.wtype == LR_NONE ? 0 : (o.wtype == LR_I32 ? 4 : 8);
  p->rbytes = o.rtype == LR_I32 ? 4 : 8;
  const size_t n = (size_t)max_n;
  p->off_w = round_up(4 * n);
  p->off_r = p->off_w + round_up(p->wbytes * n);
  p->slot_bytes = p->off_r + round_up(p->rbytes * n);
  // With a bound on the lists the workspace is allocated here and no
  // submission allocates or waits; without one every submission counts its
  // lists first and the engine sizes its own buffers from the count.
  p->ws_bytes = o.max_lists > 0 ? lr_workspace_size(max_n, 0, &o) : 0;

  cudaError_t e = cudaStreamCreateWithFlags(&p->up, cudaStreamNonBlocking);
  for (int s = 0; s < p->ncomp && e == cudaSuccess; ++s) {
    p->comp[s].p = p;
    p->comp[s].index = s;
    e = cudaStreamCreateWithFlags(&p->comp[s].stream, cudaStreamNonBlocking);
    if (e == cudaSuccess && p->ws_bytes) e = cudaMalloc(&p->comp[s].ws, p->ws_bytes);
  }
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&p->down, cudaStreamNonBlocking);
  for (int q = 0; q < depth && e == cudaSuccess; ++q) {
    e = cudaEventCreateWithFlags(&p->in_ready[q], cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p->ranked[q], cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p->out_free[q], cudaEventDisableTiming);
  }
  if (e == cudaSuccess) e = cudaMalloc((void **)&p->slots, p->slot_bytes * depth);
  if (e != cudaSuccess) {
    st = cuda_status(e);
    pipeline_free(p);
    return st;
  }
  for (int s = 0; s < p->ncomp; ++s) {
    p->comp[s].ctx = lr::get_ctx(p->comp[s].stream, &st);
    if (!p->comp[s].ctx) {
      pipeline_free(p);
      return st;
    }
  }
  p->opts.ws_bytes = p->ws_bytes;        // each ranking stream's own workspace (NULL without a bound)
  *out = p;
  return LR_OK;
}

extern "C" lr_status lr_pipeline_submit(lr_pipeline *p, const uint32_t *succ_host,
                                        const void *weight_host, int64_t n, void *rank_host) {
  if (!p) return LR_ERR_INVALID_ARGUMENT;
  if (n < 0 || n > p->max_n) return LR_ERR_INVALID_ARGUMENT;
  if (n > 0 && (!succ_host || !rank_host)) return LR_ERR_INVALID_ARGUMENT;
  if (n > 0 && ((weight_host != nullptr) != (p->wbytes != 0))) return LR_ERR_INVALID_ARGUMENT;
  int cur = 0;
  if (cudaGetDevice(&cur) != cudaSuccess) return LR_ERR_CUDA;
  if (cur != p->device) return LR_ERR_INVALID_ARGUMENT;
  const int q = (int)(p->total % p->depth);
  const bool reused = p->total >= p->depth;
  CompLane &c = p->comp[p->since_wait % p->ncomp];
  char *slot = p->slots + (size_t)q * p->slot_bytes;
  uint32_t *dsucc = reinterpret_cast<uint32_t *>(slot);
  void *dw = p->wbytes ? slot + p->off_w : nullptr;
  void *drank = slot + p->off_r;
  cudaError_t e = cudaSuccess;
  if (n > 0) {
    // copy-in: the slot's inputs are free once submission j - depth is ranked
    if (reused) e = cudaStreamWaitEvent(p->up, p->ranked[q], 0);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dsucc, succ_host, 4 * (size_t)n, cudaMemcpyHostToDevice, p->up);
    if (e == cudaSuccess && dw)
      e = cudaMemcpyAsync(dw, weight_host, p->wbytes * (size_t)n, cudaMemcpyHostToDevice, p->up);
    if (e == cudaSuccess) e = cudaEventRecord(p->in_ready[q], p->up);
    // ranking: after the copy-in, and after submission j - depth left the slot's ranks
    if (e == cudaSuccess) e = cudaStreamWaitEvent(c.stream, p->in_ready[q], 0);
    if (e == cudaSuccess && reused) e = cudaStreamWaitEvent(c.stream, p->out_free[q], 0);
    if (e != cudaSuccess) return cuda_status(e);
    lr_opts o = p->opts;
    o.workspace = c.ws;
    const lr_status st = lr_rank_ex(dsucc, dw, n, drank, &o, (lr_stream)c.stream);
    if (st != LR_OK) return st;
  }
  e = cudaLaunchHostFunc(c.stream, pipeline_ranked, &c);
  if (e == cudaSuccess) e = cudaEventRecord(p->ranked[q], c.stream);
  if (e == cudaSuccess && n > 0) {
    // copy-out after the ranking
    e = cudaStreamWaitEvent(p->down, p->ranked[q], 0);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(rank_host, drank, p->rbytes * (size_t)n, cudaMemcpyDeviceToHost, p->down);
  }
  if (e == cudaSuccess) e = cudaEventRecord(p->out_free[q], p->down);
  if (e != cudaSuccess) return cuda_status(e);
  p->total += 1;
  p->since_wait += 1;
  return LR_OK;
}

extern "C" lr_status lr_pipeline_wait(lr_pipeline *p, int64_t *failed_index) {
  if (failed_index) *failed_index = -1;
  if (!p) return LR_ERR_INVALID_ARGUMENT;
  cudaError_t e = cudaStreamSynchronize(p->up);
  for (int s = 0; s < p->ncomp; ++s) {
    const cudaError_t e2 = cudaStreamSynchronize(p->comp[s].stream);
    if (e == cudaSuccess) e = e2;
  }
  const cudaError_t e3 = cudaStreamSynchronize(p->down);
  if (e == cudaSuccess) e = e3;
  const int64_t fail = p->first_fail.load();
  const uint32_t bits = p->fail_bits.load();
  int64_t done = 0;
  for (int s = 0; s < p->ncomp; ++s) done += p->comp[s].completed.load();
  const int64_t expect = p->since_wait;
  p->since_wait = 0;
  for (int s = 0; s < p->ncomp; ++s) p->comp[s].completed.store(0);
  p->first_fail.store(-1);
  p->fail_bits.store(0);
  if (e != cudaSuccess) return cuda_status(e);
  if (done != expect) return LR_ERR_CUDA;
  if (fail >= 0) {
    if (failed_index) *failed_index = fail;
    return lr::status_from_bits(bits);
  }
  return LR_OK;
}

extern "C" void lr_pipeline_destroy(lr_pipeline *p) {
  if (!p) return;
  pipeline_free(p);
}
