// lr_tune.cu -- autotuner for the ruling-set recursion (lr_autotune*).
//
// The best ruler fraction, base-case cutoff and chase launch shape depend on
// the list size, the weights and whether the input is a batch: small lists
// are bound by the latency of one segment's dependent exchanges, large ones
// by the random-access rate (see the level-0 chase).  lr_autotune measures
// candidates on the device, by coordinate descent from the built-in
// defaults:
//   1. level-0 ruler fraction 1/f0 in {4, 8, 16, 32, 64, 128},
//   2. deeper fraction 1/f in {4, 8, 16},
//   3. base-case cutoff in {4096, 8192, 12288},
//   4. chase block 128 / 256 / 512 threads,
//   5. level-0 fraction again next to the best,
// each timed as the fastest of a few calls with CUDA events, and checks that
// the winner's ranks equal the defaults' bit for bit.  The winner is kept in
// a table keyed by (floor(log2 n), weighted, batched); calls that pass no
// tuning use the entry of their key.  The table is saved and loaded as JSON
// (lr_autotune_save / _load; LR_TUNING_FILE is loaded on first use).
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>
#include <cuda_runtime.h>

#include "lr.h"
#include "lr_device.cuh"
#include "lr_engine.h"
#include "lr_kernels.h"

namespace lr {

namespace {

std::mutex g_tmu;
std::vector<lr_tune_entry> g_table;
bool g_env_loaded = false;

int log2_floor(int64_t n) {
  int b = 0;
  while (b < 62 && ((int64_t)1 << (b + 1)) <= n) ++b;
  return b;
}

bool same_key(const lr_tune_entry &e, int lg, int w, int b) {
  return e.log2n == lg && e.weighted == w && e.batch == b;
}

void put_entry(const lr_tune_entry &e) {
  for (auto &x : g_table)
    if (same_key(x, e.log2n, e.weighted, e.batch)) { x = e; return; }
  g_table.push_back(e);
}

// ---- JSON (this table's own flat format; one object per entry)
const char *kKeys[] = {"log2n", "weighted", "batch", "f0_inv", "f_inv", "cutoff",
                       "chase_block", "chase_ctas", "algorithm", "ms"};

bool find_number(const std::string &obj, const char *key, double *v) {
  const std::string k = std::string("\"") + key + "\"";
  size_t p = obj.find(k);
  if (p == std::string::npos) return false;
  p = obj.find(':', p + k.size());
  if (p == std::string::npos) return false;
  char *end = nullptr;
  *v = strtod(obj.c_str() + p + 1, &end);
  return end != obj.c_str() + p + 1;
}

lr_status load_file(const char *path) {
  FILE *f = fopen(path, "rb");
  if (!f) return LR_ERR_NOT_FOUND;
  std::string s;
  char buf[4096];
  size_t got;
  while ((got = fread(buf, 1, sizeof(buf), f)) > 0) s.append(buf, got);
  fclose(f);
  const size_t a = s.find("\"entries\"");
  if (a == std::string::npos) return LR_ERR_INVALID_ARGUMENT;
  size_t p = s.find('[', a);
  if (p == std::string::npos) return LR_ERR_INVALID_ARGUMENT;
  std::vector<lr_tune_entry> got_entries;
  for (;;) {
    const size_t o = s.find('{', p);
    const size_t c = o == std::string::npos ? o : s.find('}', o);
    if (o == std::string::npos || c == std::string::npos) break;
    const std::string obj = s.substr(o, c - o + 1);
    double v[10];
    for (int i = 0; i < 10; ++i)
      if (!find_number(obj, kKeys[i], &v[i])) return LR_ERR_INVALID_ARGUMENT;
    lr_tune_entry e;
    memset(&e, 0, sizeof(e));
    e.log2n = (int32_t)v[0];
    e.weighted = (int32_t)v[1];
    e.batch = (int32_t)v[2];
    e.tuning.f0_inv = (uint32_t)v[3];
    e.tuning.f_inv = (uint32_t)v[4];
    e.tuning.cutoff = (uint32_t)v[5];
    e.tuning.chase_block = (uint32_t)v[6];
    e.tuning.chase_ctas = (uint32_t)v[7];
    e.tuning.algorithm = (uint32_t)v[8];
    e.ms = (float)v[9];
    if (e.log2n < 0 || e.log2n > 40 || e.tuning.algorithm > LR_ALGO_WYLLIE) return LR_ERR_INVALID_ARGUMENT;
    got_entries.push_back(e);
    p = c + 1;
  }
  for (auto &e : got_entries) put_entry(e);
  return LR_OK;
}

void load_env_once() {
  if (g_env_loaded) return;
  g_env_loaded = true;
  const char *path = getenv("LR_TUNING_FILE");
  if (path && *path) load_file(path);
}

// ---- synthetic inputs on the device: one random-order list per instance
// (a seeded bijection of each instance's positions), weights from a hash
__global__ void k_tune_input(uint32_t *succ, void *w, int wbytes, int64_t *offsets, uint32_t n,
                             int32_t k, uint64_t seed) {
  const uint32_t per = k > 0 ? (uint32_t)(((uint64_t)n + k - 1) / k) : n;
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const uint32_t j = k > 0 ? i / per : 0u;                  // instance of i
    const uint32_t base = j * per;
    const uint32_t len = min(per, n - base);
    Perm P;
    P.init(len, seed + j);
    const uint32_t p = P.fwd(i - base);
    const uint32_t s = p + 1 == len ? i - base : P.inv(p + 1);
    succ[i] = k > 0 ? s : base + s;                           // batch form: local ids
    if (w) {
      const long long v = (long long)(splitmix64(seed ^ (0x9E37ull * i)) % 2001) - 1000;
      if (wbytes == 4) reinterpret_cast<int *>(w)[i] = (int)v;
      else reinterpret_cast<long long *>(w)[i] = v;
    }
  }
  if (k > 0 && blockIdx.x == 0)
    for (int32_t j = threadIdx.x; j <= k; j += blockDim.x)
      offsets[j] = (uint64_t)j * per < n ? (int64_t)((uint64_t)j * per) : (int64_t)n;
}

__global__ void k_tune_diff(const unsigned char *a, const unsigned char *b, size_t bytes,
                            unsigned long long *bad) {
  unsigned long long d = 0;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < bytes; i += (size_t)gridDim.x * blockDim.x)
    d += a[i] != b[i];
  if (d) atomicAdd(bad, d);
}

struct TuneRun {
  const uint32_t *succ;
  const void *weight;
  const int64_t *offsets;
  int64_t n;
  int32_t k;
  lr_opts opts;
  void *rank;
  cudaStream_t s;
  cudaEvent_t e0, e1;
  lr_status err = LR_OK;

  lr_status call(const lr_tuning *t, void *out) {
    lr_opts o = opts;
    o.tuning = t;
    o.sync = 0;
    if (k > 0) return lr_rank_batch_ex(offsets, succ, weight, out, k, &o, (lr_stream)s);
    return lr_rank_ex(succ, weight, n, out, &o, (lr_stream)s);
  }
  // fastest of `reps` timed calls after one warm-up; +inf on any error
  float time(const lr_tuning &t, int reps) {
    float best = INFINITY;
    if (call(&t, rank) != LR_OK || device_status(s) != LR_OK) return best;
    for (int r = 0; r < reps; ++r) {
      cudaEventRecord(e0, s);
      const lr_status st = call(&t, rank);
      cudaEventRecord(e1, s);
      if (st != LR_OK || device_status(s) != LR_OK) return INFINITY;
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      best = std::min(best, ms);
    }
    return best;
  }
};

}  // namespace

// Entry for a call of this shape, if one was tuned (used by resolve_tuning).
bool tuned_lookup(int64_t n, bool weighted, bool batch, lr_tuning *out) {
  std::lock_guard<std::mutex> g(g_tmu);
  load_env_once();
  const int lg = log2_floor(n);
  for (auto &e : g_table)
    if (same_key(e, lg, weighted ? 1 : 0, batch ? 1 : 0)) { *out = e.tuning; return true; }
  return false;
}

}  // namespace lr

using namespace lr;

extern "C" lr_status lr_autotune(const uint32_t *succ, const void *weight, const int64_t *offsets,
                                 int64_t n_total, int32_t k, const lr_opts *opts, lr_stream stream,
                                 lr_tuning *out) {
  if (n_total <= 0 || n_total > LR_MAX_N || k < 0) return LR_ERR_INVALID_ARGUMENT;
  if (k > 0 && succ && !offsets) return LR_ERR_INVALID_ARGUMENT;
  if (succ == nullptr && n_total > ((int64_t)1 << 31)) return LR_ERR_INVALID_ARGUMENT;
  lr_opts o;
  if (opts) o = *opts;
  else lr_opts_default(&o);
  if (o.workspace != nullptr) return LR_ERR_INVALID_ARGUMENT;   // candidates size their own buffers
  if (o.tuning && o.tuning->algorithm == LR_ALGO_WYLLIE) return LR_ERR_INVALID_ARGUMENT;
  const bool weighted = o.wtype != LR_NONE;
  o.tuning = nullptr;
  // synthetic inputs: one list per instance, so the bound is known and no
  // timed call synchronises to count lists
  if (!succ) o.max_lists = k > 0 ? k : 1;
  if (k > 0) o.n_total = n_total;
  cudaStream_t s = (cudaStream_t)stream;
  lr_status st = setup_device_once();
  if (st != LR_OK) return st;

  // inputs: the caller's, or synthetic ones of the same shape
  uint32_t *dsucc = nullptr;
  void *dw = nullptr;
  const int wbytes = o.wtype == LR_I32 ? 4 : 8;
  int64_t *doff = nullptr;
  void *rank = nullptr, *ref = nullptr;
  unsigned long long *dbad = nullptr;
  const size_t rb = o.rtype == LR_I64 ? 8 : 4;
  cudaError_t e = cudaSuccess;
  if (!succ) {
    e = cudaMalloc((void **)&dsucc, 4 * (size_t)n_total);
    if (e == cudaSuccess && weighted) e = cudaMalloc(&dw, (size_t)wbytes * n_total);
    if (e == cudaSuccess && k > 0) e = cudaMalloc((void **)&doff, 8 * ((size_t)k + 1));
    if (e == cudaSuccess) {
      k_tune_input<<<stream_grid((uint64_t)n_total, 256), 256, 0, s>>>(dsucc, dw, wbytes, doff,
                                                                      (uint32_t)n_total, k, 0x7a11ull);
      e = cudaGetLastError();
    }
  }
  if (e == cudaSuccess) e = cudaMalloc(&rank, rb * (size_t)n_total);
  if (e == cudaSuccess) e = cudaMalloc(&ref, rb * (size_t)n_total);
  if (e == cudaSuccess) e = cudaMalloc((void **)&dbad, 8);
  TuneRun R;
  R.succ = succ ? succ : dsucc;
  R.weight = succ ? weight : (const void *)dw;
  R.offsets = succ ? offsets : doff;
  R.n = n_total;
  R.k = k;
  R.opts = o;
  R.rank = rank;
  R.s = s;
  if (e == cudaSuccess) e = cudaEventCreate(&R.e0);
  if (e == cudaSuccess) e = cudaEventCreate(&R.e1);
  if (e != cudaSuccess) {
    cudaGetLastError();
    cudaFree(dsucc); cudaFree(dw); cudaFree(doff); cudaFree(rank); cudaFree(ref); cudaFree(dbad);
    return e == cudaErrorMemoryAllocation ? LR_ERR_OUT_OF_MEMORY : LR_ERR_CUDA;
  }

  // reference output with the built-in defaults (table entries ignored)
  const Tuning d = resolve_tuning_builtin(n_total, weighted, k > 0);
  lr_tuning best;
  memset(&best, 0, sizeof(best));
  best.f0_inv = d.f0_inv;
  best.f_inv = d.f_inv;
  best.cutoff = d.cutoff;
  best.chase_block = d.block;
  st = R.call(&best, ref);
  if (st == LR_OK) st = device_status(s);
  const int reps = n_total >= ((int64_t)1 << 26) ? 3 : 5;
  float best_ms = st == LR_OK ? R.time(best, reps) : INFINITY;
  if (st == LR_OK && !std::isfinite(best_ms)) st = LR_ERR_CUDA;

  auto try_field = [&](uint32_t lr_tuning::*field, const std::vector<uint32_t> &vals) {
    for (uint32_t v : vals) {
      if (best.*field == v) continue;
      lr_tuning c = best;
      c.*field = v;
      const float ms = R.time(c, reps);
      if (ms < best_ms) { best_ms = ms; best = c; }
    }
  };
  if (st == LR_OK) {
    try_field(&lr_tuning::f0_inv, {4, 8, 16, 32, 64, 128});
    try_field(&lr_tuning::f_inv, {4, 8, 16});
    try_field(&lr_tuning::cutoff, {4096, 8192, 12288});
    try_field(&lr_tuning::chase_block, {128, 256, 512});
    const uint32_t f0 = best.f0_inv;
    try_field(&lr_tuning::f0_inv, {std::max<uint32_t>(2, f0 * 2 / 3), f0 * 3 / 2});
    // the winner must rank exactly as the defaults do
    st = R.call(&best, rank);
    if (st == LR_OK) st = device_status(s);
    if (st == LR_OK) {
      cudaMemsetAsync(dbad, 0, 8, s);
      k_tune_diff<<<stream_grid(rb * (size_t)n_total, 256), 256, 0, s>>>(
          (const unsigned char *)rank, (const unsigned char *)ref, rb * (size_t)n_total, dbad);
      unsigned long long bad = 0;
      cudaMemcpyAsync(&bad, dbad, 8, cudaMemcpyDeviceToHost, s);
      if (cudaStreamSynchronize(s) != cudaSuccess) st = LR_ERR_CUDA;
      else if (bad) st = LR_ERR_INTERNAL;
    }
  }
  cudaEventDestroy(R.e0);
  cudaEventDestroy(R.e1);
  cudaFree(dsucc); cudaFree(dw); cudaFree(doff); cudaFree(rank); cudaFree(ref); cudaFree(dbad);
  if (st != LR_OK) return st;
  lr_tune_entry ent;
  memset(&ent, 0, sizeof(ent));
  ent.log2n = log2_floor(n_total);
  ent.weighted = weighted ? 1 : 0;
  ent.batch = k > 0 ? 1 : 0;
  ent.tuning = best;
  ent.ms = best_ms;
  {
    std::lock_guard<std::mutex> g(g_tmu);
    load_env_once();
    put_entry(ent);
  }
  if (out) *out = best;
  return LR_OK;
}

extern "C" lr_status lr_autotune_save(const char *path) {
  if (!path) return LR_ERR_INVALID_ARGUMENT;
  std::lock_guard<std::mutex> g(g_tmu);
  const std::string tmp = std::string(path) + ".tmp";
  FILE *f = fopen(tmp.c_str(), "wb");
  if (!f) return LR_ERR_INVALID_ARGUMENT;
  fprintf(f, "{\n \"format\": \"lr_autotune 1\",\n \"entries\": [\n");
  for (size_t i = 0; i < g_table.size(); ++i) {
    const lr_tune_entry &e = g_table[i];
    fprintf(f, "  {\"log2n\": %d, \"weighted\": %d, \"batch\": %d, \"f0_inv\": %u, \"f_inv\": %u, "
               "\"cutoff\": %u, \"chase_block\": %u, \"chase_ctas\": %u, \"algorithm\": %u, \"ms\": %.6g}%s\n",
            e.log2n, e.weighted, e.batch, e.tuning.f0_inv, e.tuning.f_inv, e.tuning.cutoff,
            e.tuning.chase_block, e.tuning.chase_ctas, e.tuning.algorithm, (double)e.ms,
            i + 1 < g_table.size() ? "," : "");
  }
  fprintf(f, " ]\n}\n");
  const bool ok = fclose(f) == 0;
  if (!ok || rename(tmp.c_str(), path) != 0) return LR_ERR_INVALID_ARGUMENT;
  return LR_OK;
}

extern "C" lr_status lr_autotune_load(const char *path) {
  if (!path) return LR_ERR_INVALID_ARGUMENT;
  std::lock_guard<std::mutex> g(g_tmu);
  g_env_loaded = true;   // an explicit load replaces the environment's file
  return load_file(path);
}

extern "C" int32_t lr_autotune_entries(lr_tune_entry *out, int32_t cap) {
  std::lock_guard<std::mutex> g(g_tmu);
  load_env_once();
  const int32_t n = (int32_t)g_table.size();
  for (int32_t i = 0; out && i < n && i < cap; ++i) out[i] = g_table[i];
  return n;
}

extern "C" void lr_autotune_clear(void) {
  std::lock_guard<std::mutex> g(g_tmu);
  g_table.clear();
  g_env_loaded = true;
}
