// lr_engine.cu -- host engine of liblr.so: argument checks, the static level
// plan, workspace layout, per-stream contexts, launch sequence, device status
// and profiling.  Implements the C ABI declared in include/lr.h.
//
// Recursion plan (Section 2.1: rank the rulers' list recursively, then
// propagate; Section 3 runs a few sparse ruling-set rounds before pointer
// doubling).  The number of levels and every array size are fixed on the host
// from n and a bound h on the number of lists:
//   cap_0 = n,  cap_{l+1} = min(cap_l, ceil(cap_l / f_l) + h),
// until a level fits the single-CTA base case.  The actual sizes are decided
// on the device (each level's head scan writes the next level's size and
// mode), so a call never waits for the device unless h has to be counted
// first, and a call with a known bound can be captured in a CUDA graph.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <nvtx3/nvToolsExt.h>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <utility>
#include <vector>

#include "lr.h"
#include "lr_engine.h"
#include "lr_kernels.h"

namespace lr {

// ---------------------------------------------------------------- tuning
static uint32_t env_u32(const char *spec, const char *key, uint32_t dflt) {
  if (!spec) return dflt;
  std::string s(spec), k = std::string(key) + "=";
  size_t p = 0;
  while ((p = s.find(k, p)) != std::string::npos) {
    if (p == 0 || s[p - 1] == ',') return (uint32_t)strtoul(s.c_str() + p + k.size(), nullptr, 10);
    p += k.size();
  }
  return dflt;
}

// Default ruler fraction at level 0 by size (measured on GB300, random
// order, f = 1/8 above level 0).  Small lists are bound by the latency of
// the dependent exchanges along one segment, so they take more rulers and
// shorter segments; from 2^27 up the chase is bound by the random-access
// rate, and fewer rulers shrink the recursion more than their longer
// segments lengthen the chase's tail (1/48 at 2^28, 1/96 at 2^30).
static uint32_t default_f0_inv(int64_t n) {
  if (n < ((int64_t)1 << 16)) return 4;
  if (n < ((int64_t)1 << 22)) return 8;
  if (n < ((int64_t)1 << 27)) return 16;
  if (n < ((int64_t)1 << 29)) return 48;
  return 96;
}

// A batch chases level 0 in element order: its records stay in L2 only if
// the front (threads x ruler spacing) is narrow, so it keeps 1/16 from 2^22
// up (on the 1024-instance batch of 4.3e8 elements: 17.3 ms at 1/16 and
// 1/24, 17.8 at 1/32, 18.8 at 1/48).
static uint32_t default_f0_inv_batch(int64_t n) {
  return n < ((int64_t)1 << 22) ? default_f0_inv(n) : 16;
}

Tuning resolve_tuning_builtin(int64_t n, bool weighted, bool batch) {
  (void)weighted;
  Tuning u;
  u.f0_inv = batch ? default_f0_inv_batch(n) : default_f0_inv(n);
  u.f_inv = 8;
  u.cutoff = kMaxCutoff;
  u.block = 256;
  u.ctas = 0;
  u.xchg = 1;
  u.chase0 = LR_CHASE0_AUTO;
  u.algo = LR_ALGO_SRS;
  u.contract = LR_CONTRACT_AUTO;
  u.spawn = 0;
  u.ord = 2;              // batches: every level of 2^20 or more in element order
  u.pf = 4;               // ... prefetching its records 4K elements ahead of each draw
  return u;
}

Tuning resolve_tuning(const lr_tuning *t, int64_t n, bool weighted, bool batch) {
  Tuning u = resolve_tuning_builtin(n, weighted, batch);
  lr_tuning tt;
  if (tuned_lookup(n, weighted, batch, &tt)) {
    if (tt.f0_inv) u.f0_inv = tt.f0_inv;
    if (tt.f_inv) u.f_inv = tt.f_inv;
    if (tt.cutoff) u.cutoff = tt.cutoff;
    if (tt.chase_block) u.block = tt.chase_block;
    if (tt.chase_ctas) u.ctas = tt.chase_ctas;
  }
  const char *env = getenv("LR_TUNING");
  u.f0_inv = env_u32(env, "f0", u.f0_inv);
  u.f_inv = env_u32(env, "f", u.f_inv);
  u.cutoff = env_u32(env, "cutoff", u.cutoff);
  u.block = env_u32(env, "block", u.block);
  u.ctas = env_u32(env, "ctas", u.ctas);
  u.xchg = env_u32(env, "xchg", 1);
  const uint32_t env_log = env_u32(env, "log", 2);      // log=1 / log=0: force a level-0 form
  if (env_log < 2) u.chase0 = env_log ? LR_CHASE0_LOG : LR_CHASE0_EXCHANGE;
  u.algo = env_u32(env, "algo", LR_ALGO_SRS);
  u.contract = env_u32(env, "contract", u.contract);
  u.spawn = env_u32(env, "spawn", u.spawn);
  u.ord = env_u32(env, "ord", u.ord);
  u.pf = env_u32(env, "pf", u.pf);
  if (t) {
    if (t->spawn) u.spawn = t->spawn;
    if (t->chase0) u.chase0 = t->chase0;
    if (t->algorithm) u.algo = t->algorithm;
    if (t->contract) u.contract = t->contract;
    if (t->f0_inv) u.f0_inv = t->f0_inv;
    if (t->f_inv) u.f_inv = t->f_inv;
    if (t->cutoff) u.cutoff = t->cutoff;
    if (t->chase_block) u.block = t->chase_block;
    if (t->chase_ctas) u.ctas = t->chase_ctas;
  }
  u.f0_inv = std::max<uint32_t>(2, u.f0_inv);
  u.f_inv = std::max<uint32_t>(2, u.f_inv);
  u.cutoff = std::min<uint32_t>(std::max<uint32_t>(u.cutoff, 64), kMaxCutoff);
  if (u.block != 128 && u.block != 256 && u.block != 512) u.block = 256;
  return u;
}

// Level-0 chase form: the log form (lr_log.cu) needs an unweighted single
// instance with int32 ranks and n <= 2^30; auto takes it from 2^25 on, where
// its one random access per element beats the exchange form's two, unless
// spawning (an exchange-form feature) was asked for.
constexpr uint64_t kLogAutoMin = 1ull << 25;
static bool use_log0(const Tuning &u, uint64_t n, bool weighted, int rank_bytes, bool extras, bool multi) {
  if (weighted || rank_bytes != 4 || extras || multi || n <= u.cutoff || n > (1ull << 30) || !u.xchg)
    return false;
  if (u.chase0 == LR_CHASE0_LOG) return true;
  return u.chase0 == LR_CHASE0_AUTO && n >= kLogAutoMin && !u.spawn;
}

// Level 0 of a set of contiguous instances (a batch) chases its rulers in
// element order: a front that crosses the instances a few at a time keeps
// the records it touches, the reduced records it writes and, in the final
// pass, the rank gathers within a footprint the L2 holds.
static bool use_ord0(const Tuning &u, uint64_t n, bool log0, bool spawn0, bool extras, bool multi) {
  return u.ord != 0 && multi && !log0 && !spawn0 && !extras && n <= 0x7FFFFFFFull;
}

static uint32_t ceil_log2(uint64_t x) {
  uint32_t b = 0;
  while ((1ull << b) < x) ++b;
  return b;
}

static size_t align_up(size_t x, size_t a = 256) { return (x + a - 1) / a * a; }

// CTAs of 256 threads per SM for the chase in element order: the front's
// width (threads x ruler spacing) must stay small enough that the instances
// it crosses fit in L2; more threads only queue at the memory system.
constexpr int kOrdCtasPerSm = 4;
// Deeper levels of a batch keep each instance's rulers together too; from
// this size on they are chased in order as well (LR_TUNING ord=1: level 0
// only; ord=0: no level).
constexpr uint32_t kOrdMinLevel = 1u << 20;

int chase_grid_for(const Tuning &u, bool rec16, bool log0, bool ord0) {
  int per = u.ctas ? (int)u.ctas : (log0 ? chase_log_occupancy((int)u.block) : chase_occupancy(rec16, (int)u.block));
  if (ord0 && !u.ctas) per = std::min(per, kOrdCtasPerSm * 256 / (int)u.block);
  return device_sm_count() * std::max(1, per);
}

// Static plan for n elements and at most h lists.
// Spawned rulers provided for at level 0: t waves leave about t ln(n/t)
// rulers in all (Section 2.5 cites this for spawning); a few t more as slack.
static uint32_t spawn_capacity(uint64_t n, uint64_t threads) {
  if (threads == 0) threads = 1;
  const double ratio = n > threads ? (double)n / (double)threads : 1.0;
  const double want = (double)threads * (std::ceil(std::log(ratio)) + 4.0);
  return (uint32_t)std::min<double>((double)n, want);
}

Plan make_plan(uint64_t n, uint64_t h, const Tuning &u, bool rec16_0, int rank_bytes,
               uint64_t seed, int chase_grid, bool force_srs, bool log0, bool term, bool t0ws,
               bool spawn0, bool ord0) {
  Plan p;
  memset(&p, 0, sizeof(p));
  p.n = n;
  p.rec16_0 = rec16_0;
  p.log0 = log0;
  p.rank_bytes = rank_bytes;
  p.cutoff = u.cutoff;
  p.chase_grid = chase_grid;
  p.chase_block = (int)u.block;
  p.hcap = (uint32_t)std::max<uint64_t>(1, std::min<uint64_t>(h, std::max<uint64_t>(n, 1)));
  p.cap[0] = (uint32_t)n;
  p.f_inv[0] = u.f0_inv;
  int L = 0;
  const bool sp = spawn0 && (n > u.cutoff || force_srs);
  p.spawn_cap = sp ? spawn_capacity(n, (uint64_t)chase_grid * u.block) : 0;
  if (n > u.cutoff || force_srs) {
    for (;;) {
      const uint64_t r = (p.cap[L] + p.f_inv[L] - 1) / p.f_inv[L];
      uint64_t nc = std::min<uint64_t>(p.cap[L], r + p.hcap);
      if (L == 0 && sp) {
        p.raw_cap = (uint32_t)std::min<uint64_t>(0xFFFFFFF0ull, nc + p.spawn_cap);
        nc = std::min<uint64_t>(p.cap[0], nc + p.spawn_cap);
      }
      ++L;
      p.cap[L] = (uint32_t)nc;
      p.f_inv[L] = u.f_inv;
      if (nc <= u.cutoff) break;
      if (L == kMaxLevels) break;
      if (L == 1 && p.cap[0] <= u.cutoff) break;
      if (L >= 3 && (uint64_t)p.cap[L] * 4 > (uint64_t)p.cap[L - 1] * 3) break;  // stalled
    }
  }
  p.nlev = L + 1;
  p.has_pd = p.cap[L] > u.cutoff;
  p.pd_rounds = p.has_pd ? ceil_log2(p.cap[L]) + 1 : 0;
  for (int l = 0; l <= L; ++l) p.seed[l] = splitmix64(seed + 0x9E37ull * (uint64_t)(l + 1));

  // fixed part: independent of h
  size_t o = 0;
  p.off_desc = o; o = align_up(o + sizeof(LevelDesc) * (kMaxLevels + 1));
  p.off_zero = o;
  p.off_err = o; o = align_up(o + 16);
  p.off_hcount = o; o = align_up(o + 16);
  p.off_acc = o; o = align_up(o + 32);        // sums of terminals, successors; local links
  p.off_logctr = o; o = align_up(o + 16);
  p.off_bctr = o; o = align_up(o + sizeof(uint32_t) * 256);
  p.off_q = o; o = align_up(o + sizeof(uint32_t) * (size_t)chase_grid * kMaxLevels);
  p.off_bcnt = o; o = align_up(o + sizeof(uint64_t) * kHeadBlocks);
  p.zero_bytes = o - p.off_zero;
  p.off_bitmap = o; o = align_up(o + sizeof(uint32_t) * ((n + 31) / 32));
  if (!log0) { p.off_work[0] = o; o = align_up(o + (rec16_0 ? 16 : 8) * (size_t)n); }
  p.fixed_bytes = o;
  // variable part
  o = 0;
  for (int l = 1; l <= L; ++l) {
    p.off_work[l] = o; o = align_up(o + 16 * (size_t)p.cap[l]);
    p.off_R[l] = o; o = align_up(o + (size_t)rank_bytes * p.cap[l]);
  }
  if (log0) {
    // log entries: every element once plus one mark per ruler, in 32-entry
    // chunks handed out from one counter; each thread leaves at most one
    // chunk partly filled, and each CTA at most the rest of one window of
    // kLogWindow chunks, however long the segments are
    const uint64_t rulers = (n + p.f_inv[0] - 1) / p.f_inv[0] + p.hcap;
    const uint64_t need = (n + rulers + 31) / 32;
    const uint64_t threads = (uint64_t)chase_grid * u.block;
    const uint64_t total = need + threads + (uint64_t)chase_grid * kLogWindow + 4096;
    p.total_chunks = (uint32_t)std::min<uint64_t>(total, 0xFFFFFFF0ull);
    uint32_t lg = 0;
    while ((1ull << lg) < n) ++lg;
    p.shift = lg > 8 ? lg - 8 : 0;
    p.off_log = o; o = align_up(o + (size_t)p.total_chunks * 32 * 4);
    p.off_hdr = o; o = align_up(o + (size_t)p.total_chunks * 8);
    p.lg = log_geometry((uint32_t)n);
    p.off_pairs = o; o = align_up(o + (size_t)p.lg.na * p.lg.capA * 8);
    p.off_pairsB = o; o = align_up(o + (size_t)p.lg.nw * p.lg.capB * 8);
    p.off_cur = o;
    p.cur_bytes = 4 * ((size_t)p.lg.na + p.lg.nbB);           // claimed slots per region
    o = align_up(o + p.cur_bytes);
  }
  p.off_hA = o; o = align_up(o + 4 * (size_t)p.hcap);
  p.off_hB = o; o = align_up(o + 4 * (size_t)p.hcap);
  p.off_ns = o; o = align_up(o + 4 * (size_t)p.hcap);
  if (p.has_pd) {
    p.off_pd[0] = o; o = align_up(o + 4 * (size_t)p.cap[L]);
    p.off_pd[1] = o; o = align_up(o + 4 * (size_t)p.cap[L]);
    p.off_pd[2] = o; o = align_up(o + 8 * (size_t)p.cap[L]);
    p.off_pd[3] = o; o = align_up(o + 8 * (size_t)p.cap[L]);
  }
  if (p.spawn_cap) {
    const size_t words = (p.spawn_cap + 31) / 32;
    p.off_sraw = o; o = align_up(o + 16 * (size_t)p.raw_cap);
    p.off_srraw = o; o = align_up(o + (size_t)rank_bytes * p.raw_cap);
    p.off_supre = o; o = align_up(o + 4 * words);
    p.off_sctr = o; o = align_up(o + 16 + 4 * (size_t)chase_grid);
    p.off_sused = o; o = align_up(o + 4 * words);
    p.spawn_zero = o - p.off_sctr;                // counter, cursors, claimed bitmap
  }
  p.ord0 = ord0 && p.nlev > 1;
  if (p.ord0) {
    // one set of arrays serves every level chased in order, one at a time:
    // marks and block counts for level 0's n, positions for the most
    // sampled rulers of any level
    uint64_t rmax = 0;
    for (int l = 0; l < L; ++l) rmax = std::max<uint64_t>(rmax, (p.cap[l] + p.f_inv[l] - 1) / p.f_inv[l]);
    p.off_ord = o; o = align_up(o + 4 * (size_t)rmax);
    p.off_cum = o; o = align_up(o + 4 * (size_t)((n + 255) / 256));
  }
  p.term = term;
  if (term) {
    for (int l = 1; l <= L; ++l) {
      p.off_T[l] = o; o = align_up(o + 4 * (size_t)p.cap[l]);
      p.off_tid[l] = o; o = align_up(o + 4 * (size_t)p.cap[l]);
    }
    p.off_hC = o; o = align_up(o + 4 * (size_t)p.hcap);   // keeps level 0's head list intact
    if (p.has_pd) {
      p.off_pdt[0] = o; o = align_up(o + 4 * (size_t)p.cap[L]);
      p.off_pdt[1] = o; o = align_up(o + 4 * (size_t)p.cap[L]);
    }
    if (t0ws) { p.off_T0 = o; o = align_up(o + 4 * (size_t)n); }
  }
  p.var_bytes = std::max<size_t>(o, 256);
  return p;
}

// ---------------------------------------------------------------- contexts
static std::mutex g_mu;
static std::map<std::pair<int, uintptr_t>, Ctx *> g_ctx;
static bool g_setup_done[64];

static lr_status from_cuda(cudaError_t e) {
  if (e == cudaSuccess) return LR_OK;
  if (e == cudaErrorMemoryAllocation) return LR_ERR_OUT_OF_MEMORY;
  if (e == cudaErrorStreamCaptureUnsupported || e == cudaErrorStreamCaptureInvalidated)
    return LR_ERR_CAPTURE;
  return LR_ERR_CUDA;
}

lr_status setup_device_once() {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return from_cuda(e);
  std::lock_guard<std::mutex> g(g_mu);
  if (dev >= 0 && dev < 64 && !g_setup_done[dev]) {
    e = kernels_setup();
    if (e == cudaSuccess) e = log_setup();
    if (e == cudaSuccess) e = lc_setup();
    if (e != cudaSuccess) return from_cuda(e);
    // Place lr_rank_noalloc's scratch array on this device now, while the
    // process can still spare its 64 MiB: under lazy module loading it would
    // otherwise be placed only at the first lr_rank_noalloc call, which may
    // come after the caller's allocator has taken all free memory.  Best
    // effort: a failure here surfaces at that call, with its status.
    (void)noalloc_resolve_scratch();
    g_setup_done[dev] = true;
  }
  return LR_OK;
}

Ctx *get_ctx(cudaStream_t stream, lr_status *st) {
  *st = setup_device_once();
  if (*st != LR_OK) return nullptr;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) { *st = from_cuda(e); return nullptr; }
  std::lock_guard<std::mutex> g(g_mu);
  auto key = std::make_pair(dev, (uintptr_t)stream);
  auto it = g_ctx.find(key);
  if (it != g_ctx.end()) { *st = LR_OK; return it->second; }
  Ctx *c = new Ctx();
  c->device = dev;
  e = cudaMallocHost((void **)&c->host_words, 64);
  if (e != cudaSuccess) { delete c; *st = LR_ERR_OUT_OF_MEMORY; return nullptr; }
  memset(c->host_words, 0, 64);
  g_ctx[key] = c;
  *st = LR_OK;
  return c;
}

void release_ctx(cudaStream_t stream) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return;
  Ctx *c = nullptr;
  {
    std::lock_guard<std::mutex> g(g_mu);
    auto it = g_ctx.find(std::make_pair(dev, (uintptr_t)stream));
    if (it == g_ctx.end()) return;
    c = it->second;
    g_ctx.erase(it);
  }
  cudaStreamSynchronize(stream);
  if (c->fixed) cudaFree(c->fixed);
  if (c->var) cudaFree(c->var);
  if (c->hostpath) cudaFree(c->hostpath);
  if (c->contract) cudaFree(c->contract);
  if (c->contract2) cudaFree(c->contract2);
  cudaFreeHost(c->host_words);
  delete c;
}

static bool stream_capturing(cudaStream_t s) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &cs) != cudaSuccess) return false;
  return cs != cudaStreamCaptureStatusNone;
}

// Grow-only device buffer.
// Fault injection on the host (tests): with LR_INJECT_ALLOC_FAIL=1 in the
// environment every request for library workspace fails as a cudaMalloc
// that ran out of memory would, whether or not the arena had to grow, and
// without calling it.
static bool inject_alloc_failure() {
  const char *v = getenv("LR_INJECT_ALLOC_FAIL");
  return v && v[0] == '1';
}

lr_status ensure_buffer(void **buf, size_t *cur, size_t want, cudaStream_t s) {
  if (inject_alloc_failure()) return LR_ERR_OUT_OF_MEMORY;
  if (*cur >= want && *buf) return LR_OK;
  if (stream_capturing(s)) return LR_ERR_CAPTURE;
  if (*buf) {
    cudaStreamSynchronize(s);
    cudaFree(*buf);
    *buf = nullptr;
    *cur = 0;
  }
  size_t sz = std::max(want, (size_t)1 << 20);
  cudaError_t e = cudaMalloc(buf, sz);
  if (e != cudaSuccess) { cudaGetLastError(); *buf = nullptr; return LR_ERR_OUT_OF_MEMORY; }
  *cur = sz;
  return LR_OK;
}

// ---------------------------------------------------------------- profiling
static bool g_prof = false;
struct ProfMark { cudaEvent_t ev; int phase; };  // phase of the interval ending here
struct ProfCall { std::vector<ProfMark> marks; int64_t n; int64_t launches; bool log0 = false; };
static std::vector<ProfCall> g_prof_pending;
static lr_profile g_prof_acc;

// Per call: an NVTX range (always; free without an attached tool) whose
// payload is n, NVTX marks at the phase boundaries, and, when profiling is
// on, CUDA events at the same boundaries for lr_profile_read.
static const char *const kPhaseNames[] = {"lr.prep", "lr.select", "lr.chase0", "lr.chase",
                                          "lr.base", "lr.finalize"};

struct Profiler {
  bool on = false;
  bool ranged = false;
  ProfCall call;
  cudaStream_t s = nullptr;
  void begin(cudaStream_t st, int64_t n) {
    nvtxEventAttributes_t a;
    memset(&a, 0, sizeof(a));
    a.version = NVTX_VERSION;
    a.size = NVTX_EVENT_ATTRIB_STRUCT_SIZE;
    a.messageType = NVTX_MESSAGE_TYPE_ASCII;
    a.message.ascii = "lr.call";
    a.payloadType = NVTX_PAYLOAD_TYPE_INT64;
    a.payload.llValue = n;
    nvtxRangePushEx(&a);
    ranged = true;
    on = g_prof && !stream_capturing(st);
    s = st;
    if (!on) return;
    call.n = n;
    call.launches = launch_count();
    mark(-1);
  }
  void mark(int phase) {
    if (ranged && phase >= 0) nvtxMarkA(kPhaseNames[phase]);
    if (!on) return;
    ProfMark m;
    m.phase = phase;
    cudaEventCreate(&m.ev);
    cudaEventRecord(m.ev, s);
    call.marks.push_back(m);
  }
  void end() {
    if (ranged) { nvtxRangePop(); ranged = false; }
    if (!on) return;
    on = false;
    call.launches = launch_count() - call.launches;
    std::lock_guard<std::mutex> g(g_mu);
    g_prof_pending.push_back(call);
  }
  // drop a call that turned out not to happen (its marks are not recorded)
  void cancel() {
    if (ranged) { nvtxRangePop(); ranged = false; }
    if (!on) return;
    for (auto &m : call.marks) cudaEventDestroy(m.ev);
    call.marks.clear();
    on = false;
  }
  // a call that returns early (an error) closes its range and drops its marks
  ~Profiler() { cancel(); }
};
enum { PH_PREP = 0, PH_SELECT, PH_CHASE0, PH_CHASE, PH_BASE, PH_FINAL };

// ---------------------------------------------------------------- the run
struct Inputs {
  const uint32_t *succ;
  const void *weight;
  int wtype;          // 0 none, 1 i32, 2 i64
  void *rank;
  int rank_bytes;
  uint64_t n;
  const int64_t *offsets;  // batched form
  int32_t k;
  int validate;
  uint64_t seed;
  int64_t max_lists;
  int sync;
  void *ws;
  size_t ws_bytes;
  const uint32_t *const *sptr;   // per-instance pointer tables (device), or null
  const void *const *wptr;
  void *const *rptr;
  Ctx *ctx;                      // use this context instead of the per-stream one
  int count_in_ws;               // caller workspace, but still count the lists first
  uint32_t *term;                // extra outputs (device, optional): terminal ids,
  void *prefix;                  // head-relative ranks,
  int incl;                      // inclusive-tail ranks
  uint32_t *err_ext;             // record device errors here (and do not clear it)
  int no_contract;               // never contract (the contracted list itself)
  int builtin_tuning;            // ignore LR_TUNING and the autotuned table
};

static lr_status map_device_bits(uint32_t bits) {
  if (bits & kErrDebug) return LR_ERR_INTERNAL;      // a debug build's index check
  if (bits & kErrRange) return LR_ERR_OUT_OF_RANGE;
  if (bits & kErrNotList) return LR_ERR_NOT_A_LIST;
  if (bits & kErrCycle) return LR_ERR_CYCLE;
  if (bits & kErrCapacity) return LR_ERR_CAPACITY;
  if (bits & kErrInternal) return LR_ERR_NOT_A_LIST;
  return LR_OK;
}

#define LR_TRY(expr)                                   \
  do {                                                 \
    cudaError_t e__ = (expr);                          \
    if (e__ != cudaSuccess) return from_cuda(e__);     \
  } while (0)

// Copy the call's device error word to the context's pinned status word;
// with sync, wait and return the status it encodes.
static lr_status finish_call(Ctx *c, const uint32_t *err, int sync, cudaStream_t s) {
  LR_TRY(cudaMemcpyAsync(c->host_words, err, 4, cudaMemcpyDeviceToHost, s));
  c->pending_status = true;
  if (sync) {
    LR_TRY(cudaStreamSynchronize(s));
    c->pending_status = false;
    const uint32_t bits = c->host_words[0];
    c->host_words[0] = 0;
    return map_device_bits(bits);
  }
  return LR_OK;
}

// Workspace of the pointer-doubling algorithm: error word and scratch sums,
// the has-predecessor bitmap (validation), two record arrays.
struct WyPlan {
  size_t off_err, off_sums, off_bitmap, off_a, off_b, zero_bytes, bytes;
};

static WyPlan wyllie_plan(uint64_t n, bool w16) {
  WyPlan q;
  size_t o = 0;
  q.off_err = o; o = align_up(o + 16);
  q.off_sums = o; o = align_up(o + 16);
  q.zero_bytes = o;
  q.off_bitmap = o; o = align_up(o + sizeof(uint32_t) * ((n + 31) / 32));
  q.off_a = o; o = align_up(o + (w16 ? 16 : 8) * n);
  q.off_b = o; o = align_up(o + (w16 ? 16 : 8) * n);
  q.bytes = o;
  return q;
}

// 16-byte records exactly when weighted: the layout k_prep0 writes.
static bool wyllie_w16(const Inputs &in) { return in.wtype != 0; }

// Whole-list pointer doubling (lr_wyllie.cu) on the same inputs and outputs.
static lr_status run_wyllie(const Inputs &in, Ctx *c, cudaStream_t s) {
  c->last_nlev = 0;
  const bool w16 = wyllie_w16(in);
  const WyPlan q = wyllie_plan(in.n, w16);
  char *base = nullptr;
  if (in.ws) {
    if (in.ws_bytes < q.bytes) return LR_ERR_INVALID_ARGUMENT;
    base = (char *)in.ws;
  } else {
    const lr_status st = ensure_buffer(&c->var, &c->var_bytes, q.bytes, s);
    if (st != LR_OK) return st;
    base = (char *)c->var;
  }
  uint32_t *err = (uint32_t *)(base + q.off_err);
  uint32_t *bitmap = (uint32_t *)(base + q.off_bitmap);
  unsigned long long *sums = (unsigned long long *)(base + q.off_sums);
  void *A = base + q.off_a, *B = base + q.off_b;
  Profiler prof;
  if (!in.ctx) prof.begin(s, (int64_t)in.n);
  LR_TRY(cudaMemsetAsync(base, 0, in.validate ? q.off_a : q.zero_bytes, s));
  // without validation the scratch sums stand in for the bitmap, so the
  // pass issues no per-element atomics
  LR_TRY(launch_prep0(in.succ, in.weight, in.wtype, (uint32_t)in.n, A, bitmap, err, in.validate,
                      in.offsets, in.k, in.validate ? nullptr : sums, nullptr, s));
  prof.mark(PH_PREP);
  LR_TRY(launch_wyllie(A, B, w16, (uint32_t)in.n, in.rank, in.rank_bytes, err, s));
  prof.mark(PH_BASE);
  prof.end();
  return finish_call(c, err, in.sync, s);
}

lr_status run(const Inputs &in, const lr_tuning *tuning, cudaStream_t s);

// Tile-local contraction (lr_contract.cu) around the ruling set: count the
// local heads of every tile, build the contracted list, rank it (inclusive
// form, through run() itself), restore every element.  Returns
// LR_ERR_NOT_FOUND (nothing enqueued that writes outputs) when the exact
// count shows that contraction would not shrink the list enough.
static lr_status run_contracted(const Inputs &in, const lr_tuning *tuning, Ctx *c, bool forced,
                                cudaStream_t s) {
  const uint32_t n = (uint32_t)in.n;
  const uint32_t nt = lc_tiles(n);
  const size_t words = (size_t)nt * lc_tile_words();
  size_t o = 0;
  const size_t off_err = o; o = align_up(o + 16);
  const size_t off_hb = o; o = align_up(o + 4 * words);
  const size_t off_wpre = o; o = align_up(o + 2 * words);
  const size_t off_tcnt = o; o = align_up(o + 4 * (size_t)nt);
  const size_t off_tpre = o; o = align_up(o + 4 * ((size_t)nt + 1));
  const size_t off_tail = o; o = align_up(o + 2 * (size_t)n);
  lr_status st = ensure_buffer(&c->contract, &c->contract_bytes, o, s);
  if (st != LR_OK) return st;
  char *b = (char *)c->contract;
  uint32_t *err = (uint32_t *)(b + off_err);
  LR_TRY(cudaMemsetAsync(b, 0, off_hb, s));
  Profiler prof;
  prof.begin(s, (int64_t)in.n);
  c->last_nlev = 0;
  uint32_t *hb = (uint32_t *)(b + off_hb);
  uint16_t *wpre = (uint16_t *)(b + off_wpre);
  uint32_t *tcnt = (uint32_t *)(b + off_tcnt);
  uint32_t *tpre = (uint32_t *)(b + off_tpre);
  uint16_t *tail16 = (uint16_t *)(b + off_tail);
  LR_TRY(launch_lc_solve(in.succ, in.weight, in.wtype, n, in.rank, in.rank_bytes, tail16, hb, wpre, tcnt,
                         tpre, err, s));
  LR_TRY(cudaMemcpyAsync(c->host_words + 1, tpre + nt, 4, cudaMemcpyDeviceToHost, s));
  LR_TRY(cudaStreamSynchronize(s));
  const uint64_t m = c->host_words[1];
  if (!forced && m * 5 > (uint64_t)n * 3) { prof.cancel(); return LR_ERR_NOT_FOUND; }
  // the contracted list: successors, weights (int32 unweighted: at most one
  // tile's links; int64 weighted), ranks in the caller's type
  const int wc = in.wtype == 0 ? 1 : 2;
  const size_t wb = wc == 1 ? 4 : 8;
  size_t o2 = 0;
  const size_t off_sc = o2; o2 = align_up(o2 + 4 * std::max<uint64_t>(m, 1));
  const size_t off_wc = o2; o2 = align_up(o2 + wb * std::max<uint64_t>(m, 1));
  const size_t off_rc = o2; o2 = align_up(o2 + (size_t)in.rank_bytes * std::max<uint64_t>(m, 1));
  st = ensure_buffer(&c->contract2, &c->contract2_bytes, o2, s);
  if (st != LR_OK) return st;
  char *b2 = (char *)c->contract2;
  LR_TRY(launch_lc_nodes(in.succ, in.weight, in.wtype, n, in.rank, in.rank_bytes, tail16, hb, wpre, tpre,
                         (uint32_t *)(b2 + off_sc), b2 + off_wc, err, s));
  prof.mark(PH_PREP);
  if (m > 0) {
    Inputs sub;
    memset(&sub, 0, sizeof(sub));
    sub.succ = (const uint32_t *)(b2 + off_sc);
    sub.weight = b2 + off_wc;
    sub.wtype = wc;
    sub.rank = b2 + off_rc;
    sub.rank_bytes = in.rank_bytes;
    sub.n = m;
    sub.validate = in.validate;
    sub.seed = in.seed;
    sub.ctx = c;
    sub.incl = 1;
    sub.err_ext = err;
    sub.no_contract = 1;
    st = run(sub, tuning, s);
    if (st != LR_OK) return st;
  }
  prof.mark(PH_CHASE0);
  LR_TRY(launch_lc_finish(in.succ, in.weight, in.wtype, n, in.rank, in.rank_bytes, tail16, hb, wpre, tpre,
                          b2 + off_rc, s));
  prof.mark(PH_FINAL);
  prof.end();
  return finish_call(c, err, in.sync, s);
}

lr_status run(const Inputs &in, const lr_tuning *tuning, cudaStream_t s) {
  const bool ptrs = in.sptr != nullptr;
  lr_status st = LR_OK;
  Ctx *c = in.ctx ? in.ctx : get_ctx(s, &st);
  if (!c) return st;
  if (in.n == 0) {
    // nothing to rank; still clear the stream's recorded status
    c->host_words[0] = 0;
    c->pending_status = false;
    return LR_OK;
  }
  const bool capturing = stream_capturing(s);
  const Tuning u = in.builtin_tuning ? resolve_tuning_builtin((int64_t)in.n, in.wtype != 0, false)
                                     : resolve_tuning(tuning, (int64_t)in.n, in.wtype != 0,
                                                      in.offsets != nullptr || ptrs);
  if (u.algo == LR_ALGO_WYLLIE && !ptrs) {
    if (in.term || in.prefix || in.incl) return LR_ERR_INVALID_ARGUMENT;   // default algorithm only
    return run_wyllie(in, c, s);
  }
  if (u.algo != LR_ALGO_SRS && u.algo != LR_ALGO_WYLLIE) return LR_ERR_INVALID_ARGUMENT;
  const bool rec16_0 = in.wtype != 0;
  const bool extras = in.term != nullptr || in.prefix != nullptr || in.incl != 0;
  if (extras && ptrs) return LR_ERR_INVALID_ARGUMENT;
  const bool log0 = use_log0(u, in.n, in.wtype != 0, in.rank_bytes, extras, ptrs || in.offsets != nullptr);
  const bool t0ws = extras && in.term == nullptr;
  const bool spawn0 = u.spawn != 0 && u.xchg != 0 && !log0 && !extras && !ptrs;
  // a batch chases its level-0 rulers in element order (the has-predecessor
  // bitmap, free once the heads are chosen, holds the ruler marks; level 1's
  // rank array, written only after the chase, holds the order)
  const bool ord0 = use_ord0(u, in.n, log0, spawn0, extras, ptrs || in.offsets != nullptr);
  // tile-local contraction: forced, or decided from the count of links that
  // stay inside their tile (the log form's first pass counts them and they
  // are read with the list count; otherwise a sample of the tiles decides)
  const bool contractible = u.contract != LR_CONTRACT_OFF && !in.no_contract && !ptrs &&
                            in.offsets == nullptr && !extras && in.ws == nullptr && in.ctx == nullptr &&
                            !capturing && in.max_lists <= 0 && in.n >= 16384 && in.n <= 0xFFFFFFFEull;
  if (contractible && u.contract == LR_CONTRACT_ON) {
    const lr_status cs = run_contracted(in, tuning, c, true, s);
    if (cs != LR_ERR_NOT_FOUND) return cs;
  }
  const bool count_local = contractible && u.contract == LR_CONTRACT_AUTO;
  const int grid = chase_grid_for(u, rec16_0, log0, ord0);
  const bool need_count = in.max_lists <= 0 && (in.ws == nullptr || in.count_in_ws) &&
                          (in.n > u.cutoff || ptrs);
  if (need_count && capturing) return LR_ERR_CAPTURE;
  uint64_t hb = in.max_lists > 0 ? (uint64_t)in.max_lists : in.n;
  Plan p = make_plan(in.n, hb, u, rec16_0, in.rank_bytes, in.seed, grid, ptrs, log0, extras, t0ws, spawn0,
                     ord0);

  // fixed part (level 0)
  char *fixed = nullptr;
  char *var = nullptr;
  if (in.ws) {
    if (in.ws_bytes < p.fixed_bytes + (need_count ? 0 : p.var_bytes)) return LR_ERR_INVALID_ARGUMENT;
    fixed = (char *)in.ws;
    var = fixed + p.fixed_bytes;
  } else {
    st = ensure_buffer(&c->fixed, &c->fixed_bytes, p.fixed_bytes, s);
    if (st != LR_OK) return st;
    fixed = (char *)c->fixed;
  }
  LevelDesc *desc = (LevelDesc *)(fixed + p.off_desc);
  uint32_t *err = in.err_ext ? in.err_ext : (uint32_t *)(fixed + p.off_err);
  uint32_t *hcount = (uint32_t *)(fixed + p.off_hcount);
  uint32_t *qctr = (uint32_t *)(fixed + p.off_q);
  uint64_t *bcnt = (uint64_t *)(fixed + p.off_bcnt);
  uint32_t *bitmap = (uint32_t *)(fixed + p.off_bitmap);
  void *work0 = fixed + p.off_work[0];

  // Single instance, no validation: heads from the streaming sums (one list)
  // with the bitmap as the fallback, instead of atomics for every element.
  const bool sums0 = !log0 && !ptrs && in.offsets == nullptr && !in.validate && in.n > u.cutoff;
  // A batch (contiguous or one pointer per instance): per-instance sums (kept
  // at the start of the bitmap's memory, which must hold 16 bytes per
  // instance) give one head per instance and the number of lists, with the
  // bitmap as the fallback for the heads.
  const bool sums0b = !log0 && in.offsets != nullptr && !in.validate && !extras && !spawn0 &&
                      in.n > u.cutoff && in.k > 0 && (uint64_t)in.k * 16 <= 4 * ((in.n + 31) / 32);
  Profiler prof;
  if (!in.ctx) prof.begin(s, (int64_t)in.n);
  unsigned long long *acc = (unsigned long long *)(fixed + p.off_acc);
  LR_TRY(cudaMemsetAsync(fixed + p.off_zero, 0, p.zero_bytes, s));
  // A first pass that packs records (the exchange form) would pack them in
  // vain for an input that is then contracted: decide from a sample of the
  // tiles first.  (The log form's first pass only reads succ, and counts
  // every tile on the way.)
  const bool local_exact = count_local && log0;
  if (count_local && !log0) {
    LR_TRY(launch_local_sample(in.succ, (uint32_t)in.n, acc + 2, s));
    LR_TRY(cudaMemcpyAsync(c->host_words + 4, acc + 2, 16, cudaMemcpyDeviceToHost, s));
    LR_TRY(cudaStreamSynchronize(s));
    uint64_t smp[2];
    memcpy(smp, c->host_words + 4, 16);
    if (smp[0] * 2 >= smp[1]) {                // at least half the sampled links stay in their tile
      prof.cancel();
      const lr_status cs = run_contracted(in, tuning, c, false, s);
      if (cs != LR_ERR_NOT_FOUND) return cs;
      prof.begin(s, (int64_t)in.n);            // not contracted after all: carry on
    }
  }
  LR_TRY(cudaMemsetAsync(bitmap, 0, sizeof(uint32_t) * ((in.n + 31) / 32), s));
  if (log0)
    LR_TRY(launch_sum0(in.succ, (uint32_t)in.n, acc, local_exact ? acc + 2 : nullptr, err, s));
  else if (ptrs && sums0b)
    LR_TRY(launch_prep0_ptrs_sums(in.sptr, in.wptr, in.wtype, (uint32_t)in.n, work0, err, in.offsets, in.k,
                                  reinterpret_cast<unsigned long long *>(bitmap), s));
  else if (ptrs)
    LR_TRY(launch_prep0_ptrs(in.sptr, in.wptr, in.wtype, (uint32_t)in.n, work0, bitmap, err,
                             in.validate, in.offsets, in.k, s));
  else if (sums0b)
    LR_TRY(launch_prep0_sums(in.succ, in.weight, in.wtype, (uint32_t)in.n, work0, err, in.offsets, in.k,
                             reinterpret_cast<unsigned long long *>(bitmap), s));
  else
    LR_TRY(launch_prep0(in.succ, in.weight, in.wtype, (uint32_t)in.n, work0, bitmap, err,
                        in.validate, in.offsets, in.k, sums0 ? acc : nullptr, nullptr, s));
  if (need_count) {
    // count the lists (one wait), then size the recursion for exactly that many:
    // a single-instance pass counts terminals in its reduction, a batch adds
    // its instances' terminal counts, the other passes count zero bits of the
    // has-predecessor bitmap
    if (log0 || sums0) {
      LR_TRY(cudaMemcpyAsync(c->host_words + 1, acc, 4, cudaMemcpyDeviceToHost, s));
    } else if (sums0b) {
      LR_TRY(launch_count_batch(reinterpret_cast<const unsigned long long *>(bitmap), in.k, hcount, s));
      LR_TRY(cudaMemcpyAsync(c->host_words + 1, hcount, 4, cudaMemcpyDeviceToHost, s));
    } else {
      LR_TRY(launch_count_heads(bitmap, (uint32_t)in.n, hcount, s));
      LR_TRY(cudaMemcpyAsync(c->host_words + 1, hcount, 4, cudaMemcpyDeviceToHost, s));
    }
    if (local_exact)
      LR_TRY(cudaMemcpyAsync(c->host_words + 2, acc + 2, 8, cudaMemcpyDeviceToHost, s));
    LR_TRY(cudaStreamSynchronize(s));
    if (local_exact) {
      uint64_t local_links;
      memcpy(&local_links, c->host_words + 2, 8);
      if (local_links * 2 >= in.n) {           // at least half the links stay in their tile
        prof.cancel();
        const lr_status cs = run_contracted(in, tuning, c, false, s);
        if (cs != LR_ERR_NOT_FOUND) return cs;
        prof.begin(s, (int64_t)in.n);          // not contracted after all: carry on
      }
    }
    hb = std::max<uint64_t>(1, c->host_words[1]);
    p = make_plan(in.n, hb, u, rec16_0, in.rank_bytes, in.seed, grid, ptrs, log0, extras, t0ws, spawn0,
                  ord0);
  }
  if (!in.ws) {
    st = ensure_buffer(&c->var, &c->var_bytes, p.var_bytes, s);
    if (st != LR_OK) return st;
    var = (char *)c->var;
  } else if (in.ws_bytes < p.fixed_bytes + p.var_bytes) {
    LR_TRY(cudaStreamSynchronize(s));     // nothing else may still write the caller's memory
    return LR_ERR_CAPACITY;               // the lists need more workspace than was given
  }
  prof.mark(PH_PREP);

  InitParams ip;
  memset(&ip, 0, sizeof(ip));
  ip.nlev = p.nlev;
  ip.n0 = (uint32_t)in.n;
  ip.mode0 = p.nlev == 1 ? kModeBase : kModeSrs;
  ip.cutoff = p.cutoff;
  for (int l = 0; l < p.nlev; ++l) {
    ip.f_inv[l] = p.f_inv[l];
    ip.cap[l] = p.cap[l];
    ip.seed[l] = p.seed[l];
  }
  ip.pd_rounds = p.pd_rounds;
  ip.has_pd = p.has_pd;
  ip.hcap = p.hcap;
  LR_TRY(launch_init(desc, ip, s));
  if (!in.ctx) { c->last_desc = desc; c->last_nlev = p.nlev; }
  if (p.spawn_cap) LR_TRY(cudaMemsetAsync(var + p.off_sctr, 0, p.spawn_zero, s));
  SpawnArgs spa;
  memset(&spa, 0, sizeof(spa));
  if (p.spawn_cap) {
    spa.ctr = (uint32_t *)(var + p.off_sctr);
    spa.cap = p.spawn_cap;
    spa.used = (uint32_t *)(var + p.off_sused);
    spa.cursor = (uint32_t *)(var + p.off_sctr + 16);
  }
  uint32_t *hA0 = (uint32_t *)(var + p.off_hA);
  if (log0) {
    LR_TRY(cudaMemsetAsync(var + p.off_hdr, 0xFF, (size_t)p.total_chunks * 8, s));
    LR_TRY(cudaMemsetAsync(var + p.off_cur, 0, p.cur_bytes, s));
  }
  if (log0 || sums0)
    LR_TRY(launch_heads0_log(desc, acc, hA0, in.succ, (uint32_t)in.n, bitmap, err, in.validate, s));
  else if (sums0b)
    LR_TRY(launch_heads0_batch(desc, reinterpret_cast<unsigned long long *>(bitmap), in.offsets, in.k, hA0,
                               p.hcap, work0, rec16_0, (uint32_t)in.n, bitmap, s));

  auto work_of = [&](int l) -> void * { return l == 0 ? work0 : (void *)(var + p.off_work[l]); };
  auto R_of = [&](int l) -> void * { return l == 0 ? in.rank : (void *)(var + p.off_R[l]); };
  // terminal ids: T_l of every element of level l (the caller's array, or
  // workspace, at level 0), tid_l of every terminal of level l >= 1
  uint32_t *T0 = extras ? (in.term ? in.term : (uint32_t *)(var + p.off_T0)) : nullptr;
  auto T_of = [&](int l) -> uint32_t * {
    if (!extras) return nullptr;
    return l == 0 ? T0 : (uint32_t *)(var + p.off_T[l]);
  };
  auto tid_of = [&](int l) -> uint32_t * {
    return (extras && l > 0) ? (uint32_t *)(var + p.off_tid[l]) : nullptr;
  };
  uint32_t *hA = (uint32_t *)(var + p.off_hA);
  uint32_t *hB = (uint32_t *)(var + p.off_hB);
  uint32_t *hC = extras ? (uint32_t *)(var + p.off_hC) : hA;
  uint32_t *ns = (uint32_t *)(var + p.off_ns);
  const int L = p.nlev - 1;
  for (int l = 0; l < L; ++l) {
    const bool r16 = l > 0 || rec16_0;
    // head lists alternate between buffers; with extra outputs level 0's
    // list (hA) stays intact for the prefix pass
    uint32_t *hin = l == 0 ? hA : ((l & 1) ? hB : hC);
    uint32_t *hout = l == 0 ? hB : ((l & 1) ? hC : hB);
    if (l > 0) {
      LR_TRY(launch_base(desc, l, work_of(l), r16, R_of(l), p.rank_bytes, p.cutoff, err, tid_of(l),
                         T_of(l), s));
      prof.mark(PH_BASE);
    }
    const int kind = (l == 0 && log0) ? kRecKindSucc : (r16 ? kRecKind16 : kRecKind8);
    LR_TRY(launch_heads(desc, l, p.nlev, bitmap, hin, (l == 0 && log0) ? (void *)in.succ : work_of(l),
                        kind, ns, hout, bcnt, err, p.cutoff, p.hcap, p.has_pd ? 1u : 0u, s));
    prof.mark(PH_SELECT);
    if (l == 0 && log0)
      LR_TRY(launch_chase_log(desc, in.succ, work_of(1), ns, qctr, p.chase_grid, p.chase_block, err,
                              (uint32_t *)(var + p.off_log), (uint2 *)(var + p.off_hdr),
                              p.total_chunks, (uint32_t *)(fixed + p.off_logctr), s));
    else if (l == 0 && p.spawn_cap) {
      // spawning: reduced records at uncompacted ids, then compacted into level 1
      LR_TRY(launch_chase(desc, 0, work0, r16, var + p.off_sraw, ns, qctr, p.chase_grid, p.chase_block,
                          err, (int)u.xchg, nullptr, nullptr, &spa, nullptr, s));
      LR_TRY(launch_spawn_compact(desc, 0, p.nlev, spa.ctr, spa.cap, spa.used, (uint32_t *)(var + p.off_supre),
                                  var + p.off_sraw, work_of(1), p.raw_cap, p.cutoff, p.has_pd ? 1u : 0u,
                                  err, s));
    } else {
      OrdArgs oa;
      memset(&oa, 0, sizeof(oa));
      if (p.ord0 && (l == 0 || (u.ord >= 2 && p.cap[l] >= kOrdMinLevel))) {
        oa.ord = (uint32_t *)(var + p.off_ord);
        oa.cum = (uint32_t *)(var + p.off_cum);
        oa.bits = bitmap;        // the has-predecessor bitmap is free once level 0's heads are chosen
        oa.pf_lead = u.pf << 10;
        LR_TRY(launch_order(desc, l, p.cap[l], bcnt, &oa, hout, p.hcap, err, s));
      }
      LR_TRY(launch_chase(desc, l, work_of(l), r16, work_of(l + 1), ns,
                          qctr + (size_t)l * p.chase_grid, p.chase_grid, p.chase_block, err,
                          (int)u.xchg, tid_of(l), tid_of(l + 1), nullptr, oa.ord ? &oa : nullptr, s));
    }
    if (l == 0) prof.call.log0 = log0;
    prof.mark(l == 0 ? PH_CHASE0 : PH_CHASE);
  }
  LR_TRY(launch_base(desc, L, work_of(L), L > 0 || rec16_0, R_of(L), p.rank_bytes, p.cutoff, err,
                     tid_of(L), T_of(L), s));
  if (p.has_pd) {
    uint32_t *pt0 = extras ? (uint32_t *)(var + p.off_pdt[0]) : nullptr;
    uint32_t *pt1 = extras ? (uint32_t *)(var + p.off_pdt[1]) : nullptr;
    LR_TRY(launch_pd(desc, L, work_of(L), p.cap[L], p.pd_rounds, (uint32_t *)(var + p.off_pd[0]),
                     (uint32_t *)(var + p.off_pd[1]), (uint64_t *)(var + p.off_pd[2]),
                     (uint64_t *)(var + p.off_pd[3]), R_of(L), p.rank_bytes, err, tid_of(L), pt0, pt1,
                     T_of(L), s));
  }
  prof.mark(PH_BASE);
  for (int l = L - 1; l >= 0; --l) {
    if (l == 0 && log0)
      LR_TRY(launch_finalize_log(desc, (const uint32_t *)(var + p.off_log), (const uint2 *)(var + p.off_hdr),
                                 p.total_chunks, (const uint32_t *)(fixed + p.off_logctr), R_of(1),
                                 (uint2 *)(var + p.off_pairs),
                                 (uint2 *)(var + p.off_pairsB), (uint32_t *)(var + p.off_cur),
                                 (uint32_t *)(var + p.off_cur) + p.lg.na, p.lg, (uint32_t *)in.rank, err, s));
    else if (l == 0 && ptrs)
      LR_TRY(launch_finalize_ptrs(desc, work0, rec16_0, R_of(1), in.rptr, p.rank_bytes, p.cap[0],
                                  in.offsets, in.k, err, s));
    else if (l == 0 && p.spawn_cap) {
      LR_TRY(launch_spawn_scatter(desc, 0, R_of(1), var + p.off_srraw, p.rank_bytes, spa.used,
                                  (uint32_t *)(var + p.off_supre), p.raw_cap, s));
      LR_TRY(launch_finalize(desc, 0, work0, rec16_0, var + p.off_srraw, R_of(0), p.rank_bytes, p.cap[0],
                             err, nullptr, nullptr, nullptr, s));
    } else
      LR_TRY(launch_finalize(desc, l, work_of(l), l > 0 || rec16_0, R_of(l + 1), R_of(l),
                             p.rank_bytes, p.cap[l], err, T_of(l + 1), T_of(l), tid_of(l), s));
  }
  if (extras)
    LR_TRY(launch_outputs(desc, bitmap, hA0, (uint32_t)in.n, T0, in.rank, in.prefix, p.rank_bytes,
                          in.incl, in.weight, in.wtype, in.offsets, in.k,
                          in.offsets != nullptr && in.term != nullptr, s));
  prof.mark(PH_FINAL);
  prof.end();
  return finish_call(c, err, in.sync, s);
}

lr_status run_fixed_scratch(const uint32_t *succ, int64_t n, int32_t *rank, void *scratch,
                            size_t scratch_bytes, Ctx *ctx, cudaStream_t s) {
  Inputs in;
  memset(&in, 0, sizeof(in));
  in.succ = succ;
  in.rank = rank;
  in.rank_bytes = 4;
  in.n = (uint64_t)n;
  in.seed = 0x5eedull;
  in.sync = 1;
  in.ws = scratch;
  in.ws_bytes = scratch_bytes;
  in.ctx = ctx;
  in.count_in_ws = 1;
  // fixed settings: whether a valid list fits the scratch must not depend on
  // LR_TUNING or on what the autotuner stored in this process
  in.builtin_tuning = 1;
  return run(in, nullptr, s);
}

lr_status run_single(const uint32_t *succ, const void *weight, int wtype, void *rank, int rank_bytes,
                     int64_t n, uint64_t seed, cudaStream_t s) {
  Inputs in;
  memset(&in, 0, sizeof(in));
  in.succ = succ;
  in.weight = weight;
  in.wtype = wtype;
  in.rank = rank;
  in.rank_bytes = rank_bytes;
  in.n = (uint64_t)n;
  in.seed = seed;
  in.sync = 1;
  return run(in, nullptr, s);
}

lr_status run_ptr_batch(const int64_t *offsets, int32_t k, int64_t n_total,
                        const uint32_t *const *sptr, const void *const *wptr, void *const *rptr,
                        int wtype, int rank_bytes, uint64_t seed, cudaStream_t s) {
  Inputs in;
  memset(&in, 0, sizeof(in));
  in.n = (uint64_t)n_total;
  in.offsets = offsets;
  in.k = k;
  in.sptr = sptr;
  in.wptr = wptr;
  in.rptr = rptr;
  in.wtype = wtype;
  in.rank_bytes = rank_bytes;
  in.seed = seed;
  in.sync = 1;
  return run(in, nullptr, s);
}

lr_status status_from_bits(uint32_t bits) { return map_device_bits(bits); }

lr_status device_status(cudaStream_t s) {
  lr_status st;
  Ctx *c = get_ctx(s, &st);
  if (!c) return st;
  cudaError_t e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return from_cuda(e);
  const uint32_t bits = c->host_words[0];
  c->host_words[0] = 0;
  c->pending_status = false;
  return map_device_bits(bits);
}

}  // namespace lr

// ================================================================ C ABI
using namespace lr;

extern "C" {

void lr_opts_default(lr_opts *o) {
  if (!o) return;
  memset(o, 0, sizeof(*o));
  o->wtype = LR_NONE;
  o->rtype = LR_I32;
  o->seed = 0x5eedull;
}

const char *lr_version(void) { return "lr-gb300 0.1 (sparse ruling set, sm_103a)"; }

const char *lr_status_string(lr_status s) {
  switch (s) {
    case LR_OK: return "LR_OK";
    case LR_ERR_INVALID_ARGUMENT: return "LR_ERR_INVALID_ARGUMENT";
    case LR_ERR_OUT_OF_RANGE: return "LR_ERR_OUT_OF_RANGE";
    case LR_ERR_CYCLE: return "LR_ERR_CYCLE";
    case LR_ERR_NOT_A_LIST: return "LR_ERR_NOT_A_LIST";
    case LR_ERR_OUT_OF_MEMORY: return "LR_ERR_OUT_OF_MEMORY";
    case LR_ERR_BUDGET: return "LR_ERR_BUDGET";
    case LR_ERR_TIMEOUT: return "LR_ERR_TIMEOUT";
    case LR_ERR_CUDA: return "LR_ERR_CUDA";
    case LR_ERR_CAPACITY: return "LR_ERR_CAPACITY";
    case LR_ERR_NOT_FOUND: return "LR_ERR_NOT_FOUND";
    case LR_ERR_CANCELLED: return "LR_ERR_CANCELLED";
    case LR_ERR_CAPTURE: return "LR_ERR_CAPTURE";
    case LR_ERR_INTERNAL: return "LR_ERR_INTERNAL";
  }
  return "LR_ERR_UNKNOWN";
}

static lr_status check_types(const void *weight, lr_dtype wtype, lr_dtype rtype, int *wcode, int *rbytes) {
  if (rtype != LR_I32 && rtype != LR_I64) return LR_ERR_INVALID_ARGUMENT;
  if (wtype != LR_NONE && wtype != LR_I32 && wtype != LR_I64) return LR_ERR_INVALID_ARGUMENT;
  if ((wtype == LR_NONE) != (weight == nullptr)) return LR_ERR_INVALID_ARGUMENT;
  *wcode = (int)wtype;
  *rbytes = rtype == LR_I32 ? 4 : 8;
  return LR_OK;
}

static void set_outputs(Inputs &in, const lr_outputs *outs) {
  if (!outs) return;
  in.term = outs->term;
  in.prefix = outs->prefix;
  in.incl = outs->inclusive_tail != 0;
}

static lr_status rank_ex_impl(const uint32_t *succ, const void *weight, int64_t n, void *rank,
                              const lr_outputs *outs, const lr_opts *opts, lr_stream stream) {
  lr_opts d;
  if (!opts) { lr_opts_default(&d); if (weight) { d.wtype = LR_I64; d.rtype = LR_I64; } opts = &d; }
  if (n < 0 || n > LR_MAX_N) return LR_ERR_INVALID_ARGUMENT;
  if (n > 0 && (!succ || !rank)) return LR_ERR_INVALID_ARGUMENT;
  int wc, rb;
  lr_status st = check_types(n > 0 ? weight : (opts->wtype ? (const void *)1 : nullptr),
                             opts->wtype, opts->rtype, &wc, &rb);
  if (st != LR_OK) return st;
  Inputs in;
  memset(&in, 0, sizeof(in));
  in.succ = succ;
  in.weight = weight;
  in.wtype = wc;
  in.rank = rank;
  in.rank_bytes = rb;
  in.n = (uint64_t)n;
  in.validate = opts->validate;
  in.seed = opts->seed;
  in.max_lists = opts->max_lists;
  in.sync = opts->sync;
  in.ws = opts->workspace;
  in.ws_bytes = opts->ws_bytes;
  set_outputs(in, outs);
  return run(in, opts->tuning, (cudaStream_t)stream);
}

lr_status lr_rank_ex(const uint32_t *succ, const void *weight, int64_t n, void *rank,
                     const lr_opts *opts, lr_stream stream) {
  return rank_ex_impl(succ, weight, n, rank, nullptr, opts, stream);
}

lr_status lr_rank_outputs(const uint32_t *succ, const void *weight, int64_t n, void *rank,
                          const lr_outputs *outs, const lr_opts *opts, lr_stream stream) {
  return rank_ex_impl(succ, weight, n, rank, outs, opts, stream);
}

lr_status lr_rank(const uint32_t *succ, const void *weight, int64_t n, void *rank, lr_stream stream) {
  lr_opts o;
  lr_opts_default(&o);
  if (weight) { o.wtype = LR_I64; o.rtype = LR_I64; }
  else if (n >= ((int64_t)1 << 31)) return LR_ERR_INVALID_ARGUMENT;  // int32 ranks
  return lr_rank_ex(succ, weight, n, rank, &o, stream);
}

// The element total of a batch: n_total when given (> 0), else offsets[k]
// read back from the device (one wait on the stream).
static lr_status batch_total(const int64_t *offsets, int32_t k, int64_t n_total, cudaStream_t s, int64_t *n) {
  if (n_total > 0) {
    *n = n_total;
    return LR_OK;
  }
  if (stream_capturing(s)) return LR_ERR_CAPTURE;
  lr_status st;
  Ctx *c = get_ctx(s, &st);
  if (!c) return st;
  int64_t *h = (int64_t *)(c->host_words + 8);
  cudaError_t e = cudaMemcpyAsync(h, offsets + k, 8, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return from_cuda(e);
  *n = *h;
  return LR_OK;
}

static lr_status rank_batch_impl(const int64_t *offsets, const uint32_t *succ, const void *weight,
                                 void *rank, int32_t k, const lr_outputs *outs, const lr_opts *opts,
                                 lr_stream stream) {
  lr_opts d;
  if (!opts) { lr_opts_default(&d); if (weight) { d.wtype = LR_I64; d.rtype = LR_I64; } opts = &d; }
  if (k < 0 || (k > 0 && !offsets)) return LR_ERR_INVALID_ARGUMENT;
  if (k == 0) return LR_OK;
  cudaStream_t s = (cudaStream_t)stream;
  int64_t n = 0;
  const lr_status nst = batch_total(offsets, k, opts->n_total, s, &n);
  if (nst != LR_OK) return nst;
  if (n < 0 || n > LR_MAX_N) return LR_ERR_INVALID_ARGUMENT;
  if (n > 0 && (!succ || !rank)) return LR_ERR_INVALID_ARGUMENT;
  int wc, rb;
  lr_status st = check_types(n > 0 ? weight : (opts->wtype ? (const void *)1 : nullptr),
                             opts->wtype, opts->rtype, &wc, &rb);
  if (st != LR_OK) return st;
  Inputs in;
  memset(&in, 0, sizeof(in));
  in.succ = succ;
  in.weight = weight;
  in.wtype = wc;
  in.rank = rank;
  in.rank_bytes = rb;
  in.n = (uint64_t)n;
  in.offsets = offsets;
  in.k = k;
  in.validate = opts->validate;
  in.seed = opts->seed;
  in.max_lists = opts->max_lists;
  in.sync = opts->sync;
  in.ws = opts->workspace;
  in.ws_bytes = opts->ws_bytes;
  set_outputs(in, outs);
  return run(in, opts->tuning, s);
}

lr_status lr_rank_batch_ex(const int64_t *offsets, const uint32_t *succ, const void *weight,
                           void *rank, int32_t k, const lr_opts *opts, lr_stream stream) {
  return rank_batch_impl(offsets, succ, weight, rank, k, nullptr, opts, stream);
}

lr_status lr_rank_batch_outputs(const int64_t *offsets, const uint32_t *succ, const void *weight,
                                void *rank, int32_t k, const lr_outputs *outs, const lr_opts *opts,
                                lr_stream stream) {
  return rank_batch_impl(offsets, succ, weight, rank, k, outs, opts, stream);
}

lr_status lr_rank_batch(const int64_t *offsets, const uint32_t *succ, const void *weight,
                        void *rank, int32_t k, lr_stream stream) {
  lr_opts o;
  lr_opts_default(&o);
  if (weight) { o.wtype = LR_I64; o.rtype = LR_I64; }
  return lr_rank_batch_ex(offsets, succ, weight, rank, k, &o, stream);
}

lr_status lr_rank_batch_ptrs(const int64_t *offsets, const uint32_t *const *succ_ptrs,
                             const void *const *weight_ptrs, void *const *rank_ptrs, int32_t k,
                             const lr_opts *opts, lr_stream stream) {
  lr_opts d;
  if (!opts) {
    lr_opts_default(&d);
    if (weight_ptrs) { d.wtype = LR_I64; d.rtype = LR_I64; }
    opts = &d;
  }
  if (k < 0 || (k > 0 && (!offsets || !succ_ptrs || !rank_ptrs))) return LR_ERR_INVALID_ARGUMENT;
  if (k == 0) return LR_OK;
  if (opts->workspace) return LR_ERR_INVALID_ARGUMENT;   // the pointer form keeps its own workspace
  cudaStream_t s = (cudaStream_t)stream;
  // the kernels index the caller's buffers through the offset table, so it is
  // read back and checked here before any of them runs (one wait)
  if (stream_capturing(s)) return LR_ERR_CAPTURE;
  std::vector<int64_t> h((size_t)k + 1);
  cudaError_t e = cudaMemcpyAsync(h.data(), offsets, 8 * ((size_t)k + 1), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return from_cuda(e);
  if (h[0] != 0) return LR_ERR_INVALID_ARGUMENT;
  for (int32_t j = 0; j < k; ++j)
    if (h[j + 1] < h[j]) return LR_ERR_INVALID_ARGUMENT;
  const int64_t n = h[k];
  if (n > LR_MAX_N || (opts->n_total > 0 && opts->n_total != n)) return LR_ERR_INVALID_ARGUMENT;
  int wc, rb;
  lr_status st = check_types(weight_ptrs, opts->wtype, opts->rtype, &wc, &rb);
  if (st != LR_OK) return st;
  if (n == 0) return LR_OK;
  Inputs in;
  memset(&in, 0, sizeof(in));
  in.sptr = succ_ptrs;
  in.wptr = weight_ptrs;
  in.rptr = rank_ptrs;
  in.wtype = wc;
  in.rank_bytes = rb;
  in.n = (uint64_t)n;
  in.offsets = offsets;
  in.k = k;
  in.validate = opts->validate;
  in.seed = opts->seed;
  in.max_lists = opts->max_lists;
  in.sync = opts->sync;
  return run(in, opts->tuning, s);
}

// Enqueue copy-in, ranking and copy-out on `stream` through the stream's own
// device staging buffers; `sync` waits and returns the final status.
static lr_status rank_host_impl(const uint32_t *succ_host, const void *weight_host, int64_t n,
                                void *rank_host, const lr_opts *opts, lr_stream stream, bool sync);

lr_status lr_rank_host(const uint32_t *succ_host, const void *weight_host, int64_t n,
                       void *rank_host, const lr_opts *opts, lr_stream stream) {
  return rank_host_impl(succ_host, weight_host, n, rank_host, opts, stream, true);
}

lr_status lr_rank_host_async(const uint32_t *succ_host, const void *weight_host, int64_t n,
                             void *rank_host, const lr_opts *opts, lr_stream stream) {
  return rank_host_impl(succ_host, weight_host, n, rank_host, opts, stream, false);
}

static lr_status rank_host_impl(const uint32_t *succ_host, const void *weight_host, int64_t n,
                                void *rank_host, const lr_opts *opts, lr_stream stream, bool sync) {
  lr_opts d;
  if (!opts) { lr_opts_default(&d); if (weight_host) { d.wtype = LR_I64; d.rtype = LR_I64; } opts = &d; }
  if (n < 0 || n > LR_MAX_N) return LR_ERR_INVALID_ARGUMENT;
  if (n == 0) return LR_OK;
  if (!succ_host || !rank_host) return LR_ERR_INVALID_ARGUMENT;
  int wc, rb;
  lr_status st = check_types(weight_host, opts->wtype, opts->rtype, &wc, &rb);
  if (st != LR_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  if (stream_capturing(s)) return LR_ERR_CAPTURE;
  Ctx *c = get_ctx(s, &st);
  if (!c) return st;
  const size_t wb = wc == 0 ? 0 : (wc == 1 ? 4 : 8);
  const size_t bs = align_up(4 * (size_t)n), bw = align_up(wb * (size_t)n), br = align_up((size_t)rb * n);
  st = ensure_buffer(&c->hostpath, &c->hostpath_bytes, bs + bw + br, s);
  if (st != LR_OK) return st;
  char *b = (char *)c->hostpath;
  uint32_t *dsucc = (uint32_t *)b;
  void *dw = wb ? (void *)(b + bs) : nullptr;
  void *drank = b + bs + bw;
  LR_TRY(cudaMemcpyAsync(dsucc, succ_host, 4 * (size_t)n, cudaMemcpyHostToDevice, s));
  if (wb) LR_TRY(cudaMemcpyAsync(dw, weight_host, wb * (size_t)n, cudaMemcpyHostToDevice, s));
  lr_opts o = *opts;
  o.sync = 0;
  st = lr_rank_ex(dsucc, dw, n, drank, &o, stream);
  if (st != LR_OK) return st;
  LR_TRY(cudaMemcpyAsync(rank_host, drank, (size_t)rb * n, cudaMemcpyDeviceToHost, s));
  return sync ? device_status(s) : LR_OK;
}

size_t lr_workspace_size(int64_t n_total, int32_t k, const lr_opts *opts) {
  return lr_workspace_size_outputs(n_total, k, nullptr, opts);
}

size_t lr_workspace_size_outputs(int64_t n_total, int32_t k, const lr_outputs *outs,
                                 const lr_opts *opts) {
  lr_opts d;
  if (!opts) { lr_opts_default(&d); opts = &d; }
  if (n_total <= 0) return 0;
  const Tuning u = resolve_tuning(opts->tuning, n_total, opts->wtype != LR_NONE, k > 0);
  // The chase grid depends on the device; size for a generous upper bound so
  // the answer needs no GPU: 256 SMs x 16 CTAs.
  if (u.algo == LR_ALGO_WYLLIE) {
    Inputs in;
    memset(&in, 0, sizeof(in));
    in.wtype = opts->wtype != LR_NONE;
    in.rank_bytes = opts->rtype == LR_I64 ? 8 : 4;
    return wyllie_plan((uint64_t)n_total, wyllie_w16(in)).bytes;
  }
  const uint64_t h = opts->max_lists > 0 ? (uint64_t)opts->max_lists : (uint64_t)n_total;
  const bool extras = outs && (outs->term || outs->prefix || outs->inclusive_tail);
  const bool log0 = use_log0(u, (uint64_t)n_total, opts->wtype != LR_NONE, opts->rtype == LR_I64 ? 8 : 4,
                             extras, k != 0);
  const bool spawn0 = u.spawn != 0 && u.xchg != 0 && !log0 && !extras;
  const bool ord0 = use_ord0(u, (uint64_t)n_total, log0, spawn0, extras, k != 0);
  Plan p = make_plan((uint64_t)n_total, h, u, opts->wtype != LR_NONE,
                     opts->rtype == LR_I64 ? 8 : 4, opts->seed, 256 * 16, false, log0, extras,
                     extras && !outs->term, spawn0, ord0);
  return p.fixed_bytes + p.var_bytes;
}

lr_status lr_get_device_status(lr_stream stream) { return device_status((cudaStream_t)stream); }

int32_t lr_level_sizes(lr_stream stream, int64_t *sizes, int32_t max_levels) {
  lr_status st;
  Ctx *c = get_ctx((cudaStream_t)stream, &st);
  if (!c || !c->last_desc || c->last_nlev <= 0) return 0;
  LevelDesc d[kMaxLevels + 1];
  if (cudaMemcpyAsync(d, c->last_desc, sizeof(LevelDesc) * c->last_nlev, cudaMemcpyDeviceToHost,
                      (cudaStream_t)stream) != cudaSuccess ||
      cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess)
    return -1;
  int32_t used = 0;
  for (int l = 0; l < c->last_nlev; ++l) {
    if (d[l].mode == kModeOff) break;
    if (sizes && used < max_levels) sizes[used] = d[l].n;
    ++used;
  }
  return used;
}

lr_status lr_profile_enable(int32_t on) {
  std::lock_guard<std::mutex> g(g_mu);
  g_prof = on != 0;
  return LR_OK;
}

lr_status lr_profile_read(lr_profile *out, int32_t reset) {
  std::vector<ProfCall> pend;
  {
    std::lock_guard<std::mutex> g(g_mu);
    pend.swap(g_prof_pending);
  }
  for (auto &call : pend) {
    for (size_t i = 1; i < call.marks.size(); ++i) {
      float ms = 0.f;
      cudaEventSynchronize(call.marks[i].ev);
      cudaEventElapsedTime(&ms, call.marks[i - 1].ev, call.marks[i].ev);
      switch (call.marks[i].phase) {
        case PH_PREP: g_prof_acc.ms_prep += ms; break;
        case PH_SELECT: g_prof_acc.ms_select += ms; break;
        case PH_CHASE0:
          g_prof_acc.ms_chase0 += ms;
          g_prof_acc.chase0_launches += 1;
          g_prof_acc.chase0_log_launches += call.log0 ? 1 : 0;
          break;
        case PH_CHASE: g_prof_acc.ms_chase_rest += ms; break;
        case PH_BASE: g_prof_acc.ms_base += ms; break;
        case PH_FINAL: g_prof_acc.ms_finalize += ms; break;
      }
    }
    for (auto &m : call.marks) cudaEventDestroy(m.ev);
    g_prof_acc.calls += 1;
    g_prof_acc.kernel_launches += call.launches;
    g_prof_acc.elements += call.n;
  }
  if (out) *out = g_prof_acc;
  if (reset) memset(&g_prof_acc, 0, sizeof(g_prof_acc));
  return LR_OK;
}

int64_t lr_kernel_launch_count(void) { return launch_count(); }

}  // extern "C"
