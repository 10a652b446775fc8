// lr_probe.cu -- memory-system probes behind lr_probe_memory (measurement only).
//
// The level-0 chase is a dependent random walk, so its ceiling is not the
// streaming HBM bandwidth but the rate at which the GPU serves random
// accesses.  That rate depends on the footprint the accesses cover (the part
// that L2 holds, the page-table reach) and, on GB300, hardly at all on how
// many accesses are in flight.  These probes measure, over the caller's
// buffer (its size is the footprint):
//   copy         streaming read + write, bytes per second;
//   gather       one dependent random 4-byte load per step over 4-byte slots
//                (the log-form chase's gather of succ[x]), steps per second;
//   indep        independent random 4-byte loads, kIndepIlp in flight per
//                thread, indices from a hash (no dependence, no index
//                stream): the rate with as much memory-level parallelism as
//                the loads can have;
//   region       the same, but every warp draws a random 2 MiB-aligned
//                region per round and its lanes gather inside it: what the
//                rate becomes when each warp's accesses share one page;
//   gather_xchg  one dependent random 8-byte atomic exchange per step over
//                8-byte slots (the exchange-form chase), steps per second.
// Each walk visits every slot of one seeded random cycle once.
#include <cuda_runtime.h>

#include <algorithm>

#include "lr.h"
#include "lr_device.cuh"
#include "lr_kernels.h"

namespace lr {

constexpr int kIndepIlp = 8;
constexpr uint32_t kRegionShift = 21;      // 2 MiB regions

__global__ void k_probe_setup4(uint32_t *A, uint32_t n, uint64_t seed) {
  Perm P;
  P.init(n, seed);
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const uint32_t p = P.fwd(i);
    A[i] = P.inv(p + 1 == n ? 0u : p + 1);
  }
}

__global__ void k_probe_setup8(uint2 *A, uint32_t n, uint64_t seed) {
  Perm P;
  P.init(n, seed);
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const uint32_t p = P.fwd(i);
    A[i] = make_uint2(P.inv(p + 1 == n ? 0u : p + 1), 0u);
  }
}

// Dependent walk over 4-byte slots: x = A[x], `steps` times per thread.
__global__ void k_probe_walk4(const uint32_t *__restrict__ A, uint32_t n, uint64_t seed, uint32_t steps,
                              uint32_t *sink) {
  Perm P;
  P.init(n, seed);
  const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
  uint32_t x = P.inv((uint32_t)(((uint64_t)t * steps) % n));
  for (uint32_t s = 0; s < steps; ++s) x = __ldcg(A + x);
  if (x == 0xFFFFFFFFu) *sink = x;
}

// Dependent walk over 8-byte slots with an atomic exchange per step: write
// back the true successor with this walker's tag and continue from the
// returned word, so the chain stays dependent and the cycle intact.
__global__ void k_probe_xchg8(uint2 *A, uint32_t n, uint64_t seed, uint32_t steps, uint32_t *sink) {
  Perm P;
  P.init(n, seed);
  const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
  uint32_t x = P.inv((uint32_t)(((uint64_t)t * steps) % n));
  uint32_t acc = 0;
  for (uint32_t s = 0; s < steps; ++s) {
    const uint32_t p = P.fwd(x);
    const uint32_t nx = P.inv(p + 1 == n ? 0u : p + 1);
    const unsigned long long o =
        atomicExch(reinterpret_cast<unsigned long long *>(A + x), ((unsigned long long)t << 32) | nx);
    acc += (uint32_t)(o >> 32);
    x = (uint32_t)o;
  }
  if (acc == 0x7FFFFFFFu) *sink = acc;
}

__device__ __forceinline__ uint32_t probe_hash(uint32_t x) {
  x ^= x >> 16;
  x *= 0x7feb352du;
  x ^= x >> 15;
  x *= 0x846ca68bu;
  x ^= x >> 16;
  return x;
}

// Independent gathers: kIndepIlp loads issued before any is used.  With
// region_slots > 0 the warp draws one region of that many slots per load
// round (all lanes of the warp the same region) and gathers inside it.
__global__ void k_probe_indep4(const uint32_t *__restrict__ A, uint32_t n, uint32_t rounds,
                               uint32_t region_slots, uint32_t *sink) {
  const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
  const uint32_t w = t >> 5;
  const uint32_t nreg = region_slots ? n / region_slots : 0;
  uint32_t acc = 0;
  for (uint32_t it = 0; it < rounds; ++it) {
    uint32_t v[kIndepIlp];
#pragma unroll
    for (int j = 0; j < kIndepIlp; ++j) {
      const uint32_t k = it * kIndepIlp + (uint32_t)j;
      const uint32_t h = probe_hash(t * 0x9E3779B1u + k * 0x85EBCA77u + 0x3243F6A9u);
      uint32_t idx;
      if (nreg == 0) {
        idx = (uint32_t)(((uint64_t)h * n) >> 32);
      } else {
        const uint32_t hr = probe_hash(w * 0x27D4EB2Fu + k * 0x165667B1u + 0x13198A2Eu);
        const uint32_t reg = (uint32_t)(((uint64_t)hr * nreg) >> 32);
        idx = reg * region_slots + (uint32_t)(((uint64_t)h * region_slots) >> 32);
      }
      v[j] = __ldcg(A + idx);
    }
#pragma unroll
    for (int j = 0; j < kIndepIlp; ++j) acc += v[j];
  }
  if (acc == 0x7FFFFFFFu) *sink = acc;
}

__global__ void k_probe_copy(const uint4 *a, uint4 *b, size_t n4) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n4; i += (size_t)gridDim.x * blockDim.x)
    b[i] = __ldcs(a + i);
}

}  // namespace lr

extern "C" lr_status lr_probe_memory(void *buf, size_t bytes, lr_probe_result *out, lr_stream stream) {
  using namespace lr;
  if (!buf || !out || bytes < ((size_t)16 << 20) || ((uintptr_t)buf & 255u)) return LR_ERR_INVALID_ARGUMENT;
  cudaStream_t s = (cudaStream_t)stream;
  // 4-byte slots for the gathers, 8-byte slots for the exchanges, then one
  // 256-byte sink; the walk arrays stay below 2^32 slots
  const size_t usable = (bytes - 256) & ~(size_t)255;
  uint64_t n4l = usable / 4, n8l = usable / 8;
  if (n4l > 0xFFFFFFF0ull) n4l = 0xFFFFFFF0ull;
  if (n8l > 0xFFFFFFF0ull) n8l = 0xFFFFFFF0ull;
  const uint32_t n4 = (uint32_t)n4l, n8 = (uint32_t)n8l;
  uint32_t *A4 = reinterpret_cast<uint32_t *>(buf);
  uint2 *A8 = reinterpret_cast<uint2 *>(buf);
  uint32_t *sink = reinterpret_cast<uint32_t *>(reinterpret_cast<char *>(buf) + usable);
  const int sms = device_sm_count();
  const uint32_t threads = (uint32_t)sms * 1024u;
  const uint32_t steps4 = n4 / threads, steps8 = n8 / threads;
  if (steps4 == 0 || steps8 == 0) return LR_ERR_INVALID_ARGUMENT;
  const uint32_t region_slots = 1u << (kRegionShift - 2);
  const uint32_t rounds = std::max<uint32_t>(1u, (uint32_t)(((uint64_t)n4 / kIndepIlp) / threads));
  const uint64_t seed = 0x9e0be;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return LR_ERR_CUDA;
  float ms[5] = {0, 0, 0, 0, 0};
  lr_status st = LR_OK;
  auto timed = [&](int slot, auto launch) {
    cudaEventRecord(e0, s);
    launch();
    cudaEventRecord(e1, s);
    cudaEventSynchronize(e1);
    cudaEventElapsedTime(&ms[slot], e0, e1);
  };
  for (int rep = 0; rep < 2 && st == LR_OK; ++rep) {      // the first pass warms up
    k_probe_setup4<<<sms * 8, 256, 0, s>>>(A4, n4, seed);
    timed(0, [&] { k_probe_walk4<<<threads / 256, 256, 0, s>>>(A4, n4, seed, steps4, sink); });
    timed(1, [&] { k_probe_indep4<<<threads / 256, 256, 0, s>>>(A4, n4, rounds, 0u, sink); });
    if (n4 >= 2 * region_slots)
      timed(2, [&] { k_probe_indep4<<<threads / 256, 256, 0, s>>>(A4, n4, rounds, region_slots, sink); });
    k_probe_setup8<<<sms * 8, 256, 0, s>>>(A8, n8, seed);
    timed(3, [&] { k_probe_xchg8<<<threads / 256, 256, 0, s>>>(A8, n8, seed, steps8, sink); });
    const size_t half = (usable / 2) & ~(size_t)255;
    timed(4, [&] {
      k_probe_copy<<<sms * 8, 256, 0, s>>>(reinterpret_cast<const uint4 *>(buf),
                                          reinterpret_cast<uint4 *>(reinterpret_cast<char *>(buf) + half),
                                          half / 16);
    });
    out->copy_gbs = 2.0 * (double)half / (ms[4] * 1e-3) / 1e9;
    if (cudaGetLastError() != cudaSuccess) st = LR_ERR_CUDA;
  }
  count_launch(n4 >= 2 * region_slots ? 14 : 12);
  out->gather_gsteps = (double)threads * steps4 / (ms[0] * 1e-3) / 1e9;
  out->indep_gather_gsteps = (double)threads * rounds * kIndepIlp / (ms[1] * 1e-3) / 1e9;
  out->region_gather_gsteps =
      n4 >= 2 * region_slots ? (double)threads * rounds * kIndepIlp / (ms[2] * 1e-3) / 1e9 : 0.0;
  out->gather_xchg_gsteps = (double)threads * steps8 / (ms[3] * 1e-3) / 1e9;
  out->footprint_bytes = usable;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return st;
}
