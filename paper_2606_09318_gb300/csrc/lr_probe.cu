// lr_probe.cu -- memory-system probes behind lr_probe_memory (measurement only).
//
// The level-0 chase is a dependent random walk, so its ceiling is not the
// streaming HBM bandwidth but the rate at which the GPU serves random
// 32-byte accesses that miss L2.  These probes measure, on the caller's
// buffer (far larger than L2):
//   copy        streaming read + write, bytes per second;
//   gather      one dependent random 8-byte load per step (a chase that only
//               reads), steps per second;
//   gather_xchg one dependent random 8-byte atomic exchange per step (a chase
//               that rewrites what it reads), steps per second.
// Each walk visits every slot of one seeded random cycle once.
#include <cuda_runtime.h>

#include "lr.h"
#include "lr_device.cuh"
#include "lr_kernels.h"

namespace lr {

__global__ void k_probe_setup(uint2 *A, uint32_t n, uint64_t seed) {
  Perm P;
  P.init(n, seed);
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const uint32_t p = P.fwd(i);
    A[i] = make_uint2(P.inv(p + 1 == n ? 0u : p + 1), 0u);
  }
}

template <bool XCHG>
__global__ void k_probe_walk(uint2 *A, uint32_t n, uint64_t seed, uint32_t steps, uint32_t *sink) {
  Perm P;
  P.init(n, seed);
  const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
  uint32_t x = P.inv((uint32_t)(((uint64_t)t * steps) % n));
  uint32_t acc = 0;
  for (uint32_t s = 0; s < steps; ++s) {
    if constexpr (XCHG) {
      // write back the true successor with this walker's tag, continue from
      // the returned word: still a dependent chain, and the cycle stays intact
      const uint32_t p = P.fwd(x);
      const uint32_t nx = P.inv(p + 1 == n ? 0u : p + 1);
      const unsigned long long o =
          atomicExch(reinterpret_cast<unsigned long long *>(A + x), ((unsigned long long)t << 32) | nx);
      acc += (uint32_t)(o >> 32);
      x = (uint32_t)o;
    } else {
      const uint2 v = __ldcg(A + x);
      acc += v.y;
      x = v.x;
    }
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
  if (!buf || !out || bytes < ((size_t)64 << 20) || ((uintptr_t)buf & 255u)) return LR_ERR_INVALID_ARGUMENT;
  cudaStream_t s = (cudaStream_t)stream;
  uint64_t slots = bytes / 8 - 1;               // one uint32 sink after the walk array
  if (slots > 0xFFFFFFF0ull) slots = 0xFFFFFFF0ull;
  const uint32_t n = (uint32_t)slots;
  uint2 *A = reinterpret_cast<uint2 *>(buf);
  uint32_t *sink = reinterpret_cast<uint32_t *>(A + n);
  const int sms = device_sm_count();
  const uint32_t threads = (uint32_t)sms * 1024u;
  const uint32_t steps = n / threads;
  if (steps == 0) return LR_ERR_INVALID_ARGUMENT;
  const uint64_t seed = 0x9e0be;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return LR_ERR_CUDA;
  float ms[3] = {0, 0, 0};
  lr_status st = LR_OK;
  for (int rep = 0; rep < 2 && st == LR_OK; ++rep) {      // first pass warms up
    k_probe_setup<<<sms * 8, 256, 0, s>>>(A, n, seed);
    cudaEventRecord(e0, s);
    k_probe_walk<false><<<threads / 256, 256, 0, s>>>(A, n, seed, steps, sink);
    cudaEventRecord(e1, s);
    cudaEventSynchronize(e1);
    cudaEventElapsedTime(&ms[0], e0, e1);
    cudaEventRecord(e0, s);
    k_probe_walk<true><<<threads / 256, 256, 0, s>>>(A, n, seed, steps, sink);
    cudaEventRecord(e1, s);
    cudaEventSynchronize(e1);
    cudaEventElapsedTime(&ms[1], e0, e1);
    const size_t half = ((size_t)n * 8 / 2) & ~(size_t)255;
    cudaEventRecord(e0, s);
    k_probe_copy<<<sms * 8, 256, 0, s>>>(reinterpret_cast<const uint4 *>(A),
                                        reinterpret_cast<uint4 *>(reinterpret_cast<char *>(A) + half), half / 16);
    cudaEventRecord(e1, s);
    cudaEventSynchronize(e1);
    cudaEventElapsedTime(&ms[2], e0, e1);
    out->copy_gbs = 2.0 * (double)half / (ms[2] * 1e-3) / 1e9;
    if (cudaGetLastError() != cudaSuccess) st = LR_ERR_CUDA;
  }
  count_launch(8);
  const double visits = (double)threads * steps;
  out->gather_gsteps = visits / (ms[0] * 1e-3) / 1e9;
  out->gather_xchg_gsteps = visits / (ms[1] * 1e-3) / 1e9;
  out->footprint_bytes = (size_t)n * 8;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return st;
}
