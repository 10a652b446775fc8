// lr_noalloc.cu -- lr_rank_noalloc: list ranking that allocates nothing.
//
// Some callers cannot call cudaMalloc at the point where they need a ranking:
// a process whose caching allocator has already reserved all free device
// memory, a latency-critical loop that must not risk the implicit device
// synchronisation and unbounded latency of an allocation, or a plug-in loaded
// into a host that forbids allocations after start-up.  For them this entry
// point runs the same ranking pipeline as lr_rank in a fixed scratch area
// that is part of the library image: a file-scope __device__ array of
// kNoAllocScratchBytes that every GPU which loads the library holds until the
// process exits.
//
// Host code must not take the array's name as a device address (in host code
// it names a host-side stand-in), so the library's set-up on each device (the
// first lr_* call made with that device current) asks the runtime for the
// array's device address with cudaGetSymbolAddress and keeps it.  That lookup
// is also what places the array on the device under lazy module loading, so
// it happens as early as the library can make it, not at the first
// lr_rank_noalloc call; if it failed there (no memory left), the first
// lr_rank_noalloc call tries again and returns LR_ERR_OUT_OF_MEMORY or
// LR_ERR_CUDA.  All calls share the one array and it
// keeps the last call's contents; the pipeline clears what has to start at
// zero on every call.  Calls whose work overlaps on the GPU race on the
// scratch, so callers must serialise them (one stream, or wait between calls);
// the host side keeps one status buffer per device and is not thread-safe
// either.
#include <cuda_runtime.h>

#include <cstring>
#include <mutex>

#include "lr.h"
#include "lr_engine.h"

namespace {

constexpr size_t kNoAllocScratchBytes = (size_t)64 << 20;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

struct DeviceScratch {
  void *ptr = nullptr;           // device address of g_noalloc_scratch on this device
  lr::Ctx ctx;                   // host-side status words (no pinned allocation)
  uint32_t words[16];
};

std::mutex g_mu;
DeviceScratch g_dev[64];

lr_status scratch_for_current_device(DeviceScratch **out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return LR_ERR_CUDA;
  if (dev < 0 || dev >= 64) return LR_ERR_CUDA;
  std::lock_guard<std::mutex> g(g_mu);
  DeviceScratch &d = g_dev[dev];
  if (!d.ptr) {
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || p == nullptr) {
      cudaGetLastError();
      return e == cudaErrorMemoryAllocation ? LR_ERR_OUT_OF_MEMORY : LR_ERR_CUDA;
    }
    memset(d.words, 0, sizeof(d.words));
    d.ctx.device = dev;
    d.ctx.host_words = d.words;
    d.ptr = p;
  }
  *out = &d;
  return LR_OK;
}

}  // namespace

namespace lr {
lr_status noalloc_resolve_scratch() {
  DeviceScratch *d = nullptr;
  return scratch_for_current_device(&d);
}
}  // namespace lr

extern "C" lr_status lr_rank_noalloc(const uint32_t *succ, int64_t n, int32_t *rank, lr_stream stream) {
  if (n < 0 || n > LR_NOALLOC_MAX_N) return LR_ERR_INVALID_ARGUMENT;
  if (n == 0) return LR_OK;
  if (!succ || !rank) return LR_ERR_INVALID_ARGUMENT;
  lr_status st = lr::setup_device_once();
  if (st != LR_OK) return st;
  DeviceScratch *d = nullptr;
  st = scratch_for_current_device(&d);
  if (st != LR_OK) return st;
  return lr::run_fixed_scratch(succ, n, rank, d->ptr, kNoAllocScratchBytes, &d->ctx,
                               (cudaStream_t)stream);
}
