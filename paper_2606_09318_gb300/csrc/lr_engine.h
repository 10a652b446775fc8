// lr_engine.h -- host engine internals shared by lr_engine.cu and the server.
#pragma once
#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "lr.h"
#include "lr_device.cuh"
#include "lr_kernels.h"

namespace lr {

struct Tuning {
  uint32_t f0_inv, f_inv, cutoff, block, ctas, xchg, chase0, algo, contract, spawn, ord, pf;
};

struct Plan {
  uint64_t n;
  int nlev;                         // levels 0..nlev-1; the last one is base or fallback
  uint32_t cap[kMaxLevels + 1];
  uint32_t f_inv[kMaxLevels + 1];
  uint64_t seed[kMaxLevels + 1];
  bool has_pd;
  uint32_t pd_rounds;
  uint32_t hcap;                    // head-list capacity (bound on lists)
  uint32_t cutoff;
  bool rec16_0;
  bool log0;                        // level 0 on the log path (lr_log.cu)
  int rank_bytes;
  int chase_grid, chase_block;
  // fixed part (does not depend on the list bound)
  size_t off_desc, off_zero, zero_bytes, off_err, off_hcount, off_acc, off_logctr, off_bctr, off_q,
      off_bcnt, off_bitmap;
  size_t fixed_bytes;
  // variable part
  size_t off_work[kMaxLevels + 1], off_R[kMaxLevels + 1];
  size_t off_hA, off_hB, off_ns, off_pd[4];
  uint32_t spawn_cap;               // ruler spawning at level 0: most spawned rulers (0: off)
  uint32_t raw_cap;                 //   ids of level 1 before compaction
  size_t off_sraw, off_sused, off_supre, off_sctr, off_srraw, spawn_zero;
  bool ord0;                        // level 0 chased in element order (a batch)
  size_t off_ord, off_cum;          // its ruler positions, rulers before every 256 positions
  bool term;                        // terminal ids carried through the levels
  size_t off_T[kMaxLevels + 1], off_tid[kMaxLevels + 1], off_T0, off_hC, off_pdt[2];
  size_t off_log, off_hdr, off_pairs, off_pairsB, off_cur;   // log path
  uint32_t total_chunks, shift;
  size_t cur_bytes;
  LogGeom lg;
  size_t var_bytes;
};

// One per (device, stream): grow-only workspaces and a pinned status word.
struct Ctx {
  int device = 0;
  void *fixed = nullptr;
  size_t fixed_bytes = 0;
  void *var = nullptr;
  size_t var_bytes = 0;
  void *hostpath = nullptr;
  size_t hostpath_bytes = 0;
  void *contract = nullptr;         // tile-local contraction: bitmap, prefixes
  size_t contract_bytes = 0;
  void *contract2 = nullptr;        // and the contracted list
  size_t contract2_bytes = 0;
  uint32_t *host_words = nullptr;   // [0] device error bits, [1] head count, [2..3] tile-local
                                    // links, [4..7] sampled tile-local links and elements,
                                    // [8..9] int64 scratch
  bool pending_status = false;
  const LevelDesc *last_desc = nullptr;   // level descriptors of the last ruling-set call
  int last_nlev = 0;
};

// Tuning of a call: the caller's fields, else LR_TUNING, else the autotuned
// entry for (n, weighted, batch), else the built-in defaults.
Tuning resolve_tuning(const lr_tuning *t, int64_t n, bool weighted, bool batch);
// The built-in defaults alone.
Tuning resolve_tuning_builtin(int64_t n, bool weighted, bool batch = false);
// Autotuned entry for a call of this shape (lr_tune.cu).
bool tuned_lookup(int64_t n, bool weighted, bool batch, lr_tuning *out);
// term: also lay out the terminal-id arrays of every level; t0ws: and the
// level-0 terminal ids (when the caller does not receive them).
Plan make_plan(uint64_t n, uint64_t h, const Tuning &u, bool rec16_0, int rank_bytes,
               uint64_t seed, int chase_grid, bool force_srs, bool log0, bool term = false,
               bool t0ws = false, bool spawn0 = false, bool ord0 = false);
int chase_grid_for(const Tuning &u, bool rec16, bool log0, bool ord0 = false);
Ctx *get_ctx(cudaStream_t stream, lr_status *st);
// Forget the context of a stream that is about to be destroyed (waits for
// the stream, frees the context's buffers).
void release_ctx(cudaStream_t stream);
// Status for the error bits a call leaves in Ctx::host_words[0].
lr_status status_from_bits(uint32_t bits);
lr_status ensure_buffer(void **buf, size_t *cur, size_t want, cudaStream_t s);
lr_status device_status(cudaStream_t s);
// Unweighted int32 ranking inside caller-provided scratch with a caller-provided
// host context (no allocation); counts the lists first and waits for the result.
lr_status run_fixed_scratch(const uint32_t *succ, int64_t n, int32_t *rank, void *scratch,
                            size_t scratch_bytes, Ctx *ctx, cudaStream_t s);
// Kernel attributes (shared-memory limits) for the current device, once.
lr_status setup_device_once();
// Device address of lr_rank_noalloc's fixed scratch array on the current
// device, looked up once per device (lr_noalloc.cu).  setup_device_once calls
// it, so the array is placed on the device by the first lr_* call there.
lr_status noalloc_resolve_scratch();
// One list in device memory, ranked on its own (the single-instance path,
// with its automatic choices: tile-local contraction, the level-0 form);
// waits for the result and returns the status.
lr_status run_single(const uint32_t *succ, const void *weight, int wtype, void *rank, int rank_bytes,
                     int64_t n, uint64_t seed, cudaStream_t s);
// Rank k instances given by per-instance device pointers (tables in device
// memory); waits for the result and returns the status.
lr_status run_ptr_batch(const int64_t *offsets, int32_t k, int64_t n_total,
                        const uint32_t *const *sptr, const void *const *wptr, void *const *rptr,
                        int wtype, int rank_bytes, uint64_t seed, cudaStream_t s);

}  // namespace lr
