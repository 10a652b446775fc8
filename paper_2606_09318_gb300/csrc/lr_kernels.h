// lr_kernels.h -- host-side launchers of the list-ranking kernels (C++ linkage,
// internal to liblr.so).
#pragma once
#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "lr_device.cuh"

namespace lr {

enum : int { kRecKind8 = 0, kRecKind16 = 1, kRecKindSucc = 2 };

struct InitParams {
  int32_t nlev;                       // levels in the plan (0..nlev-1)
  uint32_t n0;                        // elements at level 0
  uint32_t mode0;                     // kModeSrs or kModeBase
  uint32_t cutoff;                    // base-case bound
  uint32_t f_inv[kMaxLevels + 1];
  uint32_t cap[kMaxLevels + 1];
  uint64_t seed[kMaxLevels + 1];
  uint32_t pd_rounds;                 // rounds of the pointer-doubling fallback
  uint32_t has_pd;                    // the last level may fall back to pointer doubling
  uint32_t hcap;                      // capacity of the head lists
};

// Kernel launch counter (all streams).
void count_launch(int k = 1);
int64_t launch_count();

int device_sm_count();
int stream_grid(uint64_t work_items, int block);

cudaError_t launch_init(LevelDesc *desc, const InitParams &p, cudaStream_t s);

// Level-0 pass.  wtype 0/1/2 (none/i32/i64).  offsets != nullptr: batched
// input with local successor ids (k instances).
// local (optional): counts the links that stay inside their contraction tile.
cudaError_t launch_prep0(const uint32_t *succ, const void *weight, int wtype, uint32_t n,
                         void *work, uint32_t *bitmap, uint32_t *err, int validate,
                         const int64_t *offsets, int32_t k, unsigned long long *sums,
                         unsigned long long *local, cudaStream_t s);

// Batched prep that sums each instance's terminals and local successors
// (isums[2k], zeroed) instead of marking predecessors; then the level-0 head
// list from those sums, or the bitmap from the records when some instance is
// not one list.
cudaError_t launch_prep0_sums(const uint32_t *succ, const void *weight, int wtype, uint32_t n, void *work,
                              uint32_t *err, const int64_t *offsets, int32_t k, unsigned long long *isums,
                              cudaStream_t s);
cudaError_t launch_count_batch(const unsigned long long *isums, int32_t k, uint32_t *out, cudaStream_t s);
cudaError_t launch_heads0_batch(LevelDesc *desc, unsigned long long *isums, const int64_t *offsets, int32_t k,
                                uint32_t *hlist0, uint32_t hcap, const void *work, bool rec16, uint32_t n,
                                uint32_t *bitmap, cudaStream_t s);
cudaError_t launch_prep0_ptrs(const uint32_t *const *sptr, const void *const *wptr, int wtype,
                              uint32_t n, void *work, uint32_t *bitmap, uint32_t *err, int validate,
                              const int64_t *offsets, int32_t k, cudaStream_t s);

// The same sums for a batch given as one pointer per instance.
cudaError_t launch_prep0_ptrs_sums(const uint32_t *const *sptr, const void *const *wptr, int wtype, uint32_t n,
                                   void *work, uint32_t *err, const int64_t *offsets, int32_t k,
                                   unsigned long long *isums, cudaStream_t s);

cudaError_t launch_finalize_ptrs(LevelDesc *desc, const void *work, bool rec16, const void *rnext,
                                 void *const *rptr, int rank_bytes, uint32_t cap,
                                 const int64_t *offsets, int32_t k, uint32_t *err, cudaStream_t s);

cudaError_t launch_count_heads(const uint32_t *bitmap, uint32_t n, uint32_t *out, cudaStream_t s);
// Tile-local links over a sample of the contraction tiles: out[0] += local
// links, out[1] += elements sampled.
cudaError_t launch_local_sample(const uint32_t *succ, uint32_t n, unsigned long long *out, cudaStream_t s);

// Head selection of level `lev` (reads the bitmap at level 0, the head list
// otherwise), then the exclusive scan and the writes.
cudaError_t launch_heads(LevelDesc *desc, int lev, int nlev, const uint32_t *bitmap,
                         const uint32_t *hlist, void *work, int rec_kind, uint32_t *ns,
                         uint32_t *hnext, uint64_t *blockcnt, uint32_t *err, uint32_t cutoff,
                         uint32_t hcap, uint32_t has_pd, cudaStream_t s);

// Terminal ids (all optional; null when the call does not ask for them):
// tid_cur/tid_next hold the original id of each terminal of this/the next
// level (written by the chase), tout/tnext the terminal of every element.
// Ruler spawning at one level (k_chase with SPAWN): spawned ids are
// R + k for k < cap, R = the level's initial rulers.
struct SpawnArgs {
  uint32_t *ctr;      // ids handed out so far
  uint32_t cap;       // most spawned ids
  uint32_t *used;     // bitmap: spawned id R + k became a ruler
  uint32_t *cursor;   // per CTA: candidates examined in its slice of ids
};

// A level in element order (a batch): the sampled rulers' positions,
// ascending (ord[0 .. r)), and a rank table over their marks (bits: n bits;
// cum[b]: rulers before position 256 b), so that a sampled ruler's id is its
// index in ord.
struct OrdArgs {
  uint32_t *ord;
  uint32_t *cum;
  uint32_t *bits;
  uint32_t pf_lead;          // prefetch the records this many elements ahead of the front (0: off)
};

// After a spawning chase at level lev: compact the next level's records
// (raw -> out, raw_cap ids at most), set its size and mode; and, once it is
// ranked, scatter its ranks back to the original ids.
cudaError_t launch_spawn_compact(LevelDesc *desc, int lev, int nlev, const uint32_t *ctr, uint32_t cap,
                                 const uint32_t *used, uint32_t *upre, const void *raw, void *out,
                                 uint32_t raw_cap, uint32_t cutoff, uint32_t has_pd, uint32_t *err,
                                 cudaStream_t s);
cudaError_t launch_spawn_scatter(LevelDesc *desc, int lev, const void *rc, void *rraw, int rank_bytes,
                                 const uint32_t *used, const uint32_t *upre, uint32_t raw_cap,
                                 cudaStream_t s);

// Build the OrdArgs arrays of level lev (at most cap elements; bits
// overwritten; per-CTA counts in cnt, kHeadBlocks of them) and rename the
// sampled heads in the next level's head list (hnext, hcap entries at most).
// bits must hold ceil(cap / 256) * 8 words, cum ceil(cap / 256), ord the
// level's sampled rulers.
cudaError_t launch_order(LevelDesc *desc, int lev, uint32_t cap, uint64_t *cnt, const OrdArgs *oa,
                         uint32_t *hnext, uint32_t hcap, uint32_t *err, cudaStream_t s);

// ord: nullptr (per-CTA slices of ruler ids, sampled ids pi(x)) or
// launch_order's arrays: the chase takes its rulers in element order and
// gives the sampled ones their ids in that order (no spawning).
cudaError_t launch_chase(LevelDesc *desc, int lev, void *work, bool rec16, void *next_work,
                         const uint32_t *ns, uint32_t *qctr, int grid, int block, uint32_t *err,
                         int xchg, const uint32_t *tid_cur, uint32_t *tid_next, const SpawnArgs *spawn,
                         const OrdArgs *ord, cudaStream_t s);

cudaError_t launch_base(LevelDesc *desc, int lev, const void *work, bool rec16, void *rout,
                        int rank_bytes, uint32_t cutoff, uint32_t *err, const uint32_t *tid,
                        uint32_t *tout, cudaStream_t s);

cudaError_t launch_pd(LevelDesc *desc, int lev, const void *work, uint32_t cap, uint32_t rounds,
                      uint32_t *nxt0, uint32_t *nxt1, uint64_t *val0, uint64_t *val1, void *rout,
                      int rank_bytes, uint32_t *err, const uint32_t *tid, uint32_t *t0, uint32_t *t1,
                      uint32_t *tout, cudaStream_t s);

// Level-0 extra outputs after the ranks and terminal ids are written:
// prefix (head-relative) ranks, the inclusive-tail form, local terminal ids.
cudaError_t launch_outputs(const LevelDesc *desc, const uint32_t *bitmap, const uint32_t *hlist0,
                           uint32_t n, uint32_t *term, void *rank, void *prefix, int rank_bytes,
                           int incl, const void *weight, int wtype, const int64_t *offsets, int32_t k,
                           int local, cudaStream_t s);

// Whole-list Wyllie pointer doubling (lr_wyllie.cu).  bufA holds k_prep0's
// records (8 B, or 16 B when weighted: w16), bufB the same size; ranks go
// to `rank` (4 or 8 bytes each).
uint32_t wyllie_rounds(uint64_t n);
cudaError_t launch_wyllie(void *bufA, void *bufB, bool w16, uint32_t n, void *rank, int rank_bytes,
                          uint32_t *err, cudaStream_t s);

cudaError_t launch_finalize(LevelDesc *desc, int lev, const void *work, bool rec16,
                            const void *rnext, void *rout, int rank_bytes, uint32_t cap,
                            uint32_t *err, const uint32_t *tnext, uint32_t *tout,
                            const uint32_t *tid_cur, cudaStream_t s);

// Log path (unweighted level 0, see lr_log.cu).  The log's chunks go to the
// chasing CTAs in windows of kLogWindow chunks.
constexpr uint32_t kLogWindow = 32;
cudaError_t launch_sum0(const uint32_t *succ, uint32_t n, unsigned long long *acc, unsigned long long *local,
                        uint32_t *err, cudaStream_t s);
cudaError_t launch_heads0_log(LevelDesc *desc, const unsigned long long *acc, uint32_t *hlist0,
                              const uint32_t *succ, uint32_t n, uint32_t *bitmap, uint32_t *err,
                              int validate, cudaStream_t s);
cudaError_t launch_chase_log(LevelDesc *desc, const uint32_t *succ, void *next_work, const uint32_t *ns,
                             uint32_t *qctr, int grid, int block, uint32_t *err, uint32_t *log,
                             uint2 *hdr, uint32_t total_chunks, uint32_t *ctr, cudaStream_t s);
// Geometry of the log path's propagation (lr_log.cu): windows of 2^14 ranks;
// level A partitions into na buckets of 2^shiftA ids (regions of capA pairs,
// gridA CTAs, claims of claimA slots); with sB > 0, level B splits each
// A-bucket into its 2^sB windows (kb CTAs per A-bucket, regions of capB).
struct LogGeom {
  uint32_t nw, sB, na, shiftA, gridA, claimA, capA, kb, claimB, capB, nbB;
};
LogGeom log_geometry(uint32_t n);
cudaError_t launch_finalize_log(LevelDesc *desc, const uint32_t *log, const uint2 *hdr, uint32_t total_chunks,
                                const uint32_t *chunk_ctr, const void *r1, uint2 *pairsA, uint2 *pairsB,
                                uint32_t *curA, uint32_t *curB, const LogGeom &g, uint32_t *rank, uint32_t *err,
                                cudaStream_t s);
cudaError_t log_setup();
int chase_log_occupancy(int block);

int chase_occupancy(bool rec16, int block);
cudaError_t kernels_setup();

// Tile-local contraction (lr_contract.cu).
uint32_t lc_tiles(uint64_t n);
uint32_t lc_tile_words();
cudaError_t lc_setup();
// Solve every tile (distances to the local tails into rank, tails into
// tail16, the local-head bitmap and counts), then the tile prefixes.
cudaError_t launch_lc_solve(const uint32_t *succ, const void *weight, int wtype, uint32_t n, void *rank,
                            int rank_bytes, uint16_t *tail16, uint32_t *hb, uint16_t *wpre, uint32_t *tcnt,
                            uint32_t *tpre, uint32_t *err, cudaStream_t s);
// The contracted list: one node per local head.
cudaError_t launch_lc_nodes(const uint32_t *succ, const void *weight, int wtype, uint32_t n, const void *rank,
                            int rank_bytes, const uint16_t *tail16, const uint32_t *hb, const uint16_t *wpre,
                            const uint32_t *tpre, uint32_t *succ_c, void *w_c, uint32_t *err, cudaStream_t s);
// Ranks of every element from the contracted ranks rc.
cudaError_t launch_lc_finish(const uint32_t *succ, const void *weight, int wtype, uint32_t n, void *rank,
                             int rank_bytes, const uint16_t *tail16, const uint32_t *hb, const uint16_t *wpre,
                             const uint32_t *tpre, const void *rc, cudaStream_t s);

}  // namespace lr
