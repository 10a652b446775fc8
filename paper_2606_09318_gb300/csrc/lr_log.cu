// lr_log.cu -- level 0 of the unweighted path with one random DRAM access per
// element.
//
// On GB300 a random 32-byte DRAM access costs the same whether it reads or
// writes back a dirty sector, and the part sustains about 40 G such accesses
// per second once the working set exceeds L2.  Rewriting each visited record
// in place (the chase in lr_kernels.cu) therefore costs two accesses per
// element: the gather and the later write-back.  Here the level-0 chase only
// gathers succ[y]; what it learns about y (its ruler and offset) is appended
// to a per-thread log whose writes fill whole sectors in L2.  Ruler
// propagation (the last step of Algorithm 1) then becomes a radix partition of
// the log into 256 buckets of the index space and a scatter whose writes stay
// inside one L2-resident window of rank[] at a time.
//
// Heads (Algorithm 1's findInit) come from one streaming reduction when the
// input holds a single list: the successors of the non-terminal elements are
// every element except the head, so head = n(n-1)/2 - sum(succ[i] != i).
// Anything else (several lists, validation) falls back to the
// has-predecessor bitmap.
#include <algorithm>

#include "lr_kernels.h"

namespace lr {

constexpr uint32_t kMark = 0x80000000u;    // log entry: a new segment of ruler (entry & ~kMark)
constexpr uint32_t kLogEnd = 0xFFFFFFFFu;  // log entry: unused slot
constexpr uint32_t kChunk = 32;            // entries per log chunk (128 bytes)
constexpr int kBuckets = 256;

// ---------------------------------------------------------------- heads by sums
__global__ void __launch_bounds__(256)
k_sum0(const uint32_t *__restrict__ succ, uint32_t n, unsigned long long *__restrict__ acc,
       uint32_t *__restrict__ err, int vec) {
  unsigned long long S = 0, T = 0;
  uint32_t bad = 0;
  const uint32_t ngroups = (uint32_t)(((uint64_t)n + 3u) / 4u);
  for (uint32_t g = blockIdx.x * blockDim.x + threadIdx.x; g < ngroups; g += gridDim.x * blockDim.x) {
    const uint32_t i0 = g * 4u;
    uint32_t s[4];
    const uint32_t cnt = min(4u, n - i0);
    if (vec && cnt == 4u) {
      uint4 v = __ldcs(reinterpret_cast<const uint4 *>(succ + i0));
      s[0] = v.x; s[1] = v.y; s[2] = v.z; s[3] = v.w;
    } else {
      for (uint32_t j = 0; j < 4u; ++j) s[j] = j < cnt ? __ldcs(succ + i0 + j) : i0 + j;
    }
#pragma unroll
    for (uint32_t j = 0; j < 4u; ++j) {
      if (j >= cnt) break;
      if (s[j] >= n) bad = 1;
      else if (s[j] == i0 + j) T += 1;
      else S += s[j];
    }
  }
  for (int d = 16; d > 0; d >>= 1) {
    S += __shfl_down_sync(0xFFFFFFFFu, S, d);
    T += __shfl_down_sync(0xFFFFFFFFu, T, d);
  }
  if ((threadIdx.x & 31) == 0) {
    if (T) atomicAdd(acc + 0, T);
    if (S) atomicAdd(acc + 1, S);
  }
  if (bad) record_error(err, kErrRange);
}

cudaError_t launch_sum0(const uint32_t *succ, uint32_t n, unsigned long long *acc, uint32_t *err,
                        cudaStream_t s) {
  const int block = 256;
  const int vec = ((uintptr_t)succ & 15u) == 0;
  k_sum0<<<stream_grid(((uint64_t)n + 3) / 4, block), block, 0, s>>>(succ, n, acc, err, vec);
  count_launch();
  return cudaGetLastError();
}

// One thread: the single head, or a switch to the bitmap.
__global__ void k_heads_single(LevelDesc *desc, const unsigned long long *acc, uint32_t *hlist0,
                               int validate) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  LevelDesc &d = desc[0];
  const unsigned long long n = d.n;
  const unsigned long long h = n * (n - 1) / 2 - acc[1];
  if (!validate && acc[0] == 1 && h < n) {
    hlist0[0] = (uint32_t)h;
    d.h = 1;
    d.hsrc = kHeadsList;
  } else {
    d.hsrc = kHeadsBitmap;
  }
}

// Has-predecessor bitmap, only when the single-head shortcut does not apply.
__global__ void __launch_bounds__(256)
k_bitmap0(const LevelDesc *__restrict__ desc, const uint32_t *__restrict__ succ, uint32_t n,
          uint32_t *__restrict__ bitmap, uint32_t *__restrict__ err, int validate) {
  if (desc[0].hsrc != kHeadsBitmap) return;
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const uint32_t s = __ldcs(succ + i);
    if (s >= n || s == i) continue;
    const uint32_t bit = 1u << (s & 31u);
    if (validate) {
      if (atomicOr(bitmap + (s >> 5), bit) & bit) record_error(err, kErrNotList);
    } else {
      atomicOr(bitmap + (s >> 5), bit);
    }
  }
}

cudaError_t launch_heads0_log(LevelDesc *desc, const unsigned long long *acc, uint32_t *hlist0,
                              const uint32_t *succ, uint32_t n, uint32_t *bitmap, uint32_t *err,
                              int validate, cudaStream_t s) {
  k_heads_single<<<1, 32, 0, s>>>(desc, acc, hlist0, validate);
  k_bitmap0<<<stream_grid(n, 256), 256, 0, s>>>(desc, succ, n, bitmap, err, validate);
  count_launch(2);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- log writer
struct LogCfg {
  uint32_t *log;          // chunks of kChunk entries
  uint2 *hdr;             // per chunk: (ruler, offset) of its first entry, or (kLogEnd, 0)
  uint32_t per_cta;       // chunks reserved for each CTA
  uint32_t main_chunks;   // per_cta * grid
  uint32_t total_chunks;  // main + overflow pool
  uint32_t *ovf;          // overflow pool cursor
};

// Entries are buffered four at a time (a register shift buffer) and stored
// as one 16-byte vector.
struct LogWriter {
  uint32_t chunk, slot, nb;
  uint32_t b0, b1, b2, b3;
  uint32_t gc, go;   // (ruler, offset) of the buffered group's first entry
  bool ok;

  __device__ void init() {
    slot = kChunk; nb = 0; ok = true; chunk = 0; gc = kLogEnd; go = 0;
    b0 = b1 = b2 = b3 = kLogEnd;
  }
  __device__ bool alloc(const LogCfg &L, uint32_t *s_used) {
    const uint32_t i = atomicAdd(s_used, 1u);
    uint64_t id = (uint64_t)blockIdx.x * L.per_cta + i;
    if (i >= L.per_cta || id >= L.main_chunks) {
      id = (uint64_t)L.main_chunks + atomicAdd(L.ovf, 1u);
      if (id >= L.total_chunks) { ok = false; return false; }
    }
    chunk = (uint32_t)id;
    slot = 0;
    L.hdr[chunk] = make_uint2(gc, go);
    return true;
  }
  __device__ void flush(const LogCfg &L, uint32_t *s_used) {
    nb = 0;
    if (!ok || (slot == kChunk && !alloc(L, s_used))) return;
    __stcg(reinterpret_cast<uint4 *>(L.log + (size_t)chunk * kChunk + slot), make_uint4(b0, b1, b2, b3));
    slot += 4;
  }
  // v: the entry; (c, o): its ruler and offset when v is an element
  __device__ __forceinline__ void put(const LogCfg &L, uint32_t *s_used, uint32_t v, uint32_t c,
                                      uint32_t o) {
    if (nb == 0) { gc = c; go = o; }
    b0 = b1; b1 = b2; b2 = b3; b3 = v;
    if (++nb == 4) flush(L, s_used);
  }
  __device__ void finish(const LogCfg &L, uint32_t *s_used) {
    if (nb > 0) {
      while (nb < 4) { b0 = b1; b1 = b2; b2 = b3; b3 = kLogEnd; ++nb; }
      flush(L, s_used);
    }
    if (ok && slot < kChunk) {
      for (; slot < kChunk; slot += 4)
        __stcg(reinterpret_cast<uint4 *>(L.log + (size_t)chunk * kChunk + slot),
               make_uint4(kLogEnd, kLogEnd, kLogEnd, kLogEnd));
    }
  }
};

// ---------------------------------------------------------------- chase
// Level-0 ruler chasing on the raw successor array.  Each ruler c emits
// MARK(c) and then the elements of its segment in order (offsets 0, 1, ...);
// the reduced list gets {next ruler, kUnvisited, segment length} at c.
__global__ void __launch_bounds__(512)
k_chase_log(LevelDesc *__restrict__ desc, const uint32_t *__restrict__ succ, Rec16 *__restrict__ next,
            const uint32_t *__restrict__ ns, uint32_t *__restrict__ qctr, uint32_t *__restrict__ err,
            LogCfg L) {
  __shared__ uint32_t s_used;
  if (threadIdx.x == 0) s_used = 0;
  __syncthreads();
  const LevelDesc d = desc[0];
  if (d.mode != kModeSrs) return;
  const uint32_t n = d.n, r = d.r;
  const uint64_t R = (uint64_t)r + d.k;
  Perm P;
  P.init(n, d.seed);
  const uint32_t lo = (uint32_t)(R * blockIdx.x / gridDim.x);
  const uint32_t hi = (uint32_t)(R * (blockIdx.x + 1) / gridDim.x);
  uint32_t *q = qctr + blockIdx.x;
  LogWriter W;
  W.init();
  uint32_t visited = 0, added = 0, bad = 0;
  uint64_t c64 = (uint64_t)lo + atomicAdd(q, 1u);
  while (c64 < hi) {
    const uint64_t cnext = (uint64_t)lo + atomicAdd(q, 1u);
    const uint32_t c = (uint32_t)c64;
    const uint32_t rho = c < r ? P.inv(c) : __ldcg(ns + (c - r));
    W.put(L, &s_used, kMark | c, kLogEnd, 0);
    uint32_t x = rho, o = 0, nxt = c;
    for (;;) {
      const uint32_t s = __ldcg(succ + x);
      W.put(L, &s_used, x, c, o);
      ++visited;
      if (s >= n) { bad |= 8u; break; }
      if (s == x) break;                       // terminal: segment length o links
      ++o;
      const uint32_t p = P.fwd(s);
      if (p < r) {                             // next ruler
        nxt = p;
        if (p == c) bad |= 2u;                 // back at itself: a cycle
        break;
      }
      if ((visited & 4095u) == 0) {            // bound a walk on invalid input
        const uint32_t delta = visited - added;
        const uint32_t old = atomicAdd(&desc[0].visited, delta);
        added = visited;
        if ((uint64_t)old + delta > n || o > n) { bad |= 1u; break; }
      }
      x = s;
    }
    __stcg(reinterpret_cast<uint4 *>(next + c), make_uint4(nxt, kUnvisited, o, 0u));
    c64 = cnext;
  }
  W.finish(L, &s_used);
  if (!W.ok) bad |= 16u;
  if (bad & 1u) record_error(err, kErrNotList);
  if (bad & 2u) record_error(err, kErrCycle);
  if (bad & 8u) record_error(err, kErrRange);
  if (bad & 16u) record_error(err, kErrCapacity);
  uint32_t rest = visited - added;
  for (int dd = 16; dd > 0; dd >>= 1) rest += __shfl_down_sync(0xFFFFFFFFu, rest, dd);
  if ((threadIdx.x & 31) == 0 && rest) atomicAdd(&desc[0].visited, rest);
}

cudaError_t launch_chase_log(LevelDesc *desc, const uint32_t *succ, void *next_work, const uint32_t *ns,
                             uint32_t *qctr, int grid, int block, uint32_t *err, uint32_t *log,
                             uint2 *hdr, uint32_t per_cta, uint32_t total_chunks, uint32_t *ovf,
                             cudaStream_t s) {
  LogCfg L;
  L.log = log;
  L.hdr = hdr;
  L.per_cta = per_cta;
  L.main_chunks = per_cta * (uint32_t)grid;
  L.total_chunks = total_chunks;
  L.ovf = ovf;
  k_chase_log<<<grid, block, 0, s>>>(desc, succ, reinterpret_cast<Rec16 *>(next_work), ns, qctr, err, L);
  count_launch();
  return cudaGetLastError();
}

int chase_log_occupancy(int block) {
  int nb = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_chase_log, block, 0);
  return nb > 0 ? nb : 1;
}

// ---------------------------------------------------------------- propagation
// Radix partition of the log by index range, without global atomics:
//   H: every CTA decodes its contiguous share of chunks and counts entries
//      per bucket (256 buckets of 2^shift indices);
//   S: one CTA turns the per-CTA counts into write offsets, bucket by bucket
//      (a bucket's region is fixed: exactly its index range for a valid list);
//   W: every CTA decodes the same chunks again, computes rank = R_1[ruler] -
//      offset and appends (y, rank) at its own cursor inside each bucket.
// Decoding a chunk takes one warp: the last mark at or before a lane gives
// the lane's ruler and offset (ballot + shuffle).
template <class F>
__device__ __forceinline__ void decode_chunks(const uint32_t *__restrict__ log, const uint2 *__restrict__ hdr,
                                              uint32_t c0, uint32_t c1, uint32_t n, F &&f) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  for (uint32_t id = c0 + warp; id < c1; id += nwarps) {
    const uint2 h = __ldg(hdr + id);
    if (h.y == kLogEnd) continue;                      // chunk never allocated (warp-uniform)
    const uint32_t e = __ldg(log + (size_t)id * kChunk + lane);
    const bool mark = e != kLogEnd && (e & kMark);
    const uint32_t mm = __ballot_sync(0xFFFFFFFFu, mark);
    const uint32_t below = mm & ((2u << lane) - 1u);
    const int m = below ? 31 - __clz(below) : 0;
    const uint32_t em = __shfl_sync(0xFFFFFFFFu, e, m);
    const uint32_t c = below ? (em & ~kMark) : h.x;
    const uint32_t o = below ? (uint32_t)(lane - m - 1) : h.y + (uint32_t)lane;
    if (e != kLogEnd && !(e & kMark) && e < n) f(e, c, o);
  }
}

__global__ void __launch_bounds__(256)
k_part_hist(const LevelDesc *__restrict__ desc, const uint32_t *__restrict__ log,
            const uint2 *__restrict__ hdr, uint32_t total_chunks, uint32_t *__restrict__ hist,
            uint32_t shift) {
  __shared__ uint32_t sh[kBuckets];
  const LevelDesc d = desc[0];
  if (d.mode != kModeSrs) return;
  for (int b = threadIdx.x; b < kBuckets; b += blockDim.x) sh[b] = 0;
  __syncthreads();
  const uint32_t c0 = (uint32_t)((uint64_t)total_chunks * blockIdx.x / gridDim.x);
  const uint32_t c1 = (uint32_t)((uint64_t)total_chunks * (blockIdx.x + 1) / gridDim.x);
  decode_chunks(log, hdr, c0, c1, d.n, [&](uint32_t y, uint32_t, uint32_t) { atomicAdd(&sh[y >> shift], 1u); });
  __syncthreads();
  for (int b = threadIdx.x; b < kBuckets; b += blockDim.x) hist[(size_t)blockIdx.x * kBuckets + b] = sh[b];
}

__global__ void __launch_bounds__(kBuckets)
k_part_scan(const LevelDesc *__restrict__ desc, uint32_t *__restrict__ hist, int nctas, uint32_t shift,
            uint32_t *__restrict__ err) {
  const LevelDesc d = desc[0];
  if (d.mode != kModeSrs) return;
  const uint32_t b = threadIdx.x;
  const uint64_t b0 = (uint64_t)b << shift;
  uint64_t run = b0;
  for (int k = 0; k < nctas; ++k) {
    const uint32_t v = hist[(size_t)k * kBuckets + b];
    hist[(size_t)k * kBuckets + b] = (uint32_t)run;
    run += v;
  }
  const uint64_t b1 = b0 + (1ull << shift);
  if (run > (b1 < d.n ? b1 : (uint64_t)d.n) && b0 < d.n) record_error(err, kErrNotList);
}

__global__ void __launch_bounds__(256)
k_part_write(const LevelDesc *__restrict__ desc, const uint32_t *__restrict__ log,
             const uint2 *__restrict__ hdr, uint32_t total_chunks, const uint32_t *__restrict__ hist,
             const uint32_t *__restrict__ r1, uint2 *__restrict__ pairs, uint32_t shift,
             uint32_t *__restrict__ err) {
  __shared__ uint32_t cur[kBuckets];
  const LevelDesc d = desc[0];
  if (d.mode != kModeSrs) return;
  const uint32_t n = d.n, nn = desc[1].n;
  for (int b = threadIdx.x; b < kBuckets; b += blockDim.x) cur[b] = hist[(size_t)blockIdx.x * kBuckets + b];
  __syncthreads();
  const uint32_t c0 = (uint32_t)((uint64_t)total_chunks * blockIdx.x / gridDim.x);
  const uint32_t c1 = (uint32_t)((uint64_t)total_chunks * (blockIdx.x + 1) / gridDim.x);
  uint32_t bad = 0;
  decode_chunks(log, hdr, c0, c1, n, [&](uint32_t y, uint32_t c, uint32_t o) {
    uint32_t val = 0;
    if (c < nn) val = __ldcg(r1 + c) - o;
    else bad |= kErrInternal;
    const uint32_t b = y >> shift;
    const uint32_t pos = atomicAdd(&cur[b], 1u);
    const uint64_t b1 = ((uint64_t)b + 1) << shift;
    if (pos < (b1 < n ? b1 : (uint64_t)n)) pairs[pos] = make_uint2(y, val);
    else bad |= kErrNotList;                  // more entries than indices: a revisit
  });
  if (bad) record_error(err, bad);
}

// Scatter: the partitioned pairs are ordered by index range, so at any time
// the grid writes into one or two windows of rank[] that stay in L2.
__global__ void __launch_bounds__(256)
k_scatter_log(const LevelDesc *__restrict__ desc, const uint2 *__restrict__ pairs,
              uint32_t *__restrict__ rank, uint32_t *__restrict__ err) {
  const LevelDesc d = desc[0];
  if (d.mode != kModeSrs) return;
  const uint32_t n = d.n;
  uint32_t bad = 0;
  if (blockIdx.x == 0 && threadIdx.x == 0 && d.visited != n) bad |= d.visited > n ? kErrNotList : kErrCycle;
  const uint32_t npairs2 = n / 2u;
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < npairs2; i += gridDim.x * blockDim.x) {
    const uint4 v = __ldcs(reinterpret_cast<const uint4 *>(pairs) + i);
    if (v.x < n) rank[v.x] = v.y; else bad |= kErrInternal;
    if (v.z < n) rank[v.z] = v.w; else bad |= kErrInternal;
  }
  if ((n & 1u) && blockIdx.x == 0 && threadIdx.x == 0) {
    const uint2 v = pairs[n - 1];
    if (v.x < n) rank[v.x] = v.y; else bad |= kErrInternal;
  }
  if (bad) record_error(err, bad);
}

cudaError_t launch_finalize_log(LevelDesc *desc, const uint32_t *log, const uint2 *hdr,
                                uint32_t total_chunks, const void *r1, uint2 *pairs, uint32_t *hist,
                                int part_ctas, uint32_t shift, uint32_t *rank, uint32_t n, uint32_t *err,
                                cudaStream_t s) {
  k_part_hist<<<part_ctas, 256, 0, s>>>(desc, log, hdr, total_chunks, hist, shift);
  k_part_scan<<<1, kBuckets, 0, s>>>(desc, hist, part_ctas, shift, err);
  k_part_write<<<part_ctas, 256, 0, s>>>(desc, log, hdr, total_chunks, hist,
                                         reinterpret_cast<const uint32_t *>(r1), pairs, shift, err);
  k_scatter_log<<<stream_grid(n / 2 + 1, 256), 256, 0, s>>>(desc, pairs, rank, err);
  count_launch(4);
  return cudaGetLastError();
}

}  // namespace lr
