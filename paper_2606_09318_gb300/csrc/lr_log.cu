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

// Entries are buffered eight at a time (a register shift buffer) and stored
// as one 32-byte sector with a single 256-bit store: on GB300 a sector
// written in smaller pieces costs one DRAM access per piece.
struct LogWriter {
  uint32_t chunk, slot, nb;
  uint32_t b0, b1, b2, b3, b4, b5, b6, b7;
  uint32_t gc, go;   // (ruler, offset) of the buffered group's first entry
  bool ok;

  __device__ void init() {
    slot = kChunk; nb = 0; ok = true; chunk = 0; gc = kLogEnd; go = 0;
    b0 = b1 = b2 = b3 = b4 = b5 = b6 = b7 = kLogEnd;
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
    st_sector(L.log + (size_t)chunk * kChunk + slot, b0, b1, b2, b3, b4, b5, b6, b7);
    slot += 8;
  }
  __device__ __forceinline__ void shift_in(uint32_t v) {
    b0 = b1; b1 = b2; b2 = b3; b3 = b4; b4 = b5; b5 = b6; b6 = b7; b7 = v;
  }
  // v: the entry; (c, o): its ruler and offset when v is an element
  __device__ __forceinline__ void put(const LogCfg &L, uint32_t *s_used, uint32_t v, uint32_t c,
                                      uint32_t o) {
    if (nb == 0) { gc = c; go = o; }
    shift_in(v);
    if (++nb == 8) flush(L, s_used);
  }
  __device__ void finish(const LogCfg &L, uint32_t *s_used) {
    if (nb > 0) {
      while (nb < 8) { shift_in(kLogEnd); ++nb; }
      flush(L, s_used);
    }
    if (ok && slot < kChunk) {
      for (; slot < kChunk; slot += 8)
        st_sector(L.log + (size_t)chunk * kChunk + slot, kLogEnd, kLogEnd, kLogEnd, kLogEnd,
                  kLogEnd, kLogEnd, kLogEnd, kLogEnd);
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
// Ruler propagation for the log path.  Every element y appears once in the
// log with its ruler c and offset o; its rank is R_1[c] - o and must land at
// rank[y].  Writing 4-byte ranks at random y costs a DRAM access each on
// GB300, so the pairs (y, rank) are first sorted by y into windows of
// 2^kLgWin elements (a two-level radix partition whose writes are whole
// 32-byte sectors), then each window is assembled in shared memory and
// written out as whole lines.
//   level A: decode the log, partition by A-bucket (y >> (kLgWin + sB));
//   level B: partition each A-bucket by window (only when there are more
//            windows than one level can hold);
//   scatter: one CTA per window.
// Each pass is count / offsets / write, with no global atomics: the region
// of every bucket is fixed (exactly its index range, for a valid list) and
// the per-CTA offsets inside it come from a column scan of the counts.
constexpr int kLgWin = 14;                 // 16384 ranks = 64 KiB of shared memory
constexpr int kMaxBuckets = 256;
constexpr int kPartThreads = 256;
constexpr int kIpt = 8;                    // items a thread holds per partition tile
constexpr int kPartTile = kPartThreads * kIpt;
constexpr int kDecodeIlp = 4;              // chunks a warp decodes with their loads in flight

struct PartSmem {
  uint2 carry[kMaxBuckets * 4];            // < 4 leftover pairs per bucket
  uint32_t ccnt[kMaxBuckets];
  uint32_t gpos[kMaxBuckets];              // next global slot of each bucket
  uint32_t tcnt[kMaxBuckets];
  uint32_t toff[kMaxBuckets + 1];          // + total
  uint32_t tcur[kMaxBuckets];
  uint32_t fstart[kMaxBuckets + 1];        // first whole sector of each bucket in this tile
  uint2 sorted[kPartTile];
};

// Decode kDecodeIlp chunks of the log per warp: all header and entry loads
// are issued before any is used.  In a chunk, the last mark at or before a
// lane gives the lane's ruler and offset (ballot + shuffle).  Each lane gets
// at most one element per chunk: out[j] = (y, ruler), off[j] = offset, or
// y = kLogEnd.  Must be called by whole warps.
__device__ __forceinline__ void decode_ilp(const uint32_t *__restrict__ log, const uint2 *__restrict__ hdr,
                                           uint32_t base, uint32_t c1, uint32_t n, uint2 (&out)[kDecodeIlp],
                                           uint32_t (&off)[kDecodeIlp]) {
  const int lane = threadIdx.x & 31;
  uint2 h[kDecodeIlp];
  uint32_t e[kDecodeIlp];
#pragma unroll
  for (int j = 0; j < kDecodeIlp; ++j) {
    const uint32_t id = base + j;
    h[j] = id < c1 ? __ldg(hdr + id) : make_uint2(kLogEnd, kLogEnd);
    e[j] = id < c1 ? __ldg(log + (size_t)id * kChunk + lane) : kLogEnd;
  }
#pragma unroll
  for (int j = 0; j < kDecodeIlp; ++j) {
    out[j] = make_uint2(kLogEnd, 0u);
    off[j] = 0;
    if (h[j].y == kLogEnd) continue;               // chunk never allocated (warp-uniform)
    const bool mark = e[j] != kLogEnd && (e[j] & kMark);
    const uint32_t mm = __ballot_sync(0xFFFFFFFFu, mark);
    const uint32_t below = mm & ((2u << lane) - 1u);
    const int m = below ? 31 - __clz(below) : 0;
    const uint32_t em = __shfl_sync(0xFFFFFFFFu, e[j], m);
    const uint32_t c = below ? (em & ~kMark) : h[j].x;
    const uint32_t o = below ? (uint32_t)(lane - m - 1) : h[j].y + (uint32_t)lane;
    if (e[j] != kLogEnd && !(e[j] & kMark) && e[j] < n) { out[j] = make_uint2(e[j], c); off[j] = o; }
  }
}

// Whole-range decode (histogram pass): f(y) for every element.
template <class F>
__device__ __forceinline__ void decode_chunks(const uint32_t *__restrict__ log, const uint2 *__restrict__ hdr,
                                              uint32_t c0, uint32_t c1, uint32_t n, F &&f) {
  const int warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  for (uint32_t base = c0 + (uint32_t)warp * kDecodeIlp; base < c1; base += (uint32_t)nwarps * kDecodeIlp) {
    uint2 it[kDecodeIlp];
    uint32_t off[kDecodeIlp];
    decode_ilp(log, hdr, base, c1, n, it, off);
#pragma unroll
    for (int j = 0; j < kDecodeIlp; ++j)
      if (it[j].x != kLogEnd) f(it[j].x);
  }
}

// Exclusive scan of nb (<= 256) shared-memory counts by warp 0; returns the
// total through out[nb].
__device__ __forceinline__ void warp0_scan(const uint32_t *in, uint32_t *out, int nb) {
  const int lane = threadIdx.x & 31;
  if ((threadIdx.x >> 5) != 0) return;
  uint32_t run = 0;
  for (int b0 = 0; b0 < nb; b0 += 32) {
    const int b = b0 + lane;
    const uint32_t v = b < nb ? in[b] : 0u;
    uint32_t x = v;
    for (int d = 1; d < 32; d <<= 1) {
      const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, d);
      if (lane >= d) x += y;
    }
    if (b < nb) out[b] = run + x - v;
    run += __shfl_sync(0xFFFFFFFFu, x, 31);
  }
  if (lane == 0) out[nb] = run;
}

// One tile of register-held items (item[i] valid when item[i].x != kLogEnd,
// bk[i] its bucket) -> sorted by bucket in shared memory -> whole-sector
// stores.  gpos/ccnt/carry persist across tiles: each bucket's output
// continues its carry, so every store but a bucket's first (unaligned) head
// and its final tail covers a whole 32-byte sector, one thread per sector.
// lim: size of `out`; positions past it (only possible for an invalid list,
// which the count scan reports) are dropped.
__device__ void part_emit_tile(PartSmem &S, int nb, const uint2 (&item)[kIpt], const uint32_t (&bk)[kIpt],
                               uint2 *__restrict__ out, uint32_t lim, uint32_t &bad) {
  const int tid = threadIdx.x;
#pragma unroll
  for (int i = 0; i < kIpt; ++i)
    if (item[i].x != kLogEnd) atomicAdd(&S.tcnt[bk[i]], 1u);
  __syncthreads();
  warp0_scan(S.tcnt, S.toff, nb);
  __syncthreads();
#pragma unroll
  for (int i = 0; i < kIpt; ++i)
    if (item[i].x != kLogEnd) S.sorted[S.toff[bk[i]] + atomicAdd(&S.tcur[bk[i]], 1u)] = item[i];
  __syncthreads();                                   // placement done before tcur is reused
  // per bucket: pairs up to the next sector boundary (h), whole sectors (f)
  for (int b = tid; b < nb; b += blockDim.x) {
    const uint32_t m = S.ccnt[b] + S.tcnt[b], g = S.gpos[b];
    const uint32_t h = min(m, (4u - (g & 3u)) & 3u);
    S.tcur[b] = (m - h) / 4u;                        // reuse: whole sectors of bucket b
  }
  __syncthreads();
  warp0_scan(S.tcur, S.fstart, nb);
  __syncthreads();
  auto seq = [&](int b, uint32_t k) -> uint2 {
    const uint32_t c = S.ccnt[b];
    return k < c ? S.carry[b * 4 + k] : S.sorted[S.toff[b] + k - c];
  };
  const uint32_t nsec = S.fstart[nb];
  for (uint32_t sct = tid; sct < nsec; sct += blockDim.x) {
    int lo = 0, hi = nb;                              // bucket: last b with fstart[b] <= sct
    while (hi - lo > 1) {
      const int mid = (lo + hi) >> 1;
      if (S.fstart[mid] <= sct) lo = mid; else hi = mid;
    }
    const int b = lo;
    const uint32_t g = S.gpos[b];
    const uint32_t h = min(S.ccnt[b] + S.tcnt[b], (4u - (g & 3u)) & 3u);
    const uint32_t k = h + 4u * (sct - S.fstart[b]);
    const uint2 a = seq(b, k), bb = seq(b, k + 1), cc = seq(b, k + 2), dd = seq(b, k + 3);
    if ((uint64_t)g + k + 3 < lim) st_sector(out + g + k, a.x, a.y, bb.x, bb.y, cc.x, cc.y, dd.x, dd.y);
    else bad |= kErrNotList;
  }
  __syncthreads();                                   // sector writers done with carry/gpos/ccnt
  // heads and new carries: one thread per bucket (reads before it writes)
  for (int b = tid; b < nb; b += blockDim.x) {
    const uint32_t m = S.ccnt[b] + S.tcnt[b], g = S.gpos[b];
    const uint32_t h = min(m, (4u - (g & 3u)) & 3u);
    for (uint32_t k = 0; k < h; ++k)
      if ((uint64_t)g + k < lim) out[g + k] = seq(b, k);
    const uint32_t used = h + 4u * ((m - h) / 4u), rest = m - used;
    const uint2 k0 = rest > 0 ? seq(b, used) : make_uint2(0u, 0u);
    const uint2 k1 = rest > 1 ? seq(b, used + 1) : make_uint2(0u, 0u);
    const uint2 k2 = rest > 2 ? seq(b, used + 2) : make_uint2(0u, 0u);
    if (rest > 0) S.carry[b * 4 + 0] = k0;
    if (rest > 1) S.carry[b * 4 + 1] = k1;
    if (rest > 2) S.carry[b * 4 + 2] = k2;
    S.gpos[b] = g + used;
    S.ccnt[b] = rest;
    S.tcnt[b] = 0;
    S.tcur[b] = 0;
  }
  __syncthreads();
}

__device__ void part_flush(PartSmem &S, int nb, uint2 *__restrict__ out, uint32_t lim) {
  const int tid = threadIdx.x;
  for (int b = tid; b < nb; b += blockDim.x)
    for (uint32_t k = 0; k < S.ccnt[b]; ++k)
      if ((uint64_t)S.gpos[b] + k < lim) out[S.gpos[b] + k] = S.carry[b * 4 + k];
}

__device__ void part_init(PartSmem &S, int nb, const uint32_t *__restrict__ offs) {
  for (int b = threadIdx.x; b < nb; b += blockDim.x) {
    S.ccnt[b] = 0; S.tcnt[b] = 0; S.tcur[b] = 0;
    S.gpos[b] = offs[b];
  }
  __syncthreads();
}

struct PartGeom {
  uint32_t n;
  uint32_t sB;          // level-B bits (windows per A-bucket = 2^sB)
  uint32_t na;          // A-buckets
  uint32_t kb;          // level-B CTAs per A-bucket
  uint32_t nw;          // windows
};

__device__ __forceinline__ uint32_t bucket_a(uint32_t y, const PartGeom &G) { return y >> (kLgWin + G.sB); }
__device__ __forceinline__ uint32_t bucket_b(uint32_t y, const PartGeom &G) {
  return (y >> kLgWin) & ((1u << G.sB) - 1u);
}

// ---- level A
__global__ void __launch_bounds__(kPartThreads)
k_la_hist(const LevelDesc *__restrict__ desc, const uint32_t *__restrict__ log, const uint2 *__restrict__ hdr,
          uint32_t total_chunks, uint32_t *__restrict__ hist, PartGeom G) {
  __shared__ uint32_t sh[kMaxBuckets];
  if (desc[0].mode != kModeSrs) return;
  for (int b = threadIdx.x; b < kMaxBuckets; b += blockDim.x) sh[b] = 0;
  __syncthreads();
  const uint32_t c0 = (uint32_t)((uint64_t)total_chunks * blockIdx.x / gridDim.x);
  const uint32_t c1 = (uint32_t)((uint64_t)total_chunks * (blockIdx.x + 1) / gridDim.x);
  decode_chunks(log, hdr, c0, c1, G.n, [&](uint32_t y) { atomicAdd(&sh[bucket_a(y, G)], 1u); });
  __syncthreads();
  for (int b = threadIdx.x; b < (int)G.na; b += blockDim.x) hist[(size_t)blockIdx.x * G.na + b] = sh[b];
}

// Column scan: counts[cta][bucket] -> start slot of each CTA's run inside the
// bucket; bucket b's region starts at base(b).  shift: log2 of a bucket's
// index span.  groups > 1: CTAs come in groups (level B: one group per
// A-bucket, buckets are that group's windows).
__global__ void k_part_scan(const LevelDesc *__restrict__ desc, uint32_t *__restrict__ hist, int nctas_per_group,
                            int nbuckets, uint32_t shift, uint32_t n, uint32_t *__restrict__ err) {
  if (desc[0].mode != kModeSrs) return;
  const int group = blockIdx.x;
  for (int b = threadIdx.x; b < nbuckets; b += blockDim.x) {
    const uint64_t bucket = (uint64_t)group * nbuckets + b;
    const uint64_t base = bucket << shift;
    uint64_t run = base;
    for (int k = 0; k < nctas_per_group; ++k) {
      uint32_t *h = hist + ((size_t)group * nctas_per_group + k) * nbuckets + b;
      const uint32_t v = *h;
      *h = (uint32_t)run;
      run += v;
    }
    const uint64_t end = base + (1ull << shift);
    if (base < n && run > (end < n ? end : (uint64_t)n)) record_error(err, kErrNotList);
  }
}

__global__ void __launch_bounds__(kPartThreads)
k_la_write(const LevelDesc *__restrict__ desc, const uint32_t *__restrict__ log, const uint2 *__restrict__ hdr,
           uint32_t total_chunks, const uint32_t *__restrict__ offs, const uint32_t *__restrict__ r1,
           uint2 *__restrict__ out, PartGeom G, uint32_t *__restrict__ err) {
  extern __shared__ __align__(16) unsigned char smem_part[];
  PartSmem &S = *reinterpret_cast<PartSmem *>(smem_part);
  const LevelDesc d = desc[0];
  if (d.mode != kModeSrs) return;
  const uint32_t nn = desc[1].n;
  part_init(S, G.na, offs + (size_t)blockIdx.x * G.na);
  const uint32_t c0 = (uint32_t)((uint64_t)total_chunks * blockIdx.x / gridDim.x);
  const uint32_t c1 = (uint32_t)((uint64_t)total_chunks * (blockIdx.x + 1) / gridDim.x);
  // a tile: every warp decodes 2 x kDecodeIlp chunks, each lane keeps its
  // (at most one per chunk) elements in registers
  const int warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  const uint32_t per_tile = (uint32_t)nwarps * 2 * kDecodeIlp;
  uint32_t bad = 0;
  for (uint32_t t0 = c0; t0 < c1; t0 += per_tile) {
    uint2 item[kIpt];
    uint32_t off[kIpt], bk[kIpt];
#pragma unroll
    for (int r = 0; r < 2; ++r) {
      uint2 it[kDecodeIlp];
      uint32_t of[kDecodeIlp];
      decode_ilp(log, hdr, t0 + ((uint32_t)r * nwarps + warp) * kDecodeIlp, c1, G.n, it, of);
#pragma unroll
      for (int j = 0; j < kDecodeIlp; ++j) { item[r * kDecodeIlp + j] = it[j]; off[r * kDecodeIlp + j] = of[j]; }
    }
#pragma unroll
    for (int i = 0; i < kIpt; ++i) {                // rank = R_1[ruler] - offset
      if (item[i].x == kLogEnd) continue;
      const uint32_t c = item[i].y;
      uint32_t val = 0;
      if (c < nn) val = __ldcg(r1 + c) - off[i];
      else bad |= kErrInternal;
      item[i].y = val;
      bk[i] = bucket_a(item[i].x, G);
    }
    part_emit_tile(S, G.na, item, bk, out, G.n, bad);
  }
  part_flush(S, G.na, out, G.n);
  if (bad) record_error(err, bad);
}

// ---- level B: CTA (a, i) handles part i of A-bucket a's region
__device__ __forceinline__ void lb_range(const PartGeom &G, uint32_t &p0, uint32_t &p1) {
  const uint32_t a = blockIdx.x / G.kb, i = blockIdx.x % G.kb;
  const uint64_t s0 = (uint64_t)a << (kLgWin + G.sB);
  const uint64_t e0 = s0 + (1ull << (kLgWin + G.sB));
  const uint64_t s = s0 < G.n ? s0 : G.n, e = e0 < G.n ? e0 : G.n;
  p0 = (uint32_t)(s + (e - s) * i / G.kb);
  p1 = (uint32_t)(s + (e - s) * (i + 1) / G.kb);
}

__global__ void __launch_bounds__(kPartThreads)
k_lb_hist(const LevelDesc *__restrict__ desc, const uint2 *__restrict__ in, uint32_t *__restrict__ hist, PartGeom G) {
  __shared__ uint32_t sh[kMaxBuckets];
  if (desc[0].mode != kModeSrs) return;
  const uint32_t nbk = 1u << G.sB;
  for (int b = threadIdx.x; b < (int)nbk; b += blockDim.x) sh[b] = 0;
  __syncthreads();
  uint32_t p0, p1;
  lb_range(G, p0, p1);
  for (uint32_t p = p0 + threadIdx.x; p < p1; p += blockDim.x) {
    const uint32_t y = __ldcs(&in[p].x);
    if (y < G.n) atomicAdd(&sh[bucket_b(y, G)], 1u);
  }
  __syncthreads();
  for (int b = threadIdx.x; b < (int)nbk; b += blockDim.x) hist[(size_t)blockIdx.x * nbk + b] = sh[b];
}

__global__ void __launch_bounds__(kPartThreads)
k_lb_write(const LevelDesc *__restrict__ desc, const uint2 *__restrict__ in, const uint32_t *__restrict__ offs,
           uint2 *__restrict__ out, PartGeom G, uint32_t *__restrict__ err) {
  extern __shared__ __align__(16) unsigned char smem_part[];
  PartSmem &S = *reinterpret_cast<PartSmem *>(smem_part);
  if (desc[0].mode != kModeSrs) return;
  const uint32_t nbk = 1u << G.sB;
  part_init(S, nbk, offs + (size_t)blockIdx.x * nbk);
  uint32_t p0, p1;
  lb_range(G, p0, p1);
  uint32_t bad = 0;
  for (uint32_t t0 = p0; t0 < p1; t0 += kPartTile) {
    uint2 item[kIpt];
    uint32_t bk[kIpt];
#pragma unroll
    for (int i = 0; i < kIpt; ++i) {
      const uint32_t p = t0 + (uint32_t)i * blockDim.x + threadIdx.x;
      item[i] = p < p1 ? __ldcs(in + p) : make_uint2(kLogEnd, 0u);
      if (item[i].x != kLogEnd && item[i].x >= G.n) { bad |= kErrInternal; item[i].x = kLogEnd; }
      bk[i] = item[i].x != kLogEnd ? bucket_b(item[i].x, G) : 0u;
    }
    part_emit_tile(S, nbk, item, bk, out, G.n, bad);
  }
  part_flush(S, nbk, out, G.n);
  if (bad) record_error(err, bad);
}

// ---- scatter: one CTA per window of 2^kLgWin ranks assembled in shared memory
__global__ void __launch_bounds__(256)
k_win_scatter(const LevelDesc *__restrict__ desc, const uint2 *__restrict__ in, uint32_t *__restrict__ rank,
              uint32_t *__restrict__ err) {
  extern __shared__ __align__(16) uint32_t win[];
  const LevelDesc d = desc[0];
  if (d.mode != kModeSrs) return;
  const uint32_t n = d.n;
  const uint64_t w0 = (uint64_t)blockIdx.x << kLgWin;
  if (w0 >= n) return;
  const uint32_t len = (uint32_t)min((uint64_t)1 << kLgWin, (uint64_t)n - w0);
  uint32_t bad = 0;
  if (blockIdx.x == 0 && threadIdx.x == 0 && d.visited != n) bad |= d.visited > n ? kErrNotList : kErrCycle;
  for (uint32_t p = threadIdx.x; p < len; p += blockDim.x) {
    const uint2 v = __ldcs(in + w0 + p);
    const uint64_t loc = (uint64_t)v.x - w0;
    if (loc < len) win[loc] = v.y; else bad |= kErrInternal;
  }
  __syncthreads();
  uint32_t *dst = rank + w0;
  if ((len & 3u) == 0 && ((uintptr_t)dst & 15u) == 0) {
    for (uint32_t q = threadIdx.x; q < len / 4; q += blockDim.x)
      __stcs(reinterpret_cast<uint4 *>(dst) + q, reinterpret_cast<const uint4 *>(win)[q]);
  } else {
    for (uint32_t q = threadIdx.x; q < len; q += blockDim.x) dst[q] = win[q];
  }
  if (bad) record_error(err, bad);
}

// Host side: geometry and launch sequence.
void log_part_geometry(uint32_t n, uint32_t *sB, uint32_t *na, uint32_t *kb, uint32_t *nw) {
  const uint32_t w = (uint32_t)(((uint64_t)n + (1u << kLgWin) - 1) >> kLgWin);
  uint32_t lg = 0;
  while ((1ull << lg) < w) ++lg;
  *sB = lg > 8 ? lg - 8 : 0;
  *na = (w + (1u << *sB) - 1) >> *sB;
  *kb = *sB ? std::max<uint32_t>(1, 1024 / *na) : 0;
  *nw = w;
}

static size_t part_smem() { return sizeof(PartSmem); }

cudaError_t log_setup() {
  cudaError_t e = cudaFuncSetAttribute(k_la_write, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)part_smem());
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_lb_write, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)part_smem());
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_win_scatter, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(4u << kLgWin));
}

cudaError_t launch_finalize_log(LevelDesc *desc, const uint32_t *log, const uint2 *hdr,
                                uint32_t total_chunks, const void *r1, uint2 *pairsA, uint2 *pairsB,
                                uint32_t *histA, uint32_t *histB, int ga, uint32_t *rank, uint32_t n,
                                uint32_t *err, cudaStream_t s) {
  PartGeom G;
  G.n = n;
  log_part_geometry(n, &G.sB, &G.na, &G.kb, &G.nw);
  const uint32_t shiftA = kLgWin + G.sB;
  k_la_hist<<<ga, kPartThreads, 0, s>>>(desc, log, hdr, total_chunks, histA, G);
  k_part_scan<<<1, 256, 0, s>>>(desc, histA, ga, (int)G.na, shiftA, n, err);
  k_la_write<<<ga, kPartThreads, part_smem(), s>>>(desc, log, hdr, total_chunks, histA,
                                                   reinterpret_cast<const uint32_t *>(r1), pairsA, G, err);
  const uint2 *final_pairs = pairsA;
  int launches = 4;
  if (G.sB > 0) {
    const int gb = (int)(G.na * G.kb);
    k_lb_hist<<<gb, kPartThreads, 0, s>>>(desc, pairsA, histB, G);
    k_part_scan<<<G.na, 256, 0, s>>>(desc, histB, (int)G.kb, 1 << G.sB, kLgWin, n, err);
    k_lb_write<<<gb, kPartThreads, part_smem(), s>>>(desc, pairsA, histB, pairsB, G, err);
    final_pairs = pairsB;
    launches += 3;
  }
  k_win_scatter<<<G.nw, 256, 4u << kLgWin, s>>>(desc, final_pairs, rank, err);
  count_launch(launches);
  return cudaGetLastError();
}

}  // namespace lr
