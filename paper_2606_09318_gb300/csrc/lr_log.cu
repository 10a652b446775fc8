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
// (local: also count the links that stay inside their 4096-id tile, for the
// contraction decision)
__global__ void __launch_bounds__(256)
k_sum0(const uint32_t *__restrict__ succ, uint32_t n, unsigned long long *__restrict__ acc,
       unsigned long long *__restrict__ local, uint32_t *__restrict__ err, int vec) {
  unsigned long long S = 0, T = 0;
  uint32_t loc = 0;
  uint32_t bad = 0;
  auto take = [&](uint32_t i, uint32_t s) {
    if (s >= n) bad = 1;
    else if (s == i) T += 1;
    else {
      S += s;
      loc += (s >> kContractTileShift) == (i >> kContractTileShift);
    }
  };
  const uint32_t ngroups = (uint32_t)(((uint64_t)n + 3u) / 4u);
  const uint32_t stride = gridDim.x * blockDim.x;
  uint32_t g = blockIdx.x * blockDim.x + threadIdx.x;
  if (vec) {                                   // two 16-byte loads in flight per thread
    const uint4 *s4 = reinterpret_cast<const uint4 *>(succ);
    const uint32_t nfull = n / 4u;
    for (; (uint64_t)g + stride < nfull; g += 2 * stride) {
      const uint4 a = __ldcs(s4 + g), b = __ldcs(s4 + g + stride);
      const uint32_t i = g * 4u, j = (g + stride) * 4u;
      take(i, a.x); take(i + 1, a.y); take(i + 2, a.z); take(i + 3, a.w);
      take(j, b.x); take(j + 1, b.y); take(j + 2, b.z); take(j + 3, b.w);
    }
  }
  for (; g < ngroups; g += stride) {
    const uint32_t i0 = g * 4u;
    const uint32_t cnt = min(4u, n - i0);
    if (vec && cnt == 4u) {
      const uint4 v = __ldcs(reinterpret_cast<const uint4 *>(succ + i0));
      take(i0, v.x); take(i0 + 1, v.y); take(i0 + 2, v.z); take(i0 + 3, v.w);
    } else {
      for (uint32_t j = 0; j < cnt; ++j) take(i0 + j, __ldcs(succ + i0 + j));
    }
  }
  for (int d = 16; d > 0; d >>= 1) {
    S += __shfl_down_sync(0xFFFFFFFFu, S, d);
    T += __shfl_down_sync(0xFFFFFFFFu, T, d);
    loc += __shfl_down_sync(0xFFFFFFFFu, loc, d);
  }
  if ((threadIdx.x & 31) == 0) {
    if (T) atomicAdd(acc + 0, T);
    if (S) atomicAdd(acc + 1, S);
    if (local && loc) atomicAdd(local, (unsigned long long)loc);
  }
  if (bad) record_error(err, kErrRange);
}

cudaError_t launch_sum0(const uint32_t *succ, uint32_t n, unsigned long long *acc, unsigned long long *local,
                        uint32_t *err, cudaStream_t s) {
  const int block = 256;
  const int vec = ((uintptr_t)succ & 15u) == 0;
  k_sum0<<<stream_grid(((uint64_t)n + 3) / 4, block), block, 0, s>>>(succ, n, acc, local, err, vec);
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
// Chunks are handed out from one global counter, to each CTA in windows of
// kLogWindow consecutive chunks (one global atomic per window), so that the
// used chunks are exactly [0, *ctr) whatever the segments' lengths, apart
// from the unused rest of each CTA's last window (headers kLogEnd).
struct LogCfg {
  uint32_t *log;          // chunks of kChunk entries
  uint2 *hdr;             // per chunk: (ruler, offset) of its first entry, or (kLogEnd, 0)
  uint32_t total_chunks;  // capacity
  uint32_t *ctr;          // chunks handed out (zeroed per call)
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
  // s_win: the CTA's window, (end << 32) | next, in global chunk ids.  The
  // thread that draws next == end takes a new window from the global
  // counter; threads that draw past the end meanwhile take one chunk each
  // from the global counter.  Nobody waits.
  __device__ bool alloc(const LogCfg &L, unsigned long long *s_win) {
    const unsigned long long w = atomicAdd(s_win, 1ull);
    const uint32_t next = (uint32_t)w, end = (uint32_t)(w >> 32);
    uint64_t id;
    if (next < end) {
      id = next;
    } else if (next == end) {
      id = atomicAdd(L.ctr, kLogWindow);
      if (id + kLogWindow <= L.total_chunks)
        atomicExch(s_win, ((unsigned long long)(id + kLogWindow) << 32) | (id + 1));
    } else {
      id = atomicAdd(L.ctr, 1u);
    }
    if (id >= L.total_chunks) { ok = false; return false; }
    chunk = (uint32_t)id;
    slot = 0;
    L.hdr[chunk] = make_uint2(gc, go);
    return true;
  }
  __device__ void flush(const LogCfg &L, unsigned long long *s_win) {
    nb = 0;
    if (!ok || (slot == kChunk && !alloc(L, s_win))) return;
    st_sector(L.log + (size_t)chunk * kChunk + slot, b0, b1, b2, b3, b4, b5, b6, b7);
    slot += 8;
  }
  __device__ __forceinline__ void shift_in(uint32_t v) {
    b0 = b1; b1 = b2; b2 = b3; b3 = b4; b4 = b5; b5 = b6; b6 = b7; b7 = v;
  }
  // v: the entry; (c, o): its ruler and offset when v is an element
  __device__ __forceinline__ void put(const LogCfg &L, unsigned long long *s_win, uint32_t v, uint32_t c,
                                      uint32_t o) {
    if (nb == 0) { gc = c; go = o; }
    shift_in(v);
    if (++nb == 8) flush(L, s_win);
  }
  __device__ void finish(const LogCfg &L, unsigned long long *s_win) {
    if (nb > 0) {
      while (nb < 8) { shift_in(kLogEnd); ++nb; }
      flush(L, s_win);
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
  __shared__ unsigned long long s_win;
  if (threadIdx.x == 0) s_win = 0;
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
    if (dbg_fail(rho < n && c < desc[1].cap, err)) { c64 = cnext; continue; }
    W.put(L, &s_win, kMark | c, kLogEnd, 0);
    uint32_t x = rho, o = 0, nxt = c;
    for (;;) {
      const uint32_t s = __ldcg(succ + x);
      W.put(L, &s_win, x, c, o);
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
  W.finish(L, &s_win);
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
                             uint2 *hdr, uint32_t total_chunks, uint32_t *ctr, cudaStream_t s) {
  LogCfg L;
  L.log = log;
  L.hdr = hdr;
  L.total_chunks = total_chunks;
  L.ctr = ctr;
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
// 2^kLgWin elements (a radix partition, one level or two), then each window
// is assembled in shared memory and written out as whole lines.
//   level A: decode the log, partition by A-bucket (y >> (kLgWin + sB));
//   level B: partition each A-bucket by window (only when there are more
//            windows than one level can hold);
//   scatter: one CTA per window.
// No histogram pass: for a valid list a bucket receives exactly the elements
// of its index range, so each bucket owns a region of that size plus slack,
// and a CTA claims room in it with one global atomic per block of `claim`
// slots.  Every store covers a whole 32-byte sector (four pairs): a CTA
// carries fewer than four leftover pairs of a bucket into its next tile and,
// at its end, fills the unused part of its last block with empty pairs
// (y = kLogEnd), which the consumers skip.
constexpr int kLgWin = 14;                 // 16384 ranks = 64 KiB of shared memory
constexpr int kMaxBuckets = 256;
constexpr int kPartThreads = 512;
constexpr int kIpt = 8;                    // items a thread holds per partition tile
constexpr int kPartTile = kPartThreads * kIpt;
constexpr int kSortCap = kPartTile + 6 * kMaxBuckets;   // runs padded to whole quads
constexpr int kDecodeIlp = 4;              // chunks a warp decodes with their loads in flight
constexpr uint32_t kDead = 0xFFFFFFFFu;    // bucket region overflowed (invalid input)
constexpr int kScatterThreads = 512;
// The log form takes n <= 2^30: at most 2^(30 - kLgWin) windows, which two
// partition levels of at most kMaxBuckets buckets each must cover.
static_assert((1u << (30 - kLgWin)) <= (uint32_t)kMaxBuckets * kMaxBuckets,
              "two partition levels must cover every window");

struct PartSmem {
  uint2 sorted[kSortCap];                  // this tile's pairs, bucket by bucket
  uint2 carry[kMaxBuckets * 4];            // < 4 leftover pairs per bucket
  uint32_t cnt[kMaxBuckets];               // this tile's pairs per bucket (reset once read)
  uint32_t ccnt[kMaxBuckets];              // carried pairs per bucket
  uint32_t pos[kMaxBuckets];               // next free slot of the bucket's current block
  uint32_t left[kMaxBuckets];              // free slots left in it (a multiple of 4), or kDead
  // this tile, per bucket: {first slot of its run in `sorted` | run length
  // << 16, room left in the current block, its free slot, the block claimed
  // for the rest}, and where the tile's own pairs start (after the carried)
  uint4 tile[kMaxBuckets];
  uint32_t tbase[kMaxBuckets];
  uint32_t wsum[32];
};

// Output of one partition: bucket b owns out[b * cap, (b + 1) * cap); cur[b]
// counts the slots claimed in it.
struct PartOut {
  uint2 *out;
  uint32_t *cur;
  uint32_t cap;          // slots per region
  uint32_t claim;        // slots per claim (a multiple of 4)
  uint32_t nb;           // buckets (<= kMaxBuckets)
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
    uint32_t c = h[j].x, o = h[j].y + (uint32_t)lane;
    if (mm) {                                      // warp-uniform: the chunk starts a segment
      const uint32_t below = mm & ((2u << lane) - 1u);
      const int m = below ? 31 - __clz(below) : 0;
      const uint32_t em = __shfl_sync(0xFFFFFFFFu, e[j], m);
      if (below) { c = em & ~kMark; o = (uint32_t)(lane - m - 1); }
    }
    if (e[j] != kLogEnd && !(e[j] & kMark) && e[j] < n) { out[j] = make_uint2(e[j], c); off[j] = o; }
  }
}

// Bulk prefetch of [p, p + bytes) into L2, shrunk inward to 16-byte
// boundaries (a hint: the next tile's input, fetched while this one is
// partitioned).
__device__ __forceinline__ void prefetch_l2(const void *p, size_t bytes) {
  const uintptr_t a = ((uintptr_t)p + 15u) & ~(uintptr_t)15u;
  const uintptr_t e = ((uintptr_t)p + bytes) & ~(uintptr_t)15u;
  if (e > a)
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" :: "l"(a), "r"((uint32_t)(e - a)) : "memory");
}

// Exclusive scan of v over the block's threads (all threads call it, at most
// 32 warps); the total comes back through `total`.  `wsum` may be written
// again only after another barrier of the block.
__device__ __forceinline__ uint32_t block_scan_excl(uint32_t v, uint32_t *wsum, uint32_t &total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  uint32_t x = v;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, d);
    if (lane >= d) x += y;
  }
  if (lane == 31) wsum[warp] = x;
  __syncthreads();
  uint32_t t = lane < nwarps ? wsum[lane] : 0u;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, t, d);
    if (lane >= d) t += y;
  }
  const uint32_t before = __shfl_sync(0xFFFFFFFFu, t, warp > 0 ? warp - 1 : 0);
  total = __shfl_sync(0xFFFFFFFFu, t, 31);
  return (warp > 0 ? before : 0u) + x - v;
}

__device__ __forceinline__ void part_init(PartSmem &S, uint32_t nb) {
  for (uint32_t b = threadIdx.x; b < nb; b += blockDim.x) {
    S.cnt[b] = 0; S.ccnt[b] = 0; S.pos[b] = 0; S.left[b] = 0;
  }
  __syncthreads();
}

// One tile of register-held pairs (item[i].x != kLogEnd: a pair, bk[i] its
// bucket, which is (item[i].x >> kshift) & kmask) -> bucket runs in shared
// memory, laid out so that every aligned quad of `sorted` is one quad of its
// bucket's output -> whole-sector stores.  The first pair of every quad is a
// real pair (a bucket's run is padded only to the end of its last quad), so
// the quad's bucket is read off that pair's id.
// The stored value is item[i].y - sub[i]: the caller may pass item[i].y
// straight from a load still in flight, which is first used when the pair
// is placed, after the tile's counting, scan and claims.
__device__ void part_tile(PartSmem &S, const PartOut &P, const uint2 (&item)[kIpt],
                          const uint32_t (&sub)[kIpt], const uint32_t (&bk)[kIpt], uint32_t kshift,
                          uint32_t kmask, uint32_t &bad) {
  const uint32_t tid = threadIdx.x, nb = P.nb;
  uint32_t slot[kIpt];
#pragma unroll
  for (int i = 0; i < kIpt; ++i) slot[i] = item[i].x != kLogEnd ? atomicAdd(&S.cnt[bk[i]], 1u) : 0u;
  __syncthreads();
  uint32_t m = 0, alloc = 0;
  if (tid < nb) {
    m = S.ccnt[tid] + S.cnt[tid];
    alloc = (m + 3u) & ~3u;
  }
  uint32_t total;
  const uint32_t st = block_scan_excl(alloc, S.wsum, total);
  if (tid < nb) {
    const uint32_t b = tid, cc = S.ccnt[b], full = m & ~3u;
    uint32_t p = S.pos[b], l = S.left[b], np = 0;
    S.cnt[b] = 0;
    if (l != kDead && full > l) {                   // claim room for what the block lacks
      const uint32_t x = full - l;
      const uint32_t c = (x + P.claim - 1u) / P.claim * P.claim;
      const uint32_t o = atomicAdd(P.cur + b, c);
      if ((uint64_t)o + c > P.cap) {
        bad |= kErrNotList;                          // more pairs than the bucket's range holds
        l = kDead;
      } else {
        np = o;
        S.pos[b] = o + x;
        S.left[b] = c - x;
      }
    } else if (l != kDead) {
      S.pos[b] = p + full;
      S.left[b] = l - full;
    }
    if (l == kDead) S.left[b] = kDead;
    S.tile[b] = make_uint4(st | (m << 16), l, p, np);
    S.tbase[b] = st + cc;
    S.ccnt[b] = m - full;
    for (uint32_t k = 0; k < cc; ++k) S.sorted[st + k] = S.carry[b * 4 + k];
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < kIpt; ++i)
    if (item[i].x != kLogEnd) S.sorted[S.tbase[bk[i]] + slot[i]] = make_uint2(item[i].x, item[i].y - sub[i]);
  __syncthreads();
  const uint32_t nq = total / 4;
  for (uint32_t q = tid; q < nq; q += blockDim.x) {
    const uint32_t b = (S.sorted[4 * q].x >> kshift) & kmask;
    const uint4 t = S.tile[b];
    const uint32_t k = 4 * q - (t.x & 0xFFFFu), rm = t.x >> 16;
    if (k + 4 <= rm) {
      const uint32_t l = t.y;
      if (l == kDead) continue;
      const uint32_t dst = k < l ? t.z + k : t.w + (k - l);
      const uint4 *src = reinterpret_cast<const uint4 *>(S.sorted + 4 * q);
      const uint4 u = src[0], v = src[1];
      st_sector(P.out + (size_t)b * P.cap + dst, u.x, u.y, u.z, u.w, v.x, v.y, v.z, v.w);
    } else {
      for (uint32_t j = k; j < rm; ++j) S.carry[b * 4 + (j - k)] = S.sorted[4 * q + (j - k)];
    }
  }
  // no barrier here: the next tile only counts (S.cnt, which this step does
  // not touch) before its first barrier, and everything this step reads or
  // writes is next written or read after that barrier (part_flush is preceded
  // by one of its own)
}

// End of a CTA's input: the carried pairs of each bucket, padded with empty
// pairs, and empty pairs in the rest of its last block.
__device__ void part_flush(PartSmem &S, const PartOut &P, uint32_t &bad) {
  __syncthreads();                                   // the last tile's carries are written
  for (uint32_t b = threadIdx.x; b < P.nb; b += blockDim.x) {
    uint32_t l = S.left[b], p = S.pos[b];
    const uint32_t r = S.ccnt[b];
    if (l == kDead || (r == 0 && l == 0)) continue;
    if (l == 0) {
      const uint32_t o = atomicAdd(P.cur + b, P.claim);
      if ((uint64_t)o + P.claim > P.cap) {
        bad |= kErrNotList;
        continue;
      }
      p = o;
      l = P.claim;
    }
    uint2 *dst = P.out + (size_t)b * P.cap + p;
    if (r > 0) {
      uint2 q[4];
#pragma unroll
      for (uint32_t k = 0; k < 4; ++k) q[k] = k < r ? S.carry[b * 4 + k] : make_uint2(kLogEnd, 0u);
      st_sector(dst, q[0].x, q[0].y, q[1].x, q[1].y, q[2].x, q[2].y, q[3].x, q[3].y);
      dst += 4;
      l -= 4;
    }
    for (; l > 0; l -= 4, dst += 4) st_sector(dst, kLogEnd, 0u, kLogEnd, 0u, kLogEnd, 0u, kLogEnd, 0u);
  }
}

// ---- level A: decode the log, rank = R_1[ruler] - offset, partition by y >> shift
__global__ void __launch_bounds__(kPartThreads, 2)
k_part_log(const LevelDesc *__restrict__ desc, const uint32_t *__restrict__ log, const uint2 *__restrict__ hdr,
           uint32_t total_chunks, const uint32_t *__restrict__ chunk_ctr, const uint32_t *__restrict__ r1,
           PartOut P, uint32_t shift, uint32_t *__restrict__ err) {
  extern __shared__ __align__(16) unsigned char smem_part[];
  PartSmem &S = *reinterpret_cast<PartSmem *>(smem_part);
  const LevelDesc d = desc[0];
  if (d.mode != kModeSrs) return;
  const uint32_t n = d.n, nn = desc[1].n;
  part_init(S, P.nb);
  const uint32_t used = min(__ldcg(chunk_ctr), total_chunks);       // chunks the chase handed out
  const uint32_t c0 = (uint32_t)((uint64_t)used * blockIdx.x / gridDim.x);
  const uint32_t c1 = (uint32_t)((uint64_t)used * (blockIdx.x + 1) / gridDim.x);
  // a tile: every warp decodes 2 x kDecodeIlp chunks; each lane keeps its
  // (at most one per chunk) elements in registers
  const int warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  const uint32_t per_tile = (uint32_t)nwarps * 2 * kDecodeIlp;
  uint32_t bad = 0;
  for (uint32_t t0 = c0; t0 < c1; t0 += per_tile) {
    if (threadIdx.x == 0 && t0 + per_tile < c1) {
      const uint32_t nx = t0 + per_tile, ne = min(c1, nx + per_tile);
      prefetch_l2(log + (size_t)nx * kChunk, (size_t)(ne - nx) * kChunk * 4);
      prefetch_l2(hdr + nx, (size_t)(ne - nx) * 8);
    }
    uint2 item[kIpt];
    uint32_t off[kIpt], bk[kIpt];
#pragma unroll
    for (int r = 0; r < 2; ++r) {
      uint2 it[kDecodeIlp];
      uint32_t of[kDecodeIlp];
      decode_ilp(log, hdr, t0 + ((uint32_t)r * nwarps + warp) * kDecodeIlp, c1, n, it, of);
#pragma unroll
      for (int j = 0; j < kDecodeIlp; ++j) { item[r * kDecodeIlp + j] = it[j]; off[r * kDecodeIlp + j] = of[j]; }
    }
#pragma unroll
    for (int i = 0; i < kIpt; ++i) {             // issue the R_1 gathers first
      const uint32_t c = item[i].y;
      const bool ok = item[i].x != kLogEnd && c < nn;
      if (item[i].x != kLogEnd && c >= nn) bad |= kErrInternal;
      item[i].y = ok ? __ldcg(r1 + c) : 0u;
    }
#pragma unroll
    for (int i = 0; i < kIpt; ++i) bk[i] = item[i].x != kLogEnd ? item[i].x >> shift : 0u;
    part_tile(S, P, item, off, bk, shift, 0xFFFFFFFFu, bad);
  }
  part_flush(S, P, bad);
  if (bad) record_error(err, bad);
}

// ---- level B: CTA (a, i) partitions part i of A-bucket a's region by window
__global__ void __launch_bounds__(kPartThreads, 2)
k_part_win(const LevelDesc *__restrict__ desc, const uint2 *__restrict__ in, const uint32_t *__restrict__ cur_in,
           uint32_t cap_in, uint32_t kb, uint32_t sB, PartOut P, uint32_t *__restrict__ err) {
  extern __shared__ __align__(16) unsigned char smem_part[];
  PartSmem &S = *reinterpret_cast<PartSmem *>(smem_part);
  if (desc[0].mode != kModeSrs) return;
  const uint32_t a = blockIdx.x / kb, i = blockIdx.x % kb;
  const uint32_t len = min(__ldcg(cur_in + a), cap_in);
  const uint32_t p0 = (uint32_t)((uint64_t)len * i / kb), p1 = (uint32_t)((uint64_t)len * (i + 1) / kb);
  const uint2 *src = in + (size_t)a * cap_in;
  PartOut Q = P;
  Q.out = P.out + ((size_t)a << sB) * P.cap;
  Q.cur = P.cur + ((size_t)a << sB);
  part_init(S, Q.nb);
  const uint32_t wmask = (1u << sB) - 1u;
  uint32_t bad = 0;
  for (uint32_t t0 = p0; t0 < p1; t0 += kPartTile) {
    if (threadIdx.x == 0 && t0 + kPartTile < p1) {
      const uint32_t nx = t0 + kPartTile, ne = min(p1, nx + kPartTile);
      prefetch_l2(src + nx, (size_t)(ne - nx) * 8);
    }
    uint2 item[kIpt];
    uint32_t bk[kIpt];
#pragma unroll
    for (int j = 0; j < kIpt; ++j) {
      const uint32_t p = t0 + (uint32_t)j * blockDim.x + threadIdx.x;
      item[j] = p < p1 ? __ldcs(src + p) : make_uint2(kLogEnd, 0u);
      bk[j] = 0;
      if (item[j].x == kLogEnd) continue;
      if ((item[j].x >> (kLgWin + sB)) != a) {       // not this bucket's: never for pairs written above
        bad |= kErrInternal;
        item[j].x = kLogEnd;
        continue;
      }
      bk[j] = (item[j].x >> kLgWin) & wmask;
    }
    const uint32_t zero[kIpt] = {0, 0, 0, 0, 0, 0, 0, 0};
    part_tile(S, Q, item, zero, bk, kLgWin, wmask, bad);
  }
  part_flush(S, Q, bad);
  if (bad) record_error(err, bad);
}

// ---- scatter: one CTA per window of 2^kLgWin ranks assembled in shared memory
__global__ void __launch_bounds__(kScatterThreads)
k_win_scatter(const LevelDesc *__restrict__ desc, const uint2 *__restrict__ in, const uint32_t *__restrict__ cur,
              uint32_t cap, uint32_t *__restrict__ rank, uint32_t *__restrict__ err) {
  extern __shared__ __align__(16) uint32_t win[];
  uint32_t *s_count = win + (1u << kLgWin);
  const LevelDesc d = desc[0];
  if (d.mode != kModeSrs) return;
  const uint32_t n = d.n;
  const uint64_t w0 = (uint64_t)blockIdx.x << kLgWin;
  if (w0 >= n) return;
  const uint32_t len = (uint32_t)min((uint64_t)1 << kLgWin, (uint64_t)n - w0);
  if (threadIdx.x == 0) *s_count = 0;
  __syncthreads();
  uint32_t bad = 0, got = 0;
  if (blockIdx.x == 0 && threadIdx.x == 0 && d.visited != n) bad |= d.visited > n ? kErrNotList : kErrCycle;
  // a region holds whole quads of pairs (claims are multiples of four), 32-byte aligned
  const uint32_t nq = min(__ldcg(cur + blockIdx.x), cap) / 4;
  const uint4 *src = reinterpret_cast<const uint4 *>(in + (size_t)blockIdx.x * cap);
  auto put = [&](uint32_t y, uint32_t v) {
    if (y == kLogEnd) return;
    const uint64_t loc = (uint64_t)y - w0;
    if (loc < len) { win[loc] = v; ++got; } else bad |= kErrInternal;
  };
  for (uint32_t q = threadIdx.x; q < nq; q += 2 * blockDim.x) {
    const uint32_t q2 = q + blockDim.x;
    const uint4 a = __ldcs(src + 2 * q), b = __ldcs(src + 2 * q + 1);
    uint4 c = make_uint4(kLogEnd, 0u, kLogEnd, 0u), e = c;
    if (q2 < nq) { c = __ldcs(src + 2 * q2); e = __ldcs(src + 2 * q2 + 1); }
    put(a.x, a.y); put(a.z, a.w); put(b.x, b.y); put(b.z, b.w);
    put(c.x, c.y); put(c.z, c.w); put(e.x, e.y); put(e.z, e.w);
  }
  for (int dd = 16; dd > 0; dd >>= 1) got += __shfl_down_sync(0xFFFFFFFFu, got, dd);
  if ((threadIdx.x & 31) == 0 && got) atomicAdd(s_count, got);
  __syncthreads();
  // a window that did not receive each of its elements exactly once: some
  // element was reached twice (and, as the chase visited n in all, another
  // never), which only a list with in-degree > 1 produces
  if (threadIdx.x == 0 && *s_count != len && d.visited == n) bad |= kErrNotList;
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
static size_t part_smem() { return sizeof(PartSmem); }
static size_t scatter_smem() { return (4u << kLgWin) + 16; }

// Resident CTAs of the level-A kernel on the current device.  The workspace
// size depends on it, so it is computed the same way whether or not the
// device setup ran before (it sets the shared-memory attribute itself).
static int part_resident_ctas() {
  static int cached[64] = {0};
  int dev = 0, sms = 0, per = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) dev = 0;
  if (cached[dev]) return cached[dev];
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0) sms = 1;
  if (cudaFuncSetAttribute(k_part_log, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)part_smem()) !=
          cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_part_log, kPartThreads, part_smem()) != cudaSuccess ||
      per <= 0)
    per = 1;
  cached[dev] = per * sms;
  return cached[dev];
}

LogGeom log_geometry(uint32_t n) {
  LogGeom g;
  g.nw = (uint32_t)(((uint64_t)n + (1u << kLgWin) - 1) >> kLgWin);
  uint32_t lg = 0;
  while ((1ull << lg) < g.nw) ++lg;
  g.sB = lg > 8 ? lg - 8 : 0;
  g.na = (g.nw + (1u << g.sB) - 1) >> g.sB;
  g.shiftA = kLgWin + g.sB;
  const uint64_t chunks_per_cta = 32;                       // a few tiles each at least
  const uint64_t want = ((uint64_t)n / 32 + chunks_per_cta - 1) / chunks_per_cta;
  g.gridA = (uint32_t)std::max<uint64_t>(1, std::min<uint64_t>(part_resident_ctas(), want));
  g.claimA = g.sB ? 32 : 8;
  g.capA = (1u << g.shiftA) + g.gridA * g.claimA;
  g.kb = g.sB ? std::max<uint32_t>(1, 2048 / g.na) : 0;
  g.claimB = 16;
  g.capB = g.sB ? (1u << kLgWin) + g.kb * g.claimB : 0;
  g.nbB = g.sB ? (g.na << g.sB) : 0;
  return g;
}

cudaError_t log_setup() {
  cudaError_t e = cudaFuncSetAttribute(k_part_log, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)part_smem());
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_part_win, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)part_smem());
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_win_scatter, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)scatter_smem());
}

cudaError_t launch_finalize_log(LevelDesc *desc, const uint32_t *log, const uint2 *hdr, uint32_t total_chunks,
                                const uint32_t *chunk_ctr, const void *r1, uint2 *pairsA, uint2 *pairsB,
                                uint32_t *curA, uint32_t *curB, const LogGeom &g, uint32_t *rank, uint32_t *err,
                                cudaStream_t s) {
  // every partition writes into shared-memory tables of kMaxBuckets buckets
  if (g.na > (uint32_t)kMaxBuckets || (g.sB > 0 && (1u << g.sB) > (uint32_t)kMaxBuckets))
    return cudaErrorInvalidValue;
  PartOut A;
  A.out = pairsA;
  A.cur = curA;
  A.cap = g.capA;
  A.claim = g.claimA;
  A.nb = g.na;
  k_part_log<<<g.gridA, kPartThreads, part_smem(), s>>>(desc, log, hdr, total_chunks, chunk_ctr,
                                                        reinterpret_cast<const uint32_t *>(r1), A, g.shiftA, err);
  int launches = 2;
  if (g.sB > 0) {
    PartOut B;
    B.out = pairsB;
    B.cur = curB;
    B.cap = g.capB;
    B.claim = g.claimB;
    B.nb = 1u << g.sB;
    k_part_win<<<g.na * g.kb, kPartThreads, part_smem(), s>>>(desc, pairsA, curA, g.capA, g.kb, g.sB, B, err);
    k_win_scatter<<<g.nw, kScatterThreads, scatter_smem(), s>>>(desc, pairsB, curB, g.capB, rank, err);
    launches = 3;
  } else {
    k_win_scatter<<<g.nw, kScatterThreads, scatter_smem(), s>>>(desc, pairsA, curA, g.capA, rank, err);
  }
  count_launch(launches);
  return cudaGetLastError();
}

}  // namespace lr
