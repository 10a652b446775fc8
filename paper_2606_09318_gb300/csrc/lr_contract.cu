// lr_contract.cu -- tile-local contraction before the ruling set (Section 2.3).
//
// The paper contracts, on every PE, the sublists made only of local
// elements before the distributed algorithm runs, and restores them at the
// end.  On one GPU "local" becomes a tile of kTile consecutive ids held in
// shared memory:
//   local link   i -> succ[i] with both ends in the same tile;
//   local head   an element with no local predecessor;
//   local tail   an element whose link leaves the tile (or a terminal).
// Every local head h starts a local sublist that ends at a local tail t.
// The contracted list has one node per local head: its successor is the
// local head that t's link enters (an element whose only predecessor lies
// in another tile is necessarily a local head there), its weight the sum of
// the link weights from h through t's link.  A contracted terminal keeps
// the distance from its head to the list's terminal as its weight, so the
// contracted list is ranked with the inclusive-tail form.  Then
//   rank[i] = dist(i -> t) + (t terminal ? 0 : w(t) + R_c[node entered by t]).
// Contracted ids are dense: a rank/select structure over the local-head
// bitmap gives node(x) = heads in earlier tiles + heads before x in its tile.
//
// Inside a tile, t and the link count to it come from pointer doubling over
// all of the tile's elements in shared memory, each thread holding the
// words of its eight elements in registers: at most log2(tile) rounds of
// one shared-memory gather per unsettled element, with no divergence, until
// every pointer has reached a local tail.  Weighted distances then follow
// from one prefix sum of the weights in list order.  (A ruling set inside
// the tile does less work, but its walks diverge and its phases need more
// barriers; on GB300 the doubling was the faster of the two.)
//
// Passes: solve (every tile in shared memory: distances to the local tails,
// the local-head bitmap), scan (tile prefixes), nodes (the contracted
// list), the ruling set on the contracted list, tails and fix (the ranks).
// Whether to contract is decided by the caller from the count of links that
// stay inside their tile: exact from the log form's first pass, or from a
// sample of the tiles before a first pass that would pack records.
#include <algorithm>
#include <cstddef>
#include <cuda_runtime.h>

#include "lr_device.cuh"
#include "lr_kernels.h"

namespace lr {

namespace {

constexpr int kTileShift = kContractTileShift;
constexpr uint32_t kTile = 1u << kTileShift;
constexpr uint32_t kTileWords = kTile / 32;
constexpr int kLcThreads = 512;
constexpr uint16_t kEnd16 = 0xFFFF;

template <int WT>
__device__ __forceinline__ uint64_t lc_weight(const void *w, uint32_t i) {
  if constexpr (WT == 1) return (uint64_t)(int64_t)__ldg(reinterpret_cast<const int *>(w) + i);
  else if constexpr (WT == 2) return (uint64_t)__ldg(reinterpret_cast<const long long *>(w) + i);
  else return 1u;
}

// Contracted id of a local head x (rank/select over the head bitmap).
__device__ __forceinline__ uint32_t lc_node(uint32_t x, const uint32_t *hb, const uint16_t *wpre,
                                            const uint32_t *tpre) {
  const uint32_t w = x >> 5;
  return __ldg(tpre + (x >> kTileShift)) + __ldg(wpre + w) +
         (uint32_t)__popc(__ldcg(hb + w) & ((1u << (x & 31u)) - 1u));
}

__device__ __forceinline__ bool lc_is_head(uint32_t x, const uint32_t *hb) {
  return (__ldcg(hb + (x >> 5)) >> (x & 31u)) & 1u;
}

// Shared-memory state of one tile.  Every element of the tile carries a
// pointer p (first its local successor, or itself for a local tail) and the
// number of links d to p; pointer doubling (p, d) <- (p[p], d + d[p]) from
// one buffer into the other reaches the local tail and the link count to it
// in at most kTileShift rounds, because a local sublist has fewer than kTile
// links.  One 32-bit word holds d << 16 | s | p, where s is a settled bit
// set once p is a local tail; adding two words whose first has its low half
// cleared adds the counts and takes the second's pointer.
//
// With weights, the link counts place every element of a local sublist in
// list order: the sublists get consecutive ranges of positions (a scan over
// their heads, whose link count is the sublist's length less one), an
// element sits at its tail's position less its link count, and one prefix
// sum of the weights in position order gives every weighted distance as a
// difference of two sums.  A tile with an int64 weight beyond the int32
// range instead doubles separate 64-bit distances, single-buffered (two
// barriers a round).
//
// Predecessor marks are plain byte stores (one per local link), turned into
// the has-local-predecessor bitmap afterwards; fewer marked elements than
// local links means an element with two local predecessors.
struct LcMarks {
  uint8_t mark[kTile];       // 1: the element has a local predecessor
  uint32_t pred[kTileWords]; // has-local-predecessor bitmap
  uint32_t tail[kTileWords]; // local-tail bitmap (wide int64 tiles only)
  uint32_t nlinks, nmarked;  // local links; marked elements
  uint32_t wflags;           // over the tile's local links: kWBig19 | kWNeg | kWBig20
};
// A tile whose local-link weights all lie in (-2^19, 2^19), or all in
// [0, 2^20), has every distance (at most kTile - 1 links) within 32 bits,
// signed or unsigned: its prefix sums are taken modulo 2^32.
constexpr uint32_t kWBig19 = 1u, kWNeg = 2u, kWBig20 = 4u;
struct LcPos {
  union {
    uint32_t pk[2][kTile];   // the doubling's words, double-buffered
    uint64_t P[kTile];       // then the weights by list position, and their prefix sums
    uint32_t P32[kTile];     // the same modulo 2^32 (a narrow tile)
  };
  int32_t w[kTile];          // each element's link weight (0 for a local tail)
  uint16_t E[kTile];         // list position of each local tail
};
// The word arrays come first: they are read and written as 16-byte vectors.
template <int WT>
struct LcTile {
  alignas(16) LcPos q;
  LcMarks m;
};
template <>
struct LcTile<0> {
  alignas(16) uint32_t pk[2][kTile];   // unweighted: the doubling's words only
  LcMarks m;
};
template <>
struct LcTile<2> {
  union alignas(16) {
    LcPos q;                 // every weight of the tile fits in int32
    struct {
      uint64_t d[kTile];     // otherwise: distances
      uint16_t p[kTile];     // and pointers
    } w;
  };
  LcMarks m;
};
static_assert(offsetof(LcTile<0>, m) % 16 == 0 && offsetof(LcTile<1>, m) % 16 == 0 &&
                  offsetof(LcTile<2>, m) % 16 == 0 && offsetof(LcMarks, mark) == 0 &&
                  offsetof(LcPos, w) % 16 == 0 && offsetof(LcPos, E) % 16 == 0,
              "vector accesses to the tile arrays and the marks stay aligned");

template <int WT>
__device__ __forceinline__ uint32_t *lc_words(LcTile<WT> &S, int b) {
  if constexpr (WT == 0) return S.pk[b];
  else return S.q.pk[b];
}

// Elements a thread owns: two runs of four consecutive ids, 4*tid and
// kTile/2 + 4*tid, so that every run is one vector load or store.
constexpr uint32_t kLcRuns = kTile / (4 * kLcThreads);
static_assert(kLcRuns * 4 * kLcThreads == kTile, "a tile is kLcRuns runs of four per thread");
constexpr uint32_t kLcRunStride = kTile / kLcRuns;
// Low half of a packed word: the pointer, and a bit set once the pointer is
// a local tail (the pointer's own word has it then).
constexpr uint32_t kLcPtrMask = kTile - 1u;
constexpr uint32_t kLcSettled = 0x8000u;
static_assert(kTile <= kLcSettled, "pointers stay below the settled bit");
// Weighted: the prefix sums are taken by each thread over 8 consecutive
// positions, then across the threads.
static_assert(kLcThreads * 8 == kTile, "one thread per 8 positions");

// Load tile `t` (len elements) and give every element its local tail p and
// distance d to it (in the rank's arithmetic, modulo 2^64); p = kEnd16 for
// an element on, or leading into, a cycle inside the tile.  Two local links
// into one element and successors out of range are reported.  pred[] holds
// the tile's has-local-predecessor bitmap afterwards.
template <int WT>
__device__ void lc_tile_solve(LcTile<WT> &S, uint32_t t, uint32_t len, const uint32_t *succ,
                              const void *weight, uint32_t n, bool vec, uint32_t (&p)[kLcRuns][4],
                              uint64_t (&d)[kLcRuns][4], uint32_t &bad) {
  __shared__ uint64_t scan_sm[33];
  const uint32_t base = t << kTileShift;
  const uint32_t tid = threadIdx.x;
  uint32_t x[kLcRuns][4];      // d << 16 | settled | p
  uint32_t links = 0;
  uint32_t wfl = 0;            // weighted: this thread's kWBig19 | kWNeg | kWBig20
  // int64 weights: does any weight of the tile leave the int32 range?
  bool wide = false;
  if constexpr (WT == 2) {
    int any = 0;
#pragma unroll
    for (uint32_t r = 0; r < kLcRuns; ++r)
#pragma unroll
      for (uint32_t e = 0; e < 4; ++e) {
        const uint32_t j = r * kLcRunStride + 4 * tid + e;
        if (j < len) {
          const uint64_t v = lc_weight<2>(weight, base + j);
          any |= ((v + 0x80000000ull) >> 32) != 0;
        }
      }
    wide = __syncthreads_or(any) != 0;
  }
  // load: pointer = local successor, or the element itself when its link
  // leaves the tile (a local tail, distance 0); mark local predecessors
#pragma unroll
  for (uint32_t r = 0; r < kLcRuns; ++r) {
    const uint32_t j0 = r * kLcRunStride + 4 * tid;
    uint32_t s[4];
    uint64_t w[4] = {1, 1, 1, 1};
    if (vec && j0 + 4 <= len) {
      const uint4 sv = __ldcs(reinterpret_cast<const uint4 *>(succ + base + j0));
      s[0] = sv.x; s[1] = sv.y; s[2] = sv.z; s[3] = sv.w;
      if constexpr (WT == 1) {
        const int4 q = __ldcs(reinterpret_cast<const int4 *>(reinterpret_cast<const int *>(weight) + base + j0));
        w[0] = (uint64_t)(int64_t)q.x; w[1] = (uint64_t)(int64_t)q.y;
        w[2] = (uint64_t)(int64_t)q.z; w[3] = (uint64_t)(int64_t)q.w;
      } else if constexpr (WT == 2) {
        const longlong2 *wp = reinterpret_cast<const longlong2 *>(reinterpret_cast<const long long *>(weight) + base + j0);
        const longlong2 q0 = __ldcs(wp), q1 = __ldcs(wp + 1);
        w[0] = (uint64_t)q0.x; w[1] = (uint64_t)q0.y; w[2] = (uint64_t)q1.x; w[3] = (uint64_t)q1.y;
      }
    } else {
#pragma unroll
      for (uint32_t e = 0; e < 4; ++e) {
        const uint32_t j = j0 + e;
        s[e] = j < len ? __ldcs(succ + base + j) : base + j;     // beyond the tile: a lone tail
        if constexpr (WT != 0) w[e] = j < len ? lc_weight<WT>(weight, base + j) : 0u;
      }
    }
    uint32_t tails = 0;
#pragma unroll
    for (uint32_t e = 0; e < 4; ++e) {
      const uint32_t j = j0 + e, i = base + j;
      if (j < len && s[e] >= n) bad |= kErrRange;
      const bool local = j < len && s[e] < n && s[e] != i && (s[e] >> kTileShift) == t;
      p[r][e] = local ? s[e] - base : j;
      x[r][e] = (local ? 1u << 16 : kLcSettled) | p[r][e];
      if constexpr (WT != 0) {
        d[r][e] = local ? w[e] : 0u;   // exact in int32 unless the tile is wide
        const int64_t wv = (int64_t)d[r][e];
        wfl |= ((uint64_t)(wv + (1 << 19)) >= (1u << 20) ? kWBig19 : 0u) | (wv < 0 ? kWNeg : 0u) |
               ((uint64_t)wv >= (1u << 20) ? kWBig20 : 0u);
      }
      if (local) {
        S.m.mark[s[e] - base] = 1;
        ++links;
      } else {
        tails |= 1u << e;
      }
    }
    if (!wide) {
      *reinterpret_cast<uint4 *>(&lc_words(S, 0)[j0]) = make_uint4(x[r][0], x[r][1], x[r][2], x[r][3]);
      if constexpr (WT != 0)
        *reinterpret_cast<int4 *>(&S.q.w[j0]) =
            make_int4((int32_t)d[r][0], (int32_t)d[r][1], (int32_t)d[r][2], (int32_t)d[r][3]);
    } else if constexpr (WT == 2) {
      atomicOr(&S.m.tail[j0 >> 5], tails << (j0 & 31u));
      *reinterpret_cast<uint2 *>(&S.w.p[j0]) = make_uint2(p[r][0] | p[r][1] << 16, p[r][2] | p[r][3] << 16);
      *reinterpret_cast<ulonglong2 *>(&S.w.d[j0]) = make_ulonglong2(d[r][0], d[r][1]);
      *reinterpret_cast<ulonglong2 *>(&S.w.d[j0 + 2]) = make_ulonglong2(d[r][2], d[r][3]);
    }
  }
  links = __reduce_add_sync(0xFFFFFFFFu, links);
  if ((tid & 31u) == 0 && links) atomicAdd(&S.m.nlinks, links);
  if constexpr (WT != 0) {
    wfl = __reduce_or_sync(0xFFFFFFFFu, wfl);
    if ((tid & 31u) == 0 && wfl) atomicOr(&S.m.wflags, wfl);
  }
  __syncthreads();
  // marks -> bitmap: eight marks per thread, four threads per word; the
  // marks are cleared for the next tile as they are read
  {
    const uint2 mk = *reinterpret_cast<const uint2 *>(&S.m.mark[8 * tid]);
    *reinterpret_cast<uint2 *>(&S.m.mark[8 * tid]) = make_uint2(0u, 0u);
    // bytes are 0 or 1: the product gathers four of them into one nibble
    uint32_t v = (((mk.x * 0x01020408u) >> 24) | (((mk.y * 0x01020408u) >> 24) << 4)) << (8 * (tid & 3u));
    v |= __shfl_xor_sync(0xFFFFFFFFu, v, 1);
    v |= __shfl_xor_sync(0xFFFFFFFFu, v, 2);
    uint32_t c = (tid & 3u) == 0 ? (uint32_t)__popc(v) : 0u;
    if ((tid & 3u) == 0) S.m.pred[tid >> 2] = v;
    c = __reduce_add_sync(0xFFFFFFFFu, c);
    if ((tid & 31u) == 0 && c) atomicAdd(&S.m.nmarked, c);
  }
  if (!wide) {
    // Pointer doubling on the packed words.  A word whose pointer has
    // reached a local tail is final: it is not gathered again, and the
    // rounds end when every word is final (a valid tile needs at most
    // kTileShift rounds; a cycle never settles).
    int b = 0;
    for (int round = 0; round <= kTileShift; ++round) {
      uint32_t all = kLcSettled;
      const uint32_t *cur = lc_words(S, b);
      uint32_t *nxt = lc_words(S, b ^ 1);
#pragma unroll
      for (uint32_t r = 0; r < kLcRuns; ++r) {
#pragma unroll
        for (uint32_t e = 0; e < 4; ++e) {
          if (!(x[r][e] & kLcSettled)) {
            const uint32_t v = cur[x[r][e] & kLcPtrMask];
            x[r][e] = (x[r][e] & 0xFFFF0000u) + v;
          }
          all &= x[r][e];
        }
        *reinterpret_cast<uint4 *>(&nxt[r * kLcRunStride + 4 * tid]) =
            make_uint4(x[r][0], x[r][1], x[r][2], x[r][3]);
      }
      b ^= 1;
      if (__syncthreads_and(all & kLcSettled)) break;
    }
    // unpack; a word that never settled is on, or leads into, a cycle (also
    // one whose length is a power of two: its pointer comes back to itself)
#pragma unroll
    for (uint32_t r = 0; r < kLcRuns; ++r)
#pragma unroll
      for (uint32_t e = 0; e < 4; ++e) {
        p[r][e] = (x[r][e] & kLcSettled) ? (x[r][e] & kLcPtrMask) : kEnd16;
        if constexpr (WT == 0) d[r][e] = x[r][e] >> 16;
      }
    if constexpr (WT != 0) {
      // positions: every settled local head opens a range of its sublist's
      // length; its tail gets the range's last position
      uint32_t cnt = 0;
#pragma unroll
      for (uint32_t r = 0; r < kLcRuns; ++r)
#pragma unroll
        for (uint32_t e = 0; e < 4; ++e) {
          const uint32_t j = r * kLcRunStride + 4 * tid + e;
          const bool head = j < len && p[r][e] != kEnd16 && !((S.m.pred[j >> 5] >> (j & 31u)) & 1u);
          if (head) cnt += (x[r][e] >> 16) + 1u;
        }
      uint64_t total;
      uint32_t at = (uint32_t)block_exclusive_scan((uint64_t)cnt, scan_sm, &total);
      // more positions than elements: merged sublists (two predecessors,
      // reported by the marks); no weighted distances for this tile
      const bool fits = total <= kTile;
      if (fits) {
#pragma unroll
        for (uint32_t r = 0; r < kLcRuns; ++r)
#pragma unroll
          for (uint32_t e = 0; e < 4; ++e) {
            const uint32_t j = r * kLcRunStride + 4 * tid + e;
            const bool head = j < len && p[r][e] != kEnd16 && !((S.m.pred[j >> 5] >> (j & 31u)) & 1u);
            if (head) {
              at += (x[r][e] >> 16) + 1u;
              S.q.E[p[r][e]] = (uint16_t)(at - 1u);
            }
          }
      }
      __syncthreads();                       // E is written; the doubling's buffers are free
      const uint32_t wf = S.m.wflags;
      const bool nsig = !(wf & kWBig19), nuns = !(wf & (kWNeg | kWBig20));
      const bool narrow = nsig || nuns;
      if (fits) {
        // weights by position (a tail's own link does not count); ids past
        // the end of the last tile are lone tails of no sublist
#pragma unroll
        for (uint32_t r = 0; r < kLcRuns; ++r)
#pragma unroll
          for (uint32_t e = 0; e < 4; ++e) {
            const uint32_t j = r * kLcRunStride + 4 * tid + e;
            if (j < len && p[r][e] != kEnd16) {
              const uint32_t pos = ((uint32_t)S.q.E[p[r][e]] - (x[r][e] >> 16)) & kLcPtrMask;
              if (narrow) S.q.P32[pos] = (uint32_t)S.q.w[j];
              else S.q.P[pos] = (uint64_t)(int64_t)S.q.w[j];
            }
          }
      }
      __syncthreads();
      if (fits && narrow) {
        // inclusive prefix sums modulo 2^32 over the positions, 8 per thread
        uint32_t v[8];
        const uint4 *src = reinterpret_cast<const uint4 *>(&S.q.P32[8 * tid]);
        const uint4 u0 = src[0], u1 = src[1];
        v[0] = u0.x; v[1] = u0.y; v[2] = u0.z; v[3] = u0.w;
        v[4] = u1.x; v[5] = u1.y; v[6] = u1.z; v[7] = u1.w;
#pragma unroll
        for (int q = 1; q < 8; ++q) v[q] += v[q - 1];
        const uint32_t off = (uint32_t)block_exclusive_scan((uint64_t)v[7], scan_sm, nullptr);
        uint4 *dst = reinterpret_cast<uint4 *>(&S.q.P32[8 * tid]);
        dst[0] = make_uint4(v[0] + off, v[1] + off, v[2] + off, v[3] + off);
        dst[1] = make_uint4(v[4] + off, v[5] + off, v[6] + off, v[7] + off);
      } else if (fits) {
        // inclusive prefix sums over the positions, 8 per thread
        uint64_t v[8];
        const ulonglong2 *src = reinterpret_cast<const ulonglong2 *>(&S.q.P[8 * tid]);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const ulonglong2 u = src[q];
          v[2 * q] = u.x;
          v[2 * q + 1] = u.y;
        }
#pragma unroll
        for (int q = 1; q < 8; ++q) v[q] += v[q - 1];
        const uint64_t off = block_exclusive_scan(v[7], scan_sm, nullptr);
        ulonglong2 *dst = reinterpret_cast<ulonglong2 *>(&S.q.P[8 * tid]);
#pragma unroll
        for (int q = 0; q < 4; ++q) dst[q] = make_ulonglong2(v[2 * q] + off, v[2 * q + 1] + off);
      } else if (tid == 0) {
        bad |= kErrNotList;
      }
      __syncthreads();
      // distance = sum of the weights from the element's position to its tail's
#pragma unroll
      for (uint32_t r = 0; r < kLcRuns; ++r)
#pragma unroll
        for (uint32_t e = 0; e < 4; ++e) {
          d[r][e] = 0;
          if (fits && p[r][e] != kEnd16 && r * kLcRunStride + 4 * tid + e < len) {
            const uint32_t last = S.q.E[p[r][e]] & kLcPtrMask;
            const uint32_t pos = (last - (x[r][e] >> 16)) & kLcPtrMask;
            if (narrow) {
              const uint32_t d32 = S.q.P32[last] - (pos ? S.q.P32[pos - 1] : 0u);
              d[r][e] = nsig ? (uint64_t)(int64_t)(int32_t)d32 : (uint64_t)d32;
            } else {
              d[r][e] = S.q.P[last] - (pos ? S.q.P[pos - 1] : 0u);
            }
          }
        }
    }
  } else if constexpr (WT == 2) {
    // wide int64 weights: read every element's target, wait, write back
    for (int round = 0; round <= kTileShift; ++round) {
      uint32_t diff = 0;
#pragma unroll
      for (uint32_t r = 0; r < kLcRuns; ++r)
#pragma unroll
        for (uint32_t e = 0; e < 4; ++e) {
          const uint32_t q = S.w.p[p[r][e]];
          diff |= q ^ p[r][e];
          d[r][e] += S.w.d[p[r][e]];
          p[r][e] = q;
        }
      __syncthreads();
#pragma unroll
      for (uint32_t r = 0; r < kLcRuns; ++r) {
        const uint32_t j0 = r * kLcRunStride + 4 * tid;
        *reinterpret_cast<uint2 *>(&S.w.p[j0]) = make_uint2(p[r][0] | p[r][1] << 16, p[r][2] | p[r][3] << 16);
        *reinterpret_cast<ulonglong2 *>(&S.w.d[j0]) = make_ulonglong2(d[r][0], d[r][1]);
        *reinterpret_cast<ulonglong2 *>(&S.w.d[j0 + 2]) = make_ulonglong2(d[r][2], d[r][3]);
      }
      if (!__syncthreads_or(diff != 0)) break;
    }
    // a pointer that did not settle on a local tail marks a cycle
#pragma unroll
    for (uint32_t r = 0; r < kLcRuns; ++r)
#pragma unroll
      for (uint32_t e = 0; e < 4; ++e)
        if (!((S.m.tail[p[r][e] >> 5] >> (p[r][e] & 31u)) & 1u)) p[r][e] = kEnd16;
  }
}
}  // namespace

// Exclusive prefix of the tile counts (one CTA); tpre[ntiles] = total.
__global__ void __launch_bounds__(1024)
k_lc_scan(const uint32_t *__restrict__ tcnt, uint32_t ntiles, uint32_t *__restrict__ tpre) {
  __shared__ uint64_t sm[33];
  const uint32_t per = (ntiles + blockDim.x - 1) / blockDim.x;
  const uint32_t a = threadIdx.x * per, b = min(ntiles, a + per);
  uint64_t s = 0;
  for (uint32_t t = a; t < b; ++t) s += tcnt[t];
  uint64_t total;
  uint64_t run = block_exclusive_scan(s, sm, &total);
  for (uint32_t t = a; t < b; ++t) { tpre[t] = (uint32_t)run; run += tcnt[t]; }
  if (threadIdx.x == 0) tpre[ntiles] = (uint32_t)total;
}

// Solve pass: per tile, every element's distance to its local tail goes to
// rank[] (in the rank type) and its tail (local index) to tail16[]; the
// local-head bitmap, the head counts before each word of the tile and the
// heads per tile go to hb, wpre and tcnt.  vec: bit 0 = succ and weight
// 16-byte aligned, bit 1 = rank 16-byte and tail16 8-byte aligned.
template <int WT, class RT>
__global__ void __launch_bounds__(kLcThreads, WT == 2 ? 2 : 3)
k_lc_solve(const uint32_t *__restrict__ succ, const void *__restrict__ weight, uint32_t n,
           RT *__restrict__ rank, uint16_t *__restrict__ tail16, uint32_t *__restrict__ hb,
           uint16_t *__restrict__ wpre, uint32_t *__restrict__ tcnt, uint32_t *__restrict__ err, int vec) {
  extern __shared__ __align__(16) unsigned char lc_smem[];
  LcTile<WT> &S = *reinterpret_cast<LcTile<WT> *>(lc_smem);
  const uint32_t ntiles = (n + kTile - 1) >> kTileShift;
  for (uint32_t j = threadIdx.x; j < kTile / 4; j += blockDim.x) reinterpret_cast<uint32_t *>(S.m.mark)[j] = 0;
  for (uint32_t w = threadIdx.x; w < kTileWords; w += blockDim.x) S.m.tail[w] = 0;
  if (threadIdx.x == 0) { S.m.nlinks = 0; S.m.nmarked = 0; S.m.wflags = 0; }
  __syncthreads();
  for (uint32_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const uint32_t base = t << kTileShift;
    const uint32_t len = min(kTile, n - base);
    uint32_t p[kLcRuns][4];
    uint64_t d[kLcRuns][4];
    uint32_t bad = 0;
    lc_tile_solve<WT>(S, t, len, succ, weight, n, (vec & 1) != 0, p, d, bad);
    bool cyc = false;
#pragma unroll
    for (uint32_t r = 0; r < kLcRuns; ++r) {
      const uint32_t j0 = r * kLcRunStride + 4 * threadIdx.x;
      if (j0 >= len) continue;
      RT o[4];
#pragma unroll
      for (uint32_t e = 0; e < 4; ++e) {
        if (j0 + e < len && p[r][e] == kEnd16) cyc = true;
        o[e] = p[r][e] == kEnd16 ? (RT)0 : (RT)d[r][e];
      }
      if ((vec & 2) && j0 + 4 <= len) {
        if constexpr (sizeof(RT) == 4) {
          __stcs(reinterpret_cast<uint4 *>(rank + base + j0), make_uint4(o[0], o[1], o[2], o[3]));
        } else {
          __stcs(reinterpret_cast<ulonglong2 *>(rank + base + j0), make_ulonglong2(o[0], o[1]));
          __stcs(reinterpret_cast<ulonglong2 *>(rank + base + j0 + 2), make_ulonglong2(o[2], o[3]));
        }
        __stcs(reinterpret_cast<uint2 *>(tail16 + base + j0),
               make_uint2(p[r][0] | p[r][1] << 16, p[r][2] | p[r][3] << 16));
      } else {
#pragma unroll
        for (uint32_t e = 0; e < 4; ++e) {
          if (j0 + e >= len) break;
          __stcs(rank + base + j0 + e, o[e]);
          __stcs(tail16 + base + j0 + e, (uint16_t)p[r][e]);
        }
      }
    }
    if (cyc) bad |= kErrCycle;
    if (threadIdx.x == 0 && S.m.nmarked < S.m.nlinks) bad |= kErrNotList;   // two local links into one element
    if (bad) record_error(err, bad);
    if (threadIdx.x < 32) {
      // 4 words per lane; exclusive prefix of the head counts over the tile
      uint32_t h[4], c = 0;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const uint32_t w = threadIdx.x * 4 + q;
        const uint32_t lo = w * 32;
        const uint32_t valid = lo >= len ? 0u : (len - lo >= 32 ? 0xFFFFFFFFu : ((1u << (len - lo)) - 1u));
        h[q] = ~S.m.pred[w] & valid;
        c += __popc(h[q]);
      }
      uint32_t incl = c;
      for (int dd = 1; dd < 32; dd <<= 1) {
        const uint32_t v = __shfl_up_sync(0xFFFFFFFFu, incl, dd);
        if ((int)threadIdx.x >= dd) incl += v;
      }
      uint32_t run = incl - c;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const uint32_t w = threadIdx.x * 4 + q;
        hb[t * kTileWords + w] = h[q];
        wpre[t * kTileWords + w] = (uint16_t)run;
        run += __popc(h[q]);
      }
      if (threadIdx.x == 31) tcnt[t] = incl;
    }
    __syncthreads();
    if constexpr (WT == 2)
      for (uint32_t w = threadIdx.x; w < kTileWords; w += blockDim.x) S.m.tail[w] = 0;
    if (threadIdx.x == 0) { S.m.nlinks = 0; S.m.nmarked = 0; S.m.wflags = 0; }
    __syncthreads();
  }
}

// Nodes pass: one contracted node per local head h, with successor the node
// its tail t enters and weight dist(h -> t) + w(t); a list's last node is a
// contracted terminal weighing dist(h -> t).
template <int WT, class RT>
__global__ void __launch_bounds__(256)
k_lc_nodes(const uint32_t *__restrict__ succ, const void *__restrict__ weight, uint32_t n,
           const RT *__restrict__ rank, const uint16_t *__restrict__ tail16,
           const uint32_t *__restrict__ hb, const uint16_t *__restrict__ wpre,
           const uint32_t *__restrict__ tpre, uint32_t *__restrict__ succ_c, void *__restrict__ w_c,
           uint32_t *__restrict__ err) {
  const uint32_t words = (uint32_t)(((uint64_t)n + 31) / 32);
  uint32_t bad = 0;
  for (uint32_t w = blockIdx.x * blockDim.x + threadIdx.x; w < words; w += gridDim.x * blockDim.x) {
    uint32_t bits = __ldg(hb + w);
    if (!bits) continue;
    const uint32_t first = __ldg(tpre + ((w * 32) >> kTileShift)) + __ldg(wpre + w);
    uint32_t rankin = 0;
    while (bits) {
      const uint32_t b = __ffs(bits) - 1;
      bits &= bits - 1u;
      const uint32_t h = w * 32 + b, id = first + rankin++;
      const uint16_t tl = __ldg(tail16 + h);
      if (tl == kEnd16) continue;                          // leads into a cycle: reported
      const uint32_t ti = (h & ~(kTile - 1u)) + tl, z = __ldg(succ + ti);
      uint64_t wc = (uint64_t)(RT)__ldg(rank + h);
      uint32_t sc = id;                                    // a contracted terminal
      if (z < n && z != ti) {
        if (!lc_is_head(z, hb)) bad |= kErrNotList;        // entered a sublist in its middle
        else sc = lc_node(z, hb, wpre, tpre);
        wc += lc_weight<WT>(weight, ti);
      }
      succ_c[id] = sc;
      if constexpr (WT == 0) reinterpret_cast<int *>(w_c)[id] = (int)wc;
      else reinterpret_cast<long long *>(w_c)[id] = (long long)(RT)wc;
    }
  }
  if (bad) record_error(err, bad);
}

// Tails pass: the tail t of every head's sublist gets its contribution, its
// own link plus the contracted rank after it (0 for a list's terminal): its
// distance to itself is 0, so rank[t] is final.
template <int WT, class RT>
__global__ void __launch_bounds__(256)
k_lc_tails(const uint32_t *__restrict__ succ, const void *__restrict__ weight, uint32_t n,
           RT *__restrict__ rank, const uint16_t *__restrict__ tail16, const uint32_t *__restrict__ hb,
           const uint16_t *__restrict__ wpre, const uint32_t *__restrict__ tpre,
           const RT *__restrict__ rc) {
  const uint32_t words = (uint32_t)(((uint64_t)n + 31) / 32);
  for (uint32_t w = blockIdx.x * blockDim.x + threadIdx.x; w < words; w += gridDim.x * blockDim.x) {
    uint32_t bits = __ldg(hb + w);
    while (bits) {
      const uint32_t b = __ffs(bits) - 1;
      bits &= bits - 1u;
      const uint32_t h = w * 32 + b;
      const uint16_t tl = __ldg(tail16 + h);
      if (tl == kEnd16) continue;
      const uint32_t ti = (h & ~(kTile - 1u)) + tl, z = __ldg(succ + ti);
      RT c = 0;
      if (z < n && z != ti && lc_is_head(z, hb))
        c = (RT)(__ldcg(rc + lc_node(z, hb, wpre, tpre)) + (RT)lc_weight<WT>(weight, ti));
      rank[ti] = c;
    }
  }
}

// Fix pass: rank[i] = dist(i -> t) + rank[t] for every element that is not
// a tail (tails already hold their final rank).  Four elements per thread
// (a group never straddles a tile: tiles are multiples of 4).
template <class RT>
__device__ __forceinline__ RT lc_fix1(uint32_t i, uint16_t tl, RT r, const RT *rank) {
  if (tl == kEnd16) return r;
  const uint32_t ti = (i & ~(kTile - 1u)) + tl;
  return ti == i ? r : (RT)(r + __ldcg(rank + ti));
}

template <class RT>
__global__ void __launch_bounds__(256)
k_lc_fix(uint32_t n, RT *__restrict__ rank, const uint16_t *__restrict__ tail16, int vec) {
  const uint32_t groups = (n + 3) / 4;
  for (uint32_t g = blockIdx.x * blockDim.x + threadIdx.x; g < groups; g += gridDim.x * blockDim.x) {
    const uint32_t i = g * 4;
    if (vec && i + 4 <= n) {
      const uint2 tv = __ldcs(reinterpret_cast<const uint2 *>(tail16 + i));
      const uint16_t t0 = (uint16_t)tv.x, t1 = (uint16_t)(tv.x >> 16), t2 = (uint16_t)tv.y, t3 = (uint16_t)(tv.y >> 16);
      if constexpr (sizeof(RT) == 4) {
        uint4 r = __ldcs(reinterpret_cast<const uint4 *>(rank + i));
        r.x = lc_fix1<RT>(i, t0, r.x, rank); r.y = lc_fix1<RT>(i + 1, t1, r.y, rank);
        r.z = lc_fix1<RT>(i + 2, t2, r.z, rank); r.w = lc_fix1<RT>(i + 3, t3, r.w, rank);
        __stcs(reinterpret_cast<uint4 *>(rank + i), r);
      } else {
        ulonglong2 a = __ldcs(reinterpret_cast<const ulonglong2 *>(rank + i));
        ulonglong2 b = __ldcs(reinterpret_cast<const ulonglong2 *>(rank + i + 2));
        a.x = lc_fix1<RT>(i, t0, a.x, rank); a.y = lc_fix1<RT>(i + 1, t1, a.y, rank);
        b.x = lc_fix1<RT>(i + 2, t2, b.x, rank); b.y = lc_fix1<RT>(i + 3, t3, b.y, rank);
        __stcs(reinterpret_cast<ulonglong2 *>(rank + i), a);
        __stcs(reinterpret_cast<ulonglong2 *>(rank + i + 2), b);
      }
    } else {
      for (uint32_t q = i; q < min(n, i + 4); ++q) rank[q] = lc_fix1<RT>(q, tail16[q], rank[q], rank);
    }
  }
}

static size_t lc_smem_bytes(int wtype) {
  return wtype == 0 ? sizeof(LcTile<0>) : (wtype == 1 ? sizeof(LcTile<1>) : sizeof(LcTile<2>));
}

uint32_t lc_tiles(uint64_t n) { return (uint32_t)((n + kTile - 1) >> kTileShift); }
uint32_t lc_tile_words() { return kTileWords; }

cudaError_t lc_setup() {
  cudaError_t e = cudaSuccess;
#define LC_ATTR(K, BYTES) \
  if (e == cudaSuccess) e = cudaFuncSetAttribute(K, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(BYTES))
  LC_ATTR((k_lc_solve<0, uint32_t>), sizeof(LcTile<0>));
  LC_ATTR((k_lc_solve<0, unsigned long long>), sizeof(LcTile<0>));
  LC_ATTR((k_lc_solve<1, uint32_t>), sizeof(LcTile<1>));
  LC_ATTR((k_lc_solve<1, unsigned long long>), sizeof(LcTile<1>));
  LC_ATTR((k_lc_solve<2, uint32_t>), sizeof(LcTile<2>));
  LC_ATTR((k_lc_solve<2, unsigned long long>), sizeof(LcTile<2>));
#undef LC_ATTR
  return e;
}

cudaError_t launch_lc_solve(const uint32_t *succ, const void *weight, int wtype, uint32_t n, void *rank,
                            int rank_bytes, uint16_t *tail16, uint32_t *hb, uint16_t *wpre, uint32_t *tcnt,
                            uint32_t *tpre, uint32_t *err, cudaStream_t s) {
  const uint32_t nt = lc_tiles(n);
  const size_t sm = lc_smem_bytes(wtype);
  const int per_sm = wtype == 2 ? 2 : 3;
  const int grid = (int)std::min<uint32_t>(nt, (uint32_t)device_sm_count() * per_sm);
  const int vec = (((uintptr_t)succ & 15u) == 0 && ((uintptr_t)weight & 15u) == 0 ? 1 : 0) |
                  (((uintptr_t)rank & 15u) == 0 && ((uintptr_t)tail16 & 7u) == 0 ? 2 : 0);
#define LC_SOLVE(W, R)                                                                             \
  k_lc_solve<W, R><<<grid, kLcThreads, sm, s>>>(succ, weight, n, reinterpret_cast<R *>(rank), tail16, \
                                                hb, wpre, tcnt, err, vec)
  if (wtype == 0) { if (rank_bytes == 4) LC_SOLVE(0, uint32_t); else LC_SOLVE(0, unsigned long long); }
  else if (wtype == 1) { if (rank_bytes == 4) LC_SOLVE(1, uint32_t); else LC_SOLVE(1, unsigned long long); }
  else { if (rank_bytes == 4) LC_SOLVE(2, uint32_t); else LC_SOLVE(2, unsigned long long); }
#undef LC_SOLVE
  k_lc_scan<<<1, 1024, 0, s>>>(tcnt, nt, tpre);
  count_launch(2);
  return cudaGetLastError();
}

cudaError_t launch_lc_nodes(const uint32_t *succ, const void *weight, int wtype, uint32_t n, const void *rank,
                            int rank_bytes, const uint16_t *tail16, const uint32_t *hb, const uint16_t *wpre,
                            const uint32_t *tpre, uint32_t *succ_c, void *w_c, uint32_t *err, cudaStream_t s) {
  const int grid = stream_grid(((uint64_t)n + 31) / 32, 256);
#define LC_NODES(W, R)                                                                             \
  k_lc_nodes<W, R><<<grid, 256, 0, s>>>(succ, weight, n, reinterpret_cast<const R *>(rank), tail16, hb, \
                                        wpre, tpre, succ_c, w_c, err)
  if (wtype == 0) { if (rank_bytes == 4) LC_NODES(0, uint32_t); else LC_NODES(0, unsigned long long); }
  else if (wtype == 1) { if (rank_bytes == 4) LC_NODES(1, uint32_t); else LC_NODES(1, unsigned long long); }
  else { if (rank_bytes == 4) LC_NODES(2, uint32_t); else LC_NODES(2, unsigned long long); }
#undef LC_NODES
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_lc_finish(const uint32_t *succ, const void *weight, int wtype, uint32_t n, void *rank,
                             int rank_bytes, const uint16_t *tail16, const uint32_t *hb, const uint16_t *wpre,
                             const uint32_t *tpre, const void *rc, cudaStream_t s) {
  const int gw = stream_grid(((uint64_t)n + 31) / 32, 256);
  const int ge = stream_grid(((uint64_t)n + 3) / 4, 256);
#define LC_TAILS(W, R)                                                                             \
  k_lc_tails<W, R><<<gw, 256, 0, s>>>(succ, weight, n, reinterpret_cast<R *>(rank), tail16, hb, wpre, tpre, \
                                      reinterpret_cast<const R *>(rc))
  if (wtype == 0) { if (rank_bytes == 4) LC_TAILS(0, uint32_t); else LC_TAILS(0, unsigned long long); }
  else if (wtype == 1) { if (rank_bytes == 4) LC_TAILS(1, uint32_t); else LC_TAILS(1, unsigned long long); }
  else { if (rank_bytes == 4) LC_TAILS(2, uint32_t); else LC_TAILS(2, unsigned long long); }
#undef LC_TAILS
  const int vec = ((uintptr_t)rank & 15u) == 0 && ((uintptr_t)tail16 & 7u) == 0;
  if (rank_bytes == 4) k_lc_fix<uint32_t><<<ge, 256, 0, s>>>(n, reinterpret_cast<uint32_t *>(rank), tail16, vec);
  else k_lc_fix<unsigned long long><<<ge, 256, 0, s>>>(n, reinterpret_cast<unsigned long long *>(rank), tail16, vec);
  count_launch(2);
  return cudaGetLastError();
}

}  // namespace lr
