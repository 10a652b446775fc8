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
// Inside a tile, dist and t come from short bounded walks between
// sub-rulers in shared memory (every element once) and pointer doubling
// over the few sub-rulers: O(tile) work, unlike pointer doubling over the
// whole tile's O(tile log tile).
//
// Passes: solve (every tile in shared memory: distances to the local tails,
// the local-head bitmap), scan (tile prefixes), nodes (the contracted
// list), the ruling set on the contracted list, tails and fix (the ranks).
// Whether to contract is decided by the caller from the prep pass's count
// of links that stay inside their tile.
#include <algorithm>
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

constexpr uint32_t kSubDefault = 8;    // every ksub-th local id is a sub-ruler (dense tiles)
constexpr uint32_t kMaxSr = 2 * kLcThreads;   // sub-rulers ranked by pointer doubling

// Shared-memory state of one tile.
template <class VT>
struct LcTile {
  uint32_t raw[kTile];       // succ of each element of the tile
  uint16_t nxt[kTile];       // local successor or kEnd16; then per sub-ruler: next sub-ruler
  uint16_t sub[kTile];       // predecessor marks; then the element's sub-ruler; per sub-ruler:
                             // its local tail once known (kEnd16 between tiles)
  VT off[kTile];             // link weight; then offset from the sub-ruler; per sub-ruler: distance
  uint32_t pred[kTileWords]; // has-local-predecessor bitmap
  uint16_t srl[kMaxSr];      // dense tiles: heads whose id is not a multiple of ksub
  uint32_t nheads, nlinks, nextra, dense, submask;
};

template <class VT>
__device__ __forceinline__ bool lc_head(const LcTile<VT> &S, uint32_t j) {
  return !((S.pred[j >> 5] >> (j & 31u)) & 1u);
}

// Sub-rulers: the local heads, and in dense tiles (few heads, long local
// sublists) also every ksub-th id.  A walk never enters a local head, so
// "the next element is a sub-ruler" is an arithmetic test.
template <class VT>
__device__ __forceinline__ bool lc_is_sr(const LcTile<VT> &S, uint32_t j) {
  return lc_head(S, j) || (S.dense && (j & S.submask) == 0);
}

// One element of the load: succ, local link, weight; marks its target.
template <int WT, class VT>
__device__ __forceinline__ void lc_load1(LcTile<VT> &S, uint32_t j, uint32_t s, VT w, uint32_t t,
                                         uint32_t base, uint32_t n, uint32_t &bad, uint32_t &links) {
  const uint32_t i = base + j;
  const bool local = s < n && s != i && (s >> kTileShift) == t;
  if (s >= n) bad |= kErrRange;
  S.nxt[j] = local ? (uint16_t)(s - base) : kEnd16;
  S.off[j] = local ? w : (VT)0;
  if (local) { S.sub[s - base] = (uint16_t)j; ++links; }
}

// Load tile `t` and find for every element its local tail and distance to
// it.  sub[] must hold kEnd16 on entry.
//   Marks: every local link stores its source into sub[target] (plain
//   stores); one ballot per 32 elements turns them into the
//   has-local-predecessor bitmap, and fewer marked targets than local links
//   means an element with two predecessors.
//   Level 1: every sub-ruler walks to the next sub-ruler (or its local
//   tail), recording (sub-ruler, offset) in each element it passes.
//   Level 2 (dense tiles): synchronous pointer doubling over the at most
//   kMaxSr sub-rulers gives each its tail and distance.  In sparse tiles the
//   sub-rulers are the heads alone, whose walks already end at their tails.
// Walks are bounded by the tile length; an element no walk reaches lies on
// a cycle.  Returns the tile length.
template <int WT, class VT>
__device__ uint32_t lc_tile_solve(LcTile<VT> &S, uint32_t t, const uint32_t *succ, const void *weight,
                                  uint32_t n, uint32_t *err, bool vec, uint32_t ksub) {
  const uint32_t base = t << kTileShift;
  const uint32_t len = min(kTile, n - base);
  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t submask = ksub - 1u;
  // the ids of one bitmap word that are multiples of ksub (2 <= ksub <= 32)
  const uint32_t mulbits = ksub >= 32 ? 1u : (0xFFFFFFFFu / ((1u << ksub) - 1u));
  if (threadIdx.x == 0) { S.nheads = 0; S.nlinks = 0; S.nextra = 0; S.submask = submask; }
  uint32_t bad = 0, links = 0;
  // load, four elements per thread and step
  for (uint32_t g = threadIdx.x; g * 4 < len; g += blockDim.x) {
    const uint32_t j = g * 4;
    if (vec && j + 4 <= len) {
      const uint4 sv = __ldcs(reinterpret_cast<const uint4 *>(succ + base + j));
      VT w0 = 1, w1 = 1, w2 = 1, w3 = 1;
      if constexpr (WT == 1) {
        const int4 q = __ldcs(reinterpret_cast<const int4 *>(reinterpret_cast<const int *>(weight) + base + j));
        w0 = (VT)(int64_t)q.x; w1 = (VT)(int64_t)q.y; w2 = (VT)(int64_t)q.z; w3 = (VT)(int64_t)q.w;
      } else if constexpr (WT == 2) {
        const longlong2 *wp = reinterpret_cast<const longlong2 *>(reinterpret_cast<const long long *>(weight) + base + j);
        const longlong2 q0 = __ldcs(wp), q1 = __ldcs(wp + 1);
        w0 = (VT)q0.x; w1 = (VT)q0.y; w2 = (VT)q1.x; w3 = (VT)q1.y;
      }
      *reinterpret_cast<uint4 *>(&S.raw[j]) = sv;
      lc_load1<WT, VT>(S, j + 0, sv.x, w0, t, base, n, bad, links);
      lc_load1<WT, VT>(S, j + 1, sv.y, w1, t, base, n, bad, links);
      lc_load1<WT, VT>(S, j + 2, sv.z, w2, t, base, n, bad, links);
      lc_load1<WT, VT>(S, j + 3, sv.w, w3, t, base, n, bad, links);
    } else {
      for (uint32_t q = j; q < min(len, j + 4); ++q) {
        const uint32_t sq = __ldcs(succ + base + q);
        S.raw[q] = sq;
        lc_load1<WT, VT>(S, q, sq, (VT)lc_weight<WT>(weight, base + q), t, base, n, bad, links);
      }
    }
  }
  links = __reduce_add_sync(0xFFFFFFFFu, links);
  if (lane == 0 && links) atomicAdd(&S.nlinks, links);
  __syncthreads();
  // the has-local-predecessor bitmap; marks are cleared as they are read
  for (uint32_t j0 = 0; j0 < kTile; j0 += blockDim.x) {
    const uint32_t j = j0 + threadIdx.x;
    const bool has = j < len && S.sub[j] != kEnd16;
    S.sub[j] = kEnd16;
    const uint32_t word = __ballot_sync(0xFFFFFFFFu, has);
    if (lane == 0) S.pred[j >> 5] = word;
  }
  __syncthreads();
  // heads per tile; in dense tiles also the heads that are not multiples of ksub
  if (threadIdx.x < 32) {
    uint32_t hw[4], cnt = 0, extra = 0;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const uint32_t w = threadIdx.x * 4 + q, lo = w * 32;
      const uint32_t valid = lo >= len ? 0u : (len - lo >= 32 ? 0xFFFFFFFFu : ((1u << (len - lo)) - 1u));
      hw[q] = ~S.pred[w] & valid;
      cnt += __popc(hw[q]);
      extra += __popc(hw[q] & ~mulbits);              // heads off the ksub grid
    }
    const uint32_t heads = __reduce_add_sync(0xFFFFFFFFu, cnt);
    const uint32_t marked = len - heads;
    if (marked < S.nlinks) bad |= kErrNotList;            // two links into one element
    const bool dense = heads + (len + ksub - 1) / ksub <= kMaxSr;
    if (dense) {
      uint32_t incl = extra;
      for (int d = 1; d < 32; d <<= 1) {
        const uint32_t v = __shfl_up_sync(0xFFFFFFFFu, incl, d);
        if ((int)lane >= d) incl += v;
      }
      uint32_t pos = incl - extra;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        uint32_t bits = hw[q] & ~mulbits;
        while (bits) {
          const uint32_t b = __ffs(bits) - 1;
          bits &= bits - 1u;
          S.srl[pos++] = (uint16_t)((threadIdx.x * 4 + q) * 32 + b);
        }
      }
      if (lane == 31) S.nextra = incl;
    }
    if (lane == 0) { S.nheads = heads; S.dense = dense; }
  }
  __syncthreads();
  const bool dense = S.dense;
  const uint32_t nmul = (len + ksub - 1) / ksub;
  const uint32_t nsr = dense ? nmul + S.nextra : len;
  // level 1
  for (uint32_t p = threadIdx.x; p < nsr; p += blockDim.x) {
    uint32_t j = p;
    if (dense) j = p < nmul ? p * ksub : S.srl[p - nmul];
    else if (!lc_head(S, j)) continue;
    uint32_t x = j, steps = 0;
    VT o = 0;
    uint16_t nx = kEnd16, tail = kEnd16;
    for (;;) {
      const VT wx = S.off[x];
      const uint16_t y = S.nxt[x];
      S.sub[x] = (uint16_t)j;
      S.off[x] = o;
      if (y == kEnd16) { tail = (uint16_t)x; break; }
      o += wx;
      if (dense && (y & submask) == 0) { nx = y; break; }
      x = y;
      if (++steps > len) { bad |= kErrCycle; break; }
    }
    S.nxt[j] = nx;                    // per sub-ruler: the next one (kEnd16: done)
    S.off[j] = o;                     // weight to it, or distance to the tail
    S.sub[j] = tail;                  // the tail, known once nxt is kEnd16
  }
  __syncthreads();
  // level 2: synchronous pointer doubling over the sub-rulers
  if (dense) {
    uint32_t rounds = 0;
    while ((1u << rounds) < nsr) ++rounds;
    for (uint32_t r = 0; r < rounds; ++r) {
      uint16_t tn[2], tt[2];
      VT tv[2];
#pragma unroll
      for (int e = 0; e < 2; ++e) {
        const uint32_t p = threadIdx.x + e * kLcThreads;
        if (p < nsr) {
          const uint32_t j = p < nmul ? p * ksub : S.srl[p - nmul];
          const uint16_t a = S.nxt[j];
          if (a != kEnd16) { tv[e] = S.off[j] + S.off[a]; tn[e] = S.nxt[a]; tt[e] = S.sub[a]; }
          else { tv[e] = S.off[j]; tn[e] = kEnd16; tt[e] = S.sub[j]; }
        }
      }
      __syncthreads();
#pragma unroll
      for (int e = 0; e < 2; ++e) {
        const uint32_t p = threadIdx.x + e * kLcThreads;
        if (p < nsr) {
          const uint32_t j = p < nmul ? p * ksub : S.srl[p - nmul];
          S.nxt[j] = tn[e]; S.off[j] = tv[e]; S.sub[j] = tt[e];
        }
      }
      __syncthreads();
    }
  }
  if (bad) record_error(err, bad);
  return len;
}

// Distance from element j to its local tail, and the tail (kEnd16: j is on
// or leads into a cycle inside the tile).  Valid after lc_tile_solve.
template <class VT>
__device__ __forceinline__ uint16_t lc_elem(const LcTile<VT> &S, uint32_t j, VT *dist) {
  uint32_t sr = j;
  VT ox = 0;
  if (!lc_is_sr(S, j)) {
    sr = S.sub[j];
    if (sr == kEnd16) return kEnd16;
    ox = S.off[j];
  }
  if (S.nxt[sr] != kEnd16) return kEnd16;          // its sub-ruler chain never ended
  *dist = S.off[sr] - ox;
  return S.sub[sr];
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
// heads per tile go to hb, wpre and tcnt.
template <int WT, class VT, class RT>
__global__ void __launch_bounds__(kLcThreads, WT == 0 ? 4 : 3)
k_lc_solve(const uint32_t *__restrict__ succ, const void *__restrict__ weight, uint32_t n,
           RT *__restrict__ rank, uint16_t *__restrict__ tail16, uint32_t *__restrict__ hb,
           uint16_t *__restrict__ wpre, uint32_t *__restrict__ tcnt, uint32_t *__restrict__ err, int vec,
           uint32_t ksub) {
  extern __shared__ __align__(16) unsigned char lc_smem[];
  LcTile<VT> &S = *reinterpret_cast<LcTile<VT> *>(lc_smem);
  const uint32_t ntiles = (n + kTile - 1) >> kTileShift;
  for (uint32_t j = threadIdx.x; j < kTile; j += blockDim.x) S.sub[j] = kEnd16;
  __syncthreads();
  for (uint32_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const uint32_t len = lc_tile_solve<WT, VT>(S, t, succ, weight, n, err, vec != 0, ksub);
    const uint32_t base = t << kTileShift;
    bool cyc = false;
    for (uint32_t j = threadIdx.x; j < len; j += blockDim.x) {
      VT d = 0;
      const uint16_t tj = lc_elem(S, j, &d);
      if (tj == kEnd16) cyc = true;              // on or into a cycle inside the tile
      __stcs(rank + base + j, tj == j ? (RT)0 : (RT)d);
      __stcs(tail16 + base + j, tj);
    }
    if (cyc) record_error(err, kErrCycle);
    if (threadIdx.x < 32) {
      // 4 words per lane; exclusive prefix of the head counts over the tile
      uint32_t h[4], c = 0;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const uint32_t w = threadIdx.x * 4 + q;
        const uint32_t lo = w * 32;
        const uint32_t valid = lo >= len ? 0u : (len - lo >= 32 ? 0xFFFFFFFFu : ((1u << (len - lo)) - 1u));
        h[q] = ~S.pred[w] & valid;
        c += __popc(h[q]);
      }
      uint32_t incl = c;
      for (int d = 1; d < 32; d <<= 1) {
        const uint32_t v = __shfl_up_sync(0xFFFFFFFFu, incl, d);
        if ((int)threadIdx.x >= d) incl += v;
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
    for (uint32_t j = threadIdx.x; j < kTile; j += blockDim.x) S.sub[j] = kEnd16;   // for the next tile
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

size_t lc_smem_bytes(bool weighted, int rank_bytes) {
  (void)rank_bytes;
  return weighted ? sizeof(LcTile<uint64_t>) : sizeof(LcTile<uint32_t>);
}

uint32_t lc_tiles(uint64_t n) { return (uint32_t)((n + kTile - 1) >> kTileShift); }
uint32_t lc_tile_words() { return kTileWords; }

cudaError_t lc_setup() {
  cudaError_t e = cudaSuccess;
#define LC_ATTR(K, BYTES) \
  if (e == cudaSuccess) e = cudaFuncSetAttribute(K, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(BYTES))
  LC_ATTR((k_lc_solve<0, uint32_t, uint32_t>), sizeof(LcTile<uint32_t>));
  LC_ATTR((k_lc_solve<0, uint32_t, unsigned long long>), sizeof(LcTile<uint32_t>));
  LC_ATTR((k_lc_solve<1, uint64_t, uint32_t>), sizeof(LcTile<uint64_t>));
  LC_ATTR((k_lc_solve<1, uint64_t, unsigned long long>), sizeof(LcTile<uint64_t>));
  LC_ATTR((k_lc_solve<2, uint64_t, uint32_t>), sizeof(LcTile<uint64_t>));
  LC_ATTR((k_lc_solve<2, uint64_t, unsigned long long>), sizeof(LcTile<uint64_t>));
#undef LC_ATTR
  return e;
}

cudaError_t launch_lc_solve(const uint32_t *succ, const void *weight, int wtype, uint32_t n, void *rank,
                            int rank_bytes, uint16_t *tail16, uint32_t *hb, uint16_t *wpre, uint32_t *tcnt,
                            uint32_t *tpre, uint32_t *err, uint32_t ksub, cudaStream_t s) {
  if (ksub < 2 || ksub > 32 || (ksub & (ksub - 1))) ksub = kSubDefault;
  const uint32_t nt = lc_tiles(n);
  const size_t sm = lc_smem_bytes(wtype != 0, rank_bytes);
  const int per_sm = wtype ? 3 : 4;
  const int grid = (int)std::min<uint32_t>(nt, (uint32_t)device_sm_count() * per_sm);
  const int vec = ((uintptr_t)succ & 15u) == 0 && ((uintptr_t)weight & 15u) == 0;
#define LC_SOLVE(W, V, R)                                                                          \
  k_lc_solve<W, V, R><<<grid, kLcThreads, sm, s>>>(succ, weight, n, reinterpret_cast<R *>(rank), tail16, \
                                                   hb, wpre, tcnt, err, vec, ksub)
  if (wtype == 0) { if (rank_bytes == 4) LC_SOLVE(0, uint32_t, uint32_t); else LC_SOLVE(0, uint32_t, unsigned long long); }
  else if (wtype == 1) { if (rank_bytes == 4) LC_SOLVE(1, uint64_t, uint32_t); else LC_SOLVE(1, uint64_t, unsigned long long); }
  else { if (rank_bytes == 4) LC_SOLVE(2, uint64_t, uint32_t); else LC_SOLVE(2, uint64_t, unsigned long long); }
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
