// lr_kernels.cu -- CUDA kernels of the sparse ruling-set list ranker (sm_103a).
//
// Pipeline of one call (Section 2.1, Algorithm 1 of "Engineering Scalable
// Distributed List Ranking", restated for one GPU):
//   prep0      level-0 pass: range check, has-predecessor bitmap (findInit),
//              pack succ (and the link weight) into per-element records;
//   heads      per level: classify the heads (initial elements) into sampled
//              rulers, extra rulers and resolved singletons, and number the
//              extra rulers after the sampled ones (pickRulers);
//   chase      per level: one thread per ruler walks succ to the next ruler,
//              rewriting each visited record as (ruler id, offset) and
//              emitting one record of the reduced list (ruler chasing);
//   base       single-CTA pointer doubling (Wyllie) once a level is small
//              enough (the base case), or a grid-wide pointer-doubling
//              fallback for a large last level;
//   finalize   per level, deepest first: R_l[i] = R_{l+1}[ruler(i)] - offset(i)
//              (ruler propagation).
// The chase records the *next* ruler, so ranks come out relative to the
// terminal directly and the list never has to be reversed (Section 2.1 notes
// that the distributed algorithm needs a reversal or the post-processing of
// Section 2.5; walking succ forward from each ruler makes both unnecessary).
#include <atomic>
#include <cstdio>
#include <cstring>

#include "lr_kernels.h"

namespace lr {

static std::atomic<int64_t> g_launches{0};
void count_launch(int k) { g_launches.fetch_add(k, std::memory_order_relaxed); }
int64_t launch_count() { return g_launches.load(std::memory_order_relaxed); }

int device_sm_count() {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 1;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 1;
  return sms > 0 ? sms : 1;
}

int stream_grid(uint64_t work_items, int block) {
  // grid-stride kernels: enough CTAs to fill every SM, no more than needed
  uint64_t want = (work_items + block - 1) / block;
  uint64_t full = (uint64_t)device_sm_count() * (2048 / block);
  if (want < 1) want = 1;
  return (int)(want < full ? want : full);
}

// ---------------------------------------------------------------- init
__global__ void k_init(LevelDesc *desc, InitParams p) {
  const int l = threadIdx.x;
  if (l < p.nlev) {
    LevelDesc x;
    x.mode = l == 0 ? p.mode0 : (uint32_t)kModeOff;
    x.n = l == 0 ? p.n0 : 0u;
    x.f_inv = p.f_inv[l];
    x.r = l == 0 ? (uint32_t)(((uint64_t)p.n0 + p.f_inv[0] - 1) / p.f_inv[0]) : 0u;
    x.k = 0;
    x.h = 0;
    x.visited = 0;
    x.cap = p.cap[l];
    x.seed = p.seed[l];
    x.rounds = p.pd_rounds;
    x.hsrc = l == 0 ? (uint32_t)kHeadsBitmap : (uint32_t)kHeadsList;
    x.nraw = 0;
    desc[l] = x;
  }
}

cudaError_t launch_init(LevelDesc *desc, const InitParams &p, cudaStream_t s) {
  k_init<<<1, 32, 0, s>>>(desc, p);
  count_launch();
  return cudaGetLastError();
}

// ---------------------------------------------------------------- prep0
template <int WT>
__device__ __forceinline__ uint64_t load_weight(const void *w, uint32_t i) {
  if constexpr (WT == 1) return (uint64_t)(int64_t)__ldcs(reinterpret_cast<const int *>(w) + i);
  else if constexpr (WT == 2) return (uint64_t)__ldcs(reinterpret_cast<const long long *>(w) + i);
  else return 1u;
}

// One pass over the input: check every successor, mark the has-predecessor
// bit of every successor (the complement gives the heads, Algorithm 1's
// findInit), and pack {succ, kUnvisited[, link weight]} records.  A terminal's
// weight is stored as 0, so every deeper computation can treat weights
// inclusively.
// sums != nullptr: instead of the bitmap, accumulate the number of terminals
// and the sum of the other successors (single-list head, see k_heads_single).
template <int WT>
__global__ void __launch_bounds__(256)
k_prep0(const uint32_t *__restrict__ succ, const void *__restrict__ weight, uint32_t n,
        void *__restrict__ work, uint32_t *__restrict__ bitmap, uint32_t *__restrict__ err,
        int validate, int vec, const int64_t *__restrict__ offsets, int32_t k,
        unsigned long long *__restrict__ sums, unsigned long long *__restrict__ local) {
  unsigned long long sT = 0, sS = 0, sL = 0;
  const uint32_t ngroups = (uint32_t)(((uint64_t)n + 3u) / 4u);
  const uint32_t stride = gridDim.x * blockDim.x;
  for (uint32_t g = blockIdx.x * blockDim.x + threadIdx.x; g < ngroups; g += stride) {
    const uint32_t i0 = g * 4u;
    const uint32_t cnt = min(4u, n - i0);
    uint32_t s[4];
    uint64_t w[4];
    if (vec && cnt == 4u) {
      uint4 v = __ldcs(reinterpret_cast<const uint4 *>(succ + i0));
      s[0] = v.x; s[1] = v.y; s[2] = v.z; s[3] = v.w;
      if constexpr (WT == 1) {
        int4 q = __ldcs(reinterpret_cast<const int4 *>(reinterpret_cast<const int *>(weight) + i0));
        w[0] = (uint64_t)(int64_t)q.x; w[1] = (uint64_t)(int64_t)q.y;
        w[2] = (uint64_t)(int64_t)q.z; w[3] = (uint64_t)(int64_t)q.w;
      } else if constexpr (WT == 2) {
        const longlong2 *wp = reinterpret_cast<const longlong2 *>(reinterpret_cast<const long long *>(weight) + i0);
        longlong2 a = __ldcs(wp), b = __ldcs(wp + 1);
        w[0] = (uint64_t)a.x; w[1] = (uint64_t)a.y; w[2] = (uint64_t)b.x; w[3] = (uint64_t)b.y;
      } else {
        w[0] = w[1] = w[2] = w[3] = 1u;
      }
    } else {
      for (uint32_t j = 0; j < 4u; ++j) {
        s[j] = j < cnt ? __ldcs(succ + i0 + j) : 0u;
        w[j] = j < cnt ? load_weight<WT>(weight, i0 + j) : 0u;
      }
    }
    if (offsets != nullptr) {
      // batched input: instance of i0 by binary search, then walk forward
      int32_t lo = 0, hi = k;
      while (hi - lo > 1) {
        int32_t mid = (lo + hi) >> 1;
        if ((uint64_t)__ldg(offsets + mid) <= i0) lo = mid; else hi = mid;
      }
      uint64_t base = (uint64_t)__ldg(offsets + lo), end = (uint64_t)__ldg(offsets + lo + 1);
      for (uint32_t j = 0; j < cnt; ++j) {
        const uint32_t i = i0 + j;
        while (i >= end && lo + 1 < k) { ++lo; base = end; end = (uint64_t)__ldg(offsets + lo + 1); }
        const uint64_t g = base + s[j];
        if (i < base || i >= end || (uint64_t)s[j] >= end - base || g >= n) {
          record_error(err, kErrRange);   // successor outside its instance (or a bad table)
          s[j] = i;
        } else {
          s[j] = (uint32_t)g;
        }
      }
    } else {
      for (uint32_t j = 0; j < cnt; ++j)
        if (s[j] >= n) { record_error(err, kErrRange); s[j] = i0 + j; }
    }
    for (uint32_t j = 0; j < cnt; ++j) {
      const uint32_t i = i0 + j;
      if (local) sL += s[j] != i && (s[j] >> kContractTileShift) == (i >> kContractTileShift);
      if (s[j] != i) {
        if (sums) {
          sS += s[j];
        } else {
          const uint32_t bit = 1u << (s[j] & 31u);
          if (validate) {
            if (atomicOr(bitmap + (s[j] >> 5), bit) & bit) record_error(err, kErrNotList);
          } else {
            atomicOr(bitmap + (s[j] >> 5), bit);
          }
        }
      } else {
        w[j] = 0u;   // a terminal has no outgoing link
        sT += 1;
      }
    }
    if constexpr (WT == 0) {
      uint2 *out = reinterpret_cast<uint2 *>(work) + i0;
      if (cnt == 4u) {
        st_sector(out, s[0], kUnvisited, s[1], kUnvisited, s[2], kUnvisited, s[3], kUnvisited);
      } else {
        for (uint32_t j = 0; j < cnt; ++j) out[j] = make_uint2(s[j], kUnvisited);
      }
    } else {
      uint4 *out = reinterpret_cast<uint4 *>(work) + i0;
      if (cnt == 4u) {
        st_sector(out, s[0], kUnvisited, (uint32_t)w[0], (uint32_t)(w[0] >> 32),
                  s[1], kUnvisited, (uint32_t)w[1], (uint32_t)(w[1] >> 32));
        st_sector(out + 2, s[2], kUnvisited, (uint32_t)w[2], (uint32_t)(w[2] >> 32),
                  s[3], kUnvisited, (uint32_t)w[3], (uint32_t)(w[3] >> 32));
      } else {
        for (uint32_t j = 0; j < cnt; ++j)
          __stcs(out + j, make_uint4(s[j], kUnvisited, (uint32_t)w[j], (uint32_t)(w[j] >> 32)));
      }
    }
  }
  if (sums) {
    for (int d = 16; d > 0; d >>= 1) {
      sS += __shfl_down_sync(0xFFFFFFFFu, sS, d);
      sT += __shfl_down_sync(0xFFFFFFFFu, sT, d);
    }
    if ((threadIdx.x & 31) == 0) {
      if (sT) atomicAdd(sums + 0, sT);
      if (sS) atomicAdd(sums + 1, sS);
    }
  }
  if (local) {
    // links that stay inside their contraction tile (decides whether to contract)
    for (int d = 16; d > 0; d >>= 1) sL += __shfl_down_sync(0xFFFFFFFFu, sL, d);
    if ((threadIdx.x & 31) == 0 && sL) atomicAdd(local, sL);
  }
}

cudaError_t launch_prep0(const uint32_t *succ, const void *weight, int wtype, uint32_t n,
                         void *work, uint32_t *bitmap, uint32_t *err, int validate,
                         const int64_t *offsets, int32_t k, unsigned long long *sums,
                         unsigned long long *local, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  const int block = 256;
  const int grid = stream_grid(((uint64_t)n + 3) / 4, block);
  int vec = ((uintptr_t)succ & 15u) == 0;
  if (wtype == 1) vec = vec && ((uintptr_t)weight & 15u) == 0;
  if (wtype == 2) vec = vec && ((uintptr_t)weight & 15u) == 0;
  switch (wtype) {
    case 0: k_prep0<0><<<grid, block, 0, s>>>(succ, weight, n, work, bitmap, err, validate, vec, offsets, k, sums, local); break;
    case 1: k_prep0<1><<<grid, block, 0, s>>>(succ, weight, n, work, bitmap, err, validate, vec, offsets, k, sums, local); break;
    default: k_prep0<2><<<grid, block, 0, s>>>(succ, weight, n, work, bitmap, err, validate, vec, offsets, k, sums, local); break;
  }
  count_launch();
  return cudaGetLastError();
}

// Links that stay inside their contraction tile, counted over every 16th
// tile (out[0]: local links, out[1]: elements sampled).  It decides the
// automatic tile-local contraction before a first pass that would pack
// records the contraction does not use.
constexpr uint32_t kLocalSampleEvery = 16;

__global__ void __launch_bounds__(256)
k_local_sample(const uint32_t *__restrict__ succ, uint32_t n, unsigned long long *__restrict__ out) {
  constexpr uint32_t kT = 1u << kContractTileShift;
  const uint64_t tiles = ((uint64_t)n + kT - 1) / kT;
  const uint64_t items = (tiles + kLocalSampleEvery - 1) / kLocalSampleEvery * kT;
  unsigned long long loc = 0, cnt = 0;
  for (uint64_t e = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; e < items;
       e += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t i = (e / kT) * kLocalSampleEvery * kT + (e % kT);
    if (i >= n) continue;
    const uint32_t sx = __ldcs(succ + i);
    cnt += 1;
    loc += sx != (uint32_t)i && (sx >> kContractTileShift) == (uint32_t)(i >> kContractTileShift);
  }
  for (int d = 16; d > 0; d >>= 1) {
    loc += __shfl_down_sync(0xFFFFFFFFu, loc, d);
    cnt += __shfl_down_sync(0xFFFFFFFFu, cnt, d);
  }
  if ((threadIdx.x & 31) == 0 && cnt) {
    atomicAdd(out, loc);
    atomicAdd(out + 1, cnt);
  }
}

cudaError_t launch_local_sample(const uint32_t *succ, uint32_t n, unsigned long long *out, cudaStream_t s) {
  const uint64_t tiles = ((uint64_t)n + (1u << kContractTileShift) - 1) >> kContractTileShift;
  const uint64_t items = (tiles + kLocalSampleEvery - 1) / kLocalSampleEvery << kContractTileShift;
  k_local_sample<<<stream_grid(items, 256), 256, 0, s>>>(succ, n, out);
  count_launch();
  return cudaGetLastError();
}

// Batched prep without per-element atomics.  Each instance j of a batch that
// is one list has exactly one terminal, and its successors are every local id
// but the head's, so head_j = n_j (n_j - 1) / 2 - sum of its non-terminal
// successors (Section 1.1's findInit, by sums).  isums[2 j] counts instance
// j's terminals and isums[2 j + 1] sums its local successors; a warp whose
// 128 elements lie in one instance adds its sums with two atomics.  Records
// as in k_prep0.  The loop runs warp-uniformly so that the warp can combine.
template <int WT>
__global__ void __launch_bounds__(256)
k_prep0_sums(const uint32_t *__restrict__ succ, const void *__restrict__ weight, uint32_t n,
             void *__restrict__ work, uint32_t *__restrict__ err, int vec, const int64_t *__restrict__ offsets,
             int32_t k, unsigned long long *__restrict__ isums) {
  const uint32_t ngroups = (uint32_t)(((uint64_t)n + 3u) / 4u);
  const uint32_t stride = gridDim.x * blockDim.x;
  const uint32_t lane = threadIdx.x & 31u;
  for (uint32_t gw = blockIdx.x * blockDim.x + (threadIdx.x & ~31u); gw < ngroups; gw += stride) {
    const uint32_t g = gw + lane;
    const bool active = g < ngroups;
    const uint32_t i0 = g * 4u;
    // instance of the warp's first element by binary search (lane 0), then
    // each lane walks forward to its own
    int32_t lo = 0;
    if (lane == 0) {
      int32_t hi = k;
      while (hi - lo > 1) {
        const int32_t mid = (lo + hi) >> 1;
        if ((uint64_t)__ldg(offsets + mid) <= (uint64_t)gw * 4u) lo = mid; else hi = mid;
      }
    }
    lo = __shfl_sync(0xFFFFFFFFu, lo, 0);
    int32_t inst = -1;                 // the one instance of this lane's elements, or -1
    unsigned long long sT = 0, sS = 0;
    if (active) {
      const uint32_t cnt = min(4u, n - i0);
      uint32_t s[4];
      uint64_t w[4];
      if (vec && cnt == 4u) {
        const uint4 v = __ldcs(reinterpret_cast<const uint4 *>(succ + i0));
        s[0] = v.x; s[1] = v.y; s[2] = v.z; s[3] = v.w;
        if constexpr (WT == 1) {
          const int4 q = __ldcs(reinterpret_cast<const int4 *>(reinterpret_cast<const int *>(weight) + i0));
          w[0] = (uint64_t)(int64_t)q.x; w[1] = (uint64_t)(int64_t)q.y;
          w[2] = (uint64_t)(int64_t)q.z; w[3] = (uint64_t)(int64_t)q.w;
        } else if constexpr (WT == 2) {
          const longlong2 *wp = reinterpret_cast<const longlong2 *>(reinterpret_cast<const long long *>(weight) + i0);
          const longlong2 a = __ldcs(wp), b = __ldcs(wp + 1);
          w[0] = (uint64_t)a.x; w[1] = (uint64_t)a.y; w[2] = (uint64_t)b.x; w[3] = (uint64_t)b.y;
        } else {
          w[0] = w[1] = w[2] = w[3] = 1u;
        }
      } else {
        for (uint32_t j = 0; j < 4u; ++j) {
          s[j] = j < cnt ? __ldcs(succ + i0 + j) : 0u;
          w[j] = j < cnt ? load_weight<WT>(weight, i0 + j) : 0u;
        }
      }
      uint64_t base = (uint64_t)__ldg(offsets + lo), end = (uint64_t)__ldg(offsets + lo + 1);
      int32_t first = -2;
      for (uint32_t j = 0; j < cnt; ++j) {
        const uint32_t i = i0 + j;
        while (i >= end && lo + 1 < k) { ++lo; base = end; end = (uint64_t)__ldg(offsets + lo + 1); }
        const uint64_t gl = base + s[j];
        bool term;
        if (i < base || i >= end || (uint64_t)s[j] >= end - base || gl >= n) {
          record_error(err, kErrRange);   // successor outside its instance (or a bad table)
          s[j] = i;
          term = true;
        } else {
          term = gl == i;
          if (!term) sS += s[j];          // local id
          s[j] = (uint32_t)gl;
        }
        if (term) { w[j] = 0u; sT += 1; }
        if (first == -2) first = lo;
        else if (first != lo) first = -1;  // the group straddles two instances
      }
      if (first >= 0) {
        inst = first;
      } else if (first == -1) {            // rare: add each element's share alone
        sT = 0; sS = 0;
        uint64_t b2 = (uint64_t)__ldg(offsets + lo);
        int32_t l2 = lo;
        for (int32_t jj = (int32_t)cnt - 1; jj >= 0; --jj) {
          const uint32_t i = i0 + (uint32_t)jj;
          while (i < b2 && l2 > 0) { --l2; b2 = (uint64_t)__ldg(offsets + l2); }
          if (s[jj] == i) atomicAdd(isums + 2 * (size_t)l2, 1ull);
          else atomicAdd(isums + 2 * (size_t)l2 + 1, (unsigned long long)(s[jj] - b2));
        }
      }
      if constexpr (WT == 0) {
        uint2 *out = reinterpret_cast<uint2 *>(work) + i0;
        if (cnt == 4u) {
          st_sector(out, s[0], kUnvisited, s[1], kUnvisited, s[2], kUnvisited, s[3], kUnvisited);
        } else {
          for (uint32_t j = 0; j < cnt; ++j) out[j] = make_uint2(s[j], kUnvisited);
        }
      } else {
        uint4 *out = reinterpret_cast<uint4 *>(work) + i0;
        if (cnt == 4u) {
          st_sector(out, s[0], kUnvisited, (uint32_t)w[0], (uint32_t)(w[0] >> 32),
                    s[1], kUnvisited, (uint32_t)w[1], (uint32_t)(w[1] >> 32));
          st_sector(out + 2, s[2], kUnvisited, (uint32_t)w[2], (uint32_t)(w[2] >> 32),
                    s[3], kUnvisited, (uint32_t)w[3], (uint32_t)(w[3] >> 32));
        } else {
          for (uint32_t j = 0; j < cnt; ++j)
            __stcs(out + j, make_uint4(s[j], kUnvisited, (uint32_t)w[j], (uint32_t)(w[j] >> 32)));
        }
      }
    }
    // combine: one pair of atomics per warp when all its lanes share an instance
    const int32_t inst0 = __shfl_sync(0xFFFFFFFFu, inst, 0);
    if (__all_sync(0xFFFFFFFFu, inst == inst0 || (inst == -1 && sT == 0 && sS == 0)) && inst0 >= 0) {
      for (int d = 16; d > 0; d >>= 1) {
        sT += __shfl_down_sync(0xFFFFFFFFu, sT, d);
        sS += __shfl_down_sync(0xFFFFFFFFu, sS, d);
      }
      if (lane == 0) {
        if (sT) atomicAdd(isums + 2 * (size_t)inst0, sT);
        if (sS) atomicAdd(isums + 2 * (size_t)inst0 + 1, sS);
      }
    } else if (inst >= 0) {
      if (sT) atomicAdd(isums + 2 * (size_t)inst, sT);
      if (sS) atomicAdd(isums + 2 * (size_t)inst + 1, sS);
    }
  }
}

cudaError_t launch_prep0_sums(const uint32_t *succ, const void *weight, int wtype, uint32_t n, void *work,
                              uint32_t *err, const int64_t *offsets, int32_t k, unsigned long long *isums,
                              cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  const int block = 256;
  const int grid = stream_grid(((uint64_t)n + 3) / 4, block);
  int vec = ((uintptr_t)succ & 15u) == 0;
  if (wtype != 0) vec = vec && ((uintptr_t)weight & 15u) == 0;
  switch (wtype) {
    case 0: k_prep0_sums<0><<<grid, block, 0, s>>>(succ, weight, n, work, err, vec, offsets, k, isums); break;
    case 1: k_prep0_sums<1><<<grid, block, 0, s>>>(succ, weight, n, work, err, vec, offsets, k, isums); break;
    default: k_prep0_sums<2><<<grid, block, 0, s>>>(succ, weight, n, work, err, vec, offsets, k, isums); break;
  }
  count_launch();
  return cudaGetLastError();
}

// Level-0 heads of a batch from its per-instance sums (one CTA): the head of
// every non-empty instance that has exactly one terminal, listed in instance
// order.  If any non-empty instance has another number of terminals, or the
// heads would not fit the list (capacity hcap), the has-predecessor bitmap
// is used instead: the sums are cleared (they share its memory) and
// k_bitmap0_recs fills it.
__global__ void __launch_bounds__(1024)
k_heads0_batch(LevelDesc *desc, unsigned long long *isums, const int64_t *__restrict__ offsets, int32_t k,
               uint32_t *__restrict__ hlist0, uint32_t hcap, uint32_t n) {
  __shared__ uint64_t sm[33];
  LevelDesc &d = desc[0];
  int fallback = 0;
  uint32_t total = 0;
  for (int32_t j0 = 0; j0 < k; j0 += (int32_t)blockDim.x) {
    const int32_t j = j0 + (int32_t)threadIdx.x;
    uint32_t has = 0;
    uint64_t head = 0;
    if (j < k) {
      const int64_t b0 = offsets[j], b1 = offsets[j + 1];
      if (b0 < 0 || b1 < b0 || (uint64_t)b1 > n) {
        fallback = 1;                        // a bad offset table: the prep reported it
      } else if (b1 > b0) {
        const uint64_t b = (uint64_t)b0, nj = (uint64_t)(b1 - b0);
        const unsigned long long T = isums[2 * (size_t)j], S = isums[2 * (size_t)j + 1];
        const unsigned long long h = nj * (nj - 1) / 2 - S;
        if (T == 1 && h < nj) { has = 1; head = b + h; }
        else fallback = 1;
      }
    }
    uint64_t cnt;
    const uint64_t pos = block_exclusive_scan((uint64_t)has, sm, &cnt);
    if (has && total + pos < hcap) hlist0[total + pos] = (uint32_t)head;
    total += (uint32_t)cnt;
    __syncthreads();
  }
  if (total > hcap) fallback = 1;
  fallback = __syncthreads_or(fallback);
  if (fallback) {
    // the sums occupy the start of the bitmap's memory: clear them
    for (int32_t j = (int32_t)threadIdx.x; j < 2 * k; j += (int32_t)blockDim.x) isums[j] = 0ull;
    if (threadIdx.x == 0) d.hsrc = kHeadsBitmap;
  } else if (threadIdx.x == 0) {
    d.h = total;
    d.hsrc = kHeadsList;
  }
}

// Has-predecessor bitmap from the level-0 records (global successors), only
// when k_heads0_batch fell back to it.
__global__ void __launch_bounds__(256)
k_bitmap0_recs(const LevelDesc *__restrict__ desc, const uint32_t *__restrict__ recs, uint32_t words_per_rec,
               uint32_t n, uint32_t *__restrict__ bitmap) {
  if (desc[0].hsrc != kHeadsBitmap) return;
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const uint32_t s = __ldcs(recs + (size_t)i * words_per_rec);
    if (s != i) atomicOr(bitmap + (s >> 5), 1u << (s & 31u));
  }
}

// Lists of a batch from its per-instance sums: every list has one terminal.
__global__ void __launch_bounds__(1024)
k_count_batch(const unsigned long long *__restrict__ isums, int32_t k, uint32_t *__restrict__ out) {
  __shared__ uint64_t sm[33];
  uint64_t t = 0;
  for (int32_t j = (int32_t)threadIdx.x; j < k; j += (int32_t)blockDim.x) t += isums[2 * (size_t)j];
  uint64_t total;
  block_exclusive_scan(t, sm, &total);
  if (threadIdx.x == 0) *out = total > 0xFFFFFFFFull ? 0xFFFFFFFFu : (uint32_t)total;
}

cudaError_t launch_count_batch(const unsigned long long *isums, int32_t k, uint32_t *out, cudaStream_t s) {
  k_count_batch<<<1, 1024, 0, s>>>(isums, k, out);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_heads0_batch(LevelDesc *desc, unsigned long long *isums, const int64_t *offsets, int32_t k,
                                uint32_t *hlist0, uint32_t hcap, const void *work, bool rec16, uint32_t n,
                                uint32_t *bitmap, cudaStream_t s) {
  k_heads0_batch<<<1, 1024, 0, s>>>(desc, isums, offsets, k, hlist0, hcap, n);
  k_bitmap0_recs<<<stream_grid(n, 256), 256, 0, s>>>(desc, reinterpret_cast<const uint32_t *>(work),
                                                      rec16 ? 4u : 2u, n, bitmap);
  count_launch(2);
  return cudaGetLastError();
}

// Batched input given as one device pointer per instance (the serving path
// ranks requests where they already live, without gathering them first).
template <int WT>
__global__ void __launch_bounds__(256)
k_prep0_ptrs(const uint32_t *const *__restrict__ sptr, const void *const *__restrict__ wptr,
             uint32_t n, void *__restrict__ work, uint32_t *__restrict__ bitmap,
             uint32_t *__restrict__ err, int validate, const int64_t *__restrict__ offsets, int32_t k) {
  const uint32_t stride = gridDim.x * blockDim.x;
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    int32_t lo = 0, hi = k;
    while (hi - lo > 1) {
      int32_t mid = (lo + hi) >> 1;
      if ((uint64_t)__ldg(offsets + mid) <= i) lo = mid; else hi = mid;
    }
    const uint64_t base = (uint64_t)__ldg(offsets + lo), len = (uint64_t)__ldg(offsets + lo + 1) - base;
    const uint64_t loc = i - base;
    uint32_t s = __ldcs(sptr[lo] + loc);
    uint64_t w = 1u;
    if constexpr (WT == 1) w = (uint64_t)(int64_t)__ldcs(reinterpret_cast<const int *>(wptr[lo]) + loc);
    if constexpr (WT == 2) w = (uint64_t)__ldcs(reinterpret_cast<const long long *>(wptr[lo]) + loc);
    if ((uint64_t)s >= len || base + s >= n) { record_error(err, kErrRange); s = i; }
    else s = (uint32_t)(base + s);
    if (s != i) {
      const uint32_t bit = 1u << (s & 31u);
      if (validate) {
        if (atomicOr(bitmap + (s >> 5), bit) & bit) record_error(err, kErrNotList);
      } else {
        atomicOr(bitmap + (s >> 5), bit);
      }
    } else {
      w = 0u;
    }
    if constexpr (WT == 0) reinterpret_cast<uint2 *>(work)[i] = make_uint2(s, kUnvisited);
    else __stcs(reinterpret_cast<uint4 *>(work) + i, make_uint4(s, kUnvisited, (uint32_t)w, (uint32_t)(w >> 32)));
  }
}

cudaError_t launch_prep0_ptrs(const uint32_t *const *sptr, const void *const *wptr, int wtype,
                              uint32_t n, void *work, uint32_t *bitmap, uint32_t *err, int validate,
                              const int64_t *offsets, int32_t k, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  const int block = 256;
  const int grid = stream_grid(n, block);
  switch (wtype) {
    case 0: k_prep0_ptrs<0><<<grid, block, 0, s>>>(sptr, wptr, n, work, bitmap, err, validate, offsets, k); break;
    case 1: k_prep0_ptrs<1><<<grid, block, 0, s>>>(sptr, wptr, n, work, bitmap, err, validate, offsets, k); break;
    default: k_prep0_ptrs<2><<<grid, block, 0, s>>>(sptr, wptr, n, work, bitmap, err, validate, offsets, k); break;
  }
  count_launch();
  return cudaGetLastError();
}

// The instance of element `base` in a table of k nondecreasing offsets with
// offsets[0] = 0 <= base < offsets[k]: the largest j < k with offsets[j] <=
// base, found by the whole warp at once (every lane probes one of 32 points
// spread over the remaining range, the ballot keeps the last probe at or
// below base), in at most 3 rounds for up to 32768 instances.  Warp-uniform.
__device__ __forceinline__ int32_t warp_instance(const int64_t *__restrict__ offsets, int32_t k, uint64_t base,
                                                 uint32_t lane) {
  int32_t lo = 0, hi = k;
  while (hi - lo > 1) {
    const int64_t span = hi - lo;
    const int32_t q = lo + (int32_t)(((int64_t)(lane + 1) * span) / 33);
    const uint32_t le = __ballot_sync(0xFFFFFFFFu, (uint64_t)__ldg(offsets + q) <= base);
    const int t = __popc(le);
    const int32_t nlo = __shfl_sync(0xFFFFFFFFu, q, t > 0 ? t - 1 : 0);
    const int32_t nhi = __shfl_sync(0xFFFFFFFFu, q, t < 32 ? t : 31);
    if (t > 0) lo = max(lo, nlo);
    if (t < 32) hi = nhi;
  }
  return lo;
}

// Pointer batches without per-element atomics: the per-instance sums of
// k_prep0_sums (terminals, local successors), read through one pointer per
// instance.  A warp takes 128 consecutive elements (lane l: l + 32 j, so that
// loads and record stores are coalesced); the warp finds the instance of
// the first (warp_instance) and every lane walks forward from it.  A warp
// whose elements all lie in one instance adds its sums with two atomics.
template <int WT>
__global__ void __launch_bounds__(256)
k_prep0_ptrs_sums(const uint32_t *const *__restrict__ sptr, const void *const *__restrict__ wptr,
                  uint32_t n, void *__restrict__ work, uint32_t *__restrict__ err,
                  const int64_t *__restrict__ offsets, int32_t k, unsigned long long *__restrict__ isums) {
  const uint32_t lane = threadIdx.x & 31u;
  const uint64_t warp = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint64_t step = ((uint64_t)gridDim.x * blockDim.x >> 5) * 128u;
  for (uint64_t base = warp * 128u; base < n; base += step) {
    const int32_t lo0 = warp_instance(offsets, k, base, lane);
    // each of the lane's four elements: its instance, then all four loads
    // in flight together
    int32_t inst[4];
    uint64_t ibv[4], iev[4];
    int32_t lo = lo0;
    uint64_t ib = (uint64_t)__ldg(offsets + lo), ie = (uint64_t)__ldg(offsets + lo + 1);
    const bool one = ie >= min(base + 128u, (uint64_t)n);   // warp-uniform
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const uint64_t i = base + lane + 32u * j;
      while (i < n && i >= ie && lo + 1 < k) { ++lo; ib = ie; ie = (uint64_t)__ldg(offsets + lo + 1); }
      inst[j] = lo;
      ibv[j] = ib;
      iev[j] = ie;
    }
    uint32_t sv[4];
    uint64_t wv[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const uint64_t i = base + lane + 32u * j;
      sv[j] = 0u;
      wv[j] = 1u;
      if (i < n && i >= ibv[j] && i < iev[j]) {
        const uint64_t loc = i - ibv[j];
        sv[j] = __ldcs(sptr[inst[j]] + loc);
        if constexpr (WT == 1) wv[j] = (uint64_t)(int64_t)__ldcs(reinterpret_cast<const int *>(wptr[inst[j]]) + loc);
        if constexpr (WT == 2) wv[j] = (uint64_t)__ldcs(reinterpret_cast<const long long *>(wptr[inst[j]]) + loc);
      }
    }
    unsigned long long sT = 0, sS = 0;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const uint64_t i = base + lane + 32u * j;
      if (i >= n) continue;
      uint32_t s = sv[j];
      uint64_t w = wv[j];
      const uint64_t ib = ibv[j], ie = iev[j];
      bool term;
      if (i < ib || i >= ie) {
        record_error(err, kErrRange);     // a bad offset table
        s = (uint32_t)i;
        term = true;
      } else if ((uint64_t)s >= ie - ib || ib + s >= n) {
        record_error(err, kErrRange);     // successor outside its instance
        s = (uint32_t)i;
        term = true;
      } else {
        term = (uint64_t)s == i - ib;
        if (!term) {
          if (one) sS += s;
          else atomicAdd(isums + 2 * (size_t)inst[j] + 1, (unsigned long long)s);
        }
        s = (uint32_t)(ib + s);
      }
      if (term) {
        w = 0u;
        if (one) sT += 1;
        else atomicAdd(isums + 2 * (size_t)inst[j], 1ull);
      }
      if constexpr (WT == 0) reinterpret_cast<uint2 *>(work)[i] = make_uint2(s, kUnvisited);
      else __stcs(reinterpret_cast<uint4 *>(work) + i, make_uint4(s, kUnvisited, (uint32_t)w, (uint32_t)(w >> 32)));
    }
    if (one) {
      for (int d = 16; d > 0; d >>= 1) {
        sT += __shfl_down_sync(0xFFFFFFFFu, sT, d);
        sS += __shfl_down_sync(0xFFFFFFFFu, sS, d);
      }
      if (lane == 0) {
        if (sT) atomicAdd(isums + 2 * (size_t)lo0, sT);
        if (sS) atomicAdd(isums + 2 * (size_t)lo0 + 1, sS);
      }
    }
  }
}

cudaError_t launch_prep0_ptrs_sums(const uint32_t *const *sptr, const void *const *wptr, int wtype, uint32_t n,
                                   void *work, uint32_t *err, const int64_t *offsets, int32_t k,
                                   unsigned long long *isums, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  const int block = 256;
  const int grid = stream_grid(((uint64_t)n + 3) / 4, block);
  switch (wtype) {
    case 0: k_prep0_ptrs_sums<0><<<grid, block, 0, s>>>(sptr, wptr, n, work, err, offsets, k, isums); break;
    case 1: k_prep0_ptrs_sums<1><<<grid, block, 0, s>>>(sptr, wptr, n, work, err, offsets, k, isums); break;
    default: k_prep0_ptrs_sums<2><<<grid, block, 0, s>>>(sptr, wptr, n, work, err, offsets, k, isums); break;
  }
  count_launch();
  return cudaGetLastError();
}

// Number of heads (zero bits of the has-predecessor bitmap below n).
__global__ void k_count_heads(const uint32_t *__restrict__ bitmap, uint32_t n, uint32_t *out) {
  const uint32_t words = (uint32_t)(((uint64_t)n + 31u) / 32u);
  uint32_t c = 0;
  for (uint32_t w = blockIdx.x * blockDim.x + threadIdx.x; w < words; w += gridDim.x * blockDim.x) {
    uint32_t bits = ~__ldcg(bitmap + w);
    if (w == words - 1u && (n & 31u)) bits &= (1u << (n & 31u)) - 1u;
    c += __popc(bits);
  }
  for (int d = 16; d > 0; d >>= 1) c += __shfl_down_sync(0xFFFFFFFFu, c, d);
  if ((threadIdx.x & 31) == 0 && c) atomicAdd(out, c);
}

cudaError_t launch_count_heads(const uint32_t *bitmap, uint32_t n, uint32_t *out, cudaStream_t s) {
  const int block = 256;
  const int grid = stream_grid(((uint64_t)n + 31u) / 32u, block);
  k_count_heads<<<grid, block, 0, s>>>(bitmap, n, out);
  count_launch();
  return cudaGetLastError();
}

// ---------------------------------------------------------------- heads
enum : int { kCatSampled = 0, kCatNew = 1, kCatSingle = 2 };

// Classify head x of a level: a sampled ruler keeps id pi(x); a head that is
// also a terminal is a one-element list whose rank is its own weight
// (resolved here, never chased); any other head becomes an extra ruler.
template <class Rec, bool RESOLVE>
__device__ __forceinline__ int classify_head(uint32_t x, const Perm &P, uint32_t r,
                                             const Rec *work, uint32_t *pid, uint64_t *wself) {
  const uint32_t p = P.fwd(x);
  *pid = p;
  if (p < r) return kCatSampled;
  if constexpr (RESOLVE) {
    Rec v = ld_rec(work + x);
    if (rec_succ(v) == x) { *wself = rec_weight(v, x); return kCatSingle; }
  }
  return kCatNew;
}

// Visit this thread's heads in a fixed order (deterministic numbering).
template <class F>
__device__ __forceinline__ void for_each_head(const LevelDesc &d, const uint32_t *bitmap,
                                              const uint32_t *hlist, F &&f) {
  if (d.hsrc == kHeadsBitmap) {
    const uint32_t words = (uint32_t)(((uint64_t)d.n + 31u) / 32u);
    const uint32_t per = (words + gridDim.x - 1) / gridDim.x;
    const uint32_t w0 = blockIdx.x * per, w1 = min(words, w0 + per);
    for (uint32_t w = w0 + threadIdx.x; w < w1; w += blockDim.x) {
      uint32_t bits = ~__ldcg(bitmap + w);
      if (w == words - 1u && (d.n & 31u)) bits &= (1u << (d.n & 31u)) - 1u;
      while (bits) {
        const uint32_t b = __ffs(bits) - 1;
        bits &= bits - 1u;
        f(w * 32u + b);
      }
    }
  } else {
    const uint32_t cnt = d.h;
    const uint32_t per = (cnt + gridDim.x - 1) / gridDim.x;
    const uint32_t e0 = blockIdx.x * per, e1 = min(cnt, e0 + per);
    for (uint32_t e = e0 + threadIdx.x; e < e1; e += blockDim.x) f(__ldcg(hlist + e));
  }
}

template <class Rec, bool RESOLVE>
__global__ void __launch_bounds__(kHeadThreads)
k_heads_count(const LevelDesc *__restrict__ desc, int lev, const uint32_t *__restrict__ bitmap,
              const uint32_t *__restrict__ hlist, const Rec *__restrict__ work,
              uint64_t *__restrict__ blockcnt) {
  __shared__ uint64_t sm[33];
  const LevelDesc d = desc[lev];
  if (d.mode != kModeSrs) return;
  Perm P;
  P.init(d.n, d.seed);
  uint32_t nS = 0, nN = 0;
  for_each_head(d, bitmap, hlist, [&](uint32_t x) {
    uint32_t p;
    uint64_t w;
    const int c = classify_head<Rec, RESOLVE>(x, P, d.r, work, &p, &w);
    nS += c == kCatSampled;
    nN += c == kCatNew;
  });
  uint64_t total;
  block_exclusive_scan(((uint64_t)(nS + nN) << 32) | nN, sm, &total);
  if (threadIdx.x == 0) blockcnt[blockIdx.x] = total;
}

// Exclusive scan of the per-CTA counts; sizes of the next level; its mode.
__global__ void __launch_bounds__(kHeadBlocks)
k_heads_scan(LevelDesc *desc, int lev, int nlev, uint64_t *blockcnt, uint32_t *err,
             uint32_t cutoff, uint32_t hcap, uint32_t has_pd) {
  __shared__ uint64_t sm[33];
  if (desc[lev].mode != kModeSrs) return;
  uint64_t total;
  const uint64_t v = blockcnt[threadIdx.x];
  const uint64_t ex = block_exclusive_scan(v, sm, &total);
  blockcnt[threadIdx.x] = ex;
  if (threadIdx.x == 0) {
    LevelDesc &d = desc[lev];
    LevelDesc &e = desc[lev + 1];
    const uint32_t kNew = (uint32_t)total;
    const uint32_t hNext = (uint32_t)(total >> 32);
    const uint64_t n1 = (uint64_t)d.r + kNew;
    d.k = kNew;
    bool bad = hNext > hcap || n1 > e.cap;
    uint32_t mode = kModeSrs;
    if (n1 <= cutoff) mode = kModeBase;
    else if (lev + 1 >= nlev - 1) { if (has_pd) mode = kModePd; else bad = true; }
    if (bad) {
      record_error(err, kErrCapacity);
      d.mode = kModeOff;      // nothing more runs at this level or below
      return;
    }
    e.n = (uint32_t)n1;
    e.r = (uint32_t)((n1 + e.f_inv - 1) / e.f_inv);
    e.h = hNext;
    e.mode = mode;
  }
}

template <class Rec, bool RESOLVE>
__global__ void __launch_bounds__(kHeadThreads)
k_heads_write(LevelDesc *__restrict__ desc, int lev, const uint32_t *__restrict__ bitmap,
              const uint32_t *__restrict__ hlist, Rec *__restrict__ work,
              uint32_t *__restrict__ ns, uint32_t *__restrict__ hnext,
              const uint64_t *__restrict__ blockoff) {
  __shared__ uint64_t sm[33];
  const LevelDesc d = desc[lev];
  if (d.mode != kModeSrs) return;
  Perm P;
  P.init(d.n, d.seed);
  uint32_t nS = 0, nN = 0;
  for_each_head(d, bitmap, hlist, [&](uint32_t x) {
    uint32_t p;
    uint64_t w;
    const int c = classify_head<Rec, RESOLVE>(x, P, d.r, work, &p, &w);
    nS += c == kCatSampled;
    nN += c == kCatNew;
  });
  const uint64_t mine = block_exclusive_scan(((uint64_t)(nS + nN) << 32) | nN, sm, nullptr);
  const uint64_t base = blockoff[blockIdx.x] + mine;
  uint32_t posN = (uint32_t)base, posH = (uint32_t)(base >> 32), nZ = 0;
  for_each_head(d, bitmap, hlist, [&](uint32_t x) {
    uint32_t p;
    uint64_t w;
    const int c = classify_head<Rec, RESOLVE>(x, P, d.r, work, &p, &w);
    if (c == kCatSampled) {
      hnext[posH++] = p;
    } else if (c == kCatNew) {
      ns[posN] = x;
      hnext[posH++] = d.r + posN;
      ++posN;
    } else {
      st_rec(work + x, kZeroCid, (uint64_t)0 - w);   // R(x) = 0 - (-w) = w
      ++nZ;
    }
  });
  for (int dd = 16; dd > 0; dd >>= 1) nZ += __shfl_down_sync(0xFFFFFFFFu, nZ, dd);
  if ((threadIdx.x & 31) == 0 && nZ) atomicAdd(&desc[lev].visited, nZ);
}

cudaError_t launch_heads(LevelDesc *desc, int lev, int nlev, const uint32_t *bitmap,
                         const uint32_t *hlist, void *work, int rec_kind, uint32_t *ns,
                         uint32_t *hnext, uint64_t *blockcnt, uint32_t *err, uint32_t cutoff,
                         uint32_t hcap, uint32_t has_pd, cudaStream_t s) {
#define LR_HEADS(KERNEL, REC, RES)                                                                \
  KERNEL<REC, RES><<<kHeadBlocks, kHeadThreads, 0, s>>>
  switch (rec_kind) {
    case kRecKind8:
      LR_HEADS(k_heads_count, Rec8, true)(desc, lev, bitmap, hlist, reinterpret_cast<const Rec8 *>(work), blockcnt);
      break;
    case kRecKind16:
      LR_HEADS(k_heads_count, Rec16, true)(desc, lev, bitmap, hlist, reinterpret_cast<const Rec16 *>(work), blockcnt);
      break;
    default:
      LR_HEADS(k_heads_count, Succ4, false)(desc, lev, bitmap, hlist, reinterpret_cast<const Succ4 *>(work), blockcnt);
      break;
  }
  k_heads_scan<<<1, kHeadBlocks, 0, s>>>(desc, lev, nlev, blockcnt, err, cutoff, hcap, has_pd);
  switch (rec_kind) {
    case kRecKind8:
      LR_HEADS(k_heads_write, Rec8, true)(desc, lev, bitmap, hlist, reinterpret_cast<Rec8 *>(work), ns, hnext, blockcnt);
      break;
    case kRecKind16:
      LR_HEADS(k_heads_write, Rec16, true)(desc, lev, bitmap, hlist, reinterpret_cast<Rec16 *>(work), ns, hnext, blockcnt);
      break;
    default:
      LR_HEADS(k_heads_write, Succ4, false)(desc, lev, bitmap, hlist, reinterpret_cast<Succ4 *>(work), ns, hnext, blockcnt);
      break;
  }
#undef LR_HEADS
  count_launch(3);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- ruler order
// Sampled rulers in element order, for inputs made of contiguous instances
// (a batch; each of its levels keeps every instance's elements together).  A chase that takes its rulers in this order works on
// a few instances at a time, so the records it reads and rewrites at random
// stay within a footprint the L2 can hold, where the default order (ruler
// ids, i.e. random positions) touches the whole input at once.  The sampled
// rulers are the same set (pi(x) < r); only their order and ids change: the
// id of the ruler at position x is the number of sampled rulers before x, so
// the reduced records and the final pass's rank gathers are local too.
//   mark:  bit x of `bits` for every sampled ruler x = pi^{-1}(c), c < r;
//   count: set bits per CTA (a contiguous run of words per thread);
//   scan:  exclusive prefix of the per-CTA counts;
//   write: each thread lists the positions of its run's set bits, in order,
//          and the count before every 256-position block (cum).
__global__ void __launch_bounds__(256)
k_ord_mark(const LevelDesc *__restrict__ desc, int lev, uint32_t *__restrict__ bits) {
  const LevelDesc d = desc[lev];
  if (d.mode != kModeSrs) return;
  Perm P;
  P.init(d.n, d.seed);
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t c = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; c < d.r; c += stride) {
    const uint32_t x = P.inv((uint32_t)c);
    atomicOr(bits + (x >> 5), 1u << (x & 31u));
  }
}

// Words [c0, c1) of this CTA: a contiguous share, read in tiles of one word
// per thread (coalesced).
__device__ __forceinline__ void ord_range(uint32_t words, uint32_t *c0, uint32_t *c1) {
  const uint32_t per_cta = (words + gridDim.x - 1) / gridDim.x;
  *c0 = min(words, blockIdx.x * per_cta);
  *c1 = min(words, *c0 + per_cta);
}

__global__ void __launch_bounds__(kHeadThreads)
k_ord_count(const LevelDesc *__restrict__ desc, int lev, const uint32_t *__restrict__ bits,
            uint64_t *__restrict__ cnt) {
  __shared__ uint64_t sm[33];
  const LevelDesc d = desc[lev];
  if (d.mode != kModeSrs) return;
  uint32_t c0, c1, m = 0;
  ord_range((uint32_t)(((uint64_t)d.n + 31u) / 32u), &c0, &c1);
  for (uint32_t w = c0 + threadIdx.x; w < c1; w += blockDim.x) m += __popc(__ldcg(bits + w));
  uint64_t total;
  block_exclusive_scan(m, sm, &total);
  if (threadIdx.x == 0) cnt[blockIdx.x] = total;
}

__global__ void __launch_bounds__(kHeadBlocks)
k_ord_scan(const LevelDesc *__restrict__ desc, int lev, uint64_t *__restrict__ cnt, uint32_t *__restrict__ err) {
  __shared__ uint64_t sm[33];
  const LevelDesc d = desc[lev];
  if (d.mode != kModeSrs) return;
  uint64_t total;
  const uint64_t ex = block_exclusive_scan(cnt[threadIdx.x], sm, &total);
  cnt[threadIdx.x] = ex;
  if (threadIdx.x == 0 && total != d.r) record_error(err, kErrInternal);   // pi is a bijection
}

// Tile by tile: each thread one word, the tile's exclusive scan of their
// counts, then each thread lists its word's marks in ascending order.
__global__ void __launch_bounds__(kHeadThreads)
k_ord_write(const LevelDesc *__restrict__ desc, int lev, const uint32_t *__restrict__ bits,
            const uint64_t *__restrict__ cnt, uint32_t *__restrict__ ord, uint32_t *__restrict__ cum) {
  __shared__ uint64_t sm[33];
  const LevelDesc d = desc[lev];
  if (d.mode != kModeSrs) return;
  uint32_t c0, c1;
  ord_range((uint32_t)(((uint64_t)d.n + 31u) / 32u), &c0, &c1);
  uint64_t base = cnt[blockIdx.x];
  for (uint32_t t0 = c0; t0 < c1; t0 += blockDim.x) {     // uniform trip count in the CTA
    const uint32_t w = t0 + threadIdx.x;
    uint32_t b = w < c1 ? __ldcg(bits + w) : 0u;
    uint64_t tile;
    uint64_t pos = base + block_exclusive_scan(__popc(b), sm, &tile);
    if (w < c1 && (w & 7u) == 0) cum[w >> 3] = (uint32_t)pos;
    while (b) {
      const uint32_t i = __ffs(b) - 1;
      b &= b - 1u;
      if (pos < d.r) ord[pos] = w * 32u + i;
      ++pos;
    }
    base += tile;
  }
}

// Id of the sampled ruler at position y: rulers before y's 256-position
// block plus the marks before y inside it (one 32-byte read of the block's
// eight words).
__device__ __forceinline__ uint32_t ord_id(const uint32_t *__restrict__ bits, const uint32_t *__restrict__ cum,
                                           uint32_t y) {
  const uint32_t b = y >> 8;
  const uint4 *wp = reinterpret_cast<const uint4 *>(bits) + 2 * (size_t)b;
  const uint4 lo = __ldcg(wp), hi = __ldcg(wp + 1);
  uint32_t id = __ldcg(cum + b);
  const uint32_t wi = (y >> 5) & 7u;
  const uint32_t m = (1u << (y & 31u)) - 1u;
  const uint32_t w[8] = {lo.x, lo.y, lo.z, lo.w, hi.x, hi.y, hi.z, hi.w};
#pragma unroll
  for (uint32_t i = 0; i < 8; ++i) id += __popc(i < wi ? w[i] : (i == wi ? (w[i] & m) : 0u));
  return id;
}

// The next level's head list named the sampled heads by pi(x); give them
// their ids in element order.
__global__ void __launch_bounds__(256)
k_ord_heads(const LevelDesc *__restrict__ desc, int lev, uint32_t *__restrict__ hnext, OrdArgs oa) {
  const LevelDesc d = desc[lev];
  if (d.mode != kModeSrs) return;
  Perm P;
  P.init(d.n, d.seed);
  const uint32_t h = desc[lev + 1].h;
  for (uint32_t e = blockIdx.x * blockDim.x + threadIdx.x; e < h; e += gridDim.x * blockDim.x) {
    const uint32_t v = hnext[e];
    if (v < d.r) hnext[e] = ord_id(oa.bits, oa.cum, P.inv(v));
  }
}

cudaError_t launch_order(LevelDesc *desc, int lev, uint32_t cap, uint64_t *cnt, const OrdArgs *oa,
                         uint32_t *hnext, uint32_t hcap, uint32_t *err, cudaStream_t s) {
  // whole 256-position blocks, so that a lookup may read all 8 words of one
  cudaError_t e = cudaMemsetAsync(oa->bits, 0, 32 * (((uint64_t)cap + 255u) / 256u), s);
  if (e != cudaSuccess) return e;
  k_ord_mark<<<stream_grid(cap / 8 + 1, 256), 256, 0, s>>>(desc, lev, oa->bits);
  k_ord_count<<<kHeadBlocks, kHeadThreads, 0, s>>>(desc, lev, oa->bits, cnt);
  k_ord_scan<<<1, kHeadBlocks, 0, s>>>(desc, lev, cnt, err);
  k_ord_write<<<kHeadBlocks, kHeadThreads, 0, s>>>(desc, lev, oa->bits, cnt, oa->ord, oa->cum);
  k_ord_heads<<<stream_grid(hcap, 256), 256, 0, s>>>(desc, lev, hnext, *oa);
  count_launch(5);
  return cudaGetLastError();
}


// Ordered queue: CTAs draw positions of the ruler sequence from one global
// counter, kOrdChunk at a time, and hand them to their threads one by one
// through a shared-memory window (end << 32) | next.  The thread that draws
// next == end refills the window; threads that draw past its end meanwhile
// take single positions from the global counter.  Nobody waits.
constexpr uint32_t kOrdChunk = 32;

__device__ __forceinline__ uint64_t ord_take(unsigned long long *s_win, uint32_t *gq, uint64_t total,
                                             bool *refilled = nullptr) {
  const unsigned long long w = atomicAdd(s_win, 1ull);
  const uint32_t next = (uint32_t)w, end = (uint32_t)(w >> 32);
  if (next < end) return next;
  if (next == end) {
    if (refilled) *refilled = true;
    // the chunk is this CTA's whatever its length: every position of it
    // must be handed out, up to the end of the sequence
    const uint32_t j = atomicAdd(gq, kOrdChunk);
    if (j < total) {
      const uint64_t e = (uint64_t)j + kOrdChunk < total ? (uint64_t)j + kOrdChunk : total;
      atomicExch(s_win, (e << 32) | (j + 1u));
    }
    return j;
  }
  return atomicAdd(gq, 1u);
}

// ---------------------------------------------------------------- chase
// Persistent CTAs; CTA b owns a contiguous slice of ruler ids and its threads
// pull ids one at a time from a per-CTA counter (the next id is requested
// while the current chain runs, hiding the atomic's latency).  Each thread
// walks succ from its ruler until it meets the next ruler (pi(y) < r) or a
// terminal, rewriting every visited record as (ruler id, offset).
// Visit one record: return its old contents and rewrite it as (cid, off)
// unless another chase got there first.  XCHG: one atomic exchange at L2;
// otherwise the store is issued only after the load has returned (it depends
// on the loaded tag), so it always hits the sector the load just brought in.
template <bool XCHG, class Rec>
__device__ __forceinline__ Rec visit(Rec *p, uint32_t cid, uint64_t off) {
  if constexpr (XCHG) {
    return xchg_rec(p, cid, off);
  } else {
    Rec v = ld_rec(p);
    if (rec_tag(v) == kUnvisited) st_rec(p, cid, off);
    return v;
  }
}

// TERM: a ruler whose segment ends at a terminal y becomes a terminal of the
// next level; it records y's original id (y itself at level 0, tid_cur[y]
// deeper) in tid_next, so the terminal of every element can be carried back.
//
// SPAWN (Section 2.2, ruler spawning; exchange chase only): a thread whose
// CTA has no queued ruler left claims an unvisited, unsampled element of its
// CTA's slice of ids as a new ruler (one exchange writes the claim mark and
// the thread's reserved id R + k), and chases from it.  A wave that meets a
// claimed element stops there, its next ruler; a queued head that a spawner
// claimed first becomes a zero-weight link to the spawned ruler.  Ids that
// were reserved but never claimed leave holes, removed after the chase.
//
// ORD (ord.ord != nullptr; a level of a batch, no spawning): the rulers come
// in element order instead, from one global queue over the sequence
// heads (ids r .. r+k-1, in head-list order) then ord[0 .. r) (positions of
// the sampled rulers, ascending), so all CTAs advance one front across the
// instances together; the sampled ruler ord[i] has id i (ord_id of its
// position).  The thread that draws a CTA's next rulers also asks L2 for
// the records of the elements its draw covers, pf_lead elements ahead:
// streamed in order, they are mostly in L2 when the chases reach them.
template <class Rec, bool XCHG, bool TERM, bool SPAWN>
__global__ void __launch_bounds__(512)
k_chase(LevelDesc *__restrict__ desc, int lev, Rec *__restrict__ work, Rec16 *__restrict__ next,
        const uint32_t *__restrict__ ns, uint32_t *__restrict__ qctr, uint32_t *__restrict__ err,
        const uint32_t *__restrict__ tid_cur, uint32_t *__restrict__ tid_next, SpawnArgs sp,
        OrdArgs oa) {
  const uint32_t *__restrict__ ord = oa.ord;
  __shared__ unsigned long long s_win;
  if (threadIdx.x == 0) s_win = 0;
  __syncthreads();
  const LevelDesc d = desc[lev];
  if (d.mode != kModeSrs) return;
  const uint32_t n = d.n, r = d.r;
  const uint64_t R = (uint64_t)r + d.k;
  Perm P;
  P.init(n, d.seed);
  const uint32_t lo = ord ? 0u : (uint32_t)(R * blockIdx.x / gridDim.x);
  const uint64_t hi = ord ? R : (uint32_t)(R * (blockIdx.x + 1) / gridDim.x);
  uint32_t *q = qctr + blockIdx.x;
  // the next position of this thread's ruler sequence: a ruler id, or (ORD)
  // an index of the ordered sequence
  auto take = [&]() -> uint64_t {
    if (ord) {
      bool refilled = false;
      const uint64_t j = ord_take(&s_win, qctr, R, &refilled);
      if (refilled && oa.pf_lead && j >= d.k && j < R) {
        // the CTA took the rulers from j on: bring the records of the
        // elements up to its next draw's first ruler, pf_lead elements ahead,
        // into L2 before the front reaches them
        const uint64_t a = (uint64_t)__ldcg(ord + (j - d.k)) + oa.pf_lead;
        const uint64_t jb = j - d.k + kOrdChunk;
        const uint64_t b = (jb < r ? (uint64_t)__ldcg(ord + jb) : (uint64_t)n) + oa.pf_lead;
        if (a < n && b > a) {
          const uintptr_t pa = ((uintptr_t)(work + a) + 15u) & ~(uintptr_t)15u;
          const uintptr_t pb = (uintptr_t)(work + (b < n ? b : n)) & ~(uintptr_t)15u;
          if (pb > pa && pb - pa <= (1u << 20))
            asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" :: "l"(pa), "r"((uint32_t)(pb - pa)) : "memory");
        }
      }
      return j;
    }
    return (uint64_t)lo + atomicAdd(q, 1u);
  };
  auto ord_pos = [&](uint64_t j) -> uint32_t {
    return (j >= d.k && j < R) ? __ldcg(ord + (j - d.k)) : 0u;
  };
  const uint32_t ncap = desc[lev + 1].cap;             // records of the next level (debug checks)
  uint32_t visited = 0, bad = 0;
  uint32_t myid = kEnd;                                  // SPAWN: reserved, not yet claimed
  const uint32_t slo = (uint32_t)((uint64_t)n * blockIdx.x / gridDim.x);
  const uint32_t shi = (uint32_t)((uint64_t)n * (blockIdx.x + 1) / gridDim.x);
  uint64_t c64 = take();
  uint32_t xo = ord ? ord_pos(c64) : 0u;                 // ORD: position of c64's ruler, loaded ahead
  for (;;) {
    uint32_t c, rho;
    Rec v;
    if (c64 < hi) {
      const uint64_t cnext = take();
      if (!ord) {
        c = (uint32_t)c64;
        rho = c < r ? P.inv(c) : __ldcg(ns + (c - r));
      } else if (c64 < d.k) {
        c = r + (uint32_t)c64;
        rho = __ldcg(ns + c64);
        xo = ord_pos(cnext);
      } else {
        rho = xo;
        c = (uint32_t)(c64 - d.k);
        xo = ord_pos(cnext);
      }
      c64 = cnext;
      if (dbg_fail(rho < n && c < ncap, err)) continue;
      v = visit<XCHG>(work + rho, c, 0);
      if constexpr (SPAWN) {
        if (rec_is_claim(v)) {                           // a spawner took this head first
          const uint32_t cs = rec_tag(v);
          st_rec(work + rho, cs, 0);                     // it stays the spawned ruler's
          __stcg(reinterpret_cast<uint4 *>(next + c), make_uint4(cs, kUnvisited, 0u, 0u));
          continue;
        }
      }
    } else if constexpr (SPAWN) {
      bool got = false;
      for (;;) {
        if (myid == kEnd) {
          const uint32_t k = atomicAdd(sp.ctr, 1u);
          if (k >= sp.cap) break;                        // out of ids: the wave dies
          myid = (uint32_t)R + k;
        }
        const uint32_t u = slo + atomicAdd(sp.cursor + blockIdx.x, 1u);
        if (u >= shi) break;                             // nothing unvisited left here
        if (P.fwd(u) < r) continue;                      // a sampled ruler: the queue chases it
        if (rec_tag(ld_rec(work + u)) != kUnvisited) continue;
        const Rec old = claim_rec(work + u, myid);
        if (rec_tag(old) != kUnvisited) { st_raw(work + u, old); continue; }   // lost it: put it back
        const uint32_t k = myid - (uint32_t)R;
        atomicOr(sp.used + (k >> 5), 1u << (k & 31u));
        c = myid;
        rho = u;
        v = old;
        myid = kEnd;
        got = true;
        break;
      }
      if (!got) break;
    } else {
      break;
    }
    uint64_t o = rec_weight(v, rho);
    uint32_t steps = 1, nxt = c;
    bad |= rec_tag(v) != kUnvisited;
    uint32_t y = rec_succ(v);
    uint32_t tend = (TERM && y == rho && rec_tag(v) == kUnvisited) ? rho : kEnd;
    if (y != rho && rec_tag(v) == kUnvisited) {
      for (;;) {
        if (y >= n) { bad |= 4u; break; }   // never produced by prep or a chase
        const uint32_t p = P.fwd(y);
        if (p < r) {                 // reached the next ruler
          nxt = ord ? ord_id(oa.bits, oa.cum, y) : p;
          if (dbg_fail(nxt < r, err)) nxt = c;
          if (nxt == c) bad |= 2u;   // came back to itself: a cycle
          break;
        }
        v = visit<XCHG>(work + y, c, o);
        if constexpr (SPAWN) {
          if (rec_is_claim(v)) {     // reached a spawned ruler
            const uint32_t cs = rec_tag(v);
            st_rec(work + y, cs, 0);
            nxt = cs;
            if (cs == c) bad |= 2u;  // its own: a cycle
            break;
          }
        }
        ++steps;
        if (rec_tag(v) != kUnvisited) { bad |= 1u; break; }   // second predecessor
        o += rec_weight(v, y);
        const uint32_t s = rec_succ(v);
        if (s == y) {                // terminal: the reduced element is terminal too
          if constexpr (TERM) tend = y;
          break;
        }
        if (steps > n) { bad |= 2u; break; }
        y = s;
      }
    }
    __stcg(reinterpret_cast<uint4 *>(next + c),
           make_uint4(nxt, kUnvisited, (uint32_t)o, (uint32_t)(o >> 32)));
    if constexpr (TERM) {
      if (tend != kEnd) tid_next[c] = tid_cur ? __ldcg(tid_cur + tend) : tend;
    }
    visited += steps;
  }
  if (bad & 1u) record_error(err, kErrNotList);
  if (bad & 2u) record_error(err, kErrCycle);
  if (bad & 4u) record_error(err, kErrInternal);
  for (int dd = 16; dd > 0; dd >>= 1) visited += __shfl_down_sync(0xFFFFFFFFu, visited, dd);
  if ((threadIdx.x & 31) == 0 && visited) atomicAdd(&desc[lev].visited, visited);
}

cudaError_t launch_chase(LevelDesc *desc, int lev, void *work, bool rec16, void *next_work,
                         const uint32_t *ns, uint32_t *qctr, int grid, int block, uint32_t *err,
                         int xchg, const uint32_t *tid_cur, uint32_t *tid_next, const SpawnArgs *spawn,
                         const OrdArgs *ord, cudaStream_t s) {
  if (ord && spawn) return cudaErrorInvalidValue;   // spawning needs the per-CTA slices
  Rec16 *nx = reinterpret_cast<Rec16 *>(next_work);
  SpawnArgs sp;
  memset(&sp, 0, sizeof(sp));
  if (spawn) sp = *spawn;
  OrdArgs oa;
  memset(&oa, 0, sizeof(oa));
  if (ord) oa = *ord;
#define LR_CHASE(REC, X, T, SP) \
  k_chase<REC, X, T, SP><<<grid, block, 0, s>>>(desc, lev, reinterpret_cast<REC *>(work), nx, ns, qctr, err, \
                                                tid_cur, tid_next, sp, oa)
  if (spawn) {
    if (rec16) LR_CHASE(Rec16, true, false, true);
    else LR_CHASE(Rec8, true, false, true);
  } else if (tid_next) {
    if (rec16) { if (xchg) LR_CHASE(Rec16, true, true, false); else LR_CHASE(Rec16, false, true, false); }
    else { if (xchg) LR_CHASE(Rec8, true, true, false); else LR_CHASE(Rec8, false, true, false); }
  } else {
    if (rec16) { if (xchg) LR_CHASE(Rec16, true, false, false); else LR_CHASE(Rec16, false, false, false); }
    else { if (xchg) LR_CHASE(Rec8, true, false, false); else LR_CHASE(Rec8, false, false, false); }
  }
#undef LR_CHASE
  count_launch();
  return cudaGetLastError();
}

int chase_occupancy(bool rec16, int block) {
  int nb = 0;
  if (rec16) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_chase<Rec16, false, false, false>, block, 0);
  else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_chase<Rec8, false, false, false>, block, 0);
  return nb > 0 ? nb : 1;
}

// ---------------------------------------------------------------- finalize
template <class RT>
__device__ __forceinline__ RT propagate(uint32_t c, uint64_t o, uint32_t nn, const RT *rnext,
                                        uint32_t &bad) {
  RT base = 0;
  if (c < nn) base = __ldcg(rnext + c);
  else if (c != kZeroCid) bad |= c == kUnvisited ? kErrCycle : kErrInternal;
  return (RT)(base - (RT)o);
}

// Terminal of element i at this level: its ruler's, or its own original id
// for a resolved singleton (a head that is its own terminal).
__device__ __forceinline__ uint32_t propagate_term(uint32_t c, uint32_t i, uint32_t nn,
                                                   const uint32_t *tnext, const uint32_t *tid_cur) {
  if (c < nn) return __ldcg(tnext + c);
  if (c == kZeroCid) return tid_cur ? __ldcg(tid_cur + i) : i;
  return kEnd;
}

// A record's last read (evict-first: the lines it frees in L2 serve the
// gathers of the next level's ranks).
template <class Rec>
__device__ __forceinline__ Rec ld_rec_last(const Rec *p) {
  Rec r;
  if constexpr (sizeof(Rec) == 8) {
    const uint2 a = __ldcs(reinterpret_cast<const uint2 *>(p));
    r.lo = a.x;
    r.hi = a.y;
  } else {
    const uint4 a = __ldcs(reinterpret_cast<const uint4 *>(p));
    r.succ = a.x;
    r.tag = a.y;
    r.w = ((uint64_t)a.w << 32) | a.z;
  }
  return r;
}

// Ruler propagation: every element gets its ruler's rank minus its offset
// (TERM: and its ruler's terminal).
template <class Rec, class RT, bool TERM>
__global__ void __launch_bounds__(256)
k_finalize(const LevelDesc *__restrict__ desc, int lev, const Rec *__restrict__ work,
           const RT *__restrict__ rnext, RT *__restrict__ rout, uint32_t *__restrict__ err,
           const uint32_t *__restrict__ tnext, uint32_t *__restrict__ tout,
           const uint32_t *__restrict__ tid_cur) {
  const LevelDesc d = desc[lev];
  if (d.mode != kModeSrs) return;
  const uint32_t n = d.n, nn = d.nraw ? d.nraw : desc[lev + 1].n;
  uint32_t bad = 0;
  if (blockIdx.x == 0 && threadIdx.x == 0 && d.visited != n) bad |= kErrCycle;
  // each warp takes 128 consecutive elements at a time and lane l the
  // elements base + l + 32 j: every record load and rank store of the warp
  // is one contiguous run, and a lane's four gathers are in flight together
  const uint32_t lane = threadIdx.x & 31u;
  const uint64_t warp = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint64_t step = ((uint64_t)gridDim.x * blockDim.x >> 5) * 128u;
  for (uint64_t base = warp * 128u; base < n; base += step) {
    Rec v[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const uint64_t i = base + lane + 32u * j;
      if (i < n) v[j] = ld_rec_last(work + i);
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const uint64_t i = base + lane + 32u * j;
      if (i < n) {
        const RT r = propagate<RT>(done_cid(v[j]), done_off(v[j]), nn, rnext, bad);
        if constexpr (TERM) __stcs(tout + i, propagate_term(done_cid(v[j]), (uint32_t)i, nn, tnext, tid_cur));
        __stcs(rout + i, r);
      }
    }
  }
  if (bad) record_error(err, bad);
}

// Level-0 propagation into per-instance output buffers.
template <class Rec, class RT>
__global__ void __launch_bounds__(256)
k_finalize_ptrs(const LevelDesc *__restrict__ desc, const Rec *__restrict__ work,
                const RT *__restrict__ rnext, RT *const *__restrict__ rptr,
                const int64_t *__restrict__ offsets, int32_t k, uint32_t *__restrict__ err) {
  const LevelDesc d = desc[0];
  if (d.mode != kModeSrs) return;
  const uint32_t n = d.n, nn = desc[1].n;
  uint32_t bad = 0;
  if (blockIdx.x == 0 && threadIdx.x == 0 && d.visited != n) bad |= kErrCycle;
  // each warp takes 128 consecutive elements (lane l: l + 32 j, coalesced
  // record loads and rank stores); the four records, then the four gathers
  // of the next level's ranks are in flight together, and the instances are
  // found meanwhile (the warp's first by a warp-wide search, the others by
  // walking forward from it).  Element ids and offsets fit 32 bits here.
  const uint32_t lane = threadIdx.x & 31u;
  const uint64_t warp = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint64_t step = ((uint64_t)gridDim.x * blockDim.x >> 5) * 128u;
  for (uint64_t b64 = warp * 128u; b64 < n; b64 += step) {
    const uint32_t base = (uint32_t)b64, rem = n - base;
    Rec v[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const uint32_t t = lane + 32u * j;
      if (t < rem) v[j] = ld_rec_last(work + base + t);
    }
    RT val[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      if (lane + 32u * j < rem) val[j] = propagate<RT>(done_cid(v[j]), done_off(v[j]), nn, rnext, bad);
    }
    int32_t lo = warp_instance(offsets, k, base, lane);
    uint32_t ib = (uint32_t)__ldg(offsets + lo), ie = (uint32_t)__ldg(offsets + lo + 1);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const uint32_t t = lane + 32u * j;
      if (t < rem) {
        const uint32_t i = base + t;
        while (i >= ie && lo + 1 < k) { ++lo; ib = ie; ie = (uint32_t)__ldg(offsets + lo + 1); }
        __stcs(rptr[lo] + (i - ib), val[j]);
      }
    }
  }
  if (bad) record_error(err, bad);
}

cudaError_t launch_finalize_ptrs(LevelDesc *desc, const void *work, bool rec16, const void *rnext,
                                 void *const *rptr, int rank_bytes, uint32_t cap,
                                 const int64_t *offsets, int32_t k, uint32_t *err, cudaStream_t s) {
  const int block = 256;
  const int grid = stream_grid(((uint64_t)cap + 3) / 4, block);
#define LR_FINP(REC, RT)                                                                          \
  k_finalize_ptrs<REC, RT><<<grid, block, 0, s>>>(desc, reinterpret_cast<const REC *>(work),      \
                                                  reinterpret_cast<const RT *>(rnext),            \
                                                  reinterpret_cast<RT *const *>(rptr), offsets, k, err)
  if (rec16) { if (rank_bytes == 4) LR_FINP(Rec16, uint32_t); else LR_FINP(Rec16, unsigned long long); }
  else { if (rank_bytes == 4) LR_FINP(Rec8, uint32_t); else LR_FINP(Rec8, unsigned long long); }
#undef LR_FINP
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_finalize(LevelDesc *desc, int lev, const void *work, bool rec16,
                            const void *rnext, void *rout, int rank_bytes, uint32_t cap,
                            uint32_t *err, const uint32_t *tnext, uint32_t *tout,
                            const uint32_t *tid_cur, cudaStream_t s) {
  const int block = 256;
  const int grid = stream_grid(((uint64_t)cap + 3) / 4, block);
#define LR_FIN(REC, RT, T)                                                                      \
  k_finalize<REC, RT, T><<<grid, block, 0, s>>>(desc, lev, reinterpret_cast<const REC *>(work), \
                                                reinterpret_cast<const RT *>(rnext),            \
                                                reinterpret_cast<RT *>(rout), err, tnext,       \
                                                tout, tid_cur)
  if (tout) {
    if (rec16) { if (rank_bytes == 4) LR_FIN(Rec16, uint32_t, true); else LR_FIN(Rec16, unsigned long long, true); }
    else { if (rank_bytes == 4) LR_FIN(Rec8, uint32_t, true); else LR_FIN(Rec8, unsigned long long, true); }
  } else {
    if (rec16) { if (rank_bytes == 4) LR_FIN(Rec16, uint32_t, false); else LR_FIN(Rec16, unsigned long long, false); }
    else { if (rank_bytes == 4) LR_FIN(Rec8, uint32_t, false); else LR_FIN(Rec8, unsigned long long, false); }
  }
#undef LR_FIN
  count_launch();
  return cudaGetLastError();
}

// ---------------------------------------------------------------- spawning: compaction
// Spawned ruler ids R + k that were handed out but never claimed leave holes.
// The next level is compacted: id c keeps c below R, and a claimed spawned
// id R + k becomes R + (claimed spawned ids before it).  The ranks are
// scattered back to the original ids before this level's propagation.
__device__ __forceinline__ uint32_t spawn_map(uint32_t c, uint32_t R, const uint32_t *used,
                                              const uint32_t *upre) {
  if (c < R) return c;
  const uint32_t k = c - R;
  return R + __ldg(upre + (k >> 5)) + (uint32_t)__popc(__ldcg(used + (k >> 5)) & ((1u << (k & 31u)) - 1u));
}

// Prefix of the claimed-id bitmap (one CTA) and the next level's size and mode.
__global__ void __launch_bounds__(1024)
k_spawn_scan(LevelDesc *desc, int lev, int nlev, const uint32_t *__restrict__ ctr, uint32_t cap,
             const uint32_t *__restrict__ used, uint32_t *__restrict__ upre, uint32_t cutoff,
             uint32_t has_pd, uint32_t *__restrict__ err) {
  __shared__ uint64_t sm[33];
  LevelDesc &d = desc[lev];
  if (d.mode != kModeSrs) return;
  const uint32_t handed = min(*ctr, cap);
  const uint32_t words = (handed + 31) / 32;
  const uint32_t per = (words + blockDim.x - 1) / blockDim.x;
  const uint32_t a = threadIdx.x * per, b = min(words, a + per);
  uint64_t s = 0;
  for (uint32_t w = a; w < b; ++w) s += __popc(used[w]);
  uint64_t total;
  uint64_t run = block_exclusive_scan(s, sm, &total);
  for (uint32_t w = a; w < b; ++w) { upre[w] = (uint32_t)run; run += __popc(used[w]); }
  if (threadIdx.x == 0) {
    LevelDesc &e = desc[lev + 1];
    const uint64_t R = (uint64_t)d.r + d.k;
    const uint64_t n1 = R + total;
    d.nraw = (uint32_t)(R + handed);
    if (n1 > e.cap) { record_error(err, kErrCapacity); d.mode = kModeOff; return; }
    uint32_t mode = kModeSrs;
    if (n1 <= cutoff) mode = kModeBase;
    else if (lev + 1 >= nlev - 1) { if (has_pd) mode = kModePd; else { record_error(err, kErrCapacity); d.mode = kModeOff; return; } }
    e.n = (uint32_t)n1;
    e.r = (uint32_t)((n1 + e.f_inv - 1) / e.f_inv);
    e.mode = mode;
  }
}

// The next level's records at compacted ids, successors remapped.
__global__ void k_spawn_compact(const LevelDesc *__restrict__ desc, int lev, const Rec16 *__restrict__ raw,
                                Rec16 *__restrict__ out, const uint32_t *__restrict__ used,
                                const uint32_t *__restrict__ upre) {
  const LevelDesc d = desc[lev];
  if (d.mode != kModeSrs || d.nraw == 0) return;
  const uint32_t R = d.r + d.k;
  for (uint32_t c = blockIdx.x * blockDim.x + threadIdx.x; c < d.nraw; c += gridDim.x * blockDim.x) {
    if (c >= R && !((__ldcg(used + ((c - R) >> 5)) >> ((c - R) & 31u)) & 1u)) continue;   // a hole
    const uint4 v = __ldcg(reinterpret_cast<const uint4 *>(raw + c));
    const uint32_t s = v.x < d.nraw ? spawn_map(v.x, R, used, upre) : v.x;
    __stcg(reinterpret_cast<uint4 *>(out + spawn_map(c, R, used, upre)), make_uint4(s, v.y, v.z, v.w));
  }
}

// Ranks of the compacted next level back at the original ids.
template <class RT>
__global__ void k_spawn_scatter(const LevelDesc *__restrict__ desc, int lev, const RT *__restrict__ rc,
                                RT *__restrict__ rraw, const uint32_t *__restrict__ used,
                                const uint32_t *__restrict__ upre) {
  const LevelDesc d = desc[lev];
  if (d.mode != kModeSrs || d.nraw == 0) return;
  const uint32_t R = d.r + d.k;
  for (uint32_t c = blockIdx.x * blockDim.x + threadIdx.x; c < d.nraw; c += gridDim.x * blockDim.x) {
    if (c >= R && !((__ldcg(used + ((c - R) >> 5)) >> ((c - R) & 31u)) & 1u)) continue;
    rraw[c] = __ldcg(rc + spawn_map(c, R, used, upre));
  }
}

cudaError_t launch_spawn_compact(LevelDesc *desc, int lev, int nlev, const uint32_t *ctr, uint32_t cap,
                                 const uint32_t *used, uint32_t *upre, const void *raw, void *out,
                                 uint32_t raw_cap, uint32_t cutoff, uint32_t has_pd, uint32_t *err,
                                 cudaStream_t s) {
  k_spawn_scan<<<1, 1024, 0, s>>>(desc, lev, nlev, ctr, cap, used, upre, cutoff, has_pd, err);
  k_spawn_compact<<<stream_grid(raw_cap, 256), 256, 0, s>>>(desc, lev, reinterpret_cast<const Rec16 *>(raw),
                                                           reinterpret_cast<Rec16 *>(out), used, upre);
  count_launch(2);
  return cudaGetLastError();
}

cudaError_t launch_spawn_scatter(LevelDesc *desc, int lev, const void *rc, void *rraw, int rank_bytes,
                                 const uint32_t *used, const uint32_t *upre, uint32_t raw_cap,
                                 cudaStream_t s) {
  const int grid = stream_grid(raw_cap, 256);
  if (rank_bytes == 4)
    k_spawn_scatter<uint32_t><<<grid, 256, 0, s>>>(desc, lev, reinterpret_cast<const uint32_t *>(rc),
                                                   reinterpret_cast<uint32_t *>(rraw), used, upre);
  else
    k_spawn_scatter<unsigned long long><<<grid, 256, 0, s>>>(
        desc, lev, reinterpret_cast<const unsigned long long *>(rc),
        reinterpret_cast<unsigned long long *>(rraw), used, upre);
  count_launch();
  return cudaGetLastError();
}

// ---------------------------------------------------------------- extra outputs (level 0)
// The paper's output also names each element's terminal (Section 1.1) and
// its in-place form counts the terminal's own weight; the head-relative
// (prefix) rank is the list's total minus the rank.  term[] holds global
// terminal ids when these passes run.
//
// Head pass: the total of each list (the rank of its head) is stored at its
// terminal's entry of prefix.
template <class RT>
__global__ void __launch_bounds__(kHeadThreads)
k_out_heads(const LevelDesc *__restrict__ desc, const uint32_t *__restrict__ bitmap,
            const uint32_t *__restrict__ hlist, const uint32_t *__restrict__ term,
            const RT *__restrict__ rank, RT *__restrict__ prefix) {
  const LevelDesc d = desc[0];
  for_each_head(d, bitmap, hlist, [&](uint32_t h) {
    const uint32_t t = __ldcg(term + h);
    if (t < d.n) prefix[t] = __ldcg(rank + h);
  });
}

// Streaming pass: prefix[i] = total - rank[i] (a terminal's entry holds the
// total and keeps it, its rank being 0, so the pass may run in place); the
// inclusive form adds the terminal's weight (weighted input only: unweighted,
// the terminal weighs 0, Section 1.1); in the batched form terminal ids
// become local to their instance.
template <class RT>
__global__ void __launch_bounds__(256)
k_out_fix(uint32_t n, uint32_t *__restrict__ term, RT *__restrict__ rank, RT *__restrict__ prefix,
          int incl, const void *__restrict__ weight, int wtype, const int64_t *__restrict__ offsets,
          int32_t k, int local) {
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const uint32_t t = term[i];
    if (t >= n) continue;                       // an error the device already recorded
    const RT r = rank[i];
    if (prefix) prefix[i] = (RT)(__ldcg(prefix + t) - r);
    if (incl) {
      uint64_t wt = 0u;
      if (wtype == 1) wt = (uint64_t)(int64_t)__ldg(reinterpret_cast<const int *>(weight) + t);
      else if (wtype == 2) wt = (uint64_t)__ldg(reinterpret_cast<const long long *>(weight) + t);
      rank[i] = (RT)(r + (RT)wt);
    }
    if (local) {
      int32_t lo = 0, hi = k;
      while (hi - lo > 1) {
        const int32_t mid = (lo + hi) >> 1;
        if ((uint64_t)__ldg(offsets + mid) <= i) lo = mid; else hi = mid;
      }
      term[i] = (uint32_t)(t - (uint64_t)__ldg(offsets + lo));
    }
  }
}

cudaError_t launch_outputs(const LevelDesc *desc, const uint32_t *bitmap, const uint32_t *hlist0,
                           uint32_t n, uint32_t *term, void *rank, void *prefix, int rank_bytes,
                           int incl, const void *weight, int wtype, const int64_t *offsets, int32_t k,
                           int local, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  if (wtype == 0) incl = 0;                     // an unweighted terminal weighs 0
  const int grid = stream_grid(n, 256);
  int launches = 0;
  if (rank_bytes == 4) {
    uint32_t *r = reinterpret_cast<uint32_t *>(rank), *p = reinterpret_cast<uint32_t *>(prefix);
    if (p) { k_out_heads<uint32_t><<<kHeadBlocks, kHeadThreads, 0, s>>>(desc, bitmap, hlist0, term, r, p); ++launches; }
    if (p || incl || local) { k_out_fix<uint32_t><<<grid, 256, 0, s>>>(n, term, r, p, incl, weight, wtype, offsets, k, local); ++launches; }
  } else {
    unsigned long long *r = reinterpret_cast<unsigned long long *>(rank);
    unsigned long long *p = reinterpret_cast<unsigned long long *>(prefix);
    if (p) { k_out_heads<unsigned long long><<<kHeadBlocks, kHeadThreads, 0, s>>>(desc, bitmap, hlist0, term, r, p); ++launches; }
    if (p || incl || local) { k_out_fix<unsigned long long><<<grid, 256, 0, s>>>(n, term, r, p, incl, weight, wtype, offsets, k, local); ++launches; }
  }
  count_launch(launches);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- base case
// Pointer doubling (Wyllie) inside one CTA: nxt/val live in shared memory;
// every round each element adds its successor's value and jumps to its
// successor's successor, reading the old values before anyone writes.
// Values are inclusive (a terminal starts with its own weight), so after
// ceil(log2 n) rounds val[i] is the rank of i at this level.
// With tout, term[] follows the same rounds: a terminal starts with its
// original id (tid, or its own index at level 0) and every other element
// with kEnd; an element takes its successor's entry, which is known exactly
// when that successor has reached the end, i.e. when the element does.
template <class Rec, class RT>
__global__ void __launch_bounds__(kBaseThreads)
k_base(LevelDesc *__restrict__ desc, int lev, const Rec *__restrict__ work, RT *__restrict__ rout,
       uint32_t *__restrict__ err, const uint32_t *__restrict__ tid, uint32_t *__restrict__ tout) {
  extern __shared__ unsigned char smem_raw[];
  LevelDesc &d = desc[lev];
  if (d.mode != kModeBase) return;
  const uint32_t n = d.n;
  const bool with_term = tout != nullptr;
  uint32_t *nxt = reinterpret_cast<uint32_t *>(smem_raw);
  RT *val = reinterpret_cast<RT *>(smem_raw + ((kMaxCutoff * 4 + 15) & ~15));
  uint32_t *term = reinterpret_cast<uint32_t *>(reinterpret_cast<unsigned char *>(val) + (size_t)kMaxCutoff * sizeof(RT));
  constexpr int PER = (kMaxCutoff + kBaseThreads - 1) / kBaseThreads;
  for (uint32_t j = threadIdx.x; j < n; j += blockDim.x) {
    Rec v = ld_rec(work + j);
    const uint32_t s = rec_succ(v);
    nxt[j] = (s == j || s >= n) ? kEnd : s;
    val[j] = (RT)rec_weight(v, j);
    if (with_term) term[j] = s == j ? (tid ? __ldcg(tid + j) : j) : kEnd;
    if (s >= n) record_error(err, kErrInternal);
  }
  __syncthreads();
  uint32_t rounds = 0;
  while ((1ull << rounds) < n) ++rounds;
  for (uint32_t it = 0; it < rounds; ++it) {
    uint32_t tn[PER], tt[PER];
    RT tv[PER];
#pragma unroll
    for (int e = 0; e < PER; ++e) {
      const uint32_t j = threadIdx.x + e * kBaseThreads;
      if (j < n) {
        const uint32_t a = nxt[j];
        if (a != kEnd) {
          tv[e] = val[j] + val[a];
          tn[e] = nxt[a];
          tt[e] = with_term ? term[a] : 0u;
        } else {
          tv[e] = val[j];
          tn[e] = kEnd;
          tt[e] = with_term ? term[j] : 0u;
        }
      }
    }
    __syncthreads();
#pragma unroll
    for (int e = 0; e < PER; ++e) {
      const uint32_t j = threadIdx.x + e * kBaseThreads;
      if (j < n) {
        nxt[j] = tn[e];
        val[j] = tv[e];
        if (with_term) term[j] = tt[e];
      }
    }
    __syncthreads();
  }
  uint32_t bad = 0;
  for (uint32_t j = threadIdx.x; j < n; j += blockDim.x) {
    if (nxt[j] != kEnd) bad = 1;
    rout[j] = val[j];
    if (with_term) tout[j] = term[j];
  }
  if (bad) record_error(err, kErrCycle);
  if (threadIdx.x == 0) d.visited = n;
}

static size_t base_smem(int rank_bytes) {
  // nxt, val and the terminal ids of up to kMaxCutoff elements
  return ((kMaxCutoff * 4 + 15) & ~15) + (size_t)kMaxCutoff * rank_bytes + (size_t)kMaxCutoff * 4;
}

cudaError_t launch_base(LevelDesc *desc, int lev, const void *work, bool rec16, void *rout,
                        int rank_bytes, uint32_t cutoff, uint32_t *err, const uint32_t *tid,
                        uint32_t *tout, cudaStream_t s) {
  (void)cutoff;
  const size_t sm = base_smem(rank_bytes);
#define LR_BASE(REC, RT)                                                                         \
  k_base<REC, RT><<<1, kBaseThreads, sm, s>>>(desc, lev, reinterpret_cast<const REC *>(work), \
                                              reinterpret_cast<RT *>(rout), err, tid, tout)
  if (rec16) { if (rank_bytes == 4) LR_BASE(Rec16, uint32_t); else LR_BASE(Rec16, unsigned long long); }
  else { if (rank_bytes == 4) LR_BASE(Rec8, uint32_t); else LR_BASE(Rec8, unsigned long long); }
#undef LR_BASE
  count_launch();
  return cudaGetLastError();
}

// ---------------------------------------------------------------- grid-wide pointer doubling
// Fallback base case for a last level larger than one CTA can hold (many
// lists whose heads keep the levels from shrinking).  Same rounds as the
// single-CTA version, one kernel per round, ping-pong buffers.
// With term arrays (t0/t1 non-null) the terminal ids follow the rounds as in
// the single-CTA base case.
__global__ void k_pd_init(const LevelDesc *__restrict__ desc, int lev, const Rec16 *__restrict__ work,
                          uint32_t *__restrict__ nxt, uint64_t *__restrict__ val,
                          const uint32_t *__restrict__ tid, uint32_t *__restrict__ term) {
  const LevelDesc d = desc[lev];
  if (d.mode != kModePd) return;
  for (uint32_t j = blockIdx.x * blockDim.x + threadIdx.x; j < d.n; j += gridDim.x * blockDim.x) {
    Rec16 v = ld_rec(work + j);
    nxt[j] = (v.succ == j || v.succ >= d.n) ? kEnd : v.succ;
    val[j] = v.w;
    if (term) term[j] = v.succ == j ? (tid ? __ldcg(tid + j) : j) : kEnd;
  }
}

__global__ void k_pd_round(const LevelDesc *__restrict__ desc, int lev, const uint32_t *__restrict__ nin,
                           const uint64_t *__restrict__ vin, uint32_t *__restrict__ nout,
                           uint64_t *__restrict__ vout, const uint32_t *__restrict__ tin,
                           uint32_t *__restrict__ tout) {
  const LevelDesc d = desc[lev];
  if (d.mode != kModePd) return;
  for (uint32_t j = blockIdx.x * blockDim.x + threadIdx.x; j < d.n; j += gridDim.x * blockDim.x) {
    const uint32_t a = nin[j];
    if (a != kEnd) {
      vout[j] = vin[j] + vin[a];
      nout[j] = nin[a];
      if (tout) tout[j] = tin[a];
    } else {
      vout[j] = vin[j];
      nout[j] = kEnd;
      if (tout) tout[j] = tin[j];
    }
  }
}

template <class RT>
__global__ void k_pd_out(LevelDesc *__restrict__ desc, int lev, const uint32_t *__restrict__ nxt,
                         const uint64_t *__restrict__ val, RT *__restrict__ rout, uint32_t *__restrict__ err,
                         const uint32_t *__restrict__ term, uint32_t *__restrict__ tout) {
  const LevelDesc d = desc[lev];
  if (d.mode != kModePd) return;
  uint32_t bad = 0;
  for (uint32_t j = blockIdx.x * blockDim.x + threadIdx.x; j < d.n; j += gridDim.x * blockDim.x) {
    bad |= nxt[j] != kEnd;
    rout[j] = (RT)val[j];
    if (tout) tout[j] = term[j];
  }
  if (bad) record_error(err, kErrCycle);
  if (blockIdx.x == 0 && threadIdx.x == 0) desc[lev].visited = d.n;
}

cudaError_t launch_pd(LevelDesc *desc, int lev, const void *work, uint32_t cap, uint32_t rounds,
                      uint32_t *nxt0, uint32_t *nxt1, uint64_t *val0, uint64_t *val1, void *rout,
                      int rank_bytes, uint32_t *err, const uint32_t *tid, uint32_t *t0, uint32_t *t1,
                      uint32_t *tout, cudaStream_t s) {
  const int block = 256;
  const int grid = stream_grid(cap, block);
  if (!tout) t0 = t1 = nullptr;
  k_pd_init<<<grid, block, 0, s>>>(desc, lev, reinterpret_cast<const Rec16 *>(work), nxt0, val0, tid, t0);
  uint32_t *na = nxt0, *nb = nxt1, *ta = t0, *tb = t1;
  uint64_t *va = val0, *vb = val1;
  for (uint32_t it = 0; it < rounds; ++it) {
    k_pd_round<<<grid, block, 0, s>>>(desc, lev, na, va, nb, vb, ta, tb);
    uint32_t *tn = na; na = nb; nb = tn;
    uint64_t *tv = va; va = vb; vb = tv;
    uint32_t *tt = ta; ta = tb; tb = tt;
  }
  if (rank_bytes == 4)
    k_pd_out<uint32_t><<<grid, block, 0, s>>>(desc, lev, na, va, reinterpret_cast<uint32_t *>(rout), err,
                                              ta, tout);
  else
    k_pd_out<unsigned long long><<<grid, block, 0, s>>>(desc, lev, na, va,
                                                        reinterpret_cast<unsigned long long *>(rout), err,
                                                        ta, tout);
  count_launch(2 + (int)rounds);
  return cudaGetLastError();
}

cudaError_t kernels_setup() {
  cudaError_t e;
  e = cudaFuncSetAttribute(k_base<Rec8, uint32_t>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)base_smem(4));
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_base<Rec8, unsigned long long>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)base_smem(8));
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_base<Rec16, uint32_t>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)base_smem(4));
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_base<Rec16, unsigned long long>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)base_smem(8));
}

}  // namespace lr
