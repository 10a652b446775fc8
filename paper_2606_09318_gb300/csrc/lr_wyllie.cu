// lr_wyllie.cu -- Wyllie pointer doubling over the whole list: the
// comparison algorithm of Sections 1 and 3 (the paper's PD), run as a second
// algorithm behind lr_tuning.algorithm = 1.
//
// State of element j after round r: nxt = its 2^r-th successor, or kEnd once
// that would lie past the terminal; val = sum of the link weights from j up
// to nxt (to the terminal once nxt == kEnd).  A round replaces (nxt, val) by
// (nxt[nxt], val + val[nxt]) from the previous round's array (double
// buffered, so every round reads one consistent state).  An element at
// distance d from its terminal reaches kEnd in the first round with 2^r > d,
// so after ceil(log2 n) rounds every element of a list has its rank and an
// element still short of kEnd lies on or leads into a cycle.
//
// One record per element holds both fields, so an active element costs one
// random gather per round (8 B records {nxt, val32} when unweighted, where a
// rank is at most n - 1 < 2^32; 16 B {nxt, -, val64} when weighted, the
// layout of k_prep0's records in either case); finished elements are copied
// without a gather.  The first round reads k_prep0's records (range-checked
// successors, weights with the terminal's set to 0) and converts them on the
// fly; the last round writes the ranks in the caller's type.
#include <cuda_runtime.h>

#include "lr_device.cuh"
#include "lr_kernels.h"

namespace lr {

// (nxt, val) of element j from a record of the previous round; in the first
// round the record is k_prep0's {succ, tag[, w]}, where succ == j marks the
// terminal.
template <bool W16, bool FIRST>
__device__ __forceinline__ void wy_decode(uint4 r, uint32_t j, uint32_t &nxt, uint64_t &val) {
  if constexpr (W16) {
    val = (uint64_t)r.z | ((uint64_t)r.w << 32);
    nxt = (FIRST && r.x == j) ? kEnd : r.x;
  } else if constexpr (FIRST) {
    nxt = r.x == j ? kEnd : r.x;
    val = r.x == j ? 0u : 1u;
  } else {
    nxt = r.x;
    val = r.y;
  }
}

template <bool W16>
__device__ __forceinline__ uint4 wy_load_stream(const void *p, uint32_t j) {
  if constexpr (W16) return __ldcs(reinterpret_cast<const uint4 *>(p) + j);
  const uint2 v = __ldcs(reinterpret_cast<const uint2 *>(p) + j);
  return make_uint4(v.x, v.y, 0u, 0u);
}

template <bool W16>
__device__ __forceinline__ uint4 wy_gather(const void *p, uint32_t a) {
  if constexpr (W16) return __ldcg(reinterpret_cast<const uint4 *>(p) + a);
  const uint2 v = __ldcg(reinterpret_cast<const uint2 *>(p) + a);
  return make_uint4(v.x, v.y, 0u, 0u);
}

template <bool W16, bool FIRST, bool LAST, class RT>
__global__ void __launch_bounds__(256)
k_wyllie(const void *__restrict__ src, void *__restrict__ dst, RT *__restrict__ rank, uint32_t n,
         uint32_t *__restrict__ err) {
  bool open = false;
  for (uint32_t j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
    uint32_t nj;
    uint64_t vj;
    wy_decode<W16, FIRST>(wy_load_stream<W16>(src, j), j, nj, vj);
    if (nj != kEnd) {
      uint32_t na;
      uint64_t va;
      wy_decode<W16, FIRST>(wy_gather<W16>(src, nj), nj, na, va);
      vj += va;
      nj = na;
    }
    if constexpr (LAST) {
      rank[j] = (RT)vj;
      open |= nj != kEnd;
    } else if constexpr (W16) {
      __stcs(reinterpret_cast<uint4 *>(dst) + j, make_uint4(nj, 0u, (uint32_t)vj, (uint32_t)(vj >> 32)));
    } else {
      __stcs(reinterpret_cast<uint2 *>(dst) + j, make_uint2(nj, (uint32_t)vj));
    }
  }
  if (open) record_error(err, kErrCycle);
}

template <bool W16, class RT>
static void wy_round(bool first, bool last, const void *src, void *dst, void *rank, uint32_t n,
                     uint32_t *err, int grid, cudaStream_t s) {
  RT *r = reinterpret_cast<RT *>(rank);
  if (first && last) k_wyllie<W16, true, true, RT><<<grid, 256, 0, s>>>(src, dst, r, n, err);
  else if (first) k_wyllie<W16, true, false, RT><<<grid, 256, 0, s>>>(src, dst, r, n, err);
  else if (last) k_wyllie<W16, false, true, RT><<<grid, 256, 0, s>>>(src, dst, r, n, err);
  else k_wyllie<W16, false, false, RT><<<grid, 256, 0, s>>>(src, dst, r, n, err);
}

uint32_t wyllie_rounds(uint64_t n) {
  uint32_t b = 0;
  while ((1ull << b) < n) ++b;
  return b < 1 ? 1u : b;
}

cudaError_t launch_wyllie(void *bufA, void *bufB, bool w16, uint32_t n, void *rank, int rank_bytes,
                          uint32_t *err, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  const uint32_t rounds = wyllie_rounds(n);
  const int grid = stream_grid(n, 256);
  void *src = bufA, *dst = bufB;
  for (uint32_t r = 0; r < rounds; ++r) {
    const bool first = r == 0, last = r + 1 == rounds;
    if (!w16 && rank_bytes == 4) wy_round<false, uint32_t>(first, last, src, dst, rank, n, err, grid, s);
    else if (!w16) wy_round<false, unsigned long long>(first, last, src, dst, rank, n, err, grid, s);
    else if (rank_bytes == 4) wy_round<true, uint32_t>(first, last, src, dst, rank, n, err, grid, s);
    else wy_round<true, unsigned long long>(first, last, src, dst, rank, n, err, grid, s);
    void *t = src; src = dst; dst = t;
  }
  count_launch((int)rounds);
  return cudaGetLastError();
}

}  // namespace lr
