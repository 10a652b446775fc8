// lr_device.cuh -- device-side definitions shared by the list-ranking kernels.
//
// Sparse ruling set on one GPU (Section 2.1, Algorithm 1 of "Engineering
// Scalable Distributed List Ranking"), restated for HBM:
//   level l works on n_l elements stored as fixed-size records;
//   rulers = heads (forced, Algorithm 1's ruler-selection step) plus the
//   elements x with pi_l(x) < r_l, where pi_l is a seeded bijection of
//   [0, n_l) and r_l = ceil(n_l / f_inv).  A sampled ruler's compact id is
//   pi_l(x) itself, so the hot loop tests "is y a ruler" and finds its id
//   with a few integer operations instead of a memory lookup.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace lr {

// ---------------------------------------------------------------- constants
constexpr uint32_t kUnvisited = 0xFFFFFFFFu;   // tag word of a record not yet chased
constexpr uint32_t kZeroCid = 0xFFFFFFFEu;     // "ruler" of a resolved singleton: R = 0
constexpr uint32_t kEnd = 0xFFFFFFFFu;         // no successor (pointer doubling)
constexpr int kMaxLevels = 12;                 // SRS levels in a static plan
constexpr int kHeadBlocks = 512;               // CTAs of the head-selection kernels
constexpr int kHeadThreads = 256;
constexpr int kBaseThreads = 1024;             // single-CTA base case
constexpr uint32_t kMaxCutoff = 12288;         // largest base-case level (SMEM bound)
constexpr int kContractTileShift = 12;         // tile-local contraction: tiles of 4096 ids

// error bits recorded on the device (mapped to lr_status by the host)
enum : uint32_t {
  kErrRange = 1u,      // successor out of range
  kErrCycle = 2u,      // an element unreachable from a head
  kErrNotList = 4u,    // an element with two predecessors
  kErrCapacity = 8u,   // more rulers than the static plan provided for
  kErrInternal = 16u,  // a record or id the pipeline never produces
  kErrDebug = 32u,     // a debug build's index check failed (LR_DEBUG)
};

// Debug build (-DLR_DEBUG, build.py's debug=True): the kernels check the
// indices they derive from their own structures (a ruler's position, a
// reduced record's id, a queue position) before using them; a failed check
// records kErrDebug and skips the access instead of faulting, which makes
// the build a stand-in for a memory checker.  Without LR_DEBUG every check
// folds away.
#ifdef LR_DEBUG
constexpr bool kDebugChecks = true;
#else
constexpr bool kDebugChecks = false;
#endif

// per-level mode, decided on the device by the previous level
enum : uint32_t { kModeOff = 0, kModeSrs = 1, kModeBase = 2, kModePd = 3 };

// Level descriptor (device memory).  n/r/mode of level l+1 are written by the
// head-selection scan of level l; the host writes level 0 and the static
// fields through the init kernel.
struct LevelDesc {
  uint32_t mode;
  uint32_t n;        // elements at this level
  uint32_t r;        // sampled rulers: ceil(n / f_inv)
  uint32_t k;        // extra rulers: heads that were not sampled and are not singletons
  uint32_t h;        // entries of this level's head list (levels >= 1)
  uint32_t visited;  // records written at this level (must end equal to n)
  uint32_t f_inv;    // static: 1/f
  uint32_t cap;      // static: capacity of this level's arrays
  uint64_t seed;     // static: permutation seed
  uint32_t rounds;   // static: pointer-doubling rounds of the fallback base
  uint32_t hsrc;     // where this level's heads come from: kHeadsBitmap or kHeadsList
  uint32_t nraw;     // with spawning: ruler ids of the next level before compaction (else 0)
};

enum : uint32_t { kHeadsBitmap = 0, kHeadsList = 1 };

// ---------------------------------------------------------------- permutation
// A keyed bijection of [0, 2^b) built from invertible steps (multiply by an
// odd constant, xor-shift by at least half the width, add and xor a key),
// restricted to [0, n) by cycle walking.  Host and device compute it alike.
__host__ __device__ inline uint64_t splitmix64(uint64_t x) {
  x += 0x9E3779B97F4A7C15ull;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  return x ^ (x >> 31);
}

__host__ __device__ inline uint32_t inverse_odd(uint32_t a) {
  uint32_t x = a;                 // correct to 3 bits; Newton doubles the bits
  for (int i = 0; i < 5; ++i) x *= 2u - a * x;
  return x;
}

struct Perm {
  uint32_t n, mask, s, a, ai, b, bi, k1, k2;

  __host__ __device__ void init(uint32_t n_, uint64_t seed) {
    n = n_;
    uint32_t bits = 1;
    while (bits < 32 && (1ull << bits) < (uint64_t)n_) ++bits;
    mask = bits >= 32 ? 0xFFFFFFFFu : ((1u << bits) - 1u);
    s = (bits + 1) / 2;
    uint64_t z0 = splitmix64(seed), z1 = splitmix64(seed ^ 0xA5A5A5A5DEADBEEFull);
    a = (uint32_t)z0 | 1u;
    b = (uint32_t)(z0 >> 32) | 1u;
    ai = inverse_odd(a);
    bi = inverse_odd(b);
    k1 = (uint32_t)z1 & mask;
    k2 = (uint32_t)(z1 >> 32) & mask;
  }
  __host__ __device__ uint32_t round_fwd(uint32_t x) const {
    x = (x * a) & mask;
    x ^= x >> s;
    x = (x + k1) & mask;
    x = (x * b) & mask;
    x ^= x >> s;
    return x ^ k2;
  }
  __host__ __device__ uint32_t round_inv(uint32_t y) const {
    y ^= k2;
    y ^= y >> s;                  // s >= bits/2: one step undoes the xor-shift
    y = (y * bi) & mask;
    y = (y - k1) & mask;
    y ^= y >> s;
    return (y * ai) & mask;
  }
  // pi(x) for x < n
  __host__ __device__ uint32_t fwd(uint32_t x) const {
    do { x = round_fwd(x); } while (x >= n);
    return x;
  }
  // pi^{-1}(y) for y < n
  __host__ __device__ uint32_t inv(uint32_t y) const {
    do { y = round_inv(y); } while (y >= n);
    return y;
  }
};

// ---------------------------------------------------------------- records
// Level-0 unweighted record, 8 bytes: before the chase {succ, tag=kUnvisited},
// after it {offset, ruler id}.  The chase reads and rewrites the same 8 bytes,
// so one element costs one 32-byte sector read and its write-back.
struct __align__(8) Rec8 {
  uint32_t lo;   // succ, then offset
  uint32_t hi;   // kUnvisited, then ruler id
};

// Weighted level-0 and all deeper levels, 16 bytes:
// before {succ, kUnvisited, weight}, after {0, ruler id, offset}.
struct __align__(16) Rec16 {
  uint32_t succ;
  uint32_t tag;
  uint64_t w;    // weight (wrapping), then offset
};

__device__ __forceinline__ void record_error(uint32_t *err, uint32_t bits) {
  atomicOr(err, bits);
}

// True (after recording kErrDebug) when a debug build's check fails.
__device__ __forceinline__ bool dbg_fail(bool ok, uint32_t *err) {
  if (kDebugChecks && !ok) {
    atomicOr(err, kErrDebug);
    return true;
  }
  return false;
}

// L2-only loads/stores for data with no reuse in L1.
__device__ __forceinline__ Rec8 ld_rec(const Rec8 *p) {
  uint2 v = __ldcg(reinterpret_cast<const uint2 *>(p));
  return Rec8{v.x, v.y};
}
__device__ __forceinline__ void st_rec(Rec8 *p, uint32_t cid, uint64_t off) {
  __stcg(reinterpret_cast<uint2 *>(p), make_uint2((uint32_t)off, cid));
}
__device__ __forceinline__ Rec16 ld_rec(const Rec16 *p) {
  uint4 v = __ldcg(reinterpret_cast<const uint4 *>(p));
  Rec16 r;
  r.succ = v.x;
  r.tag = v.y;
  r.w = ((uint64_t)v.w << 32) | v.z;
  return r;
}
__device__ __forceinline__ void st_rec(Rec16 *p, uint32_t cid, uint64_t off) {
  __stcg(reinterpret_cast<uint4 *>(p), make_uint4(0u, cid, (uint32_t)off, (uint32_t)(off >> 32)));
}
// One 32-byte store: a whole sector in a single request.  On GB300 two
// 16-byte stores to one sector cost two DRAM accesses; this costs one.
__device__ __forceinline__ void st_sector(void *p, uint32_t a, uint32_t b, uint32_t c, uint32_t d,
                                          uint32_t e, uint32_t f, uint32_t g, uint32_t h) {
  asm volatile("st.global.v8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};"
               :: "l"(p), "r"(a), "r"(b), "r"(c), "r"(d), "r"(e), "r"(f), "r"(g), "r"(h)
               : "memory");
}

// Swap in (ruler id, offset) and return the old record in one L2 atomic
// (8-byte records only).
__device__ __forceinline__ Rec8 xchg_rec(Rec8 *p, uint32_t cid, uint64_t off) {
  const unsigned long long nv = ((unsigned long long)cid << 32) | (uint32_t)off;
  const unsigned long long ov = atomicExch(reinterpret_cast<unsigned long long *>(p), nv);
  return Rec8{(uint32_t)ov, (uint32_t)(ov >> 32)};
}
// 16-byte records: one 128-bit atomic exchange at L2 (sm_90 and later).
__device__ __forceinline__ Rec16 xchg_rec(Rec16 *p, uint32_t cid, uint64_t off) {
  const unsigned long long nlo = (unsigned long long)cid << 32, nhi = off;
  unsigned long long olo, ohi;
  asm volatile("{\n\t.reg .b128 d, b;\n\tmov.b128 b, {%2, %3};\n\t"
               "atom.global.exch.b128 d, [%4], b;\n\tmov.b128 {%0, %1}, d;\n\t}"
               : "=l"(olo), "=l"(ohi) : "l"(nlo), "l"(nhi), "l"(p) : "memory");
  Rec16 r;
  r.succ = (uint32_t)olo;
  r.tag = (uint32_t)(olo >> 32);
  r.w = ohi;
  return r;
}

// Ruler spawning (Section 2.2).  A spawner claims an unvisited element as a
// new ruler c by exchanging in a claim mark, which no visited record can
// equal: an 8-byte record {offset, id} never carries offset 0xFFFFFFFF (an
// offset is below n <= 2^32 - 2); a 16-byte record carries successor word 0
// once visited, and kClaimMark in a claim.
constexpr uint32_t kClaimMark = 0xFFFFFFFFu;

__device__ __forceinline__ Rec8 claim_rec(Rec8 *p, uint32_t cid) { return xchg_rec(p, cid, kClaimMark); }
__device__ __forceinline__ Rec16 claim_rec(Rec16 *p, uint32_t cid) {
  const unsigned long long nlo = ((unsigned long long)cid << 32) | kClaimMark, nhi = 0;
  unsigned long long olo, ohi;
  asm volatile("{\n\t.reg .b128 d, b;\n\tmov.b128 b, {%2, %3};\n\t"
               "atom.global.exch.b128 d, [%4], b;\n\tmov.b128 {%0, %1}, d;\n\t}"
               : "=l"(olo), "=l"(ohi) : "l"(nlo), "l"(nhi), "l"(p) : "memory");
  Rec16 r;
  r.succ = (uint32_t)olo;
  r.tag = (uint32_t)(olo >> 32);
  r.w = ohi;
  return r;
}
__device__ __forceinline__ bool rec_is_claim(const Rec8 &r) { return r.hi != kUnvisited && r.lo == kClaimMark; }
__device__ __forceinline__ bool rec_is_claim(const Rec16 &r) { return r.tag != kUnvisited && r.succ == kClaimMark; }
// Put back a record exactly as it was (a spawner that lost its candidate).
__device__ __forceinline__ void st_raw(Rec8 *p, const Rec8 &r) {
  __stcg(reinterpret_cast<uint2 *>(p), make_uint2(r.lo, r.hi));
}
__device__ __forceinline__ void st_raw(Rec16 *p, const Rec16 &r) {
  __stcg(reinterpret_cast<uint4 *>(p), make_uint4(r.succ, r.tag, (uint32_t)r.w, (uint32_t)(r.w >> 32)));
}

// The raw successor array read as a record (level 0 of the log path): no tag,
// unit link weight, 0 at a terminal.
struct Succ4 {
  uint32_t s;
};
__device__ __forceinline__ Succ4 ld_rec(const Succ4 *p) {
  return Succ4{__ldcg(reinterpret_cast<const uint32_t *>(p))};
}
__device__ __forceinline__ uint64_t rec_weight(const Succ4 &r, uint32_t self) {
  return r.s == self ? 0u : 1u;
}
__device__ __forceinline__ uint32_t rec_succ(const Succ4 &r) { return r.s; }
__device__ __forceinline__ uint32_t rec_tag(const Succ4 &) { return kUnvisited; }
__device__ __forceinline__ void st_rec(Succ4 *, uint32_t, uint64_t) {}

// Link weight carried by a record (level-0 unweighted: 1, or 0 at a terminal).
__device__ __forceinline__ uint64_t rec_weight(const Rec8 &r, uint32_t self) {
  return r.lo == self ? 0u : 1u;
}
__device__ __forceinline__ uint64_t rec_weight(const Rec16 &r, uint32_t) { return r.w; }
__device__ __forceinline__ uint32_t rec_succ(const Rec8 &r) { return r.lo; }
__device__ __forceinline__ uint32_t rec_succ(const Rec16 &r) { return r.succ; }
__device__ __forceinline__ uint32_t rec_tag(const Rec8 &r) { return r.hi; }
__device__ __forceinline__ uint32_t rec_tag(const Rec16 &r) { return r.tag; }
// After the chase: (ruler id, offset)
__device__ __forceinline__ uint32_t done_cid(const Rec8 &r) { return r.hi; }
__device__ __forceinline__ uint32_t done_cid(const Rec16 &r) { return r.tag; }
__device__ __forceinline__ uint64_t done_off(const Rec8 &r) { return r.lo; }
__device__ __forceinline__ uint64_t done_off(const Rec16 &r) { return r.w; }

// ---------------------------------------------------------------- block scan
// Exclusive scan of one 64-bit value per thread across a CTA (warp shuffles,
// then a scan of the warp totals).  `smem` holds >= 33 entries.
__device__ inline uint64_t block_exclusive_scan(uint64_t v, uint64_t *smem, uint64_t *total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nwarps = (blockDim.x + 31) >> 5;
  uint64_t x = v;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    uint64_t y = __shfl_up_sync(0xFFFFFFFFu, x, d);
    if (lane >= d) x += y;
  }
  if (lane == 31) smem[warp] = x;
  __syncthreads();
  if (warp == 0) {
    uint64_t t = lane < nwarps ? smem[lane] : 0;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      uint64_t y = __shfl_up_sync(0xFFFFFFFFu, t, d);
      if (lane >= d) t += y;
    }
    smem[lane] = t;  // inclusive warp-total prefix
  }
  __syncthreads();
  uint64_t warp_base = warp > 0 ? smem[warp - 1] : 0;
  if (total) *total = smem[nwarps - 1];
  uint64_t r = warp_base + x - v;
  __syncthreads();
  return r;
}

}  // namespace lr
