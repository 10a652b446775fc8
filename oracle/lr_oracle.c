/*
 * lr_oracle.c -- sequential CPU oracle for (weighted) list ranking.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the checker that the GPU library is
 * compared against.  Only the test suite, the smoke check and the benchmark's
 * CPU-baseline leg load it; the library under test never includes, links or
 * calls it, and it shares no code, header or constant with the library.
 *
 * What it computes is the plain definition of the problem (Section 1.1 of
 * "Engineering Scalable Distributed List Ranking"):
 *
 *   - succ[0..n-1] is a successor array; a terminal element points to itself
 *     (succ[t] == t); an initial element (a head) has no predecessor.
 *   - rank[i] is the number of links (unweighted) or the sum of the link
 *     weights (weighted) on the path from i to the terminal of its list.
 *   - The unweighted problem is the weighted one with weight 1 on every link
 *     and weight 0 on the terminal (Section 1.1, last paragraph).
 *
 * Readings where the paper is silent:
 *   - weight[i] is the weight of the link i -> succ[i]; a terminal has no
 *     outgoing link, so its weight is ignored and rank[t] == 0.
 *   - Sums wrap around in two's complement in the rank type; int32 weights
 *     are sign-extended first.
 *   - Invalid inputs are reported, checked in this order: a successor out of
 *     range, an element with two or more predecessors, an element that is not
 *     reachable from any head (a cycle).  rank is unspecified on error.
 *
 * Algorithm (linear time, one thread):
 *   1. range check;
 *   2. count predecessors (self-loops excluded); heads have count 0;
 *   3. for every head in ascending index order, walk succ to the terminal and
 *      record the visiting order;
 *   4. walk that order backwards, accumulating the weights: the terminal gets
 *      0, every other element gets its own weight plus its successor's rank;
 *   5. if fewer than n elements were visited, some element lies on a cycle.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

enum { LRO_OK = 0, LRO_INVALID = 1, LRO_OUT_OF_RANGE = 2, LRO_CYCLE = 3,
       LRO_NOT_A_LIST = 4, LRO_NO_MEMORY = 5 };
enum { LRO_W_NONE = 0, LRO_W_I32 = 1, LRO_W_I64 = 2 };
enum { LRO_R_I32 = 1, LRO_R_I64 = 2 };

/* Weight of element i as an unsigned 64-bit value (mod 2^64 arithmetic). */
static uint64_t weight_of(const void *w, int wtype, int64_t i)
{
    if (wtype == LRO_W_NONE) return 1u;
    if (wtype == LRO_W_I32) return (uint64_t)(int64_t)((const int32_t *)w)[i];
    return (uint64_t)((const int64_t *)w)[i];
}

static void store_rank(void *rank, int rtype, int64_t i, uint64_t v)
{
    if (rtype == LRO_R_I32) ((uint32_t *)rank)[i] = (uint32_t)v;
    else ((uint64_t *)rank)[i] = v;
}

int lro_rank(const uint32_t *succ, const void *weight, int wtype, int64_t n,
             void *rank, int rtype)
{
    if (n < 0) return LRO_INVALID;
    if (n == 0) return LRO_OK;
    if (!succ || !rank) return LRO_INVALID;
    if (wtype != LRO_W_NONE && !weight) return LRO_INVALID;
    if (wtype < LRO_W_NONE || wtype > LRO_W_I64) return LRO_INVALID;
    if (rtype != LRO_R_I32 && rtype != LRO_R_I64) return LRO_INVALID;

    /* 1. every successor must name an element */
    for (int64_t i = 0; i < n; ++i)
        if ((int64_t)succ[i] >= n) return LRO_OUT_OF_RANGE;

    /* 2. predecessor counts, saturating at 2 */
    uint8_t *npred = (uint8_t *)calloc((size_t)n, 1);
    uint32_t *order = (uint32_t *)malloc((size_t)n * sizeof(uint32_t));
    if (!npred || !order) { free(npred); free(order); return LRO_NO_MEMORY; }
    for (int64_t i = 0; i < n; ++i) {
        uint32_t s = succ[i];
        if ((int64_t)s != i && npred[s] < 2) npred[s]++;
    }
    for (int64_t i = 0; i < n; ++i)
        if (npred[i] >= 2) { free(npred); free(order); return LRO_NOT_A_LIST; }

    /* 3.+4. walk each list from its head, then accumulate backwards */
    int64_t visited = 0;
    int status = LRO_OK;
    for (int64_t h = 0; h < n && status == LRO_OK; ++h) {
        if (npred[h] != 0) continue;
        int64_t len = 0;
        uint32_t x = (uint32_t)h;
        for (;;) {
            if (visited + len >= n) { status = LRO_CYCLE; break; }
            order[len++] = x;
            if (succ[x] == x) break;      /* reached the terminal */
            x = succ[x];
        }
        if (status != LRO_OK) break;
        uint64_t acc = 0;                 /* rank of the terminal */
        store_rank(rank, rtype, order[len - 1], acc);
        for (int64_t k = len - 2; k >= 0; --k) {
            acc += weight_of(weight, wtype, order[k]);
            store_rank(rank, rtype, order[k], acc);
        }
        visited += len;
    }
    /* 5. anything not reached from a head lies on a cycle */
    if (status == LRO_OK && visited != n) status = LRO_CYCLE;
    free(npred);
    free(order);
    return status;
}

/*
 * Batched form: k independent instances stored back to back.  Instance j owns
 * elements offsets[j] .. offsets[j+1]-1; its successors are local ids in
 * [0, offsets[j+1]-offsets[j]).  Each instance is ranked on its own.  Returns
 * the first error met (instances are checked in order).
 */
int lro_rank_batch(const int64_t *offsets, int32_t k, const uint32_t *succ,
                   const void *weight, int wtype, void *rank, int rtype)
{
    if (k < 0 || !offsets) return LRO_INVALID;
    if (k > 0 && offsets[0] != 0) return LRO_INVALID;
    for (int32_t j = 0; j < k; ++j)
        if (offsets[j + 1] < offsets[j]) return LRO_INVALID;
    size_t wsz = wtype == LRO_W_I32 ? 4 : 8;
    size_t rsz = rtype == LRO_R_I32 ? 4 : 8;
    for (int32_t j = 0; j < k; ++j) {
        int64_t a = offsets[j], len = offsets[j + 1] - offsets[j];
        const void *wj = wtype == LRO_W_NONE ? NULL
                         : (const void *)((const char *)weight + (size_t)a * wsz);
        int st = lro_rank(succ + a, wj, wtype, len,
                          (void *)((char *)rank + (size_t)a * rsz), rtype);
        if (st != LRO_OK) return st;
    }
    return LRO_OK;
}

/*
 * Full output of Section 1.1: besides the rank, the paper's result names for
 * every element the terminal of its list (it overwrites succ[i] with it), and
 * its in-place form leaves the terminal's own weight in rank[t].  Computed
 * here straight from those definitions, after lro_rank has validated the
 * input and produced the (exclusive) ranks:
 *   term[i]   = the element reached from i by following succ until
 *               succ[x] == x;
 *   prefix[i] = the sum of the link weights from the head of i's list up to
 *               i, not counting i's own link (0 at a head);
 *   inclusive: rank[i] += weight of the terminal, i.e. the terminal's weight
 *               is no longer ignored.  In the unweighted problem the terminal
 *               weighs 0 (Section 1.1: unweighted means weight 1 on every
 *               element except the terminal, which gets 0), so there the
 *               inclusive form equals the plain rank.
 * term and prefix may be NULL (not produced); prefix has the rank type.
 */
int lro_rank_ext(const uint32_t *succ, const void *weight, int wtype, int64_t n,
                 void *rank, int rtype, uint32_t *term, void *prefix, int inclusive)
{
    int st = lro_rank(succ, weight, wtype, n, rank, rtype);
    if (st != LRO_OK || n == 0) return st;
    uint8_t *haspred = (uint8_t *)calloc((size_t)n, 1);
    if (!haspred) return LRO_NO_MEMORY;
    for (int64_t i = 0; i < n; ++i)
        if ((int64_t)succ[i] != i) haspred[succ[i]] = 1;
    for (int64_t h = 0; h < n; ++h) {
        if (haspred[h]) continue;
        /* find the terminal of h's list */
        uint32_t t = (uint32_t)h;
        while (succ[t] != t) t = succ[t];
        /* walk again from the head: terminal, running prefix, inclusive rank */
        uint64_t acc = 0;
        uint64_t wt = wtype == LRO_W_NONE ? 0u : weight_of(weight, wtype, t);
        uint32_t x = (uint32_t)h;
        for (;;) {
            if (term) term[x] = t;
            if (prefix) store_rank(prefix, rtype, x, acc);
            if (inclusive) {
                uint64_t r = rtype == LRO_R_I32 ? (uint64_t)((uint32_t *)rank)[x]
                                                : ((uint64_t *)rank)[x];
                store_rank(rank, rtype, x, r + wt);
            }
            if (succ[x] == x) break;
            acc += weight_of(weight, wtype, x);
            x = succ[x];
        }
    }
    free(haspred);
    return LRO_OK;
}

/* Batched form of lro_rank_ext: terminal ids are local to their instance. */
int lro_rank_ext_batch(const int64_t *offsets, int32_t k, const uint32_t *succ,
                       const void *weight, int wtype, void *rank, int rtype,
                       uint32_t *term, void *prefix, int inclusive)
{
    if (k < 0 || !offsets) return LRO_INVALID;
    if (k > 0 && offsets[0] != 0) return LRO_INVALID;
    for (int32_t j = 0; j < k; ++j)
        if (offsets[j + 1] < offsets[j]) return LRO_INVALID;
    size_t wsz = wtype == LRO_W_I32 ? 4 : 8;
    size_t rsz = rtype == LRO_R_I32 ? 4 : 8;
    for (int32_t j = 0; j < k; ++j) {
        int64_t a = offsets[j], len = offsets[j + 1] - offsets[j];
        const void *wj = wtype == LRO_W_NONE ? NULL
                         : (const void *)((const char *)weight + (size_t)a * wsz);
        int st = lro_rank_ext(succ + a, wj, wtype, len,
                              (void *)((char *)rank + (size_t)a * rsz), rtype,
                              term ? term + a : NULL,
                              prefix ? (void *)((char *)prefix + (size_t)a * rsz) : NULL,
                              inclusive);
        if (st != LRO_OK) return st;
    }
    return LRO_OK;
}
