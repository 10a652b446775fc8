"""Seeded synthetic inputs for list ranking.

This module only builds inputs: successor arrays, weights, batch offset tables
and request traces.  It contains no ranking arithmetic; the oracle and the GPU
library both consume what it returns.

Input families follow the shapes of the paper's workloads (Section 3, "Input
Instances"): lists whose order is a random permutation (the paper's
List(n, gamma=1)), lists with window-local disorder (a stand-in for small
gamma), the plain identity order, forests of many lists, and Euler tours of
random trees.  The paper's KaGen graphs are not available; the random recursive
tree below stands in for its BFS trees.

All generators use numpy's PCG64 with an explicit seed, which gives the same
numbers on x86-64 and aarch64.
"""
import numpy as np

__all__ = [
    "rng", "succ_from_order", "random_order", "locality_order", "identity_order",
    "random_list", "locality_list", "identity_list", "list_of_order_kind",
    "weights_i32", "weights_i64", "forest", "random_recursive_tree", "euler_tour",
    "batch_lengths", "batch_instances", "serving_trace", "config_seed",
]


def config_seed(config: int, rep: int = 0) -> int:
    """Seed convention: 1000 * config + repetition."""
    return 1000 * int(config) + int(rep)


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(int(seed)))


def succ_from_order(order: np.ndarray, list_ends=None) -> np.ndarray:
    """Successor array of the list(s) visiting ``order`` front to back.

    ``list_ends`` (bool array, same length) marks positions that end a list;
    by default only the last position does.  A list end points to itself.
    """
    order = np.ascontiguousarray(order, dtype=np.uint32)
    n = order.shape[0]
    succ = np.empty(n, dtype=np.uint32)
    if n == 0:
        return succ
    nxt = np.empty(n, dtype=np.uint32)
    nxt[:-1] = order[1:]
    nxt[-1] = order[-1]
    if list_ends is not None:
        ends = np.asarray(list_ends, dtype=bool)
        nxt = np.where(ends, order, nxt)
    succ[order] = nxt
    return succ


def random_order(n: int, seed: int) -> np.ndarray:
    """A uniformly random visiting order of 0..n-1 (no locality)."""
    return rng(seed).permutation(np.arange(n, dtype=np.uint32))


def locality_order(n: int, seed: int, window: int = 256) -> np.ndarray:
    """Identity order, shuffled uniformly inside each aligned window."""
    g = rng(seed)
    order = np.arange(n, dtype=np.uint32)
    full = (n // window) * window
    if full:
        order[:full] = g.permuted(order[:full].reshape(-1, window), axis=1).reshape(-1)
    if full < n:
        order[full:] = g.permutation(order[full:])
    return order


def identity_order(n: int) -> np.ndarray:
    return np.arange(n, dtype=np.uint32)


def random_list(n: int, seed: int) -> np.ndarray:
    return succ_from_order(random_order(n, seed))


def locality_list(n: int, seed: int, window: int = 256) -> np.ndarray:
    return succ_from_order(locality_order(n, seed, window))


def identity_list(n: int) -> np.ndarray:
    return succ_from_order(identity_order(n))


def list_of_order_kind(kind: str, n: int, seed: int) -> np.ndarray:
    if kind == "random":
        return random_list(n, seed)
    if kind == "locality":
        return locality_list(n, seed)
    if kind == "identity":
        return identity_list(n)
    raise ValueError("unknown order kind %r" % kind)


def weights_i32(n: int, seed: int, lo: int = -1000, hi: int = 1000) -> np.ndarray:
    """Uniform int32 weights in [lo, hi] (both ends included)."""
    return rng(seed).integers(lo, hi + 1, size=n, dtype=np.int32)


def weights_i64(n: int, seed: int, lo: int = 0, hi: int = 1 << 20) -> np.ndarray:
    """Uniform int64 weights in [lo, hi) (upper end excluded)."""
    return rng(seed).integers(lo, hi, size=n, dtype=np.int64)


def forest(n_total: int, seed: int, n_long: int = 16, long_len: int = 1 << 22,
           mean_short: int = 64):
    """Many lists in one successor array, labels randomly interleaved.

    ``n_long`` lists of ``long_len`` elements, then lists of geometric length
    (success probability 1/mean_short, at least one element) filling the rest;
    the last short list is truncated.  Returns (succ, number_of_lists).
    """
    g = rng(seed)
    long_total = n_long * long_len
    if long_total > n_total:
        raise ValueError("long lists exceed the total size")
    rest = n_total - long_total
    lens = [np.full(n_long, long_len, dtype=np.int64)]
    if rest > 0:
        parts, acc = [], 0
        while acc < rest:
            chunk = g.geometric(1.0 / mean_short, size=(rest - acc) // mean_short + 1024)
            parts.append(chunk.astype(np.int64))
            acc += int(chunk.sum())
        short = np.concatenate(parts)
        cs = np.cumsum(short)
        m = int(np.searchsorted(cs, rest, side="left"))   # first prefix reaching rest
        short = short[: m + 1]
        short[-1] -= int(cs[m]) - rest                     # truncate the last list
        lens.append(short)
    lens = np.concatenate(lens)
    lens = lens[lens > 0]
    ends = np.zeros(n_total, dtype=bool)
    ends[np.cumsum(lens) - 1] = True
    labels = g.permutation(np.arange(n_total, dtype=np.uint32))
    return succ_from_order(labels, ends), int(lens.shape[0])


def random_recursive_tree(n_vertices: int, seed: int) -> np.ndarray:
    """parent[v] uniform in [0, v-1] for v >= 1; parent[0] = 0 (the root)."""
    g = rng(seed)
    parent = np.zeros(n_vertices, dtype=np.int64)
    if n_vertices > 1:
        v = np.arange(1, n_vertices, dtype=np.int64)
        parent[1:] = np.minimum((g.random(n_vertices - 1) * v).astype(np.int64), v - 1)
    return parent


def euler_tour(parent: np.ndarray):
    """Euler tour of a rooted tree as a weighted list.

    Arc labels: down(v) = 2(v-1) (parent -> v, weight +1) and
    up(v) = 2(v-1)+1 (v -> parent, weight -1), for v = 1..V-1.  The tour
    starts at the root and visits children in ascending id; it ends with the
    up-arc of the root's last child, which points to itself.
    Returns (succ uint32, weight int32).
    """
    parent = np.asarray(parent, dtype=np.int64)
    V = parent.shape[0]
    if V < 2:
        raise ValueError("a tour needs at least one edge")
    kids = np.arange(1, V, dtype=np.int64)
    by_parent = kids[np.argsort(parent[1:], kind="stable")]   # children grouped, ascending
    par_sorted = parent[by_parent]
    first_child = np.full(V, -1, dtype=np.int64)
    is_first = np.ones(V - 1, dtype=bool)
    is_first[1:] = par_sorted[1:] != par_sorted[:-1]
    first_child[par_sorted[is_first]] = by_parent[is_first]
    next_sib = np.full(V, -1, dtype=np.int64)
    same = par_sorted[1:] == par_sorted[:-1]
    next_sib[by_parent[:-1][same]] = by_parent[1:][same]

    down = 2 * (kids - 1)
    up = down + 1
    succ = np.empty(2 * (V - 1), dtype=np.int64)
    fc = first_child[kids]
    succ[down] = np.where(fc >= 0, 2 * (fc - 1), up)
    ns = next_sib[kids]
    pv = parent[kids]
    succ_up = np.where(ns >= 0, 2 * (ns - 1), np.where(pv == 0, up, 2 * (pv - 1) + 1))
    succ[up] = succ_up
    weight = np.empty(2 * (V - 1), dtype=np.int32)
    weight[down] = 1
    weight[up] = -1
    return succ.astype(np.uint32), weight


def batch_lengths(k: int, seed: int, lo_exp: float = 8.0, hi_exp: float = 22.0) -> np.ndarray:
    """Instance sizes floor(2^U) with U uniform in [lo_exp, hi_exp]."""
    u = rng(seed).uniform(lo_exp, hi_exp, size=k)
    return np.floor(np.exp2(u)).astype(np.int64)


def batch_instances(k: int, seed: int, lo_exp: float = 8.0, hi_exp: float = 22.0,
                    weighted: bool = True, order: str = "random"):
    """k independent random-order lists back to back with local successor ids.

    Returns (offsets int64[k+1], succ uint32[total], weight int64[total] or None).
    """
    lens = batch_lengths(k, seed, lo_exp, hi_exp)
    offsets = np.zeros(k + 1, dtype=np.int64)
    np.cumsum(lens, out=offsets[1:])
    total = int(offsets[-1])
    succ = np.empty(total, dtype=np.uint32)
    for j in range(k):
        a, b = int(offsets[j]), int(offsets[j + 1])
        succ[a:b] = list_of_order_kind(order, b - a, seed * 7919 + j + 1)
    weight = weights_i64(total, seed + 17) if weighted else None
    return offsets, succ, weight


def serving_trace(num: int, seed: int, rate_per_s: float, lo_exp: float = 10.0,
                  hi_exp: float = 26.0, p_random: float = 0.5):
    """Poisson arrival trace: returns (arrival_s float64[num], sizes int64[num],
    kinds list of 'random'/'locality', per-request seeds int64[num])."""
    g = rng(seed)
    gaps = g.exponential(1.0 / rate_per_s, size=num)
    arrivals = np.cumsum(gaps) - gaps[0]
    sizes = np.floor(np.exp2(g.uniform(lo_exp, hi_exp, size=num))).astype(np.int64)
    kinds = ["random" if x < p_random else "locality" for x in g.random(num)]
    seeds = g.integers(1, 2**62, size=num, dtype=np.int64)
    return arrivals, sizes, kinds, seeds
