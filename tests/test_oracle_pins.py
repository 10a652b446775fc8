"""Pins for the CPU oracle (no GPU).

The oracle is checked against things fixed by the paper's definition
(Section 1.1) and by mathematics, never against itself:
  - hand-derived fixtures (tests/golden/small_cases.json);
  - brute force: from every element, follow succ to the terminal and add up;
  - closed forms for the identity order (rank = n-1-i, weighted suffix sums);
  - invariants (tail rank 0, the recurrence, per-list permutations, sum of
    head ranks);
  - the unweighted == weight-1 equivalence stated in Section 1.1;
  - Euler-tour depths, computed from the tree without any list ranking;
  - batch == per-instance.
A mutation test then plants plausible mistakes in a copy of the oracle and
checks that at least one pin fails for each.
"""
import ctypes
import json
import os
import shutil
import subprocess

import numpy as np
import pytest

import gen
import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "small_cases.json")
_DT = {"i32": np.int32, "i64": np.int64}


def brute_force(succ, weight=None, rank_dtype=np.int64):
    """From every element follow succ until the terminal, summing link weights.

    Vectorised over elements; n rounds, so O(n^2) work.  Wraps modulo 2^64,
    then the result is cast to the rank type (modulo 2^32 for int32).
    """
    succ = np.asarray(succ, dtype=np.int64)
    n = succ.shape[0]
    w = (np.ones(n, dtype=np.uint64) if weight is None
         else np.asarray(weight).astype(np.int64).astype(np.uint64))
    cur = np.arange(n, dtype=np.int64)
    acc = np.zeros(n, dtype=np.uint64)
    for _ in range(n):
        moving = succ[cur] != cur
        if not moving.any():
            break
        acc[moving] += w[cur[moving]]
        cur = np.where(moving, succ[cur], cur)
    return acc.astype(rank_dtype)


def test_golden_fixtures():
    data = json.load(open(GOLDEN))
    for case in data["cases"]:
        succ = np.array(case["succ"], dtype=np.uint32)
        w = None if "weight" not in case else np.array(case["weight"], dtype=_DT[case["wtype"]])
        rdt = _DT[case.get("rtype", "i32")]
        got = oracle.rank(succ, w, rdt)
        assert got.tolist() == case["rank"], case["name"]
    for case in data["invalid"]:
        st, _ = oracle.rank_status(np.array(case["succ"], dtype=np.uint32))
        assert oracle.STATUS_NAMES[st] == case["status"], case["name"]


def test_empty_input():
    st, out = oracle.rank_status(np.zeros(0, dtype=np.uint32))
    assert st == oracle.OK and out.shape == (0,)


@pytest.mark.parametrize("n", [1, 2, 3, 31, 32, 33, 257, 1000])
def test_brute_force_random_lists(n):
    for rep in range(3):
        succ = gen.random_list(n, 11 * n + rep)
        np.testing.assert_array_equal(oracle.rank(succ), brute_force(succ, None, np.int32))
        w = gen.weights_i32(n, 5 + rep)
        np.testing.assert_array_equal(oracle.rank(succ, w, np.int64), brute_force(succ, w, np.int64))
        w64 = gen.weights_i64(n, 9 + rep, -(1 << 40), 1 << 40)
        np.testing.assert_array_equal(oracle.rank(succ, w64, np.int64), brute_force(succ, w64, np.int64))


def test_brute_force_forest_and_wrap():
    succ, nlists = gen.forest(3000, 4, n_long=3, long_len=400, mean_short=8)
    assert nlists > 3
    np.testing.assert_array_equal(oracle.rank(succ), brute_force(succ, None, np.int32))
    big = np.full(3000, np.iinfo(np.int32).max, dtype=np.int32)
    np.testing.assert_array_equal(oracle.rank(succ, big, np.int32), brute_force(succ, big, np.int32))
    w64 = np.full(3000, np.iinfo(np.int64).max, dtype=np.int64)
    np.testing.assert_array_equal(oracle.rank(succ, w64, np.int64), brute_force(succ, w64, np.int64))


@pytest.mark.parametrize("n", [1, 2, 17, 4096, 100003])
def test_identity_closed_form(n):
    succ = gen.identity_list(n)
    np.testing.assert_array_equal(oracle.rank(succ), n - 1 - np.arange(n, dtype=np.int64))
    w = gen.weights_i32(n, 3)
    # rank[i] = w[i] + w[i+1] + ... + w[n-2]  (the terminal's weight is not a link)
    suffix = np.zeros(n, dtype=np.int64)
    if n > 1:
        suffix[:-1] = np.cumsum(w[:-1][::-1].astype(np.int64))[::-1]
    np.testing.assert_array_equal(oracle.rank(succ, w, np.int64), suffix)


def _check_invariants(succ, rank, weight=None):
    n = succ.shape[0]
    idx = np.arange(n)
    term = succ.astype(np.int64) == idx
    assert (rank[term] == 0).all()
    w = np.ones(n, dtype=np.int64) if weight is None else weight.astype(np.int64)
    nt = ~term
    assert (rank[nt].astype(np.int64) == w[nt] + rank[succ[nt]].astype(np.int64)).all()


@pytest.mark.parametrize("kind", ["random", "locality", "identity"])
def test_invariants(kind):
    n = 1 << 16
    succ = gen.list_of_order_kind(kind, n, 21)
    r = oracle.rank(succ)
    _check_invariants(succ, r)
    # a single list: ranks are a permutation of 0..n-1, head at n-1
    assert np.array_equal(np.sort(r), np.arange(n))
    haspred = np.zeros(n, dtype=bool)
    haspred[succ[succ != np.arange(n)]] = True
    assert r[~haspred].tolist() == [n - 1]
    w = gen.weights_i32(n, 22)
    _check_invariants(succ, oracle.rank(succ, w, np.int64), w)


def test_forest_invariants():
    succ, nlists = gen.forest(1 << 17, 8, n_long=4, long_len=1 << 13, mean_short=64)
    n = succ.shape[0]
    r = oracle.rank(succ)
    _check_invariants(succ, r)
    haspred = np.zeros(n, dtype=bool)
    idx = np.arange(n)
    haspred[succ[succ != idx]] = True
    heads = np.flatnonzero(~haspred)
    assert heads.shape[0] == nlists
    # every element is counted once: sum over heads of (list length) = n
    assert int((r[heads].astype(np.int64) + 1).sum()) == n


def test_unweighted_equals_unit_weights():
    n = 5000
    succ = gen.random_list(n, 31)
    ones = np.ones(n, dtype=np.int32)
    # the terminal's weight is not a link: any value there gives the same ranks
    tail = int(np.flatnonzero(succ == np.arange(n))[0])
    ones[tail] = 12345
    np.testing.assert_array_equal(oracle.rank(succ, ones, np.int32), oracle.rank(succ))


@pytest.mark.parametrize("V", [2, 3, 50, 20000])
def test_euler_tour_depths(V):
    parent = gen.random_recursive_tree(V, 40 + V)
    succ, w = gen.euler_tour(parent)
    r = oracle.rank(succ, w, np.int32).astype(np.int64)
    depth = np.zeros(V, dtype=np.int64)
    for v in range(1, V):                  # parent[v] < v: one ascending pass
        depth[v] = depth[parent[v]] + 1
    v = np.arange(1, V)
    down, up = 2 * (v - 1), 2 * (v - 1) + 1
    np.testing.assert_array_equal(2 - r[down], depth[v])
    np.testing.assert_array_equal(-r[up], depth[parent[v]])


def test_batch_matches_single():
    offsets, succ, w = gen.batch_instances(12, 77, lo_exp=0.0, hi_exp=9.0)
    got = oracle.rank_batch(offsets, succ, w, np.int64)
    for j in range(12):
        a, b = offsets[j], offsets[j + 1]
        np.testing.assert_array_equal(got[a:b], oracle.rank(succ[a:b], w[a:b], np.int64))


def test_invalid_inputs():
    st, _ = oracle.rank_status(np.array([0, 3], dtype=np.uint32))
    assert st == oracle.OUT_OF_RANGE
    n = 1000
    succ = gen.random_list(n, 3).copy()
    head = int(np.setdiff1d(np.arange(n), succ[succ != np.arange(n)])[0])
    tail = int(np.flatnonzero(succ == np.arange(n))[0])
    bad = succ.copy()
    bad[tail] = head                           # closes the list into a cycle
    assert oracle.rank_status(bad)[0] == oracle.CYCLE
    bad = succ.copy()
    bad[tail] = succ[head]                     # tail -> second element: in-degree 2
    assert oracle.rank_status(bad)[0] == oracle.NOT_A_LIST


# ---------------------------------------------------------------- mutation test
_MUTATIONS = {
    "weight_sign": ("acc += weight_of(weight, wtype, order[k]);",
                    "acc -= weight_of(weight, wtype, order[k]);"),
    "terminal_weight_counted": ("for (int64_t k = len - 2; k >= 0; --k) {",
                                "acc += weight_of(weight, wtype, order[len - 1]);\n"
                                "        for (int64_t k = len - 2; k >= 0; --k) {"),
    "successor_weight": ("acc += weight_of(weight, wtype, order[k]);",
                         "acc += weight_of(weight, wtype, order[k + 1]);"),
    "rank_from_head": ("store_rank(rank, rtype, order[k], acc);",
                       "store_rank(rank, rtype, order[len - 2 - k], acc);"),
    "unit_weight_two": ("if (wtype == LRO_W_NONE) return 1u;",
                        "if (wtype == LRO_W_NONE) return 2u;"),
    "zero_extend_i32": ("return (uint64_t)(int64_t)((const int32_t *)w)[i];",
                        "return (uint64_t)((const uint32_t *)w)[i];"),
    "heads_inverted": ("if (npred[h] != 0) continue;", "if (npred[h] == 0) continue;"),
    "no_cycle_check": ("if (status == LRO_OK && visited != n) status = LRO_CYCLE;", ""),
    "terminal_test_swapped": ("if (succ[x] == x) break;", "if (succ[x] != x) break;"),
}


def _pins_pass(lib):
    """Run a compact set of the pins above against a given oracle library."""
    lib.lro_rank.restype = ctypes.c_int
    lib.lro_rank.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_int64,
                             ctypes.c_void_p, ctypes.c_int]

    def run(succ, w=None, rdt=np.int64):
        succ = np.ascontiguousarray(succ, dtype=np.uint32)
        out = np.zeros(succ.shape[0], dtype=rdt)
        wc = 0 if w is None else (1 if w.dtype == np.int32 else 2)
        st = lib.lro_rank(succ.ctypes.data, None if w is None else w.ctypes.data, wc,
                          succ.shape[0], out.ctypes.data, 1 if rdt == np.int32 else 2)
        return st, out

    data = json.load(open(GOLDEN))
    for case in data["cases"]:
        w = None if "weight" not in case else np.array(case["weight"], dtype=_DT[case["wtype"]])
        st, out = run(case["succ"], w, _DT[case.get("rtype", "i32")])
        if st != 0 or out.tolist() != case["rank"]:
            return False
    for case in data["invalid"]:
        if oracle.STATUS_NAMES.get(run(case["succ"])[0]) != case["status"]:
            return False
    for n in (2, 33, 300):
        succ = gen.random_list(n, n)
        w = gen.weights_i32(n, n + 1)
        st, out = run(succ, w, np.int64)
        if st != 0 or not np.array_equal(out, brute_force(succ, w, np.int64)):
            return False
    return True


@pytest.mark.skipif(shutil.which("gcc") is None, reason="needs gcc")
def test_mutants_are_caught(tmp_path):
    src = open(os.path.join(os.path.dirname(oracle.__file__), "lr_oracle.c")).read()
    assert _pins_pass(ctypes.CDLL(oracle.build()))
    for name, (old, new) in _MUTATIONS.items():
        assert old in src, "mutation site for %s is gone from the oracle" % name
        mutant_c = tmp_path / ("m_%s.c" % name)
        mutant_c.write_text(src.replace(old, new, 1))
        so = tmp_path / ("m_%s.so" % name)
        subprocess.check_call(["gcc", "-std=c11", "-O1", "-fPIC", "-shared", "-o", str(so), str(mutant_c)])
        assert not _pins_pass(ctypes.CDLL(str(so))), "pins did not catch mutant %s" % name


# ---------------------------------------------------------------- extra outputs
# Section 1.1 also names each element's terminal as part of the result, and
# the in-place form counts the terminal's weight.  Pins for oracle.rank_ext.

def brute_force_ext(succ, weight=None):
    """term[i]: the end of the walk from i.  prefix[x]: the sum of w[j] over
    every strict ancestor j of x (every j whose walk passes through x).
    O(n^2) walks from every element; a formulation unlike the oracle's."""
    succ = np.asarray(succ, dtype=np.int64)
    n = succ.shape[0]
    w = np.ones(n, dtype=np.int64) if weight is None else np.asarray(weight, dtype=np.int64)
    term = np.zeros(n, dtype=np.int64)
    prefix = np.zeros(n, dtype=np.int64)
    for j in range(n):
        x = j
        while succ[x] != x:
            x = succ[x]
            prefix[x] += w[j]
        term[j] = x
    return term, prefix


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_ext_brute_force_forest(seed):
    succ, _ = gen.forest(400, seed, n_long=2, long_len=60, mean_short=7)
    w = gen.weights_i32(400, seed + 10)
    for weight in (None, w):
        r, t, p = oracle.rank_ext(succ, weight, np.int64)
        bt, bp = brute_force_ext(succ, weight)
        np.testing.assert_array_equal(t, bt)
        np.testing.assert_array_equal(p, bp)
        np.testing.assert_array_equal(r, brute_force(succ, weight, np.int64))
        ri, ti, pi = oracle.rank_ext(succ, weight, np.int64, inclusive=True)
        # Section 1.1: the unweighted problem gives the terminal weight 0
        wt = np.zeros(400, dtype=np.int64) if weight is None else weight.astype(np.int64)
        np.testing.assert_array_equal(ri, r + wt[bt])
        np.testing.assert_array_equal(ti, bt)
        np.testing.assert_array_equal(pi, bp)


@pytest.mark.parametrize("n", [1, 2, 5, 1000])
def test_ext_identity_closed_form(n):
    succ = gen.identity_list(n)
    r, t, p = oracle.rank_ext(succ)
    np.testing.assert_array_equal(t, np.full(n, n - 1))
    np.testing.assert_array_equal(p, np.arange(n))
    ri, _, _ = oracle.rank_ext(succ, inclusive=True)
    np.testing.assert_array_equal(ri, n - 1 - np.arange(n))  # unweighted terminal weighs 0
    w = gen.weights_i64(n, n, lo=-50, hi=50)
    r, t, p = oracle.rank_ext(succ, w, np.int64)
    excl = np.concatenate([[0], np.cumsum(w[:-1])])          # sum of the links before i
    np.testing.assert_array_equal(p, excl)
    ri, _, _ = oracle.rank_ext(succ, w, np.int64, inclusive=True)
    np.testing.assert_array_equal(ri, np.cumsum(w[::-1])[::-1])   # suffix sums including the tail


def test_ext_invariants_forest():
    succ, nl = gen.forest(1 << 16, 9, n_long=4, long_len=1 << 12, mean_short=32)
    w = gen.weights_i32(1 << 16, 10)
    r, t, p = oracle.rank_ext(succ, w, np.int64)
    s = succ.astype(np.int64)
    idx = np.arange(s.shape[0])
    assert np.all(s[t] == t)                                 # a terminal ends every walk
    assert np.all(t[s] == t)                                 # the terminal is shared along a list
    tot = p[t]                                               # the total sits at the terminal
    np.testing.assert_array_equal(p + r, tot)
    nt = s != idx
    np.testing.assert_array_equal(p[s[nt]], p[nt] + w[nt])   # forward recurrence
    heads = np.setdiff1d(idx, s[nt])
    assert heads.shape[0] == nl and np.all(p[heads] == 0)
    assert np.unique(t).shape[0] == nl


@pytest.mark.parametrize("V", [2, 3, 50, 20000])
def test_ext_euler_tour_depths(V):
    """Euler-tour technique: the prefix sum of the +-1 arcs before an arc is
    the depth of the node the tour stands on."""
    parent = gen.random_recursive_tree(V, 50 + V)
    succ, w = gen.euler_tour(parent)
    _, t, p = oracle.rank_ext(succ, w, np.int32)
    depth = np.zeros(V, dtype=np.int64)
    for v in range(1, V):
        depth[v] = depth[parent[v]] + 1
    v = np.arange(1, V)
    down, up = 2 * (v - 1), 2 * (v - 1) + 1
    np.testing.assert_array_equal(p[down], depth[parent[v]])
    np.testing.assert_array_equal(p[up], depth[v])
    assert np.all(t == t[0]) and succ[t[0]] == t[0]


def test_ext_batch_local_terminals():
    offsets, succ, w = gen.batch_instances(10, 78, lo_exp=0.0, hi_exp=9.0)
    r, t, p = oracle.rank_ext_batch(offsets, succ, w, np.int64, inclusive=True)
    for j in range(10):
        a, b = offsets[j], offsets[j + 1]
        rj, tj, pj = oracle.rank_ext(succ[a:b], w[a:b], np.int64, inclusive=True)
        np.testing.assert_array_equal(r[a:b], rj)
        np.testing.assert_array_equal(t[a:b], tj)
        np.testing.assert_array_equal(p[a:b], pj)
        assert np.all(t[a:b] < b - a)


_EXT_MUTATIONS = {
    "prefix_counts_own_link": ("            acc += weight_of(weight, wtype, x);\n            x = succ[x];",
                               "            x = succ[x];\n            acc += weight_of(weight, wtype, x);"),
    "inclusive_uses_head_weight": ("0u : weight_of(weight, wtype, t);",
                                   "0u : weight_of(weight, wtype, h);"),
    "unweighted_terminal_weighs_one": ("wtype == LRO_W_NONE ? 0u :", "wtype == LRO_W_NONE ? 1u :"),
    "term_is_head": ("if (term) term[x] = t;", "if (term) term[x] = (uint32_t)h;"),
    "prefix_starts_at_head_weight": ("        uint64_t acc = 0;\n        uint64_t wt",
                                     "        uint64_t acc = weight_of(weight, wtype, h);\n        uint64_t wt"),
}


def _ext_pins_pass(lib):
    lib.lro_rank_ext.restype = ctypes.c_int
    lib.lro_rank_ext.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_int64,
                                 ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                                 ctypes.c_int]
    for seed in (1, 2):
        succ, _ = gen.forest(300, seed, n_long=2, long_len=50, mean_short=6)
        succ = np.ascontiguousarray(succ, dtype=np.uint32)
        w = gen.weights_i32(300, seed + 20)
        bt, bp = brute_force_ext(succ, w)
        for incl in (0, 1):
            r = np.zeros(300, dtype=np.int64)
            t = np.zeros(300, dtype=np.uint32)
            p = np.zeros(300, dtype=np.int64)
            st = lib.lro_rank_ext(succ.ctypes.data, w.ctypes.data, 1, 300, r.ctypes.data, 2,
                                  t.ctypes.data, p.ctypes.data, incl)
            want_r = brute_force(succ, w, np.int64) + (w.astype(np.int64)[bt] if incl else 0)
            if st != 0 or not (np.array_equal(t, bt) and np.array_equal(p, bp) and np.array_equal(r, want_r)):
                return False
            # unweighted: the terminal weighs 0 (Section 1.1), so the
            # inclusive form is the plain link count
            r = np.zeros(300, dtype=np.int64)
            st = lib.lro_rank_ext(succ.ctypes.data, None, 0, 300, r.ctypes.data, 2,
                                  t.ctypes.data, p.ctypes.data, incl)
            if st != 0 or not np.array_equal(r, brute_force(succ, None, np.int64)):
                return False
    return True


@pytest.mark.skipif(shutil.which("gcc") is None, reason="needs gcc")
def test_ext_mutants_are_caught(tmp_path):
    src = open(os.path.join(os.path.dirname(oracle.__file__), "lr_oracle.c")).read()
    assert _ext_pins_pass(ctypes.CDLL(oracle.build()))
    for name, (old, new) in _EXT_MUTATIONS.items():
        assert src.count(old) == 1, "mutation site for %s is gone from the oracle" % name
        mutant_c = tmp_path / ("e_%s.c" % name)
        mutant_c.write_text(src.replace(old, new, 1))
        so = tmp_path / ("e_%s.so" % name)
        subprocess.check_call(["gcc", "-std=c11", "-O1", "-fPIC", "-shared", "-o", str(so), str(mutant_c)])
        assert not _ext_pins_pass(ctypes.CDLL(str(so))), "pins did not catch mutant %s" % name
