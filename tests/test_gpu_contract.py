"""Tile-local contraction (Section 2.3) on the GPU.

Contraction changes the route, never the result: every case is compared
with the oracle, with contraction left to the automatic choice, forced on
(also on inputs where it does not pay) and forced off.
"""
import numpy as np
import pytest

import gen
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2606_09318_gb300 as lr  # noqa: E402

ON = lr.Tuning(contract=lr.CONTRACT_ON)
OFF = lr.Tuning(contract=lr.CONTRACT_OFF)
TILE = 4096


def dev(a):
    a = np.ascontiguousarray(a)
    if a.dtype == np.uint32:
        a = a.view(np.int32)
    return torch.from_numpy(a).cuda()


def rank(succ, w=None, rdt=torch.int32, **kw):
    return lr.rank(dev(succ), None if w is None else dev(w), rank_dtype=rdt, **kw).cpu().numpy()


@pytest.mark.parametrize("n", [16384, 3 * TILE + 17, (1 << 20) + 5, (1 << 22) + 4097])
@pytest.mark.parametrize("kind", ["locality", "identity"])
def test_local_orders(n, kind):
    succ = gen.list_of_order_kind(kind, n, 500 + n % 89)
    want = oracle.rank(succ)
    for t in (None, ON, OFF):
        np.testing.assert_array_equal(rank(succ, tuning=t), want)


@pytest.mark.parametrize("n", [16384, (1 << 20) + 3])
def test_forced_on_random_and_forest(n):
    succ = gen.random_list(n, 501)
    np.testing.assert_array_equal(rank(succ, tuning=ON), oracle.rank(succ))
    fs, _ = gen.forest(n, 502, n_long=2, long_len=n // 8, mean_short=16)
    np.testing.assert_array_equal(rank(fs, tuning=ON), oracle.rank(fs))


def test_local_forest():
    """Many short lists, each inside a few tiles: runs of a locality order cut
    into pieces (terminals inside tiles, contracted terminals)."""
    n = (1 << 20) + 77
    order = np.asarray(gen.locality_order(n, 503), dtype=np.int64)
    ends = np.zeros(n, dtype=bool)
    ends[np.random.default_rng(504).choice(n, 3000, replace=False)] = True
    ends[-1] = True
    succ = gen.succ_from_order(order, ends)
    want = oracle.rank(succ)
    for t in (None, ON):
        np.testing.assert_array_equal(rank(succ, tuning=t), want)


@pytest.mark.parametrize("wkind,rdt", [("i32", np.int64), ("i64", np.int64), ("i32", np.int32)])
def test_weighted(wkind, rdt):
    n = (1 << 20) + 1023
    succ = gen.locality_list(n, 505)
    w = gen.weights_i32(n, 506) if wkind == "i32" else gen.weights_i64(n, 507, lo=-(1 << 40), hi=1 << 40)
    tdt = torch.int32 if rdt == np.int32 else torch.int64
    want = oracle.rank(succ, w, rdt)
    for t in (None, ON):
        np.testing.assert_array_equal(rank(succ, w, tdt, tuning=t), want)


def test_weighted_extreme_int32():
    # int32 weights over their whole range: in-tile distances reach about
    # 2^43 in magnitude, the largest the packed in-tile form must carry
    n = 5 * TILE + 3
    for kind in ("locality", "identity"):
        succ = gen.list_of_order_kind(kind, n, 509)
        w = np.random.default_rng(510).integers(-(1 << 31), 1 << 31, size=n, dtype=np.int64).astype(np.int32)
        w[:TILE] = np.int32(-(1 << 31))                   # one tile of the most negative weight
        want = oracle.rank(succ, w, np.int64)
        for t in (None, ON):
            np.testing.assert_array_equal(rank(succ, w, torch.int64, tuning=t), want)


def test_weighted_int64_mixed_tiles():
    # int64 weights: tiles whose weights all fit in int32 take the packed
    # in-tile form, the tile holding a wider weight the separate one
    n = 6 * TILE + 9
    for kind in ("locality", "identity"):
        succ = gen.list_of_order_kind(kind, n, 511)
        w = gen.weights_i64(n, 512)
        w[TILE + 7] = 1 << 50
        w[3 * TILE + 100] = -(1 << 62)
        want = oracle.rank(succ, w, np.int64)
        for t in (None, ON):
            np.testing.assert_array_equal(rank(succ, w, torch.int64, tuning=t), want)
    # a cycle inside a tile with a wide weight is still found
    succ = gen.identity_list(n).astype(np.int64)
    succ[999] = 1101
    succ[1100] = 1000
    w = gen.weights_i64(n, 513)
    w[1050] = 1 << 45
    try:
        lr.rank(dev(succ.astype(np.uint32)), dev(w), tuning=ON)
        got = "LR_OK"
    except lr.LRError as e:
        got = e.name
    assert got == "LR_ERR_CYCLE"


@pytest.mark.parametrize("wdt", [np.int32, np.int64])
def test_weighted_narrow_limits(wdt):
    # A tile whose weights all lie in (-2^19, 2^19), or all in [0, 2^20),
    # takes its in-tile prefix sums modulo 2^32; identity order makes every
    # tile one chain of 4095 local links, so its distances reach 4095 times
    # the weight: just inside 2^31 (signed) and 2^32 (unsigned).  A tile with
    # one weight past either limit takes 64-bit sums.
    n = 6 * TILE + 11
    succ = gen.identity_list(n)
    w = np.zeros(n, dtype=np.int64)
    w[0 * TILE:1 * TILE] = (1 << 19) - 1                 # signed limit
    w[1 * TILE:2 * TILE] = -((1 << 19) - 1)
    w[2 * TILE:3 * TILE] = (1 << 20) - 1                 # unsigned limit
    w[3 * TILE:4 * TILE] = (1 << 19) - 1
    w[3 * TILE + 5] = -(1 << 19)                         # just past the signed limit, negative: 64-bit
    w[4 * TILE:5 * TILE] = (1 << 20) - 1
    w[4 * TILE + 9] = 1 << 20                            # just past the unsigned limit: 64-bit
    rng = np.random.default_rng(514)
    w[5 * TILE:] = rng.integers(-(1 << 19) + 1, 1 << 19, size=n - 5 * TILE)
    w = w.astype(wdt)
    want = oracle.rank(succ, w, np.int64)
    for t in (None, ON):
        np.testing.assert_array_equal(rank(succ, w, torch.int64, tuning=t), want)
    # locality order: many short local sublists per tile, same weights
    succ = gen.locality_list(n, 515)
    want = oracle.rank(succ, w, np.int64)
    np.testing.assert_array_equal(rank(succ, w, torch.int64, tuning=ON), want)


def test_euler_tour_forced():
    parent = gen.random_recursive_tree(1 << 16, 508)
    succ, w = gen.euler_tour(parent)
    np.testing.assert_array_equal(rank(succ, w, torch.int32, tuning=ON), oracle.rank(succ, w, np.int32))


def _status(succ, **kw):
    try:
        lr.rank(dev(succ), **kw)
        return "LR_OK"
    except lr.LRError as e:
        return e.name


def test_errors_with_contraction():
    n = 8 * TILE + 5
    succ = gen.identity_list(n).astype(np.int64)
    bad = succ.copy()
    bad[100] = n + 3
    assert _status(bad.astype(np.uint32), tuning=ON) == "LR_ERR_OUT_OF_RANGE"
    cyc = succ.copy()
    cyc[200] = 150                         # a cycle inside tile 0 (150..200), rest is a list
    assert oracle.rank_status(cyc.astype(np.uint32))[0] != oracle.OK
    assert _status(cyc.astype(np.uint32), tuning=ON) != "LR_OK"
    for a, b in ((1000, 1100), (1025, 1055), (2000, 2001), (3000, 3063)):   # headless cycles
        hc = succ.copy()                      # inside tile 0, of lengths 101, 31, 2 and 64
        hc[a - 1] = b + 1                     # the list skips a..b
        hc[b] = a                             # which close on themselves
        assert oracle.rank_status(hc.astype(np.uint32))[0] == oracle.CYCLE
        assert _status(hc.astype(np.uint32), tuning=ON) == "LR_ERR_CYCLE"
    cross = succ.copy()
    cross[n - 1] = 0                       # close the whole list into a cycle across tiles
    assert _status(cross.astype(np.uint32), tuning=ON) == "LR_ERR_CYCLE"
    two = succ.copy()
    two[3 * TILE + 10] = 50                # enters tile 0 in the middle: 50 has two predecessors
    assert oracle.rank_status(two.astype(np.uint32))[0] == oracle.NOT_A_LIST
    assert _status(two.astype(np.uint32), tuning=ON) != "LR_OK"
    assert _status(two.astype(np.uint32), tuning=ON, validate=True) == "LR_ERR_NOT_A_LIST"
    inner = succ.copy()
    inner[30] = 20                         # two predecessors of 20 inside tile 0
    assert _status(inner.astype(np.uint32), tuning=ON, validate=True) == "LR_ERR_NOT_A_LIST"
    # the stream still works
    np.testing.assert_array_equal(rank(succ.astype(np.uint32), tuning=ON), oracle.rank(succ.astype(np.uint32)))
