"""Whole-list pointer doubling (lr_tuning.algorithm = LR_ALGO_WYLLIE) on the GPU.

The comparison algorithm must return exactly the oracle's ranks on every
input the default algorithm accepts, report the same errors, and agree with
the default algorithm element by element.
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

PD = lr.Tuning(algorithm=lr.ALGO_WYLLIE)


def dev(a):
    a = np.ascontiguousarray(a)
    if a.dtype == np.uint32:
        a = a.view(np.int32)
    return torch.from_numpy(a).cuda()


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 1000, 4096, (1 << 20) + 7])
@pytest.mark.parametrize("kind", ["random", "locality", "identity"])
def test_unweighted(n, kind):
    succ = gen.list_of_order_kind(kind, n, 70 + n % 97)
    got = lr.rank(dev(succ), tuning=PD).cpu().numpy()
    np.testing.assert_array_equal(got, oracle.rank(succ))


@pytest.mark.parametrize("wkind,rdt", [("i32", np.int64), ("i64", np.int64), ("i32", np.int32)])
def test_weighted(wkind, rdt):
    n = (1 << 19) + 11
    succ = gen.random_list(n, 71)
    w = gen.weights_i32(n, 72) if wkind == "i32" else gen.weights_i64(n, 73, lo=-(1 << 40), hi=1 << 40)
    tdt = torch.int32 if rdt == np.int32 else torch.int64
    got = lr.rank(dev(succ), dev(w), rank_dtype=tdt, tuning=PD).cpu().numpy()
    np.testing.assert_array_equal(got, oracle.rank(succ, w, rdt))


def test_unweighted_int64_ranks_and_forest():
    succ, _ = gen.forest(1 << 20, 74, n_long=3, long_len=1 << 16, mean_short=64)
    got = lr.rank(dev(succ), rank_dtype=torch.int64, tuning=PD).cpu().numpy()
    np.testing.assert_array_equal(got, oracle.rank(succ, None, np.int64))
    np.testing.assert_array_equal(lr.rank(dev(succ), tuning=PD).cpu().numpy(), oracle.rank(succ))


def test_batch_and_agreement_with_default():
    k = 50
    offsets, succ, w = gen.batch_instances(k, 75, lo_exp=1.0, hi_exp=17.0)
    a = lr.rank_batch(dev(offsets), dev(succ), dev(w), tuning=PD).cpu().numpy()
    b = lr.rank_batch(dev(offsets), dev(succ), dev(w)).cpu().numpy()
    np.testing.assert_array_equal(a, oracle.rank_batch(offsets, succ, w, np.int64))
    np.testing.assert_array_equal(a, b)


def _status(succ, **kw):
    try:
        lr.rank(dev(succ), tuning=PD, **kw)
        return "LR_OK"
    except lr.LRError as e:
        return e.name


@pytest.mark.parametrize("cyc", [2, 3, 4, 8, 1000, 1 << 12])
def test_cycles_of_every_length(cyc):
    """Headless cycles beside a valid list, including lengths that are powers
    of two (a cycle of length 2^j returns to its start after 2^j steps)."""
    n = 5000
    a = gen.random_list(n, 76).astype(np.int64)
    order = np.random.default_rng(cyc).permutation(cyc) + n
    c = np.empty(cyc, dtype=np.int64)
    c[order - n] = np.roll(order, -1)
    succ = np.concatenate([a, c]).astype(np.uint32)
    assert oracle.rank_status(succ)[0] == oracle.CYCLE
    assert _status(succ) == "LR_ERR_CYCLE"
    # the next call still works
    good = gen.random_list(n, 77)
    np.testing.assert_array_equal(lr.rank(dev(good), tuning=PD).cpu().numpy(), oracle.rank(good))


def test_closed_cycle_and_range_and_two_predecessors():
    n = (1 << 16) + 3
    succ = gen.random_list(n, 78).copy()
    hp = np.zeros(n, dtype=bool)
    hp[succ[succ != np.arange(n)]] = True
    head, tail = int(np.flatnonzero(~hp)[0]), int(np.flatnonzero(succ == np.arange(n))[0])
    closed = succ.copy()
    closed[tail] = head
    assert _status(closed) == "LR_ERR_CYCLE"
    bad = succ.copy()
    bad[n // 2] = n + 5
    assert _status(bad) == "LR_ERR_OUT_OF_RANGE"
    rho = succ.copy()
    rho[tail] = succ[succ[head]]      # the tail joins the list again
    assert oracle.rank_status(rho)[0] == oracle.NOT_A_LIST
    assert _status(rho, validate=True) == "LR_ERR_NOT_A_LIST"
    assert _status(rho) == "LR_ERR_CYCLE"   # no terminal: caught without validation too
    skip = succ.copy()
    skip[head] = tail                 # the tail gets two predecessors
    assert oracle.rank_status(skip)[0] == oracle.NOT_A_LIST
    assert _status(skip, validate=True) == "LR_ERR_NOT_A_LIST"


def test_workspace_and_stream_forms():
    n = (1 << 18) + 1
    succ = gen.random_list(n, 79)
    ws = torch.empty(lr.workspace_size(n, tuning=PD), dtype=torch.uint8, device="cuda")
    s = torch.cuda.Stream()
    out = torch.empty(n, dtype=torch.int32, device="cuda")
    lr.rank_ex(dev(succ), out=out, tuning=PD, workspace=ws, sync=False, stream=s)
    assert lr.device_status(s) == 0
    np.testing.assert_array_equal(out.cpu().numpy(), oracle.rank(succ))
    small = torch.empty(1024, dtype=torch.uint8, device="cuda")
    with pytest.raises(lr.LRError):
        lr.rank_ex(dev(succ), tuning=PD, workspace=small)
