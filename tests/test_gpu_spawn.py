"""Ruler spawning (Section 2.2) on the GPU (lr_tuning.spawn = 1).

Spawning changes how many rulers there are and where, never the ranks:
every case is compared with the oracle, including runs with so few initial
rulers that spawned ones do nearly all the work, forests (spawners may claim
heads that are still queued) and every error case.  The ruler count is
checked against Section 2.5's estimate for t waves, t ln(n / t).
"""
import math

import numpy as np
import pytest

import gen
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2606_09318_gb300 as lr  # noqa: E402


def dev(a):
    a = np.ascontiguousarray(a)
    if a.dtype == np.uint32:
        a = a.view(np.int32)
    return torch.from_numpy(a).cuda()


def sp(**kw):
    return lr.Tuning(spawn=1, contract=lr.CONTRACT_OFF, **kw)


@pytest.mark.parametrize("n", [20000, (1 << 20) + 7, (1 << 22) + 1])
def test_random_lists(n):
    succ = gen.random_list(n, 600 + n % 13)
    want = oracle.rank(succ)
    np.testing.assert_array_equal(lr.rank(dev(succ), tuning=sp()).cpu().numpy(), want)
    few = sp(f0_inv=max(2, n // 500))                      # ~500 initial rulers
    np.testing.assert_array_equal(lr.rank(dev(succ), tuning=few).cpu().numpy(), want)
    sizes = lr.level_sizes()
    assert sizes[0] == n and sizes[1] > 500                # spawned rulers were added


@pytest.mark.parametrize("kind", ["locality", "identity"])
def test_local_orders(kind):
    succ = gen.list_of_order_kind(kind, (1 << 20) + 33, 601)
    np.testing.assert_array_equal(lr.rank(dev(succ), tuning=sp(f0_inv=4096)).cpu().numpy(),
                                  oracle.rank(succ))


@pytest.mark.parametrize("wkind,rdt", [("i32", np.int64), ("i64", np.int64), ("i32", np.int32)])
def test_weighted(wkind, rdt):
    n = (1 << 20) + 3
    succ = gen.random_list(n, 602)
    w = gen.weights_i32(n, 603) if wkind == "i32" else gen.weights_i64(n, 604, lo=-(1 << 40), hi=1 << 40)
    tdt = torch.int32 if rdt == np.int32 else torch.int64
    for t in (sp(), sp(f0_inv=2048)):
        got = lr.rank(dev(succ), dev(w), rank_dtype=tdt, tuning=t).cpu().numpy()
        np.testing.assert_array_equal(got, oracle.rank(succ, w, rdt))


@pytest.mark.parametrize("mean_short", [64, 4])
def test_forests_and_batch(mean_short):
    succ, nl = gen.forest(1 << 20, 605 + mean_short, n_long=4, long_len=1 << 15, mean_short=mean_short)
    want = oracle.rank(succ)
    for t in (sp(), sp(f0_inv=1 << 14)):
        np.testing.assert_array_equal(lr.rank(dev(succ), tuning=t).cpu().numpy(), want)
        np.testing.assert_array_equal(lr.rank(dev(succ), tuning=t, max_lists=nl).cpu().numpy(), want)
    k = 40
    offsets, bs, bw = gen.batch_instances(k, 606, lo_exp=2.0, hi_exp=17.0)
    got = lr.rank_batch(dev(offsets), dev(bs), dev(bw), tuning=sp(f0_inv=4096)).cpu().numpy()
    np.testing.assert_array_equal(got, oracle.rank_batch(offsets, bs, bw, np.int64))


def test_euler_tour():
    parent = gen.random_recursive_tree(1 << 18, 607)
    succ, w = gen.euler_tour(parent)
    got = lr.rank(dev(succ), dev(w), rank_dtype=torch.int32, tuning=sp(f0_inv=1024)).cpu().numpy()
    np.testing.assert_array_equal(got, oracle.rank(succ, w, np.int32))


def _status(succ, **kw):
    try:
        lr.rank(dev(succ), **kw)
        return "LR_OK"
    except lr.LRError as e:
        return e.name


def test_errors():
    n = (1 << 18) + 5
    succ = gen.random_list(n, 608).copy()
    hp = np.zeros(n, dtype=bool)
    hp[succ[succ != np.arange(n)]] = True
    head, tail = int(np.flatnonzero(~hp)[0]), int(np.flatnonzero(succ == np.arange(n))[0])
    for t in (sp(), sp(f0_inv=4096)):
        closed = succ.copy()
        closed[tail] = head
        assert _status(closed, tuning=t) == "LR_ERR_CYCLE"
        bad = succ.copy()
        bad[n // 3] = n + 1
        assert _status(bad, tuning=t) == "LR_ERR_OUT_OF_RANGE"
        rho = succ.copy()
        rho[tail] = succ[succ[head]]
        assert _status(rho, tuning=t, validate=True) == "LR_ERR_NOT_A_LIST"
        assert _status(rho, tuning=t) != "LR_OK"
        # a headless cycle beside a list: spawned rulers may land on it
        m = 5000
        cyc = np.arange(1, m + 1, dtype=np.int64) % m + n
        both = np.concatenate([succ.astype(np.int64), cyc]).astype(np.uint32)
        assert oracle.rank_status(both)[0] == oracle.CYCLE
        assert _status(both, tuning=t) == "LR_ERR_CYCLE"
    np.testing.assert_array_equal(lr.rank(dev(succ), tuning=sp()).cpu().numpy(), oracle.rank(succ))


def test_ruler_count():
    """With about one initial ruler per chasing thread (t waves), spawning
    keeps every thread busy and leaves about t ln(n / t) rulers in all; with
    spawning off the count is the initial rulers alone."""
    n = 1 << 24
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    t = sms * 8 * 256                                      # resident chase threads (8 CTAs of 256)
    f0 = max(2, n // t)
    succ = dev(gen.random_list(n, 609))
    lr.rank(succ, tuning=lr.Tuning(f0_inv=f0, contract=lr.CONTRACT_OFF))
    plain = lr.level_sizes()
    r0 = -(-n // f0)
    assert plain[0] == n and r0 <= plain[1] <= r0 + 1      # the sampled rulers and the head
    out = lr.rank(succ, tuning=sp(f0_inv=f0))
    spawned = lr.level_sizes()
    expect = t * math.log(n / t)
    assert 0.5 * expect < spawned[1] < 2.0 * expect, (spawned, expect)
    r = out.cpu().numpy()
    assert r.max() == n - 1 and np.unique(r).shape[0] == n
