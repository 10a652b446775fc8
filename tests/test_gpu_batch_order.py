"""Level 0 of a batch in element order (GPU).

A batch chases its level-0 rulers in element order: one queue over the
heads and then the sampled rulers sorted by position, so that all CTAs
advance one front across the instances, and the sampled rulers take their
ids in that order.  LR_TUNING=ord=0 restores the per-CTA slices of ruler
ids.  Either way every instance must be ranked exactly as the oracle ranks
it: ragged and empty instances, instances shorter than the ruler spacing,
heads that are sampled rulers, instances that are forests, both record
widths, both rank widths, and inputs that are not lists.
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


def dev(a):
    a = np.ascontiguousarray(a)
    if a.dtype == np.uint32:
        a = a.view(np.int32)
    return torch.from_numpy(a).cuda()


def _lens(seed, k, hi_exp):
    rng = np.random.default_rng(seed)
    lens = np.floor(2.0 ** rng.uniform(0.0, hi_exp, size=k)).astype(np.int64)
    lens[rng.choice(k, size=k // 10, replace=False)] = 0          # empty instances
    return lens


def _batch(lens, seed, forest_at=()):
    offsets = np.zeros(len(lens) + 1, dtype=np.int64)
    np.cumsum(lens, out=offsets[1:])
    parts = []
    for j, m in enumerate(lens):
        m = int(m)
        if j in forest_at and m >= 4:
            # two lists in one instance: cut one random list in the middle
            order = np.asarray(gen.random_order(m, seed + j), dtype=np.int64)
            loc = np.empty(m, dtype=np.uint32)
            loc[order[:-1]] = order[1:]
            loc[order[-1]] = order[-1]
            loc[order[m // 2]] = order[m // 2]
            parts.append(loc)
        else:
            parts.append(gen.random_list(m, seed + j).astype(np.uint32) if m else np.zeros(0, np.uint32))
    return offsets, np.concatenate(parts).astype(np.uint32)


def _weights(kind, n, seed):
    if kind is None:
        return None
    return gen.weights_i32(n, seed) if kind == "i32" else gen.weights_i64(n, seed)


@pytest.mark.parametrize("tuning", ["ord=1,f0=2", "ord=1,f0=16", "ord=1,f0=64,ctas=1", "ord=0,f0=16"])
@pytest.mark.parametrize("wt,rdt", [(None, np.int32), (None, np.int64), ("i32", np.int64), ("i64", np.int64)])
def test_batch_order_equals_oracle(monkeypatch, tuning, wt, rdt):
    lens = _lens(41, 300, 15.0)
    offsets, succ = _batch(lens, 4100, forest_at=(7, 150))
    n = int(offsets[-1])
    assert n > 12288                                          # beyond the single-CTA base case
    w = _weights(wt, n, 4101)
    want = oracle.rank_batch(offsets, succ, w, rdt)
    lists = sum(int((succ[int(offsets[j]):int(offsets[j + 1])] ==
                     np.arange(int(offsets[j + 1] - offsets[j]))).sum()) for j in range(len(lens)))
    monkeypatch.setenv("LR_TUNING", tuning)
    tdt = torch.int32 if rdt == np.int32 else torch.int64
    for ml in (0, lists):                                     # 0: the call counts the lists
        got = lr.rank_batch(dev(offsets), dev(succ), None if w is None else dev(w), rank_dtype=tdt,
                            max_lists=ml).cpu().numpy()
        np.testing.assert_array_equal(got, want)


def test_batch_orders_agree_at_size(monkeypatch):
    # a 1024-instance batch of the benchmark's size mix, scaled down to about
    # 2^25 elements: both orders give the same ranks and the recurrence holds
    k = 1024
    lens = gen.batch_lengths(k, 43, 4.0, 18.0)
    offsets, succ = _batch(lens, 4300)
    n = int(offsets[-1])
    w = gen.weights_i64(n, 4301)
    d_off, d_succ, d_w = dev(offsets), dev(succ), dev(w)
    outs = []
    for t in ("ord=1", "ord=0"):
        monkeypatch.setenv("LR_TUNING", t)
        outs.append(lr.rank_batch(d_off, d_succ, d_w, max_lists=k).cpu().numpy())
    np.testing.assert_array_equal(outs[0], outs[1])
    inst = np.repeat(np.arange(k), lens)
    g = offsets[inst] + succ.astype(np.int64)                 # global successors
    r = outs[0]
    tail = g == np.arange(n)
    assert (r[tail] == 0).all()
    assert (r[~tail] == r[g[~tail]] + w[~tail]).all()


def test_batch_order_detects_bad_lists(monkeypatch):
    monkeypatch.setenv("LR_TUNING", "ord=1,f0=8")
    lens = np.random.default_rng(44).integers(200, 3000, size=40)
    offsets, succ = _batch(lens, 4400)
    # two predecessors inside instance 5
    bad = succ.copy()
    a, m = int(offsets[5]), int(lens[5])
    tgt = int(bad[a])
    j = next(i for i in range(m) if bad[a + i] != tgt and bad[a + i] != i)
    bad[a + j] = tgt
    assert oracle.rank_batch_status(offsets, bad, None, np.int32)[0] != oracle.OK
    with pytest.raises(lr.LRError):
        lr.rank_batch(dev(offsets), dev(bad), rank_dtype=torch.int32, max_lists=0)
    # a cycle beside a list in instance 9
    cyc = succ.copy()
    a, m = int(offsets[9]), int(lens[9])
    order = np.asarray(gen.random_order(m, 4401), dtype=np.int64)
    loc = np.empty(m, dtype=np.uint32)
    loc[order[:-1]] = order[1:]
    loc[order[-1]] = order[-1]
    loc[order[m // 2 - 1]] = order[m - 1]
    loc[order[m - 2]] = order[m // 2]
    cyc[a:a + m] = loc
    assert oracle.rank_batch_status(offsets, cyc, None, np.int32)[0] != oracle.OK
    with pytest.raises(lr.LRError):
        lr.rank_batch(dev(offsets), dev(cyc), rank_dtype=torch.int32, max_lists=len(lens))
    # a successor outside its instance
    rng_bad = succ.copy()
    rng_bad[int(offsets[3]) + 1] = int(lens[3]) + 2
    with pytest.raises(lr.LRError) as e:
        lr.rank_batch(dev(offsets), dev(rng_bad), rank_dtype=torch.int32, max_lists=len(lens))
    assert e.value.name == "LR_ERR_OUT_OF_RANGE"
    # the stream still works
    got = lr.rank_batch(dev(offsets), dev(succ), rank_dtype=torch.int32, max_lists=len(lens)).cpu().numpy()
    np.testing.assert_array_equal(got, oracle.rank_batch(offsets, succ, None, np.int32))


def test_request_forest_in_order(monkeypatch):
    # the server ranks waiting small requests as one forest of per-request
    # buffers: the same element order applies there
    monkeypatch.setenv("LR_TUNING", "ord=1,f0=8")
    reqs = []
    for i in range(24):
        m = int(2 ** np.random.default_rng(4500 + i).uniform(4, 14))
        s = gen.random_list(m, 4500 + i).astype(np.uint32)
        w = gen.weights_i64(m, 4600 + i)
        reqs.append((s, w))
    srv = lr.Server(budget_bytes=1 << 30, n_streams=1, alone_min_n=1 << 20)
    try:
        tickets = [srv.submit(dev(s), dev(w)) for s, w in reqs]
        for t, (s, w) in zip(tickets, reqs):
            got, _ = srv.wait(t)
            got = got.cpu().numpy()
            np.testing.assert_array_equal(got, oracle.rank(s, w, np.int64))
    finally:
        srv.close()


@pytest.mark.parametrize("tuning", ["ord=2,f0=8", "ord=0,f0=8"])
def test_batch_order_with_validation(monkeypatch, tuning):
    # validation marks predecessors with a bitmap during the first pass (the
    # element order then reuses that bitmap for its ruler marks)
    monkeypatch.setenv("LR_TUNING", tuning)
    lens = _lens(46, 120, 14.0)
    offsets, succ = _batch(lens, 4700, forest_at=(3,))
    n = int(offsets[-1])
    w = gen.weights_i64(n, 4701)
    for ml in (0, 200):
        got = lr.rank_batch(dev(offsets), dev(succ), dev(w), validate=True, max_lists=ml).cpu().numpy()
        np.testing.assert_array_equal(got, oracle.rank_batch(offsets, succ, w, np.int64))
    j = int(np.argmax(lens))
    a, m = int(offsets[j]), int(lens[j])
    bad = succ.copy()
    tgt = int(bad[a])
    i = next(i for i in range(m) if bad[a + i] != tgt and bad[a + i] != i)
    bad[a + i] = tgt                                           # two predecessors
    with pytest.raises(lr.LRError) as e:
        lr.rank_batch(dev(offsets), dev(bad), dev(w), validate=True)
    assert e.value.name == "LR_ERR_NOT_A_LIST"
