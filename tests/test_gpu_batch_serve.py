"""Batched form in a CUDA graph, and the serving loop (GPU).

The batch of k instances is one launch sequence over the forest they form;
with the list bound given (max_lists) and a caller workspace it neither
synchronises nor allocates, so it is captured in a CUDA graph and replayed
on new data.  The server must return, for every request, exactly what the
same request returns when ranked alone.
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


def test_batch_in_cuda_graph():
    k = 96
    offsets, succ, w = gen.batch_instances(k, 11, lo_exp=4.0, hi_exp=16.0)
    n = int(offsets[-1])
    want = oracle.rank_batch(offsets, succ, w, np.int64)
    d_off, d_succ, d_w = dev(offsets), dev(succ), dev(w)
    out = torch.empty(n, dtype=torch.int64, device="cuda")
    ws = torch.empty(lr.workspace_size(n, k, weighted=True, max_lists=k), dtype=torch.uint8, device="cuda")
    s = torch.cuda.Stream()
    kw = dict(out=out, max_lists=k, n_total=n, sync=False, stream=s, workspace=ws)
    with torch.cuda.stream(s):
        lr.rank_batch(d_off, d_succ, d_w, **kw)            # warm-up outside capture
    s.synchronize()
    assert lr.device_status(s) == 0
    np.testing.assert_array_equal(out.cpu().numpy(), want)
    g = torch.cuda.CUDAGraph()
    out.fill_(0)
    with torch.cuda.graph(g, stream=s):
        lr.rank_batch(d_off, d_succ, d_w, **kw)
    g.replay()
    torch.cuda.synchronize()
    np.testing.assert_array_equal(out.cpu().numpy(), want)
    # new data of the same shapes, same graph
    offsets2 = offsets.copy()
    succ2 = np.concatenate([gen.random_list(int(offsets[j + 1] - offsets[j]), 900 + j) for j in range(k)])
    w2 = gen.weights_i64(n, 901)
    d_succ.copy_(dev(succ2.astype(np.uint32)))
    d_w.copy_(dev(w2))
    g.replay()
    torch.cuda.synchronize()
    np.testing.assert_array_equal(out.cpu().numpy(), oracle.rank_batch(offsets2, succ2.astype(np.uint32), w2, np.int64))


def test_batch_equals_per_instance_loop():
    k = 40
    offsets, succ, w = gen.batch_instances(k, 12, lo_exp=2.0, hi_exp=17.0)
    got = lr.rank_batch(dev(offsets), dev(succ), dev(w), max_lists=k).cpu().numpy()
    for j in range(k):
        a, b = int(offsets[j]), int(offsets[j + 1])
        one = lr.rank(dev(succ[a:b]), dev(w[a:b])).cpu().numpy()
        np.testing.assert_array_equal(got[a:b], one)


def _requests(num, seed):
    g = np.random.default_rng(seed)
    reqs = []
    for i in range(num):
        m = int(2 ** g.uniform(4, 17))
        kind = "random" if i % 2 == 0 else "locality"
        succ = gen.list_of_order_kind(kind, m, seed * 100 + i)
        w = gen.weights_i64(m, seed * 100 + i + 7)
        reqs.append((succ, w))
    return reqs


@pytest.mark.parametrize("n_streams,plain", [(2, False), (3, False), (1, True)])
def test_server_alone_equals_in_mix(n_streams, plain):
    reqs = _requests(40, 5)
    srv = lr.Server(budget_bytes=2_000_000_000, n_streams=n_streams, max_batch=16, plain=plain)
    tickets = []
    for i, (succ, w) in enumerate(reqs):
        if i % 3 == 0:   # device-resident request, ranked in place
            tickets.append(srv.submit(dev(succ), dev(w)))
        else:            # host request, copied by the server
            tickets.append(srv.submit(torch.from_numpy(succ.view(np.int32)), torch.from_numpy(w)))
    for (succ, w), t in zip(reqs, tickets):
        out, info = srv.wait(t)
        alone = lr.rank(dev(succ), dev(w)).cpu().numpy()
        np.testing.assert_array_equal(out.cpu().numpy(), alone)
        np.testing.assert_array_equal(alone, oracle.rank(succ, w, np.int64))
        assert info["t_submit_ms"] <= info["t_admit_ms"] <= info["t_launch_ms"] <= info["t_done_ms"]
    st = srv.stats()
    assert st["completed"] == len(reqs) and st["p99_ms"] >= st["p50_ms"] > 0
    if not plain:
        assert st["batches"] <= len(reqs)
    else:
        assert st["ranked_alone"] == len(reqs)
    srv.close()


def test_server_large_requests_ranked_alone():
    # Requests of at least alone_min_n elements are batches of their own and
    # take the single-list path (which contracts the locality and identity
    # orders); smaller ones are batched.  Every result equals the oracle's.
    reqs = []
    for i in range(6):
        m = (1 << 17) + 1000 * i + 7
        kind = ("random", "locality", "identity")[i % 3]
        reqs.append((gen.list_of_order_kind(kind, m, 600 + i), gen.weights_i64(m, 700 + i)))
    for i in range(10):
        m = 3000 + 977 * i
        reqs.append((gen.list_of_order_kind(("random", "locality")[i % 2], m, 800 + i), gen.weights_i64(m, 900 + i)))
    order = np.random.default_rng(3).permutation(len(reqs))
    reqs = [reqs[i] for i in order]
    for alone_min, n_big in ((1 << 16, 6), (-1, 0)):
        srv = lr.Server(budget_bytes=4_000_000_000, n_streams=1, max_batch=32, alone_min_n=alone_min)
        tickets = [srv.submit(dev(s_), dev(w_)) for s_, w_ in reqs]
        for (succ, w), t in zip(reqs, tickets):
            out, _ = srv.wait(t)
            np.testing.assert_array_equal(out.cpu().numpy(), oracle.rank(succ, w, np.int64))
        st = srv.stats()
        assert st["completed"] == len(reqs)
        assert st["ranked_alone"] >= n_big       # plus small requests that happened to arrive alone
        srv.close()


def test_server_budget_and_errors():
    srv = lr.Server(budget_bytes=50_000_000, n_streams=2)
    big = torch.zeros(10_000_000, dtype=torch.int32)
    with pytest.raises(lr.LRError) as e:
        srv.submit(big)
    assert e.value.name == "LR_ERR_BUDGET"
    # an invalid request fails alone; its neighbours in the batch still succeed
    good = gen.random_list(5000, 1)
    bad = good.copy()
    bad[3] = 5000
    t1 = srv.submit(torch.from_numpy(good.view(np.int32)))
    t2 = srv.submit(torch.from_numpy(bad.view(np.int32)))
    t3 = srv.submit(torch.from_numpy(good.view(np.int32)))
    out1, _ = srv.wait(t1)
    with pytest.raises(lr.LRError) as e2:
        srv.wait(t2)
    assert e2.value.name == "LR_ERR_OUT_OF_RANGE"
    out3, _ = srv.wait(t3)
    np.testing.assert_array_equal(out1.numpy(), oracle.rank(good))
    np.testing.assert_array_equal(out3.numpy(), oracle.rank(good))
    with pytest.raises(lr.LRError):
        srv.wait(123456)
    srv.close()


def _batch(lens, seed, forest_at=()):
    """Instances of the given sizes back to back (local successor ids): random
    single lists, or a forest of short lists for the indices in forest_at."""
    offsets = np.zeros(len(lens) + 1, dtype=np.int64)
    np.cumsum(lens, out=offsets[1:])
    succ = np.empty(int(offsets[-1]), dtype=np.uint32)
    for j, m in enumerate(lens):
        a, b = int(offsets[j]), int(offsets[j + 1])
        if m == 0:
            continue
        if j in forest_at and m > 8:
            succ[a:b] = gen.forest(m, seed + j, n_long=1, long_len=m // 4, mean_short=4)[0]
        else:
            succ[a:b] = gen.random_list(m, seed + j)
    return offsets, succ


@pytest.mark.parametrize("weighted", [False, True])
def test_batch_heads_from_sums(weighted):
    # With the list bound given, a batch takes each instance's head from the
    # sums of its successors.  Ragged sizes put instance boundaries inside
    # warps and groups of four; empty instances are skipped.
    rng = np.random.default_rng(31)
    lens = rng.integers(1, 500, size=64)
    lens[[3, 10, 11]] = 0
    lens[20] = 1
    offsets, succ = _batch(lens, 900)
    n = int(offsets[-1])
    assert n > 12288
    w = gen.weights_i64(n, 901) if weighted else None
    want = oracle.rank_batch(offsets, succ, w, np.int64 if weighted else np.int32)
    rdt = torch.int64 if weighted else torch.int32
    for ml in (0, 64, 200):                                  # 0: the call counts the lists
        got = lr.rank_batch(dev(offsets), dev(succ), None if w is None else dev(w), rank_dtype=rdt,
                            max_lists=ml).cpu().numpy()
        np.testing.assert_array_equal(got, want)


def test_batch_sums_fallbacks_and_errors():
    rng = np.random.default_rng(32)
    lens = rng.integers(100, 900, size=48)
    # instances that are forests: the heads come from the bitmap instead
    offsets, succ = _batch(lens, 950, forest_at=(5, 6, 40))
    want = oracle.rank_batch(offsets, succ, None, np.int32)
    lists = sum(int((succ[int(offsets[j]):int(offsets[j + 1])] ==
                     np.arange(int(offsets[j + 1] - offsets[j]))).sum()) for j in range(len(lens)))
    for ml in (lists, 0):
        got = lr.rank_batch(dev(offsets), dev(succ), rank_dtype=torch.int32, max_lists=ml).cpu().numpy()
        np.testing.assert_array_equal(got, want)
    # more lists than the bound: a capacity error, as without the sums
    with pytest.raises(lr.LRError) as e:
        lr.rank_batch(dev(offsets), dev(succ), rank_dtype=torch.int32, max_lists=len(lens))
    assert e.value.name == "LR_ERR_CAPACITY"
    # a single-list batch with one bad instance
    offsets, succ = _batch(lens, 960)
    bad = succ.copy()
    a = int(offsets[7])
    bad[a + 3] = int(offsets[8] - offsets[7]) + 5            # out of its instance
    with pytest.raises(lr.LRError) as e:
        lr.rank_batch(dev(offsets), dev(bad), rank_dtype=torch.int32, max_lists=len(lens))
    assert e.value.name == "LR_ERR_OUT_OF_RANGE"
    cyc = succ.copy()                                        # a list plus a cycle, one terminal
    m = int(offsets[9] - offsets[8])
    order = np.asarray(gen.random_order(m, 961), dtype=np.int64)
    loc = np.empty(m, dtype=np.uint32)
    loc[order[:-1]] = order[1:]
    loc[order[-1]] = order[-1]
    loc[order[m // 2 - 1]] = order[m - 1]                    # the list skips the middle
    loc[order[m - 2]] = order[m // 2]                        # which closes on itself
    cyc[int(offsets[8]):int(offsets[9])] = loc
    assert oracle.rank_batch_status(offsets, cyc, None, np.int32)[0] != oracle.OK
    with pytest.raises(lr.LRError):
        lr.rank_batch(dev(offsets), dev(cyc), rank_dtype=torch.int32, max_lists=len(lens))
    # the stream still works
    got = lr.rank_batch(dev(offsets), dev(succ), rank_dtype=torch.int32, max_lists=len(lens)).cpu().numpy()
    np.testing.assert_array_equal(got, oracle.rank_batch(offsets, succ, None, np.int32))


def test_batch_bad_offset_table():
    # A decreasing offset table is reported, not trusted: with or without a
    # list bound the call fails with an error status.
    n = 20000
    succ = gen.random_list(n, 970)
    offsets = np.array([0, 5000, 3000, n], dtype=np.int64)
    for ml in (0, 3):
        with pytest.raises(lr.LRError):
            lr.rank_batch(dev(offsets), dev(succ), rank_dtype=torch.int32, max_lists=ml, n_total=n)
    good = np.array([0, 5000, 12000, n], dtype=np.int64)
    parts = [gen.random_list(int(good[j + 1] - good[j]), 971 + j) for j in range(3)]
    s2 = np.concatenate(parts).astype(np.uint32)
    got = lr.rank_batch(dev(good), dev(s2), rank_dtype=torch.int32, max_lists=3).cpu().numpy()
    np.testing.assert_array_equal(got, oracle.rank_batch(good, s2, None, np.int32))


@pytest.mark.parametrize("wt", [None, "i32", "i64"])
def test_server_forest_heads_from_sums(wt):
    # Waiting requests are ranked as one forest of per-request buffers; its
    # heads come from per-request sums (one head per list request).  Requests
    # shorter than a warp's 128 elements share warps; requests that are
    # forests themselves make the heads fall back to the predecessor bitmap;
    # an invalid request fails alone.
    rng = np.random.default_rng(77)
    reqs = []
    for i in range(60):
        m = int(rng.choice([1, 2, 5, 37, 130, 700, 4000, 20000]))
        if i in (11, 40) and m > 8:
            s = gen.forest(m, 7700 + i, n_long=1, long_len=m // 4, mean_short=4)[0].astype(np.uint32)
        else:
            s = gen.random_list(m, 7700 + i).astype(np.uint32)
        w = None if wt is None else (gen.weights_i32(m, 7800 + i) if wt == "i32" else gen.weights_i64(m, 7800 + i))
        reqs.append((s, w))
    bad = gen.random_list(3000, 7999).astype(np.uint32)
    bad[17] = 3000 + 4                                        # outside its request
    for with_forest in (False, True):
        use = [r for i, r in enumerate(reqs) if with_forest or i not in (11, 40)]
        srv = lr.Server(budget_bytes=1 << 30, n_streams=1, max_batch=64, alone_min_n=1 << 22)
        try:
            tickets = [srv.submit(dev(s), None if w is None else dev(w)) for s, w in use]
            tbad = srv.submit(dev(bad))
            for t, (s, w) in zip(tickets, use):
                got, _ = srv.wait(t)
                np.testing.assert_array_equal(got.cpu().numpy(),
                                              oracle.rank(s, w, np.int64 if w is not None else np.int32))
            with pytest.raises(lr.LRError) as e:
                srv.wait(tbad)
            assert e.value.name == "LR_ERR_OUT_OF_RANGE"
        finally:
            srv.close()
