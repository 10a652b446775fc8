"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle.

Integer results, so the bar is bit-exact equality on every element.  Sizes
span several tiles and ragged tails; at the full headline size the result is
checked by properties that determine it completely (tail rank 0 and the
recurrence rank[i] = w[i] + rank[succ[i]] on a single valid list).
"""
import numpy as np
import pytest

import gen
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - collected on CPU machines too
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2606_09318_gb300 as lr  # noqa: E402


def dev(a):
    a = np.ascontiguousarray(a)
    if a.dtype == np.uint32:
        a = a.view(np.int32)
    return torch.from_numpy(a).cuda()


def host(t):
    return t.cpu().numpy()


def check_equal(succ, weight=None, rank_dtype=np.int32, **kw):
    want = oracle.rank(succ, weight, rank_dtype)
    tdt = torch.int32 if rank_dtype == np.int32 else torch.int64
    got = lr.rank(dev(succ), None if weight is None else dev(weight), rank_dtype=tdt, **kw)
    np.testing.assert_array_equal(host(got), want)
    return got


@pytest.mark.parametrize("n", [1, 2, 3, 31, 32, 33, 1023, 1024, 1025, 8191, 8192, 8193,
                               12289, 65537, 1 << 20, (1 << 20) + 7])
def test_random_list_unweighted(n):
    check_equal(gen.random_list(n, 100 + n))


@pytest.mark.parametrize("kind", ["random", "locality", "identity"])
@pytest.mark.parametrize("n", [(1 << 22) + 3, 1 << 24])
def test_orders(kind, n):
    check_equal(gen.list_of_order_kind(kind, n, 7))


@pytest.mark.parametrize("wt,rt", [(np.int32, np.int64), (np.int64, np.int64),
                                   (np.int32, np.int32), (np.int64, np.int32)])
@pytest.mark.parametrize("n", [5, 4097, (1 << 20) + 1])
def test_weighted(wt, rt, n):
    succ = gen.random_list(n, 3 * n)
    if wt == np.int32:
        w = gen.weights_i32(n, 11)
    else:
        w = gen.weights_i64(n, 12, -(1 << 40), 1 << 40)
    check_equal(succ, w, rt)


def test_wraparound_extremes():
    n = 100_000
    succ = gen.random_list(n, 5)
    check_equal(succ, np.full(n, np.iinfo(np.int32).max, dtype=np.int32), np.int32)
    check_equal(succ, np.full(n, np.iinfo(np.int32).min, dtype=np.int32), np.int64)
    check_equal(succ, np.full(n, np.iinfo(np.int64).max, dtype=np.int64), np.int64)


def test_forest():
    succ, _ = gen.forest(1 << 22, 31, n_long=16, long_len=1 << 16, mean_short=64)
    check_equal(succ)


def test_forest_short_lists_and_singletons():
    succ, _ = gen.forest(1 << 20, 32, n_long=2, long_len=1 << 12, mean_short=2)
    check_equal(succ)
    check_equal(np.arange(300_000, dtype=np.uint32))          # all singletons


def test_euler_tour_depths():
    V = 1 << 18
    parent = gen.random_recursive_tree(V, 77)
    succ, w = gen.euler_tour(parent)
    r = host(check_equal(succ, w, np.int32)).astype(np.int64)
    depth = np.zeros(V, dtype=np.int64)
    for v in range(1, V):
        depth[v] = depth[parent[v]] + 1
    v = np.arange(1, V)
    np.testing.assert_array_equal(2 - r[2 * (v - 1)], depth[v])


def test_result_independent_of_seed_and_tuning():
    n = (1 << 21) + 5
    succ = gen.random_list(n, 9)
    want = oracle.rank(succ)
    s = dev(succ)
    for seed in (1, 2, 12345):
        np.testing.assert_array_equal(host(lr.rank(s, seed=seed)), want)
    for f0, f, cut in ((16, 4, 1024), (128, 16, 12288), (2, 2, 64), (32, 8, 4096)):
        t = lr.Tuning(f0_inv=f0, f_inv=f, cutoff=cut)
        np.testing.assert_array_equal(host(lr.rank(s, tuning=t)), want)
    for blk, ctas in ((128, 4), (512, 2), (256, 1)):
        t = lr.Tuning(chase_block=blk, chase_ctas=ctas)
        np.testing.assert_array_equal(host(lr.rank(s, tuning=t)), want)


def test_max_lists_path_matches_counted_path():
    succ, nl = gen.forest(1 << 20, 8, n_long=4, long_len=1 << 14, mean_short=64)
    s = dev(succ)
    a = host(lr.rank(s))
    b = host(lr.rank(s, max_lists=nl))
    np.testing.assert_array_equal(a, b)
    with pytest.raises(lr.LRError) as e:
        lr.rank(s, max_lists=max(1, nl // 4))
    assert e.value.name == "LR_ERR_CAPACITY"


def test_empty():
    out = lr.rank(torch.empty(0, dtype=torch.int32, device="cuda"))
    assert out.numel() == 0


def test_batch_matches_oracle_and_single_calls():
    offsets, succ, w = gen.batch_instances(64, 5, lo_exp=0.0, hi_exp=15.0)
    want = oracle.rank_batch(offsets, succ, w, np.int64)
    got = host(lr.rank_batch(dev(offsets), dev(succ), dev(w)))
    np.testing.assert_array_equal(got, want)
    got2 = host(lr.rank_batch(dev(offsets), dev(succ), dev(w), max_lists=64))
    np.testing.assert_array_equal(got2, want)
    for j in (0, 17, 63):
        a, b = offsets[j], offsets[j + 1]
        one = host(lr.rank(dev(succ[a:b]), dev(w[a:b])))
        np.testing.assert_array_equal(one, want[a:b])


def test_batch_unweighted_with_empty_instances():
    lens = np.array([0, 5, 0, 1, 300, 0, 70000, 2], dtype=np.int64)
    offsets = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
    succ = np.concatenate([gen.random_list(int(m), 40 + i) for i, m in enumerate(lens)]).astype(np.uint32)
    want = oracle.rank_batch(offsets, succ, None, np.int32)
    got = host(lr.rank_batch(dev(offsets), dev(succ), rank_dtype=torch.int32))
    np.testing.assert_array_equal(got, want)


def test_host_buffers_end_to_end():
    n = (1 << 20) + 3
    succ = gen.random_list(n, 44)
    np.testing.assert_array_equal(lr.rank_host(succ), oracle.rank(succ))
    w = gen.weights_i32(n, 45)
    np.testing.assert_array_equal(lr.rank_host(succ, w), oracle.rank(succ, w, np.int64))


@pytest.mark.parametrize("n", [1 << 28])
def test_full_size_properties(n):
    """Headline size: the recurrence and tail rank 0 pin the result exactly."""
    succ = torch.randperm(n, device="cuda", generator=torch.Generator("cuda").manual_seed(2028),
                          dtype=torch.int64)
    order = succ
    s = torch.empty(n, dtype=torch.int64, device="cuda")
    s[order[:-1]] = order[1:]
    s[order[-1]] = order[-1]
    s32 = s.to(torch.int32)
    del s
    r = lr.rank(s32).to(torch.int64)
    idx = torch.arange(n, device="cuda", dtype=torch.int64)
    sl = s32.to(torch.int64)
    term = sl == idx
    assert int(term.sum()) == 1
    assert int(r[term].item()) == 0
    nt = ~term
    assert bool((r[nt] == r[sl[nt]] + 1).all())
    assert int(r[order[0]].item()) == n - 1
    # sampled elements against the closed form: the element at list position p has rank n-1-p
    pos = torch.empty(n, dtype=torch.int64, device="cuda")
    pos[order] = torch.arange(n, device="cuda")
    pick = torch.randint(0, n, (4096,), device="cuda", generator=torch.Generator("cuda").manual_seed(3))
    assert bool((r[pick] == n - 1 - pos[pick]).all())


@pytest.mark.parametrize("path", ["log=0", "log=1", "log=1,f0=16,f=4", "xchg=0,log=0"])
def test_level0_paths(path, monkeypatch):
    """Both level-0 variants (log-based and in-place records) and their knobs."""
    monkeypatch.setenv("LR_TUNING", path)
    for n, seed in ((100_003, 1), ((1 << 20) + 9, 2)):
        check_equal(gen.random_list(n, seed))
        check_equal(gen.locality_list(n, seed))
    succ, _ = gen.forest(1 << 20, 3, n_long=4, long_len=1 << 14, mean_short=64)
    check_equal(succ)
    check_equal(gen.random_list(300_000, 4), rank_dtype=np.int64)


@pytest.mark.parametrize("n", [1 << 22, (1 << 22) + 12345, (1 << 24) + 3])
def test_log_path_two_level_partition(n, monkeypatch):
    """The log path at 256 windows of 2^14 ranks (the most one partition level
    holds) and past it: a level-A partition into A-buckets, then level B into
    windows (1 and 3 window bits)."""
    monkeypatch.setenv("LR_TUNING", "log=1")
    check_equal(gen.random_list(n, 48))
    check_equal(gen.locality_list(n, 49))
    succ, _ = gen.forest(n, 50, n_long=8, long_len=n // 16, mean_short=64)
    check_equal(succ)


def test_chase0_auto_and_forced():
    """The level-0 chase form: auto takes the log form for large unweighted
    single lists and the exchange form otherwise; either can be forced; the
    ranks are the same."""
    def form(succ, **kw):
        lr.profile_enable(True)
        lr.profile_read(reset=True)
        got = lr.rank(dev(succ), **kw)
        prof = lr.profile_read(reset=True)
        lr.profile_enable(False)
        assert prof["chase0_launches"] == 1
        return got, "log" if prof["chase0_log_launches"] == 1 else "exchange"
    big = gen.random_list((1 << 25) + 17, 52)
    want = oracle.rank(big)
    for t, expect in ((None, "log"), (lr.Tuning(chase0=lr.CHASE0_EXCHANGE), "exchange"),
                      (lr.Tuning(spawn=1), "exchange")):
        got, f = form(big, tuning=t)
        assert f == expect
        np.testing.assert_array_equal(host(got), want)
    got, f = form(big, rank_dtype=torch.int64)
    assert f == "exchange"
    np.testing.assert_array_equal(host(got), want.astype(np.int64))
    small = gen.random_list((1 << 20) + 5, 53)
    assert form(small)[1] == "exchange"
    got, f = form(small, tuning=lr.Tuning(chase0=lr.CHASE0_LOG))
    assert f == "log"
    np.testing.assert_array_equal(host(got), oracle.rank(small))
    # a locality order is contracted before either form is chosen
    loc = gen.locality_list((1 << 25) + 3, 54)
    lr.profile_enable(True)
    lr.profile_read(reset=True)
    np.testing.assert_array_equal(host(lr.rank(dev(loc))), oracle.rank(loc))
    prof = lr.profile_read(reset=True)
    lr.profile_enable(False)
    assert prof["chase0_log_launches"] == 0


@pytest.mark.parametrize("path,n", [
    ("log=1,f0=2", (1 << 20) + 3),            # a ruler at every other element: marks everywhere
    ("log=1,f0=65536", (1 << 22) + 1),        # segments of ~65536: mark-free chunks, long walks,
                                              # and a last window of one element after 256 full ones
    ("log=1", 12289),                         # just above the base case
    ("log=1,f0=3,f=2", 100_003),
])
def test_log_path_ruler_densities(path, n, monkeypatch):
    monkeypatch.setenv("LR_TUNING", path)
    check_equal(gen.random_list(n, 55))
    check_equal(gen.locality_list(n, 56))


@pytest.mark.parametrize("mean_short", [1, 2])
def test_log_path_forest_of_tiny_lists(mean_short, monkeypatch):
    """Mostly singletons and pairs: the heads come from the bitmap, most
    rulers are heads, and many segments are a single element."""
    monkeypatch.setenv("LR_TUNING", "log=1")
    succ, _ = gen.forest(1 << 21, 57 + mean_short, n_long=2, long_len=1 << 16, mean_short=mean_short)
    check_equal(succ)


def _status_of(succ, **kw):
    try:
        lr.rank(dev(succ), **kw)
        return "LR_OK"
    except lr.LRError as e:
        return e.name


@pytest.mark.parametrize("n", [300_007, (1 << 22) + 5])
def test_log_path_errors(n, monkeypatch):
    """Invalid lists on the log path report an error; the stream still works."""
    monkeypatch.setenv("LR_TUNING", "log=1")
    succ = gen.random_list(n, 51).astype(np.int64)
    hp = np.zeros(n, dtype=bool)
    hp[succ[succ != np.arange(n)]] = True
    head = int(np.flatnonzero(~hp)[0])
    tail = int(np.flatnonzero(succ == np.arange(n))[0])
    bad = succ.copy()
    bad[n // 3] = n + 7
    assert _status_of(bad.astype(np.uint32)) == "LR_ERR_OUT_OF_RANGE"
    closed = succ.copy()
    closed[tail] = head
    assert _status_of(closed.astype(np.uint32)) == "LR_ERR_CYCLE"
    rho = succ.copy()
    rho[tail] = succ[succ[head]]
    assert _status_of(rho.astype(np.uint32)) != "LR_OK"
    two = succ.copy()
    a = int(succ[head])
    b = int(succ[a])
    two[a] = int(succ[b])                      # b becomes a second head; succ[b] has two predecessors
    assert oracle.rank_status(two.astype(np.uint32))[0] == oracle.NOT_A_LIST
    assert _status_of(two.astype(np.uint32)) != "LR_OK"
    check_equal(succ.astype(np.uint32))


def test_host_async_two_streams():
    """lr_rank_host_async: calls alternate between two streams; each result is exact."""
    n = (1 << 20) + 3
    succ = gen.random_list(n, 46)
    want = oracle.rank(succ)
    hs = torch.from_numpy(succ.view(np.int32)).pin_memory()
    outs = [torch.empty(n, dtype=torch.int32).pin_memory() for _ in range(2)]
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    for i in range(4):
        lr.rank_host(hs, out=outs[i % 2].numpy(), stream=streams[i % 2], wait=False, max_lists=1)
    torch.cuda.synchronize()
    for j in range(2):
        assert lr.device_status(streams[j]) == 0
        np.testing.assert_array_equal(outs[j].numpy(), want)
    w = gen.weights_i32(n, 47)
    hw = torch.from_numpy(w).pin_memory()
    out64 = torch.empty(n, dtype=torch.int64).pin_memory()
    lr.rank_host(hs, hw, out=out64.numpy(), stream=streams[0], wait=False)
    torch.cuda.synchronize()
    assert lr.device_status(streams[0]) == 0
    np.testing.assert_array_equal(out64.numpy(), oracle.rank(succ, w, np.int64))


def _view(a, off):
    """A device copy of `a` that starts `off` elements into its allocation, so
    that 16-byte vector accesses cannot be used on it."""
    a = np.ascontiguousarray(a)
    if a.dtype == np.uint32:
        a = a.view(np.int32)
    buf = torch.zeros(a.size + off + 3, dtype=torch.from_numpy(a[:1]).dtype, device="cuda")
    v = buf[off:off + a.size]
    v.copy_(torch.from_numpy(a))
    return v


@pytest.mark.parametrize("kind", ["random", "locality"])
@pytest.mark.parametrize("wkind", [None, "i32", "i64"])
def test_misaligned_buffers(kind, wkind):
    """Successors, weights and ranks one or three elements past an aligned
    start: every kernel that reads or writes them in 16-byte vectors takes its
    scalar form, with the same result, whichever level-0 form or contraction
    runs."""
    n = 3 * 4096 * 8 + 13
    succ = gen.list_of_order_kind(kind, n, 60)
    w = None if wkind is None else (gen.weights_i32(n, 61) if wkind == "i32" else gen.weights_i64(n, 62))
    rdt = np.int32 if w is None else np.int64
    want = oracle.rank(succ, w, rdt)
    tunings = [None, lr.Tuning(contract=lr.CONTRACT_ON), lr.Tuning(contract=lr.CONTRACT_OFF)]
    if w is None:
        tunings.append(lr.Tuning(chase0=lr.CHASE0_LOG))
    for off in (1, 3):
        ds = _view(succ, off)
        dw = None if w is None else _view(w, off)
        for t in tunings:
            out = torch.full((n + off + 2,), -9, dtype=torch.int32 if rdt == np.int32 else torch.int64,
                             device="cuda")[off:off + n]
            lr.rank(ds, dw, out=out, tuning=t)
            np.testing.assert_array_equal(host(out), want)
