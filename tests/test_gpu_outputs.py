"""Extra outputs of Section 1.1 on the GPU (lr_rank_outputs / lr_rank_batch_outputs).

Terminal ids, head-relative ranks and the inclusive-tail form must equal the
oracle's (oracle.rank_ext) element by element, through every path the
recursion can take: the base case alone, SRS levels ending in the
single-CTA base case, and the grid-wide pointer-doubling fallback that many
short lists force; single-head and bitmap head detection; batches.
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


def check(succ, weight=None, rdt=np.int32, inclusive=False, **kw):
    want_r, want_t, want_p = oracle.rank_ext(succ, weight, rdt, inclusive=inclusive)
    tdt = torch.int32 if rdt == np.int32 else torch.int64
    r, t, p = lr.rank_outputs(dev(succ), None if weight is None else dev(weight), term=True,
                              prefix=True, inclusive_tail=inclusive, rank_dtype=tdt, **kw)
    np.testing.assert_array_equal(r.cpu().numpy(), want_r)
    np.testing.assert_array_equal(t.cpu().numpy().view(np.uint32), want_t)
    np.testing.assert_array_equal(p.cpu().numpy(), want_p)


@pytest.mark.parametrize("n", [1, 2, 3, 5000, 12288, 12289, 100003, (1 << 20) + 7])
@pytest.mark.parametrize("inclusive", [False, True])
def test_single_list(n, inclusive):
    succ = gen.random_list(n, 300 + n % 101)
    check(succ, inclusive=inclusive)
    check(succ, inclusive=inclusive, validate=True)          # bitmap head detection


@pytest.mark.parametrize("wkind,rdt", [("i32", np.int64), ("i64", np.int64), ("i32", np.int32)])
def test_weighted(wkind, rdt):
    n = (1 << 19) + 3
    succ = gen.locality_list(n, 301)
    w = gen.weights_i32(n, 302) if wkind == "i32" else gen.weights_i64(n, 303, lo=-(1 << 35), hi=1 << 35)
    check(succ, w, rdt)
    check(succ, w, rdt, inclusive=True)


@pytest.mark.parametrize("mean_short,long_len", [(64, 1 << 14), (4, 1 << 10), (2, 64)])
def test_forests_including_pd_fallback(mean_short, long_len):
    """mean_short = 2 or 4 leaves ~2^18..2^19 lists in 2^20 elements: the
    levels stop shrinking and the grid-wide pointer doubling ranks the last one."""
    succ, nl = gen.forest(1 << 20, 304 + mean_short, n_long=4, long_len=long_len, mean_short=mean_short)
    w = gen.weights_i32(1 << 20, 305)
    check(succ)
    check(succ, w, np.int64, inclusive=True)
    check(succ, max_lists=nl)


def test_batch_local_terminals():
    k = 60
    offsets, succ, w = gen.batch_instances(k, 306, lo_exp=0.0, hi_exp=16.0)
    want_r, want_t, want_p = oracle.rank_ext_batch(offsets, succ, w, np.int64, inclusive=True)
    r, t, p = lr.rank_batch_outputs(dev(offsets), dev(succ), dev(w), term=True, prefix=True,
                                    inclusive_tail=True, max_lists=k)
    np.testing.assert_array_equal(r.cpu().numpy(), want_r)
    np.testing.assert_array_equal(t.cpu().numpy().view(np.uint32), want_t)
    np.testing.assert_array_equal(p.cpu().numpy(), want_p)
    # ranks alone equal the plain batched call
    np.testing.assert_array_equal(
        lr.rank_batch(dev(offsets), dev(succ), dev(w)).cpu().numpy(),
        oracle.rank_batch(offsets, succ, w, np.int64))


def test_only_some_outputs_and_workspace():
    n = (1 << 18) + 9
    succ = gen.random_list(n, 307)
    want_r, want_t, want_p = oracle.rank_ext(succ, None, np.int32, inclusive=True)
    r, t, p = lr.rank_outputs(dev(succ), term=False, prefix=True)
    assert t is None
    np.testing.assert_array_equal(p.cpu().numpy(), want_p)
    r, t, p = lr.rank_outputs(dev(succ), term=False, prefix=False, inclusive_tail=True)
    np.testing.assert_array_equal(r.cpu().numpy(), want_r)
    # unweighted, the terminal weighs 0 (Section 1.1): the inclusive form is the plain rank
    np.testing.assert_array_equal(r.cpu().numpy(), oracle.rank(succ))
    ws = torch.empty(lr.workspace_size(n, max_lists=1, term=True), dtype=torch.uint8, device="cuda")
    s = torch.cuda.Stream()
    r, t, p = lr.rank_outputs(dev(succ), term=True, workspace=ws, max_lists=1, sync=False, stream=s)
    assert lr.device_status(s) == 0
    np.testing.assert_array_equal(t.cpu().numpy().view(np.uint32), want_t)
    small = torch.empty(lr.workspace_size(n, max_lists=1), dtype=torch.uint8, device="cuda")
    with pytest.raises(lr.LRError):
        lr.rank_outputs(dev(succ), term=True, prefix=True, workspace=small, max_lists=1)


def test_euler_tour_depths():
    """The Euler-tour technique on the GPU: depth(parent v) = prefix[down(v)]
    and depth(v) = prefix[up(v)], against depths from the tree itself."""
    V = 1 << 18
    parent = gen.random_recursive_tree(V, 308)
    succ, w = gen.euler_tour(parent)
    _, t, p = lr.rank_outputs(dev(succ), dev(w), term=True, prefix=True, rank_dtype=torch.int32)
    p = p.cpu().numpy().astype(np.int64)
    depth = np.zeros(V, dtype=np.int64)
    for v in range(1, V):
        depth[v] = depth[parent[v]] + 1
    v = np.arange(1, V)
    np.testing.assert_array_equal(p[2 * (v - 1)], depth[parent[v]])
    np.testing.assert_array_equal(p[2 * (v - 1) + 1], depth[v])
    t = t.cpu().numpy().view(np.uint32)
    assert np.all(t == t[0]) and succ[t[0]] == t[0]


def test_errors_and_unsupported():
    n = 5000
    succ = gen.random_list(n, 309).copy()
    bad = succ.copy()
    bad[7] = n + 1
    with pytest.raises(lr.LRError) as e:
        lr.rank_outputs(dev(bad), term=True, prefix=True)
    assert e.value.name == "LR_ERR_OUT_OF_RANGE"
    with pytest.raises(lr.LRError) as e:
        lr.rank_outputs(dev(succ), term=True, tuning=lr.Tuning(algorithm=lr.ALGO_WYLLIE))
    assert e.value.name == "LR_ERR_INVALID_ARGUMENT"
    # the stream is still usable
    check(succ)
