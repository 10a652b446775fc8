"""Host-buffer pipeline (lr_pipeline_*) on the GPU.

Every submission must return exactly what the oracle returns for it, whatever
its neighbours in the pipeline are; a failing submission is reported with its
index and leaves the other submissions' ranks intact.
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


def pinned(a):
    a = np.ascontiguousarray(a)
    if a.dtype == np.uint32:
        a = a.view(np.int32)
    return torch.from_numpy(a).pin_memory()


def _lists(seed):
    """Ragged sizes across the base-case cutoff, an empty list and a forest."""
    out = []
    for i, n in enumerate([1, 3000, 12289, (1 << 20) + 5, 0, 77777, (1 << 21) - 3]):
        out.append(gen.random_list(n, seed + i) if n else np.zeros(0, dtype=np.uint32))
    out.append(gen.forest(1 << 20, seed + 50, n_long=3, long_len=1 << 16, mean_short=512)[0])
    out.append(gen.locality_list(300001, seed + 60))
    return out


@pytest.mark.parametrize("depth,max_lists", [(2, 0), (3, 0), (4, 4096)])
def test_pipeline_unweighted(depth, max_lists):
    lists = _lists(10 * depth)
    pipe = lr.Pipeline(1 << 21, depth=depth, max_lists=max_lists)
    for rep in range(2):                      # the second pass reuses every slot
        outs = [pipe.submit(pinned(s)) for s in lists]
        pipe.wait()
        for s, o in zip(lists, outs):
            np.testing.assert_array_equal(o.numpy(), oracle.rank(s))
    pipe.close()


@pytest.mark.parametrize("wdt,depth", [(np.int32, 2), (np.int64, 2), (np.int64, 4)])
def test_pipeline_weighted(wdt, depth):
    lists = _lists(7)
    pipe = lr.Pipeline(1 << 21, wtype=wdt, depth=depth)
    ws, outs = [], []
    for i, s in enumerate(lists):
        w = (gen.weights_i32 if wdt == np.int32 else gen.weights_i64)(s.shape[0], 100 + i)
        ws.append(w)
        outs.append(pipe.submit(pinned(s), pinned(w)))
    pipe.wait()
    for s, w, o in zip(lists, ws, outs):
        assert o.dtype == torch.int64
        np.testing.assert_array_equal(o.numpy(), oracle.rank(s, w, np.int64))
    pipe.close()


@pytest.mark.parametrize("depth", [2, 3])
def test_pipeline_error_index_and_neighbours(depth):
    # depth 3 ranks on two streams: submissions 1 and 4 fail on different
    # streams, and the lowest index is the one reported
    n = (1 << 20) + 1
    good = gen.random_list(n, 31)
    bad = good.copy()
    bad[n // 3] = n + 9
    assert oracle.rank_status(bad)[0] == oracle.OUT_OF_RANGE
    pipe = lr.Pipeline(n, depth=depth)
    o0 = pipe.submit(pinned(good))
    pipe.submit(pinned(bad))
    o2 = pipe.submit(pinned(good))
    if depth > 2:
        o3 = pipe.submit(pinned(good))
        pipe.submit(pinned(bad))
    with pytest.raises(lr.LRError) as e:
        pipe.wait()
    assert e.value.name == "LR_ERR_OUT_OF_RANGE" and e.value.index == 1
    if depth > 2:
        np.testing.assert_array_equal(o3.numpy(), oracle.rank(good))
    want = oracle.rank(good)
    np.testing.assert_array_equal(o0.numpy(), want)
    np.testing.assert_array_equal(o2.numpy(), want)
    # the pipeline carries on after the failure
    o3 = pipe.submit(pinned(good))
    pipe.wait()
    np.testing.assert_array_equal(o3.numpy(), want)
    pipe.close()


def test_pipeline_list_bound():
    succ, nl = gen.forest(1 << 20, 8, n_long=4, long_len=1 << 14, mean_short=64)
    pipe = lr.Pipeline(1 << 20, depth=2, max_lists=max(1, nl // 4))
    one = gen.random_list(1 << 20, 9)
    o0 = pipe.submit(pinned(one))
    pipe.submit(pinned(succ))
    with pytest.raises(lr.LRError) as e:
        pipe.wait()
    assert e.value.name == "LR_ERR_CAPACITY" and e.value.index == 1
    np.testing.assert_array_equal(o0.numpy(), oracle.rank(one))
    pipe.close()


def test_pipeline_argument_errors():
    pipe = lr.Pipeline(1000, depth=2)
    with pytest.raises(lr.LRError) as e:
        pipe.submit(pinned(gen.random_list(1001, 1)))
    assert e.value.name == "LR_ERR_INVALID_ARGUMENT"
    with pytest.raises(lr.LRError):                 # weights on an unweighted pipeline
        pipe.submit(pinned(gen.random_list(10, 1)), pinned(np.ones(10, dtype=np.int64)))
    pipe.wait()                                     # nothing was enqueued
    pipe.close()
    for bad in (dict(depth=1), dict(depth=5), dict(max_lists=-1)):
        with pytest.raises(lr.LRError):
            lr.Pipeline(1000, **bad)


@pytest.mark.parametrize("depth,max_lists", [(2, 0), (3, 0), (4, 600_000)])
def test_pipeline_log_form_sizes(depth, max_lists):
    """Lists of 2^25 and more take the log form at level 0 (auto): through the
    pipeline's own workspaces (one per ranking stream, sized by
    lr_workspace_size with a list bound), in every slot, next to smaller
    lists ranked with the exchange form; depth 3 and 4 rank two at a time."""
    big = (1 << 25) + 1
    lists = [gen.random_list(big, 70), gen.random_list(100_003, 71), gen.random_list(big - 64, 72),
             gen.forest(big, 73, n_long=4, long_len=1 << 20, mean_short=64)[0]]
    pipe = lr.Pipeline(big, depth=depth, max_lists=max_lists)
    outs = [pipe.submit(pinned(s)) for s in lists]
    pipe.wait()
    for s, o in zip(lists, outs):
        np.testing.assert_array_equal(o.numpy(), oracle.rank(s))
    pipe.close()


def test_log_form_exact_workspace_and_host_buffers():
    """A caller workspace of exactly lr_workspace_size bytes suffices for the
    log form; the host-buffer entry point takes it too."""
    n = (1 << 25) + 1
    succ = gen.random_list(n, 74)
    want = oracle.rank(succ)
    ws_bytes = lr.workspace_size(n, max_lists=1)
    ws = torch.empty(ws_bytes, dtype=torch.uint8, device="cuda")
    d = torch.from_numpy(succ.view(np.int32)).cuda()
    out = torch.empty(n, dtype=torch.int32, device="cuda")
    lr.rank_ex(d, out=out, max_lists=1, workspace=ws)
    np.testing.assert_array_equal(out.cpu().numpy(), want)
    small = torch.empty(ws_bytes // 2, dtype=torch.uint8, device="cuda")
    with pytest.raises(lr.LRError):
        lr.rank_ex(d, out=out, max_lists=1, workspace=small)
    host = np.empty(n, dtype=np.int32)
    lr.rank_host(succ, out=host, max_lists=1)
    np.testing.assert_array_equal(host, want)
