"""The autotuner on the GPU (lr_autotune).

Whatever the autotuner picks, ranks stay exact: it checks its winner
against the defaults itself, and here every later call that picks the
tuned entry up from the table is compared with the oracle.
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

F0 = {4, 8, 16, 32, 64, 128, 2, 5, 6, 10, 12, 21, 24, 42, 48, 85, 96, 192}


def dev(a):
    a = np.ascontiguousarray(a)
    if a.dtype == np.uint32:
        a = a.view(np.int32)
    return torch.from_numpy(a).cuda()


@pytest.fixture(autouse=True)
def clean_table():
    lr.autotune_clear()
    yield
    lr.autotune_clear()


def test_synthetic_single_list():
    n = (1 << 20) + 17
    t = lr.autotune(n)
    assert t.f0_inv in F0 and t.f_inv in (4, 8, 16) and t.cutoff in (4096, 8192, 12288)
    assert t.chase_block in (128, 256, 512)
    ent = lr.autotune_entries()
    assert len(ent) == 1 and ent[0]["log2n"] == 20 and ent[0]["weighted"] == 0 and ent[0]["batch"] == 0
    assert ent[0]["ms"] > 0
    # later calls of this shape take the entry from the table and stay exact
    succ = gen.random_list(n, 400)
    np.testing.assert_array_equal(lr.rank(dev(succ)).cpu().numpy(), oracle.rank(succ))
    succ2 = gen.locality_list((1 << 20) + 3, 401)
    np.testing.assert_array_equal(lr.rank(dev(succ2), max_lists=1).cpu().numpy(), oracle.rank(succ2))


def test_callers_data_forest_and_weighted():
    succ, nl = gen.forest(1 << 19, 402, n_long=2, long_len=1 << 14, mean_short=16)
    w = gen.weights_i32(1 << 19, 403)
    lr.autotune(succ=dev(succ), weight=dev(w))          # counted lists, the caller's weights
    ent = lr.autotune_entries()
    assert len(ent) == 1 and ent[0]["weighted"] == 1
    got = lr.rank(dev(succ), dev(w)).cpu().numpy()
    np.testing.assert_array_equal(got, oracle.rank(succ, w, np.int64))


def test_batch_synthetic_then_real():
    lr.autotune(1 << 20, k=64, wtype="int64")
    ent = lr.autotune_entries()
    assert len(ent) == 1 and ent[0]["batch"] == 1 and ent[0]["weighted"] == 1
    offsets, succ, w = gen.batch_instances(64, 404, lo_exp=4.0, hi_exp=16.0)
    n = int(offsets[-1])
    got = lr.rank_batch(dev(offsets), dev(succ), dev(w), max_lists=64).cpu().numpy()
    np.testing.assert_array_equal(got, oracle.rank_batch(offsets, succ, w, np.int64))
    # workspace sized with the table in place, then a graph-free bound call
    ws = torch.empty(lr.workspace_size(n, 64, weighted=True, max_lists=64), dtype=torch.uint8, device="cuda")
    out = torch.empty(n, dtype=torch.int64, device="cuda")
    lr.rank_batch(dev(offsets), dev(succ), dev(w), out=out, max_lists=64, n_total=n, workspace=ws)
    np.testing.assert_array_equal(out.cpu().numpy(), oracle.rank_batch(offsets, succ, w, np.int64))


def test_small_and_invalid():
    t = lr.autotune(20000, wtype="int32")
    assert t.f0_inv in F0
    succ = gen.random_list(20000, 405)
    w = gen.weights_i32(20000, 406)
    np.testing.assert_array_equal(lr.rank(dev(succ), dev(w)).cpu().numpy(), oracle.rank(succ, w, np.int64))
    with pytest.raises(lr.LRError):
        lr.autotune(0)
    bad = gen.random_list(5000, 407).copy()
    bad[3] = 5000
    with pytest.raises(lr.LRError):
        lr.autotune(succ=dev(bad))
