"""Batches of lists in separate device buffers (lr_rank_batch_ptrs, GPU).

k instances, each in its own succ / weight / rank tensors, are ranked as one
forest in one launch sequence through device pointer tables (Section 1.1's
set of lists).  Every instance must come out exactly as the oracle ranks it
alone: empty, single-element and sub-warp instances, instances that share a
warp, instances that are forests (the heads then come from the predecessor
bitmap instead of per-instance sums), both rank widths, every weight type,
with and without a list bound, and batches below the base-case size.  Bad
inputs are reported, not trusted.
"""
import ctypes

import numpy as np
import pytest

import gen
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2606_09318_gb300 as lr  # noqa: E402

SIZES = [0, 1, 2, 5, 37, 127, 128, 129, 1000, 5000, 70000]


def dev(a):
    a = np.ascontiguousarray(a)
    if a.dtype == np.uint32:
        a = a.view(np.int32)
    return torch.from_numpy(a).cuda()


def _instances(seed, sizes, forest_at=()):
    out = []
    for j, m in enumerate(sizes):
        if m == 0:
            out.append(np.zeros(0, np.uint32))
        elif j in forest_at and m > 8:
            out.append(gen.forest(m, seed + j, n_long=1, long_len=m // 4, mean_short=4)[0].astype(np.uint32))
        else:
            out.append(gen.random_list(m, seed + j).astype(np.uint32))
    return out


def _weights(kind, sizes, seed):
    if kind is None:
        return None
    f = gen.weights_i32 if kind == "i32" else gen.weights_i64
    return [f(m, seed + j) if m else np.zeros(0, np.int32 if kind == "i32" else np.int64)
            for j, m in enumerate(sizes)]


def _lists(s):
    return int((s == np.arange(len(s))).sum())


@pytest.mark.parametrize("wt,rdt", [(None, np.int32), (None, np.int64), ("i32", np.int64), ("i64", np.int64),
                                    ("i32", np.int32)])
@pytest.mark.parametrize("forest", [False, True])
def test_ptrs_equal_oracle(wt, rdt, forest):
    rng = np.random.default_rng(5)
    sizes = SIZES + [int(x) for x in rng.integers(1, 3000, size=40)]
    succ = _instances(800, sizes, forest_at=(9, 20) if forest else ())
    w = _weights(wt, sizes, 900)
    tdt = torch.int32 if rdt == np.int32 else torch.int64
    lists = sum(_lists(s) for s in succ)
    for ml in (0, lists):
        outs = lr.rank_batch_ptrs([dev(s) for s in succ], None if w is None else [dev(x) for x in w],
                                  rank_dtype=tdt, max_lists=ml)
        for j, (s, o) in enumerate(zip(succ, outs)):
            want = oracle.rank(s, None if w is None else w[j], rdt)
            np.testing.assert_array_equal(o.cpu().numpy(), want, err_msg="instance %d" % j)


def test_ptrs_below_base_case_size():
    # a batch smaller than the single-CTA base case still chases level 0
    sizes = [0, 3, 17, 64, 200, 1]
    succ = _instances(810, sizes)
    outs = lr.rank_batch_ptrs([dev(s) for s in succ])
    for s, o in zip(succ, outs):
        np.testing.assert_array_equal(o.cpu().numpy(), oracle.rank(s))


def test_ptrs_equal_contiguous_batch():
    # the batched benchmark's size mix, scaled down: the pointer form and the
    # contiguous form give the same ranks, and both satisfy the recurrence
    k = 512
    lens = gen.batch_lengths(k, 47, 4.0, 17.0)
    succ = _instances(820, [int(m) for m in lens])
    w = [gen.weights_i64(int(m), 830 + j) for j, m in enumerate(lens)]
    outs = lr.rank_batch_ptrs([dev(s) for s in succ], [dev(x) for x in w], max_lists=k)
    offsets = np.zeros(k + 1, dtype=np.int64)
    np.cumsum(lens, out=offsets[1:])
    cat = lr.rank_batch(dev(offsets), dev(np.concatenate(succ)), dev(np.concatenate(w)), max_lists=k)
    np.testing.assert_array_equal(torch.cat(outs).cpu().numpy(), cat.cpu().numpy())
    for j in range(0, k, 61):                                   # a sample against the oracle
        np.testing.assert_array_equal(outs[j].cpu().numpy(), oracle.rank(succ[j], w[j], np.int64))


def test_ptrs_errors():
    sizes = [3000, 4000, 2500]
    succ = _instances(840, sizes)
    # a successor outside its instance
    bad = [s.copy() for s in succ]
    bad[1][17] = sizes[1] + 3
    with pytest.raises(lr.LRError) as e:
        lr.rank_batch_ptrs([dev(s) for s in bad])
    assert e.value.name == "LR_ERR_OUT_OF_RANGE"
    # two predecessors, with validation
    two = [s.copy() for s in succ]
    tgt = int(two[2][0])
    i = next(i for i in range(sizes[2]) if two[2][i] != tgt and two[2][i] != i)
    two[2][i] = tgt
    assert oracle.rank_status(two[2], None, np.int32)[0] != oracle.OK
    with pytest.raises(lr.LRError) as e:
        lr.rank_batch_ptrs([dev(s) for s in two], validate=True)
    assert e.value.name == "LR_ERR_NOT_A_LIST"
    # a decreasing offset table is refused before any kernel reads through it
    lib = lr.load()
    bufs = [torch.zeros(8000, dtype=torch.int32, device="cuda") for _ in range(3)]
    outs = [torch.zeros(8000, dtype=torch.int32, device="cuda") for _ in range(3)]
    sp = torch.tensor([b.data_ptr() for b in bufs], dtype=torch.int64, device="cuda")
    rp = torch.tensor([o.data_ptr() for o in outs], dtype=torch.int64, device="cuda")
    o = lr._opts(0, 1, sync=True)
    for table in ([0, 5000, 3000, 8000], [5, 3000, 6000, 8000]):
        off = torch.tensor(table, dtype=torch.int64, device="cuda")
        code = lib.lr_rank_batch_ptrs(ctypes.c_void_p(off.data_ptr()), ctypes.c_void_p(sp.data_ptr()), None,
                                      ctypes.c_void_p(rp.data_ptr()), 3, ctypes.byref(o),
                                      ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
        assert lr.STATUS[code] == "LR_ERR_INVALID_ARGUMENT"
    assert int(torch.count_nonzero(torch.stack(outs))) == 0        # nothing was written
    # the stream still works
    outs = lr.rank_batch_ptrs([dev(s) for s in succ])
    for s, o2 in zip(succ, outs):
        np.testing.assert_array_equal(o2.cpu().numpy(), oracle.rank(s))
