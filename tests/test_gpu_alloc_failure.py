"""Allocation failure, injected on the host (GPU).

The library allocates only its workspace (one grow-only arena per stream).
With LR_INJECT_ALLOC_FAIL=1 every request for it fails as an exhausted
cudaMalloc would, without touching the device: the call reports
LR_ERR_OUT_OF_MEMORY, writes nothing, and the same stream ranks normally
once the injection is lifted.  Nothing runs out of device memory for real.
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


@pytest.mark.parametrize("kind", ["single", "weighted", "batch"])
def test_injected_allocation_failure(monkeypatch, kind):
    n = (1 << 18) + 7
    succ = gen.random_list(n, 4800)
    w = gen.weights_i32(n, 4801) if kind == "weighted" else None
    s = torch.cuda.Stream()
    d_succ = dev(succ)
    d_w = None if w is None else dev(w)
    if kind == "batch":
        offsets = np.array([0, 1000, 1000, n], dtype=np.int64)
        parts = [gen.random_list(1000, 4802), gen.random_list(n - 1000, 4803)]
        succ = np.concatenate(parts).astype(np.uint32)
        d_succ = dev(succ)
        want = oracle.rank_batch(offsets, succ, None, np.int32)
        call = lambda out: lr.rank_batch(dev(offsets), d_succ, out=out, rank_dtype=torch.int32, stream=s)
    else:
        want = oracle.rank(succ, w, np.int32 if w is None else np.int64)
        call = lambda out: lr.rank_ex(d_succ, d_w, out=out, stream=s)
    out = torch.full((n,), -7, dtype=torch.int32 if w is None else torch.int64, device="cuda")
    monkeypatch.setenv("LR_INJECT_ALLOC_FAIL", "1")
    with pytest.raises(lr.LRError) as e:
        with torch.cuda.stream(s):
            call(out)
    assert e.value.name == "LR_ERR_OUT_OF_MEMORY"
    s.synchronize()
    assert bool((out == -7).all())                # nothing was written
    monkeypatch.delenv("LR_INJECT_ALLOC_FAIL")
    with torch.cuda.stream(s):
        call(out)
    s.synchronize()
    np.testing.assert_array_equal(out.cpu().numpy(), want)
