"""lr_rank_noalloc: ranking inside the library's fixed scratch array.

For callers that cannot allocate device memory when they need a ranking.
The entry point is called through the C ABI and its output is compared with
lr_rank's (which uses allocated workspace) on two calls in a row, bit for bit
as every other integer result here.  This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

import gen

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2606_09318_gb300 as lr  # noqa: E402


def _entry():
    lib = lr.load()
    f = lib.lr_rank_noalloc
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p]
    return f


def test_noalloc_matches_lr_rank_on_two_calls():
    f = _entry()
    stream = torch.cuda.current_stream()
    cases = [gen.random_list((1 << 22) - 5, 71), gen.locality_list(3_000_001, 72)]
    for succ in cases:                      # two calls in a row on the shared scratch
        s = torch.from_numpy(succ.view(np.int32)).cuda()
        out = torch.full((s.numel(),), -7, dtype=torch.int32, device="cuda")
        code = f(ctypes.c_void_p(s.data_ptr()), s.numel(), ctypes.c_void_p(out.data_ptr()),
                 ctypes.c_void_p(stream.cuda_stream))
        assert code == 0, lr.status_string(code)
        want = lr.rank(s)                   # the allocating entry point
        assert torch.equal(out, want)


def test_noalloc_limits():
    f = _entry()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    big = (1 << 22) + 1
    assert f(ctypes.c_void_p(1), big, ctypes.c_void_p(1), stream) == 1      # beyond the maximum
    assert f(None, 0, None, stream) == 0                                   # empty input
    assert f(None, 10, None, stream) == 1                                  # NULL pointers
