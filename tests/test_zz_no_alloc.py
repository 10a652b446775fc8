"""lr_rank_noalloc: ranking inside the library's fixed scratch array.

For callers that cannot allocate device memory when they need a ranking: a
process whose allocator already holds all free device memory, a loop that
must not risk an allocation's implicit synchronisation, a plug-in whose host
forbids allocations after start-up.  The entry point is called through the
C ABI and its output is compared with the CPU oracle, element by element (an
integer result, so bit for bit), on several calls in a row that share the
scratch: large then small, so that stale contents of a bigger call are
present.  This file is collected last on purpose.
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

LR_OK, LR_ERR_INVALID_ARGUMENT, LR_ERR_CAPACITY = 0, 1, 9


def _entry():
    lib = lr.load()
    f = lib.lr_rank_noalloc
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p]
    return f


def _call(f, s, out, stream):
    return f(ctypes.c_void_p(s.data_ptr()), s.numel(), ctypes.c_void_p(out.data_ptr()),
             ctypes.c_void_p(stream.cuda_stream))


def test_noalloc_matches_oracle_on_calls_in_a_row():
    f = _entry()
    stream = torch.cuda.current_stream()
    cases = [gen.random_list((1 << 22) - 5, 71),          # the largest size it takes
             gen.locality_list(3_000_001, 72),
             gen.random_list(777, 73),                     # small, after large ones
             gen.random_list((1 << 20) + 3, 74)]
    for succ in cases:
        s = torch.from_numpy(succ.view(np.int32)).cuda()
        out = torch.full((s.numel(),), -7, dtype=torch.int32, device="cuda")
        code = _call(f, s, out, stream)
        assert code == LR_OK, lr.status_string(code)
        np.testing.assert_array_equal(out.cpu().numpy(), oracle.rank(succ))


def test_noalloc_allocates_no_device_memory():
    f = _entry()
    succ = gen.random_list((1 << 21) + 11, 75)
    s = torch.from_numpy(succ.view(np.int32)).cuda()
    out = torch.zeros(s.numel(), dtype=torch.int32, device="cuda")
    assert _call(f, s, out, torch.cuda.current_stream()) == LR_OK      # set-up done
    fresh = torch.cuda.Stream()
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    out.fill_(-1)
    torch.cuda.synchronize()
    assert _call(f, s, out, fresh) == LR_OK                           # a stream it never saw
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    np.testing.assert_array_equal(out.cpu().numpy(), oracle.rank(succ))


def test_noalloc_capacity_leaves_rank_untouched():
    f = _entry()
    n = 1 << 22
    succ, nlists = gen.forest(n, 76, n_long=0, long_len=1, mean_short=2)   # ~2^21 lists
    assert nlists > n // 3
    s = torch.from_numpy(succ.view(np.int32)).cuda()
    out = torch.full((n,), -7, dtype=torch.int32, device="cuda")
    assert _call(f, s, out, torch.cuda.current_stream()) == LR_ERR_CAPACITY
    torch.cuda.synchronize()
    assert bool((out == -7).all())
    # the scratch is usable again right after
    small = gen.random_list(5000, 77)
    t = torch.from_numpy(small.view(np.int32)).cuda()
    o2 = torch.empty(5000, dtype=torch.int32, device="cuda")
    assert _call(f, t, o2, torch.cuda.current_stream()) == LR_OK
    np.testing.assert_array_equal(o2.cpu().numpy(), oracle.rank(small))


def test_noalloc_limits():
    f = _entry()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    big = (1 << 22) + 1
    assert f(ctypes.c_void_p(1), big, ctypes.c_void_p(1), stream) == LR_ERR_INVALID_ARGUMENT
    assert f(None, 0, None, stream) == LR_OK                               # empty input
    assert f(None, 10, None, stream) == LR_ERR_INVALID_ARGUMENT            # NULL pointers
