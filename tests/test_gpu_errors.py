"""Invalid inputs on the GPU: every case is bounded by construction (range
errors become terminals, chases stop at rulers, terminals or an element seen
before, the base case runs a fixed number of rounds), so nothing here can hang
or fault; each checks the reported status and that the next call still works."""
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
    return torch.from_numpy(np.ascontiguousarray(a).view(np.int32)).cuda()


def status_of(succ, **kw):
    try:
        lr.rank(dev(succ), **kw)
        return "LR_OK"
    except lr.LRError as e:
        return e.name


def _head_tail(succ):
    n = succ.shape[0]
    hp = np.zeros(n, dtype=bool)
    hp[succ[succ != np.arange(n)]] = True
    return int(np.flatnonzero(~hp)[0]), int(np.flatnonzero(succ == np.arange(n))[0])


@pytest.mark.parametrize("n", [1000, (1 << 20) + 1])
def test_out_of_range(n):
    succ = gen.random_list(n, 1).copy()
    succ[n // 2] = n + 3
    assert oracle.rank_status(succ)[0] == oracle.OUT_OF_RANGE
    assert status_of(succ) == "LR_ERR_OUT_OF_RANGE"
    succ[n // 2] = 0xFFFFFFFF
    assert status_of(succ) == "LR_ERR_OUT_OF_RANGE"


@pytest.mark.parametrize("n", [1000, (1 << 20) + 1, 1 << 22])
def test_closed_cycle(n):
    succ = gen.random_list(n, 2).copy()
    h, t = _head_tail(succ)
    succ[t] = h
    assert oracle.rank_status(succ)[0] == oracle.CYCLE
    assert status_of(succ) == "LR_ERR_CYCLE"
    assert status_of(succ, validate=True) == "LR_ERR_CYCLE"


@pytest.mark.parametrize("n", [5000, (1 << 20) + 1])
def test_headless_cycle_beside_a_list(n):
    a = gen.random_list(n, 3)
    cyc = np.roll(np.arange(n, 2 * n, dtype=np.uint32), -1)        # n..2n-1 in a ring
    succ = np.concatenate([a, cyc]).astype(np.uint32)
    assert oracle.rank_status(succ)[0] == oracle.CYCLE
    assert status_of(succ) == "LR_ERR_CYCLE"


@pytest.mark.parametrize("n", [1000, (1 << 20) + 1])
def test_two_predecessors(n):
    succ = gen.random_list(n, 4).copy()
    h, t = _head_tail(succ)
    succ[t] = succ[succ[h]]            # rho: the tail joins the list again
    assert oracle.rank_status(succ)[0] == oracle.NOT_A_LIST
    assert status_of(succ, validate=True) == "LR_ERR_NOT_A_LIST"
    assert status_of(succ) != "LR_OK"  # without validation it is still caught
    succ2 = gen.random_list(n, 5).copy()
    h2, t2 = _head_tail(succ2)
    succ2[h2] = t2                      # the head jumps to the tail: tail has 2 preds
    assert status_of(succ2, validate=True) == "LR_ERR_NOT_A_LIST"


def test_async_status_and_recovery():
    n = 1 << 20
    good = gen.random_list(n, 6)
    bad = good.copy()
    bad[7] = n
    lr.rank(dev(bad), sync=False)
    assert lr.status_string(lr.device_status()) == "LR_ERR_OUT_OF_RANGE"
    assert lr.device_status() == 0        # status is cleared once read
    out = lr.rank(dev(good))
    np.testing.assert_array_equal(out.cpu().numpy(), oracle.rank(good))


def test_argument_errors():
    s = torch.zeros(10, dtype=torch.int32, device="cuda")
    with pytest.raises(TypeError):
        lr.rank(s.to(torch.float32))
    lib = lr.load()
    assert lib.lr_rank(None, None, 10, None, None) == 1     # NULL pointers with n > 0
    assert lib.lr_rank(None, None, -1, None, None) == 1     # negative size
    assert lib.lr_rank(None, None, 0, None, None) == 0      # n = 0 is a no-op
