"""lr_probe_memory (measurement only): the random-access and streaming rates
the chase is held to.  Rates must be positive and ordered as the memory
system orders them (a footprint inside L2 serves random gathers faster than
one far larger than L2); bad buffers are argument errors."""
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2606_09318_gb300 as lr  # noqa: E402


def test_probe_rates_and_footprint():
    small = torch.empty((32 << 20) + 256, dtype=torch.uint8, device="cuda")
    r = lr.probe_memory(small)
    assert r["footprint_bytes"] == (32 << 20)
    for k in ("copy_gbs", "gather_gsteps", "gather_xchg_gsteps", "indep_gather_gsteps", "region_gather_gsteps"):
        assert r[k] > 0, k
    del small
    big = torch.empty((1 << 30) + 256, dtype=torch.uint8, device="cuda")
    b = lr.probe_memory(big)
    assert b["footprint_bytes"] == (1 << 30)
    # 32 MiB sits in L2; 1 GiB does not: random gathers are served faster there
    assert r["indep_gather_gsteps"] > b["indep_gather_gsteps"]
    assert r["gather_gsteps"] > b["gather_gsteps"]


def test_probe_argument_errors():
    tiny = torch.empty(1 << 20, dtype=torch.uint8, device="cuda")
    with pytest.raises(lr.LRError) as e:
        lr.probe_memory(tiny)                       # below 16 MiB
    assert e.value.name == "LR_ERR_INVALID_ARGUMENT"
    buf = torch.empty((32 << 20) + 512, dtype=torch.uint8, device="cuda")
    with pytest.raises(lr.LRError):
        lr.probe_memory(buf[1:])                    # not 256-byte aligned
