"""The debug build (GPU): every kernel path on small inputs with the index
checks of -DLR_DEBUG compiled in, in a process of its own that loads
liblr_debug.so (see _debug_cases.py).  No check may fail and every result
must equal the oracle's."""
import os
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_debug_build_cases():
    sys.path.insert(0, ROOT)
    from paper_2606_09318_gb300 import build
    build.build(debug=True)
    env = dict(os.environ, LR_DEBUG_LIB="1")
    env.pop("LR_TUNING", None)
    r = subprocess.run([sys.executable, os.path.join(ROOT, "tests", "_debug_cases.py")], env=env,
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-3000:]
    assert "all ok" in r.stdout
