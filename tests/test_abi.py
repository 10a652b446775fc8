"""The C-ABI library builds, loads and exports every function include/lr.h
declares; host-only entry points work without a GPU (no compute calls here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "lr.h")


@pytest.fixture(scope="module")
def lib():
    from paper_2606_09318_gb300 import build
    build.build()
    import paper_2606_09318_gb300 as lr
    return lr.load()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"\b(lr_[a-z0-9_]+)\s*\(", text)
    return sorted(set(names))


def test_header_declares_entry_points():
    names = declared_functions()
    for must in ("lr_rank", "lr_rank_batch", "lr_rank_ex", "lr_rank_batch_ex", "lr_workspace_size",
                 "lr_get_device_status", "lr_status_string", "lr_server_create", "lr_server_submit",
                 "lr_server_wait", "lr_server_destroy", "lr_rank_host"):
        assert must in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_host_only_calls(lib):
    import paper_2606_09318_gb300 as lr
    assert lr.status_string(0) == "LR_OK"
    assert lr.status_string(3) == "LR_ERR_CYCLE"
    assert "sm_103a" in lr.version()
    # workspace grows with n and with weights; the list bound shrinks it
    a = lr.workspace_size(1 << 20)
    b = lr.workspace_size(1 << 24)
    c = lr.workspace_size(1 << 24, weighted=True)
    d = lr.workspace_size(1 << 24, max_lists=1)
    assert 0 < a < b < c and d < b
    # level 0 dominates: the log (about 4.3 B), its partition buffer (8 B) and
    # the bitmap for an unweighted list; 16-byte records when weighted
    assert (1 << 24) * 8 < d < (1 << 24) * 24
    assert (1 << 24) * 16 < c
    assert lr.workspace_size(0) == 0


def test_library_has_no_oracle_dependency():
    """The product path never imports, links or calls the oracle."""
    src_dir = os.path.join(ROOT, "paper_2606_09318_gb300")
    for dirpath, _, files in os.walk(src_dir):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                text = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in text and "from oracle" not in text, f
                assert "lr_oracle" not in text and "lro_" not in text, f
