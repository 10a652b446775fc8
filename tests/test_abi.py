"""The C-ABI library builds, loads and exports every function include/lr.h
declares; host-only entry points work without a GPU (no compute calls here)."""
import ctypes
import os
import re
import subprocess
import sys

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


def test_batch_ptrs_argument_errors_on_host(lib):
    # lr_rank_batch_ptrs refuses bad arguments before it touches the device
    import paper_2606_09318_gb300 as lr
    o = lr._opts(0, 1)
    fake = ctypes.c_void_p(256)
    assert lib.lr_rank_batch_ptrs(fake, fake, None, fake, 0, ctypes.byref(o), None) == 0   # no instances
    assert lib.lr_rank_batch_ptrs(fake, fake, None, fake, -1, ctypes.byref(o), None) == 1
    assert lib.lr_rank_batch_ptrs(None, fake, None, fake, 2, ctypes.byref(o), None) == 1   # no offsets
    assert lib.lr_rank_batch_ptrs(fake, None, None, fake, 2, ctypes.byref(o), None) == 1   # no succ table
    assert lib.lr_rank_batch_ptrs(fake, fake, None, None, 2, ctypes.byref(o), None) == 1   # no rank table
    o.workspace = fake                                       # a caller workspace is not supported
    o.ws_bytes = 1 << 20
    assert lib.lr_rank_batch_ptrs(fake, fake, None, fake, 2, ctypes.byref(o), None) == 1


def test_workspace_counts_element_order_arrays(lib, monkeypatch):
    """A batch chases its levels in element order: its workspace holds the
    positions of the largest level's sampled rulers (4 B each) and the count
    before every 256 positions (4 B each), each region 256-byte aligned; a
    single list, and a batch with LR_TUNING=ord=0, hold neither.  Needs no
    GPU."""
    import paper_2606_09318_gb300 as lr
    n, k = 10_000_000, 100
    align = lambda x: (x + 255) // 256 * 256
    monkeypatch.delenv("LR_TUNING", raising=False)
    on = lr.workspace_size(n, k, weighted=True, max_lists=k)
    single = lr.workspace_size(n, 0, weighted=True, max_lists=k)
    monkeypatch.setenv("LR_TUNING", "ord=0")
    off = lr.workspace_size(n, k, weighted=True, max_lists=k)
    assert lr.workspace_size(n, 0, weighted=True, max_lists=k) == single
    # a batch of 10^7 elements keeps ruler spacing 16 at level 0, the largest level
    assert on - off == align(4 * -(-n // 16)) + align(4 * -(-n // 256))
    # with extra outputs a batch keeps the slice order (the outputs need the bitmap)
    monkeypatch.delenv("LR_TUNING", raising=False)
    a = lr.workspace_size(n, k, weighted=True, max_lists=k, term=True)
    monkeypatch.setenv("LR_TUNING", "ord=0")
    assert lr.workspace_size(n, k, weighted=True, max_lists=k, term=True) == a


def test_library_has_no_oracle_dependency():
    """The product path never imports, links or calls the oracle."""
    src_dir = os.path.join(ROOT, "paper_2606_09318_gb300")
    for dirpath, _, files in os.walk(src_dir):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                text = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in text and "from oracle" not in text, f
                assert "lr_oracle" not in text and "lro_" not in text, f


def test_autotune_table_roundtrip(tmp_path, lib):
    """The autotuned table: load, read back, save, reload; needs no GPU."""
    import json as _json
    import paper_2606_09318_gb300 as lr
    lr.autotune_clear()
    src = tmp_path / "tune.json"
    entries = [{"log2n": 20, "weighted": 0, "batch": 0, "f0_inv": 4, "f_inv": 16, "cutoff": 4096,
                "chase_block": 128, "chase_ctas": 0, "algorithm": 0, "ms": 0.25},
               {"log2n": 24, "weighted": 1, "batch": 1, "f0_inv": 16, "f_inv": 8, "cutoff": 12288,
                "chase_block": 256, "chase_ctas": 0, "algorithm": 0, "ms": 1.5}]
    src.write_text(_json.dumps({"format": "lr_autotune 1", "entries": entries}))
    base = lr.workspace_size(1 << 20, max_lists=1)
    lr.autotune_load(str(src))
    got = lr.autotune_entries()
    assert len(got) == 2
    for want, have in zip(entries, got):
        for key in want:
            assert abs(have[key] - want[key]) < 1e-6, key
    # the entry for (2^20, unweighted, single) now drives the plan: 1/f0 = 1/4
    assert lr.workspace_size(1 << 20, max_lists=1) > base           # more rulers per level
    assert lr.workspace_size((1 << 20) + 5, max_lists=1) == lr.workspace_size((1 << 20) + 5, max_lists=1)
    out = tmp_path / "saved.json"
    lr.autotune_save(str(out))
    lr.autotune_clear()
    assert lr.autotune_entries() == [] and lr.workspace_size(1 << 20, max_lists=1) == base
    lr.autotune_load(str(out))
    assert lr.autotune_entries() == got
    bad = tmp_path / "bad.json"
    bad.write_text('{"entries": [{"log2n": 20}]}')
    with pytest.raises(lr.LRError):
        lr.autotune_load(str(bad))
    with pytest.raises(lr.LRError):
        lr.autotune_load(str(tmp_path / "missing.json"))
    lr.autotune_clear()


def test_autotune_file_from_environment(tmp_path, lib):
    src = tmp_path / "env.json"
    src.write_text('{"entries": [{"log2n": 22, "weighted": 0, "batch": 0, "f0_inv": 8, "f_inv": 8, '
                   '"cutoff": 8192, "chase_block": 256, "chase_ctas": 0, "algorithm": 0, "ms": 1}]}')
    code = ("import paper_2606_09318_gb300 as lr; e = lr.autotune_entries(); "
            "assert len(e) == 1 and e[0]['log2n'] == 22 and e[0]['f0_inv'] == 8, e")
    env = dict(os.environ, LR_TUNING_FILE=str(src))
    subprocess.check_call([sys.executable, "-c", code], env=env, cwd=ROOT)


def test_debug_build_exports_the_same_symbols():
    """build(debug=True) cross-compiles here (no GPU needed) into a library
    of its own that exports exactly the release library's entry points."""
    import shutil
    import subprocess as sp
    if shutil.which("nm") is None:
        pytest.skip("nm not available")
    from paper_2606_09318_gb300 import build
    rel = build.build()
    dbg = build.build(debug=True)
    assert dbg != rel and dbg.endswith("liblr_debug.so")

    def exports(path):
        out = sp.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True, check=True).stdout
        return {ln.split()[-1] for ln in out.splitlines() if ln.split() and ln.split()[-1].startswith("lr_")}
    assert exports(dbg) == exports(rel) and "lr_rank" in exports(rel)
