"""The Python binding's ctypes structures against the C header's layout.

Each public struct of include/lr.h is compiled with the host C compiler,
which prints its size and every member's offset; the ctypes mirror in the
binding must agree field by field, so that a member added on one side only
cannot shift the others unnoticed.  Host only: no GPU, no library load.
"""
import ctypes
import os
import shutil
import subprocess

import pytest

import paper_2606_09318_gb300 as lr

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# C struct name -> ctypes mirror
MIRRORS = {
    "lr_tuning": lr.Tuning,
    "lr_opts": lr._Opts,
    "lr_outputs": lr._Outputs,
    "lr_tune_entry": lr._TuneEntry,
    "lr_profile": lr._Profile,
    "lr_server_config": lr._ServerConfig,
    "lr_request": lr._Request,
    "lr_result": lr._Result,
    "lr_server_stats": lr._ServerStats,
    "lr_probe_result": lr._ProbeResult,
}


def _c_layout(tmp_path):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no host C compiler")
    lines = ['#include "lr.h"', "#include <stddef.h>", "#include <stdio.h>", "int main(void) {"]
    for cname, mirror in MIRRORS.items():
        lines.append('  printf("%s size %%zu\\n", sizeof(%s));' % (cname, cname))
        for field, _ in mirror._fields_:
            lines.append('  printf("%s %s %%zu\\n", offsetof(%s, %s));' % (cname, field, cname, field))
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                   check=True, capture_output=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    got = {}
    for line in out.splitlines():
        cname, key, val = line.split()
        got[(cname, key)] = int(val)
    return got


def test_ctypes_mirrors_match_the_header(tmp_path):
    c = _c_layout(tmp_path)
    for cname, mirror in MIRRORS.items():
        assert c[(cname, "size")] == ctypes.sizeof(mirror), cname
        for field, _ in mirror._fields_:
            assert c[(cname, field)] == getattr(mirror, field).offset, (cname, field)
