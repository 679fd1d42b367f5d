"""The C-ABI library builds, loads and exports every entry point declared in
include/shaken.h, with struct layouts that match the Python binding.  CPU only:
no compute call is made (there is no GPU here)."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "shaken.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(shaken_[a-z_]+)\s*\(", text)))


def test_library_exports_every_declared_symbol():
    from paper_1904_06257_gb300 import build
    path = build.build()
    lib = ctypes.CDLL(path)
    names = declared_functions()
    assert len(names) >= 30
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_struct_layout_matches_header(tmp_path):
    from paper_1904_06257_gb300 import shaken as S
    src = tmp_path / "layout.c"
    src.write_text(
        '#include <stdio.h>\n#include <stddef.h>\n#include "shaken.h"\n'
        'int main(void){printf("%zu %zu %zu %zu %zu\\n", sizeof(shaken_problem),'
        ' offsetof(shaken_problem, beta), offsetof(shaken_problem, init_spins),'
        ' sizeof(shaken_obs), offsetof(shaken_obs, cut_weight)); return 0;}\n')
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.dirname(HEADER), str(src), "-o", str(exe)], check=True)
    got = [int(x) for x in subprocess.run([str(exe)], capture_output=True, text=True,
                                          check=True).stdout.split()]
    want = [ctypes.sizeof(S.shaken_problem), S.shaken_problem.beta.offset,
            S.shaken_problem.init_spins.offset, ctypes.sizeof(S.shaken_obs),
            S.shaken_obs.cut_weight.offset]
    assert got == want


def test_version_and_strerror():
    from paper_1904_06257_gb300 import shaken as S
    assert "sm_103a" in S.shaken_version()
    assert S._lib.shaken_strerror(-1) == b"invalid argument"


def test_invalid_problems_rejected_without_gpu():
    """Validation happens on the host before any CUDA call."""
    import numpy as np
    from paper_1904_06257_gb300 import shaken as S
    bad = [
        dict(kind=S.LATTICE, encoding=S.INT8, replicas=1, beta=0.4, q=0.0, L=64),     # q <= 0
        dict(kind=S.LATTICE, encoding=S.INT8, replicas=1, beta=0.4, q=1.0, L=48),     # L % 32
        dict(kind=S.LATTICE, encoding=S.MULTISPIN, replicas=40, beta=0.4, q=1.0, L=64),
        dict(kind=S.LATTICE, encoding=S.INT8, replicas=1, beta=float("nan"), q=1.0, L=64),
        dict(kind=S.GRAPH, encoding=S.MULTISPIN, replicas=32, beta=0.4, q=1.0, n=4,
             u=[0, 1], v=[1, 1], J_edge=[1, 1]),                                       # self-loop
        dict(kind=S.GRAPH, encoding=S.MULTISPIN, replicas=32, beta=0.4, q=1.0, n=4,
             u=[0, 1], v=[1, 7], J_edge=[1, 1]),                                       # out of range
        dict(kind=S.GRAPH, encoding=S.MULTISPIN, replicas=32, beta=0.4, q=1.0, n=4,
             u=[0, 1], v=[1, 2], J_edge=[1, 0.5], J_is_integer=True),                  # not +-1
    ]
    for kw in bad:
        kw = dict(kw)
        p = S.Problem(kw.pop("kind"), kw.pop("encoding"), kw.pop("replicas"), kw.pop("beta"),
                      kw.pop("q"), **kw)
        with pytest.raises(S.ShakenError) as ei:
            S.shaken_init(p, 1)
        assert ei.value.status == -1
