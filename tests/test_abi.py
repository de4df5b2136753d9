"""The C-ABI library builds, loads and exports every entry point include/pamd.h
declares (no compute calls: these run without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared(header):
    text = open(os.path.join(ROOT, "include", header)).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(pamd_[a-z_0-9]+)\s*\(", text)))


def test_library_builds_and_exports_every_declared_symbol():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1907_09529_gb300 import _lib
    lib = _lib.load()
    declared = _declared("pamd.h")
    assert declared, "no declarations found"
    missing = [name for name in declared if not hasattr(lib, name)]
    assert not missing, missing
    assert set(declared) == set(_lib.EXPORTS)
    assert lib.pamd_version() == 1
    assert lib.pamd_status_string(-4) == b"device wait timed out"


def test_struct_layout_matches_header():
    """ctypes mirrors of the ABI structs have the sizes a C compiler gives them."""
    from paper_1907_09529_gb300 import _lib
    import subprocess, tempfile
    src = r'''
#include <stdio.h>
#include <stddef.h>
#include "pamd.h"
int main(void){printf("%zu %zu %zu %zu %zu\n", sizeof(pamd_potential), sizeof(pamd_system),
 sizeof(pamd_problem), offsetof(pamd_system, pos_offset), offsetof(pamd_problem, systems));return 0;}
'''
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "t.c")
        open(c, "w").write(src)
        exe = os.path.join(d, "t")
        subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), c, "-o", exe], check=True)
        got = [int(v) for v in subprocess.run([exe], capture_output=True, text=True).stdout.split()]
    want = [ctypes.sizeof(_lib.pamd_potential), ctypes.sizeof(_lib.pamd_system),
            ctypes.sizeof(_lib.pamd_problem), _lib.pamd_system.pos_offset.offset,
            _lib.pamd_problem.systems.offset]
    assert got == want


def test_problem_layout_host_logic():
    import paper_1907_09529_gb300 as pamd
    p = pamd.Problem([pamd.System("lj", 108, 3, 10, 2, box=5.03, rc=2.5),
                      pamd.System("harmonic", 1, 3, 17, 3)], 1.0, 1.0, 1e-4)
    assert p.offsets[0] == 0 and p.offsets[1] % 8 == 0
    assert p.offsets[1] >= 2 * 11 * 3 * 108
    assert p.n_chains == 5 and p.chain0 == [0, 2]
    assert p.units == 108 * 10 * 2 + 17 * 3
    buf = p.empty("cpu")
    assert p.view(buf, 1).shape == (3, 18, 3, 1)


def test_tune_accepts_the_autotuner_shapes_and_rejects_bad_ones():
    """pamd_tune is host-only (no CUDA call): every autotuner shape is accepted,
    sizes that cannot work are refused with PAMD_ERR_ARG."""
    import paper_1907_09529_gb300 as pamd
    from paper_1907_09529_gb300 import _lib, autotune
    try:
        shapes = list(autotune.candidates(tiles=(32, 192), windows=(2, 12)))
        assert shapes and all(len(s) == 5 for s in shapes)
        for shape in shapes:
            pamd.tune(*shape)
        lib = _lib.load()
        for bad in [(-1, 0, 0, -1.0, 0), (0, 3, 0, -1.0, 0), (0, 0, -5, -1.0, 0),
                    (0, 0, 0, -1.0, 1), (0, 0, 0, -1.0, -2)]:
            assert lib.pamd_tune(*bad) == _lib.PAMD_ERR_ARG, bad
    finally:
        pamd.tune()
