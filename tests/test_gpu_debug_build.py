"""The bounds-checked build (libpamd_debug.so, -DPAMD_DEBUG) over the small parity
shapes: every array index of the kernels is checked on the device, and none may
fall outside its array; the results still match the oracle.  Run in a child
process so that the checked library is the one loaded."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_debug_build_records_no_out_of_bounds_index():
    torch = pytest.importorskip("torch")
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import __graft_entry__
    __graft_entry__.build()
    from paper_1907_09529_gb300 import build
    build.build(debug=True)
    env = dict(os.environ, PAMD_LIBRARY="debug")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "tests", "_debug_shapes.py")],
                       capture_output=True, text=True, env=env, cwd=ROOT, timeout=900)
    assert r.returncode == 0, r.stderr[-4000:]
    res = json.loads(r.stdout.strip().splitlines()[-1])
    assert res["checked"] == 1, "the child did not load the bounds-checked build"
    assert res["count"] == 0, res
    assert res["worst"]["fp32"] <= 1e-5 and res["worst"]["fp64"] <= 1e-12, res["worst"]
