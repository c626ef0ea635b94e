"""Programmatic dependent launch and the captured graph change when kernels are
scheduled, never what they compute: a registration run with both (the
default), one in a process with SICP_NO_PDL=1 (plain stream order) and one
with SICP_NO_GRAPH=1 (plain launches instead of the captured loop) return
bit-identical particles, for every exact search, point-to-point and
point-to-plane, Stein and independent runs.  The oracle is not involved; the
comparison is exact.
"""
import os
import subprocess
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_2106_03287_gb300 as S  # noqa: E402

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# One script, run in this process's environment and in one without the
# programmatic launches; it prints every run's particles as hex words.
SCRIPT = r"""
import sys
import numpy as np
sys.path.insert(0, sys.argv[1])
import paper_2106_03287_gb300 as S
from paper_2106_03287_gb300 import synth
c = S.sicp_create(0)
out = []
d = synth.make_box_problem(2, K=40)
S.sicp_set_reference(c, d["ref"])
S.sicp_reference_normals(c, 10, want=False)
for mode in (S.SICP_NN_GRID, S.SICP_NN_BRUTE_FP32, S.SICP_NN_BRUTE_BF16):
    for extra in (0, S.SICP_POINT_TO_PLANE, S.SICP_INDEPENDENT):
        p = S.sicp_default_params(T=25, m=100, lr=0.01, seed=3, nn_mode=mode | extra)
        th, _, _ = S.sicp_register(c, d["src"], d["particles"], p)
        out.append(np.ascontiguousarray(th, np.float32).view(np.uint32).tobytes().hex())
d = synth.make_kinect_problem(1)
S.sicp_set_reference(c, d["ref"])
th, _, _ = S.sicp_register(c, d["src"], d["particles"],
                           S.sicp_default_params(T=20, m=300, lr=0.03, seed=1, nn_mode=S.SICP_NN_GRID))
out.append(np.ascontiguousarray(th, np.float32).view(np.uint32).tobytes().hex())
S.sicp_destroy(c)
print("\n".join(out))
"""


def _run(env):
    r = subprocess.run([sys.executable, "-c", SCRIPT, ROOT], env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    return r.stdout.split()


def test_programmatic_launch_changes_no_result():
    from paper_2106_03287_gb300 import build
    build.build()
    on = dict(os.environ)
    on.pop("SICP_NO_PDL", None)
    off = dict(on, SICP_NO_PDL="1")
    a, b = _run(on), _run(off)
    assert len(a) == len(b) == 10
    for i, (x, y) in enumerate(zip(a, b)):
        assert x == y, f"run {i} differs with and without programmatic launch"


def test_uncaptured_loop_changes_no_result():
    """SICP_NO_GRAPH=1 runs the registration loop as plain launches instead of
    one captured CUDA graph: the same kernels with the same arguments, so the
    same particles bit for bit (also with the programmatic launches off)."""
    from paper_2106_03287_gb300 import build
    build.build()
    base = dict(os.environ)
    base.pop("SICP_NO_PDL", None)
    base.pop("SICP_NO_GRAPH", None)
    a = _run(base)
    b = _run(dict(base, SICP_NO_GRAPH="1"))
    c = _run(dict(base, SICP_NO_GRAPH="1", SICP_NO_PDL="1"))
    assert len(a) == len(b) == len(c) == 10
    for i, (x, y, z) in enumerate(zip(a, b, c)):
        assert x == y == z, f"run {i} differs without the captured graph"
