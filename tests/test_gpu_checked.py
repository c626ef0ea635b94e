"""The GPU suite on the bounds-checked build (build(checked=True),
-DSICP_CHECKED): every index that comes from data (cell coordinates, the
seed map, cell bounds, the row table, minibatch entries, search results,
fallback lists, batched work items) is checked before its access.  The suite
runs in a child process with SICP_CHECKED=1, which makes the binding load
the checked library and conftest's fixture assert after each GPU test that
no check failed.  This stands in for a memory checker where none can run:
the same tests, the same results, and not one access outside its buffer.
"""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_gpu_suite_passes_on_the_checked_build():
    if os.environ.get("SICP_CHECKED") == "1":
        pytest.skip("already inside the checked run")
    from paper_2106_03287_gb300 import build
    build.build()
    lib = build.build(checked=True)
    assert os.path.exists(lib)
    here = os.path.join(ROOT, "tests")
    files = sorted(f for f in os.listdir(here)
                   if (f.startswith("test_gpu_") or f.startswith("test_zz_")) and f != "test_gpu_checked.py")
    env = dict(os.environ, SICP_CHECKED="1")
    r = subprocess.run([sys.executable, "-m", "pytest", *files, "-q", "-m", "gpu", "-p", "no:cacheprovider", "-x"],
                       cwd=here, env=env, capture_output=True, text=True, timeout=1800)
    tail = (r.stdout + r.stderr)[-3000:]
    assert r.returncode == 0, tail
    assert " passed" in r.stdout and "failed" not in r.stdout, tail
    print(r.stdout.strip().splitlines()[-1])
