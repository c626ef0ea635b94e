"""The C-ABI library builds for sm_103a, loads, and exports every entry point
that include/steinicp.h declares (no compute calls: this runs without a GPU)."""
import ctypes
import os
import re

import paper_2106_03287_gb300 as S
from paper_2106_03287_gb300 import build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            text = open(os.path.join(ROOT, "include", h)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b(sicp_\w+)\s*\(", text))
    return names


def test_library_builds_and_exports_every_declared_symbol():
    path = build.build()
    assert os.path.exists(path)
    lib = ctypes.CDLL(path)
    declared = _declared()
    assert declared, "no declarations found"
    missing = [n for n in sorted(declared) if not hasattr(lib, n)]
    assert not missing, missing
    assert declared == set(S.EXPORTS)


def test_checked_library_builds_and_exports_the_same_symbols():
    """The bounds-checked variant (-DSICP_CHECKED) is the same library with
    index checks compiled in: same exports, plus a status that says so (the
    status itself needs a GPU, so only the symbol is checked here)."""
    path = build.build(checked=True)
    assert os.path.basename(path) == "libsteinicp_checked.so" and os.path.exists(path)
    lib = ctypes.CDLL(path)
    missing = [n for n in sorted(_declared()) if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_params_layout_matches_defaults():
    p = S.sicp_default_params()
    assert (p.T, p.m, p.nn_mode, p.prior, p.surrogate_iters) == (100, 100, S.SICP_NN_GRID, 0, 0)
    assert p.surrogate_min_conf == 0.5
    assert abs(p.lr - 0.01) < 1e-9 and abs(p.beta2 - 0.999) < 1e-7
    assert ctypes.sizeof(S.sicp_params) == 96
