import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built library")


@pytest.fixture(autouse=True)
def _index_checks(request):
    """With SICP_CHECKED=1 the binding loads the bounds-checked library: after
    every GPU test, no index check may have failed."""
    yield
    if os.environ.get("SICP_CHECKED") == "1" and request.node.get_closest_marker("gpu"):
        import paper_2106_03287_gb300 as S
        checked, first, count = S.sicp_check_status()
        assert checked, "SICP_CHECKED=1 but the loaded library is not the checked build"
        assert count == 0, f"{count} index checks failed; first: site {(first >> 40) & 0x7fffff}, " \
                           f"index {first & ((1 << 40) - 1)}"
