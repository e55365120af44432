import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running CPU check")


@pytest.fixture(autouse=True)
def _no_out_of_range_index(request):
    """In the bounds-checked build (KS_DEBUG_BOUNDS=1), every GPU test must
    leave no out-of-range index in the kernels' record."""
    yield
    if request.node.get_closest_marker("gpu") is None:
        return
    if os.environ.get("KS_DEBUG_BOUNDS", "0") in ("", "0"):
        return
    import paper_1308_2864_gb300 as ks
    rec = ks.debug_bounds()
    assert rec["checked"], "KS_DEBUG_BOUNDS is set but the library is not a bounds-checked build"
    assert rec["count"] == 0, (f"{rec['count']} out-of-range indices, the first at "
                               f"{rec['file']}:{rec['line']}")
