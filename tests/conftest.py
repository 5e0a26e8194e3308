import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU and the compiled sm_103a library")
    config.addinivalue_line("markers", "slow: long-running CPU oracle check")


@pytest.fixture(autouse=True)
def _debug_checks(request):
    """With MQS_DEBUG=1 (the debug library): after every GPU test, no kernel index
    may have left its array and every open solver's guard bytes must be intact."""
    yield
    if os.environ.get("MQS_DEBUG", "") in ("", "0") or request.node.get_closest_marker("gpu") is None:
        return
    import paper_1611_06721_gb300 as pkg
    rep = pkg.debug_check()
    assert rep["enabled"] == 1, "MQS_DEBUG=1 but the release library is loaded"
    assert rep["faults"] == 0, f"kernel index out of range: site {rep['site']}, index {rep['index']}"
    assert rep["canaries_bad"] == 0, f"{rep['canaries_bad']} of {rep['buffers']} buffers overran their guard bytes"
