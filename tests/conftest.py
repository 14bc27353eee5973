import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (B300) and the built library")
    config.addinivalue_line("markers", "slow: longer statistical test (still CPU-only)")


@pytest.fixture(scope="session")
def cuda_ok():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return True


@pytest.fixture(autouse=True)
def _checked_build_word(request):
    """Under the checked build (LRDMC_CHECKED=1) every GPU test must leave the
    kernels' index-violation word at zero: an out-of-extent index anywhere in
    the walker or branching kernels fails the test that caused it."""
    yield
    if os.environ.get("LRDMC_CHECKED") != "1" or request.node.get_closest_marker("gpu") is None:
        return
    if request.node.name.startswith("test_check_selftest"):
        return
    import paper_2508_12033_b300.binding as B
    if B._LIB is None:
        return
    word, checked = B.check_word(clear=True)
    assert checked, "LRDMC_CHECKED=1 but the normal library is loaded"
    assert word == 0, f"index violation at csrc line {word >> 32}, index {word & 0xffffffff}"
