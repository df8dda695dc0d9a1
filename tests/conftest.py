import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_addoption(parser):
    parser.addoption("--fx-checked", action="store_true",
                     help="run the GPU tests on the checked build (libfx_checked.so, every kernel memory index "
                          "range-checked) and require zero check failures")
    parser.addoption("--fx-lib", default=None,
                     help="run the GPU tests on the library at this path (a checked build must count zero "
                          "check failures)")


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built library")
    config.addinivalue_line("markers", "slow: long-running CPU test")


@pytest.fixture(scope="session")
def cuda_lib(request):
    """The CUDA library through its C-ABI binding (GPU tests only).  With
    --fx-checked the checked build is loaded instead, and the session ends by
    requiring that its kernels counted no range-check failure."""
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1304_3992_gb300 import fx
    checked = request.config.getoption("--fx-checked")
    if checked:
        from paper_1304_3992_gb300 import build
        fx.LIB_PATH = build.build(checked=True)
    elif request.config.getoption("--fx-lib"):
        fx.LIB_PATH = os.path.abspath(request.config.getoption("--fx-lib"))
    fx.load()
    counted = fx.checked_violations(reset=True)  # None unless a checked build is loaded
    assert counted in (None, 0)
    assert counted is not None or not checked
    yield fx
    if counted is not None:
        n = fx.checked_violations()
        assert n == 0, f"{n} kernel memory accesses failed their range check"
