import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: long oracle runs (still CPU-only)")


@pytest.fixture(scope="session")
def gpu_lib():
    """The built CUDA library; GPU tests fail loudly when it is missing."""
    import torch

    assert torch.cuda.is_available(), "GPU test run without a CUDA device"
    from paper_1805_07251_gb300 import build, capi

    build.build()
    capi.load()
    return capi


# Parity bounds applied by the GPU tests, printed in the terminal summary so that every
# run's log shows which bound each comparison used and what it measured.
_BOUNDS = []


@pytest.fixture
def parity_bound(request):
    """check(quantity, measured, bound): assert measured < bound and record both."""
    name = request.node.nodeid.split("::")[-1]

    def check(quantity, measured, bound):
        measured, bound = float(measured), float(bound)
        _BOUNDS.append((name, quantity, measured, bound))
        assert measured < bound, f"{quantity}: {measured:.3e} is not below the bound {bound:.3e}"

    return check


def pytest_terminal_summary(terminalreporter):
    if not _BOUNDS:
        return
    tr = terminalreporter
    tr.write_sep("-", "parity bounds applied (measured < bound)")
    for name, quantity, measured, bound in _BOUNDS:
        tr.write_line(f"{name[:58]:58s} {quantity[:34]:34s} {measured:9.2e} < {bound:9.2e}")
    worst = max(_BOUNDS, key=lambda b: b[2] / b[3] if b[3] > 0 else 0.0)
    tr.write_line(f"closest to its bound: {worst[0]} {worst[1]} ({worst[2]:.2e} of {worst[3]:.2e})")
