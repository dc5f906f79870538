import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: takes more than a few seconds on the CPU")


def pytest_collection_modifyitems(config, items):
    try:
        import torch
        has_gpu = torch.cuda.is_available()
    except Exception:  # pragma: no cover
        has_gpu = False
    if has_gpu:
        return
    skip = pytest.mark.skip(reason="no CUDA device")
    for it in items:
        if "gpu" in it.keywords:
            it.add_marker(skip)


def pytest_terminal_summary(terminalreporter):
    try:
        from tests.gpu_util import MEASURED
    except Exception:  # pragma: no cover
        return
    if not MEASURED:
        return
    terminalreporter.write_sep("-", "measured errors (GPU parity)")
    for test, quantity, value, bound in MEASURED:
        b = "" if bound is None else f"   (bound {bound:.1e})"
        terminalreporter.write_line(f"{test}: {quantity} = {value:.3e}{b}")
