import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built CUDA library")
    config.addinivalue_line("markers", "slow: long-running statistical or full-size test")


def pytest_collection_modifyitems(config, items):
    try:
        import torch
        have_gpu = torch.cuda.is_available()
    except Exception:  # pragma: no cover
        have_gpu = False
    if have_gpu:
        return
    skip = pytest.mark.skip(reason="no CUDA GPU in this environment")
    for it in items:
        if "gpu" in it.keywords:
            it.add_marker(skip)


def pytest_terminal_summary(terminalreporter, exitstatus, config):
    """Near-tie rates of the sampled full-size parity tests (oracle near ties over components)."""
    mod = sys.modules.get("parity_util")
    if mod is None:
        return
    for label, near, comps, mism in mod.NEAR_TIE_LOG:
        rate = near / comps if comps else 0.0
        terminalreporter.write_line(f"near ties {label}: {near} of {comps} components ({rate:.2e}), "
                                    f"{mism} exempted id mismatches")
