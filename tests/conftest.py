import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the compiled libls.so")


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


def pytest_terminal_summary(terminalreporter, exitstatus, config):
    """The parity figures the GPU tests measured (image errors, flagged and
    mismatched pixel fractions, record-field and gradient errors)."""
    try:
        from tests.gpu_helpers import PARITY_LOG
    except Exception:  # pragma: no cover
        return
    if not PARITY_LOG:
        return
    terminalreporter.write_sep("-", "measured parity")
    for test, what, fig in PARITY_LOG:
        vals = " ".join("%s=%.3g" % (k, v) if isinstance(v, float) else "%s=%s" % (k, v) for k, v in fig.items())
        terminalreporter.write_line("%s %s %s" % (test, what, vals))
