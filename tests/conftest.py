import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built rvh library")
    config.addinivalue_line("markers", "slow: longer CPU or GPU runs")


def pytest_terminal_summary(terminalreporter, exitstatus, config):
    try:
        from tests import gpu_util
    except Exception:  # the GPU helpers need numpy and the oracle
        return
    if gpu_util.PARITY_LOG:
        terminalreporter.write_sep("-", "oracle parity: clusters compared, oracle-fragile, ties")
        for line in gpu_util.PARITY_LOG:
            terminalreporter.write_line(line)
