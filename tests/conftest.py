import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: long CPU test")


def pytest_terminal_summary(terminalreporter):
    """The worst per-event parity errors seen in this session (tests/parity.py)."""
    from tests.parity import WORST
    if WORST:
        terminalreporter.write_sep("-", "parity: worst |log P_gpu - log P_orc| and stated errors")
        for k, v in WORST.items():
            terminalreporter.write_line(f"{k}: {v:.3e}")
