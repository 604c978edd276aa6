import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA device (B300); parity tests through the C ABI")


@pytest.fixture(scope="session")
def table():
    from paper_1712_05012_b300 import synth

    return synth.type_table()
