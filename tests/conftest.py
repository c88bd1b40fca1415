import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


GOLDEN = os.path.join(ROOT, "tests", "golden")


def paper_values():
    """Numbers printed in the paper (tests/golden/paper_printed_values.json)."""
    import json
    with open(os.path.join(GOLDEN, "paper_printed_values.json")) as f:
        return json.load(f)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300) and the built CUDA library")
    config.addinivalue_line("markers", "slow: long-running CPU test")
