import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

# a layout cache the autotuner may have left on this machine must not change
# the layouts the tests run (tests of the tuner point this at their own file)
os.environ.setdefault("PTA_TUNE_CACHE", os.path.join(ROOT, "tests", ".no_tune_cache.json"))


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU and the compiled library")
    config.addinivalue_line("markers", "slow: long CPU test")


def golden(name):
    """Read a whitespace table from tests/golden (comment lines start with #)."""
    rows = []
    with open(os.path.join(ROOT, "tests", "golden", name)) as fh:
        for line in fh:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line.split())
    return rows


@pytest.fixture(scope="session")
def oracle():
    import oracle as O
    O.build()
    return O
