import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300) and the built libhbe")
    config.addinivalue_line("markers", "slow: long-running CPU test")


def _golden(name):
    path = os.path.join(ROOT, "tests", "golden", name)
    out = {}
    with open(path) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if not line:
                continue
            key, val = (s.strip() for s in line.split("=", 1))
            parts = [eval(v, {"__builtins__": {}}) for v in val.split(",")]
            out[key] = parts[0] if len(parts) == 1 else tuple(parts)
    return out


@pytest.fixture(scope="session")
def paper_values():
    return _golden("paper_values.txt")
