import math
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")


def load_golden(name: str = "hand_examples.txt") -> dict:
    """Parse a golden fixture of `key = python-expression` lines."""
    path = os.path.join(ROOT, "tests", "golden", name)
    env = {"sqrt": math.sqrt, "__builtins__": {}}
    out = {}
    with open(path) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            key, expr = line.split("=", 1)
            out[key.strip()] = eval(expr.strip(), env)  # noqa: S307 - trusted fixture
    return out


@pytest.fixture(scope="session")
def golden():
    return load_golden()
