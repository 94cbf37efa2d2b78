import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built library")


@pytest.fixture(scope="session")
def golden4():
    """The exact 4x4 pencil of tests/golden/pencil4_exact.txt as float64 arrays."""
    from fractions import Fraction

    import numpy as np

    rows = {"A": [], "B": [], "U": [], "lambda": []}
    with open(os.path.join(ROOT, "tests", "golden", "pencil4_exact.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            key, *vals = line.split()
            rows[key].append([float(Fraction(v)) for v in vals])
    return (np.array(rows["A"]), np.array(rows["B"]), np.array(rows["U"]), np.array(rows["lambda"][0]))
