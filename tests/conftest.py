import os
import sys
import tempfile
from fractions import Fraction

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

GOLDEN = os.path.join(ROOT, "tests", "golden")


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    # the library's autotuner table: a file of this test session's own
    os.environ.setdefault("HIVC_TUNE_CACHE", os.path.join(tempfile.gettempdir(), f"hivc_tune_{os.getpid()}.json"))


def read_golden(name):
    """Parse a golden fixture: header ints, then tagged lines of numbers
    (fractions like 36/7 allowed).  Returns (header, {tag: [rows]})."""
    header, tags = None, {}
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            line = line.split("#", 1)[0].strip()
            if not line:
                continue
            parts = line.split()
            if header is None and parts[0][0].isdigit():
                header = [int(p) for p in parts]
                continue
            tags.setdefault(parts[0], []).append([float(Fraction(p)) for p in parts[1:]])
    return header, tags


@pytest.fixture(scope="session")
def oracle_lib():
    import oracle

    oracle.build()
    return oracle
