import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA device (GB300, sm_103a)")


def _read_paper_values():
    """name -> value from tests/golden/paper_values.txt (the values the paper prints)."""
    out = {}
    with open(os.path.join(ROOT, "tests", "golden", "paper_values.txt")) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if line:
                name, value = line.split()
                out[name] = float(value)
    return out


PAPER_VALUES = _read_paper_values()
