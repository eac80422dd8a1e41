import sys
from pathlib import Path

import pytest

ROOT = Path(__file__).resolve().parents[1]
if str(ROOT) not in sys.path:
    sys.path.insert(0, str(ROOT))


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA device and the built CUDA library")
    config.addinivalue_line("markers", "slow: longer CPU statistics test")


def load_kat():
    rows = []
    for line in (ROOT / "tests" / "golden" / "philox4x32_10_kat.txt").read_text().splitlines():
        if not line.strip() or line.startswith("#"):
            continue
        v = [int(t, 16) for t in line.split()]
        rows.append((v[0:4], v[4:6], v[6:10]))
    return rows


@pytest.fixture(scope="session")
def kat_vectors():
    return load_kat()
