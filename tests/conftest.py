import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: long CPU test")


def golden_table2():
    rows = []
    with open(os.path.join(ROOT, "tests", "golden", "table2_sog_params.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            v = line.split()
            rows.append(dict(b=float(v[0]), sigma=float(v[1]), omega=float(v[2]),
                             err_energy=float(v[3]), M_energy=int(v[4]),
                             err_force=float(v[5]), M_force=int(v[6]),
                             err_pressure=float(v[7]), M_pressure=int(v[8])))
    return rows


@pytest.fixture(scope="session")
def table2():
    return golden_table2()
