import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300) and the built CUDA library")
    config.addinivalue_line("markers", "slow: long-running CPU statistics test")


@pytest.fixture(scope="session")
def O():
    alt = os.environ.get("RT_ORACLE_PY")
    if alt:
        # a copy of oracle/oracle.py with one planted mistake (the mutation
        # tests of the oracle's pins)
        import importlib.util
        spec = importlib.util.spec_from_file_location("oracle_planted", alt)
        oracle = importlib.util.module_from_spec(spec)
        spec.loader.exec_module(oracle)
    else:
        from oracle import oracle
    oracle.build()
    return oracle
