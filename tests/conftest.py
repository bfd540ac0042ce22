import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built libcrk.so")
    config.addinivalue_line("markers", "slow: long CPU test")


@pytest.fixture(scope="session")
def orc():
    from oracle import oracle as O

    O.build()
    return O


def pytest_sessionfinish(session, exitstatus):
    out = os.environ.get("CRK_ERRORS_OUT")
    if out:
        import json

        from tests import _errors

        with open(out, "w") as fh:
            json.dump(_errors.RECORDS, fh, indent=0)
