import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300) and the built libgksl")
    config.addinivalue_line("markers", "slow: long-running CPU test")


def _has_gpu():
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False


def pytest_collection_modifyitems(config, items):
    if _has_gpu():
        return
    skip = pytest.mark.skip(reason="no CUDA device")
    for it in items:
        if "gpu" in it.keywords:
            it.add_marker(skip)


_RECORDS = {}


@pytest.fixture
def record(request):
    """record(key, value) keeps a measured error or count of the calling test.  With the
    environment variable GKSL_RECORD set to a path, every recorded value is written there as
    JSON when the session ends; without it nothing is written."""
    def put(key, value):
        _RECORDS[f"{request.node.name}:{key}"] = float(value)
    return put


def pytest_sessionfinish(session, exitstatus):
    path = os.environ.get("GKSL_RECORD")
    if path and _RECORDS:
        import json
        with open(path, "w") as f:
            json.dump(_RECORDS, f, indent=1, sort_keys=True)
