import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


@pytest.fixture()
def record(request):
    """record(name, value): appends a measured error or timing to the JSON
    lines file named by GCQ_RECORD (when set), tagged with the test id, so
    that the tolerances in the tests can be compared with measured values."""
    import json
    path = os.environ.get("GCQ_RECORD")

    def _rec(name, value):
        if path:
            with open(path, "a") as f:
                f.write(json.dumps({"test": request.node.nodeid, "name": name, "value": float(value)}) + "\n")
    return _rec


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA device (B300, sm_103a)")
    config.addinivalue_line("markers", "slow: longer CPU test")


def pytest_collection_modifyitems(config, items):
    # GPU tests need the CUDA library and a device; keep CPU runs clean
    try:
        import torch
        has_gpu = torch.cuda.is_available()
    except Exception:  # pragma: no cover
        has_gpu = False
    if has_gpu:
        return
    skip = pytest.mark.skip(reason="no CUDA device")
    for item in items:
        if "gpu" in item.keywords:
            item.add_marker(skip)
