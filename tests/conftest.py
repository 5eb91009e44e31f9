import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built libvemg")
    config.addinivalue_line("markers", "slow: larger oracle cases")


def record(name, **values):
    """Append a measured value (an achieved error, an iteration count) as one JSON line to the
    file named by VEMG_TEST_RECORD, when that variable is set; tests assert their bounds either
    way."""
    path = os.environ.get("VEMG_TEST_RECORD")
    if not path:
        return
    import json
    with open(path, "a") as f:
        f.write(json.dumps({"test": name, **{k: (float(v) if hasattr(v, "__float__") else v)
                                            for k, v in values.items()}}) + "\n")
