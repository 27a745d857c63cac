import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
for p in (ROOT, os.path.join(ROOT, "oracle")):
    if p not in sys.path:
        sys.path.insert(0, p)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a GB300 (sm_103a) and the CUDA library")


def pytest_collection_modifyitems(config, items):
    # keep GPU tests from running by accident on a box without a GPU
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


# FP32 (GPU) against FP64 (oracle) error per parity result.  GPU tests record
# each measured error with its tolerance through the `parity_report` fixture;
# with LHMM_PARITY_REPORT=<path> set, the session writes them as a markdown
# table to that path.
_PARITY_ROWS = []


@pytest.fixture
def parity_report(request):
    def record(result, error, tolerance, unit=""):
        _PARITY_ROWS.append((request.node.nodeid.split("::")[-1], result, float(error),
                             float(tolerance), unit))
    return record


def pytest_sessionfinish(session, exitstatus):
    path = os.environ.get("LHMM_PARITY_REPORT")
    if not path or not _PARITY_ROWS:
        return
    with open(path, "w") as fh:
        fh.write("| test | result | measured FP32-vs-FP64 error | tolerance | unit |\n")
        fh.write("|---|---|---|---|---|\n")
        for test, result, err, tol, unit in _PARITY_ROWS:
            fh.write("| %s | %s | %.3g | %.3g | %s |\n"
                     % (test, result, err, tol, unit.replace("|", "\\|")))
