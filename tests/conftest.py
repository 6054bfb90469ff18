import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a GB300 (sm_103a) GPU and the CUDA library")
    config.addinivalue_line("markers", "slow: statistical checks that take tens of seconds")


@pytest.fixture(scope="session")
def oracle_mod():
    import oracle

    oracle.build()
    return oracle


def pytest_sessionfinish(session, exitstatus):
    """Write the GPU parity report (intervals compared, decisions, near-edge
    decisions, partings and worst errors of every compared run) when GPU
    tests recorded any: to $LRDMC_PARITY_REPORT, else
    results/parity_report.json."""
    import json

    try:
        import _parity_util as U
    except ImportError:
        return
    if not U.REPORT:
        return
    path = os.environ.get("LRDMC_PARITY_REPORT", os.path.join(ROOT, "results", "parity_report.json"))
    os.makedirs(os.path.dirname(os.path.abspath(path)), exist_ok=True)
    summary = {
        "tolerance_rel": U.RTOL, "edge": U.EDGE, "entries": len(U.REPORT),
        "intervals_compared": sum(e.get("intervals_compared", 0) for e in U.REPORT),
        "decisions": sum(e.get("decisions", 0) for e in U.REPORT),
        "near_edge_decisions": sum(e.get("near_edge", 0) for e in U.REPORT),
        "partings": sum(1 for e in U.REPORT if e.get("parted")),
    }
    with open(path, "w") as f:
        json.dump({"summary": summary, "runs": U.REPORT}, f, indent=1, default=float)
