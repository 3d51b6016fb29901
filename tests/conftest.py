import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300) and the built library")
    config.addinivalue_line("markers", "slow: longer CPU test")


def pytest_terminal_summary(terminalreporter, exitstatus, config):
    """Print the worst measured error of every parity comparison (GPU path
    against the FP64 oracle), per test and precision policy, beside the bar
    the test held it to."""
    try:
        from tests import gpu_helpers
    except Exception:
        return
    rows = gpu_helpers.MEASURED
    if not rows:
        return
    tr = terminalreporter
    tr.section("measured parity errors (GPU path vs FP64 oracle)")
    keys = ("force", "energy", "charge", "mu", "eatom", "virial", "stationarity")
    tr.write_line("%-64s %-6s " % ("test [replica]", "policy") + " ".join("%10s" % k for k in keys))
    for name, prec, res in rows:
        tr.write_line("%-64s %-6s " % (name[-64:], prec)
                      + " ".join("%10.2e" % res[k] if k in res else "%10s" % "-" for k in keys))
    for prec in sorted({p for _, p, _ in rows}):
        worst = {k: max((r[k] for _, p, r in rows if p == prec and k in r), default=None) for k in keys}
        bar = dict(gpu_helpers.TOL[prec])
        bar["stationarity"] = 10 * bar["mu"]   # sampled local checks: dE/dq_i - mu at sampled atoms
        tr.write_line("worst %-6s: " % prec + ", ".join(
            "%s %.2e (bar %.0e)" % (k, v, bar[k]) for k, v in worst.items() if v is not None))
