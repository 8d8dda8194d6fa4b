import os
import sys

import pytest

ROOT = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(ROOT)
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)
TESTS = os.path.join(ROOT, "tests")
if TESTS not in sys.path:
    sys.path.insert(0, TESTS)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built library")
    config.addinivalue_line("markers", "slow: long-running CPU test")


def pytest_terminal_summary(terminalreporter, exitstatus, config):
    """The worst parity errors of every GPU-vs-oracle gate of this run:
    relative Frobenius and element-wise (max |x - x_o| / max |x_o|), on y and
    on Cx = y - Du, against the path's bar."""
    try:
        from _parity import RESULTS
    except Exception:
        return
    if not RESULTS:
        return
    tr = terminalreporter
    tr.section("parity: worst errors per gate (frob y, frob Cx, elem y, elem Cx | bar)")
    worst_ratio = 0.0
    for tid, what, fy, fcx, ey, ecx, bar in RESULTS:
        ratio = max(fy, fcx, ey, ecx) / bar if bar > 0 else 0.0
        worst_ratio = max(worst_ratio, ratio)
        name = tid.split("::", 1)[-1]
        tr.write_line(f"{name[:70]:70s} {what:6s} {fy:9.2e} {fcx:9.2e} {ey:9.2e} {ecx:9.2e} | "
                      f"{bar:.0e}  ({ratio:.2f} of bar)")
    tr.write_line(f"{len(RESULTS)} gates; the largest error is {worst_ratio:.3f} of its bar")
