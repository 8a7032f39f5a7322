import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)
HERE = os.path.dirname(os.path.abspath(__file__))
if HERE not in sys.path:
    sys.path.insert(0, HERE)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA device (GB300, sm_103a)")


@pytest.fixture(scope="session")
def orc():
    import oracle
    oracle.build()
    return oracle


def pytest_terminal_summary(terminalreporter):
    # the largest measured / bound-unit ratio of every parity tolerance kind,
    # so that each constant in tests/parity.py can be checked against data
    try:
        import parity
    except Exception:
        return
    if not parity.RATIOS:
        return
    terminalreporter.write_sep("-", "parity ratios (largest measured / unit)")
    for kind, (r, where) in sorted(parity.RATIOS.items()):
        terminalreporter.write_line(f"{kind}: {r:.3g}  [{where}]")
