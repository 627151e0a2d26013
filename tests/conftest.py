import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)
HERE = os.path.dirname(os.path.abspath(__file__))
if HERE not in sys.path:
    sys.path.insert(0, HERE)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (runs the sm_103a library)")
    config.addinivalue_line("markers", "slow: takes more than a few seconds")


def pytest_terminal_summary(terminalreporter):
    """Every argmax comparison of the run with the oracle's top-two gap:
    decisive ones (identical indices required) and declared near-ties."""
    gc = sys.modules.get("gpu_common")
    rec = getattr(gc, "ARGMAX_RECORD", None)
    if not rec:
        return
    ties = [r for r in rec if not r[3]]
    terminalreporter.write_sep("-", f"argmax comparisons: {len(rec)}, near-ties: {len(ties)}")
    for test, gap, tol, decisive in rec:
        terminalreporter.write_line(f"{'decisive ' if decisive else 'near-tie '} gap {gap:.3e}  bound {tol:g}  {test}")
