import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)
HERE = os.path.dirname(os.path.abspath(__file__))
if HERE not in sys.path:
    sys.path.insert(0, HERE)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a GB300 GPU and the CUDA library")
    config.addinivalue_line("markers", "slow: long-running CPU test")


def pytest_terminal_summary(terminalreporter):
    import _records

    if not _records.TENDENCY:
        return
    tr = terminalreporter
    tr.section("tendency errors against the oracle (per field h, hu, hv)")
    tr.write_line("check: plain ||k - k_oracle|| / ||k_oracle||  |  max|k - k_oracle| / max S")
    for what, row in _records.TENDENCY:
        plain = " ".join(f"{p:.2e}" for p, _ in row)
        mag = " ".join(f"{m:.2e}" for _, m in row)
        tr.write_line(f"{what}: {plain}  |  {mag}")
