"""Every command-line option the benchmark's workloads read is one its parser
defines (a workload that reads a missing option fails only when it runs)."""
import os
import re
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_every_option_read_is_defined(monkeypatch):
    monkeypatch.setattr(sys, "argv", ["bench.py"])
    if ROOT not in sys.path:
        sys.path.insert(0, ROOT)
    import bench
    defined = set(vars(bench.parse()))
    used = set()
    for rel in ("bench.py", os.path.join("paper_1808_02515_gb300", "bench_workloads.py")):
        with open(os.path.join(ROOT, rel)) as f:
            used |= set(re.findall(r"\bargs\.([a-z_0-9]+)", f.read()))
    assert used, "no options found"
    assert sorted(used - defined) == []
