"""Host helpers of bench.py: the committed ncu counters of the PROBE level kernel are used only while the kernel
source still has the hash they were captured at, and the roofline inputs parse as the summary states them."""
import hashlib
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    if ROOT not in sys.path:
        sys.path.insert(0, ROOT)
    import bench
    return bench


def test_committed_counters_match_the_current_kernel():
    bench = _bench()
    ratio, pipe = bench.recorded_pull_counters()
    assert ratio is not None and 1.0 <= ratio < 3.0  # DRAM bytes at least the compulsory ones
    assert pipe is not None and 0.0 < pipe <= 1.0


def test_counters_are_dropped_once_the_kernel_changes(tmp_path, monkeypatch):
    bench = _bench()
    (tmp_path / "paper_1709_06955_gb300" / "csrc").mkdir(parents=True)
    (tmp_path / "profiles").mkdir()
    src = tmp_path / "paper_1709_06955_gb300" / "csrc" / "pull.cu"
    src.write_text("// a kernel\n")
    h = hashlib.sha256(src.read_bytes()).hexdigest()[:16]
    (tmp_path / "profiles" / "k_pull_traffic.txt").write_text(
        "# a summary\nratio 1.25 %s\nl1pipe 0.5 %s\n" % (h, h))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.recorded_pull_counters() == (1.25, 0.5)
    src.write_text("// the kernel, edited after the capture\n")
    assert bench.recorded_pull_counters() == (None, None)
