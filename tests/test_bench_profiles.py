"""Host logic of bench.py's roofline fields: the DRAM traffic per launch is
read from the committed ncu summary of the kernel and workload, and only
while the kernel's sources still match the digest recorded with it."""
import os
import shutil
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _summary(digest, traffic):
    return ("# test summary\n\n| key | value |\n|---|---|\n"
            f"| traffic_bytes_per_launch | {traffic} |\n| sources_sha256 | `{digest}` |\n")


def test_traffic_read_only_while_sources_match(tmp_path, monkeypatch):
    # a copy of the repository layout the helpers read
    root = tmp_path / "repo"
    shutil.copytree(os.path.join(ROOT, "paper_2009_12609_gb300", "csrc"),
                    root / "paper_2009_12609_gb300" / "csrc")
    (root / "profiles").mkdir()
    monkeypatch.setattr(bench, "ROOT", str(root))
    kernel, key = "march3d_kernel", "grid3d"
    digest = bench.sources_digest(kernel)
    assert len(digest) == 16
    assert bench.committed_traffic(kernel, key) is None          # no summary
    path = root / "profiles" / f"{kernel}_{key}_traffic.md"
    path.write_text(_summary(digest, 24490000000))
    assert bench.committed_traffic(kernel, key) == 24490000000.0
    path.write_text(_summary("0" * 16, 24490000000))             # other sources
    assert bench.committed_traffic(kernel, key) is None
    path.write_text(_summary(digest, "n/a"))                      # unreadable figure
    assert bench.committed_traffic(kernel, key) is None
    # a change to any source of the kernel changes the digest
    src = root / "paper_2009_12609_gb300" / "csrc" / "k_march3d.cu"
    src.write_text(src.read_text() + "\n// edit\n")
    assert bench.sources_digest(kernel) != digest


def test_committed_profiles_name_their_commands():
    """Every committed summary gives the command that produced it."""
    d = os.path.join(ROOT, "profiles")
    names = [n for n in os.listdir(d) if n.endswith(".md")]
    assert names
    for n in names:
        text = open(os.path.join(d, n)).read()
        assert "ncu " in text and "--clock-control none" in text, n
        assert "python bench.py" in text, n
