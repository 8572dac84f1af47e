"""Host logic of bench.py that needs no GPU: the DRAM traffic figure is reported
only while the kernel source it was captured with is unchanged."""
import hashlib
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _sha(rel):
    return hashlib.sha256(open(os.path.join(ROOT, rel), "rb").read()).hexdigest()


def test_traffic_follows_the_source_hash(tmp_path, monkeypatch):
    src = "paper_1909_10286_gb300/csrc/biolog_kernels.cu"
    f = tmp_path / "traffic.txt"
    f.write_text(f"# comment\npaper {src} {_sha(src)} 12345   note\nlarge {src} {'0' * 64} 999\n")
    monkeypatch.setattr(bench, "TRAFFIC_FILE", str(f))
    assert bench._traffic("paper") == 12345
    assert bench._traffic("large") is None        # captured with another version of the source
    assert bench._traffic("batched") is None      # no capture listed
    monkeypatch.setattr(bench, "TRAFFIC_FILE", str(tmp_path / "missing.txt"))
    assert bench._traffic("paper") is None


def test_committed_traffic_file_is_well_formed():
    rows = [r.split() for r in open(bench.TRAFFIC_FILE) if r.strip() and not r.startswith("#")]
    assert {r[0] for r in rows} >= {"paper", "batched", "large", "learned"}
    for r in rows:
        assert os.path.exists(os.path.join(ROOT, r[1])) and len(r[2]) == 64 and int(r[3]) > 0
