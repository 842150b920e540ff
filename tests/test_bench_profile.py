"""The bench reports ncu DRAM traffic only for the kernel and tile shape it was captured on.

`traffic_from_profile` reads `traffic_bytes_per_launch` from a committed summary under
`profiles/` when the sha256 of the kernel's sources and the tile shape both match; otherwise the
bench's `roofline.traffic` is null. No GPU is needed.
"""
import hashlib
import os
import re

import pytest

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SUMMARIES = ["step_fused_pendulum_8192.md", "step_fused_fel_4096x2048.md"]


@pytest.mark.parametrize("name", SUMMARIES)
def test_summary_records_traffic_tile_and_hash(name):
    text = open(os.path.join(ROOT, "profiles", name)).read()
    assert re.search(r"^traffic_bytes_per_launch:\s*[0-9.eE+]+$", text, re.M)
    assert re.search(r"^tile:\s*\d+x\d+$", text, re.M)
    assert re.search(r"^source_sha256:\s*[0-9a-f]{64}$", text, re.M)
    # the summary names the command that made it, which runs committed files only
    assert "ncu --set full --clock-control none" in text and "python bench.py" in text


def test_traffic_needs_matching_sources_and_tile(tmp_path, monkeypatch):
    """A copy of the repository layout with a summary written for a known hash and tile."""
    src = tmp_path / "k.cu"
    src.write_text("kernel source\n")
    (tmp_path / "profiles").mkdir()
    digest = hashlib.sha256(b"kernel source\n").hexdigest()
    (tmp_path / "profiles" / "p.md").write_text(
        f"traffic_bytes_per_launch: 1.25e+08\ntile: 224x63\nsource_sha256: {digest}\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.traffic_from_profile("p.md", ["k.cu"], tile=(224, 63)) == 1.25e8
    assert bench.traffic_from_profile("p.md", ["k.cu"], tile=(224, 64)) is None
    assert bench.traffic_from_profile("missing.md", ["k.cu"], tile=(224, 63)) is None
    src.write_text("kernel source, changed\n")
    assert bench.traffic_from_profile("p.md", ["k.cu"], tile=(224, 63)) is None
