"""Host-side logic of bench.py that needs no GPU: the roofline's DRAM traffic is taken from the committed
ncu summary only while that summary was captured on the current kernel source, and the measured peaks
file is read when present."""
import os

import bench


def test_committed_traffic_matches_current_kernel_source():
    """The FP32 Dslash summary carries the hash of the source it was captured on; it must be the current
    one (an edit to the kernel or its helpers needs a new capture), and the traffic is then reported."""
    path = os.path.join(bench.ROOT, "profiles", "ncu_dslash_f32_48c12.txt")
    kv = dict(l.split(":", 1) for l in open(path) if ":" in l and not l.startswith("#"))
    assert kv["kernel_source_hash"].strip() == bench.kernel_source_hash()
    traffic = bench.ncu_traffic("ncu_dslash_f32_48c12.txt")
    assert traffic is not None
    # close to the algorithmic bytes of one launch (16 links + 2 vector entries per site, FP32)
    algorithmic = 663552 * (16 * 18 + 12) * 4
    assert 0.9 * algorithmic < traffic < 1.1 * algorithmic


def test_traffic_is_dropped_for_another_source(tmp_path, monkeypatch):
    src = open(os.path.join(bench.ROOT, "profiles", "ncu_dslash_f32_48c12.txt")).read()
    p = tmp_path / "profiles"
    p.mkdir()
    (p / "stale.txt").write_text(src.replace("kernel_source_hash: ", "kernel_source_hash: 0", 1))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: "5f8e32a76ed99193")
    assert bench.ncu_traffic("stale.txt") is None
    assert bench.ncu_traffic("missing.txt") is None


def test_peaks_fallback(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.peaks() == (bench.FALLBACK_HBM, "of fallback")
    (tmp_path / "MEASURED_PEAKS.json").write_text('{"hbm_gbs": 6777.3}')
    assert bench.peaks() == (6777.3, "of measured")
