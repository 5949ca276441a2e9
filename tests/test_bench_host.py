"""Host-side arithmetic of bench.py on CPU: the algorithmic byte model (the PCG at
its minimum of 6 values per cell and iteration: x, r, p read and written), the bytes
each PCG form's schedule moves, the per-kernel table the roofline line is built from
(GB/s = algorithmic bytes / event time, the persistent PCG counted per iteration), and
the rule that DRAM traffic from the committed ncu summary is used only while the
profiled kernel sources are unchanged."""
import hashlib
import os

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_byte_model():
    assert bench.bytes_per_cell("pcg", False, 0.0) == 24      # 6 FP32 values per cell
    assert bench.bytes_per_cell("pcg", True, 0.0) == 48
    # the two-launch schedule moves 10 values: the two passes of one iteration
    assert bench.bytes_per_cell("cg_a", False, 0.0) + bench.bytes_per_cell("cg_b", False, 0.0) \
        == bench.pcg_schedule_bytes(0, False) == 40
    # the streaming form: x += alpha p moved into pass A's staging of p saves p's reread
    assert bench.pcg_schedule_bytes(1, False) == 36
    # the fused single-barrier form: x, r, p in and out (q recomputed) plus the face planes
    assert bench.pcg_schedule_bytes(5, False) == 6 * 4 + 3 * 0.375 * 4
    assert bench.bytes_per_cell("momentum", False, 0.5) == 12 * 4 + 0.5 * 4


def test_kernel_table_rates():
    prof = {"pcg": (10.0, 2), "rhs": (1.0, 5), "misc": (0.1, 3), "mg": (0.0, 0)}
    t = bench.kernel_table(prof, 1000, False, 0.0, 100)
    assert "mg" not in t                                      # never launched
    p = t["pcg"]
    assert p["units"] == 100 and p["launches"] == 2
    assert p["bytes_per_launch"] == 24 * 1000 * 100 / 2
    assert abs(p["GBps"] - 24 * 1000 * 100 / 10e-3 / 1e9) < 1e-12
    assert abs(p["us_per_iter"] - 100.0) < 1e-12
    r = t["rhs"]
    assert r["units"] == 5 and abs(r["avg_us"] - 200.0) < 1e-12
    assert t["misc"]["GBps"] is None                          # no byte model: time only


def _source_hash():
    h = hashlib.sha256()
    for f in bench.PCG_SOURCES:
        with open(os.path.join(ROOT, "paper_1808_04099_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def test_profiled_traffic_only_for_matching_sources(tmp_path, monkeypatch):
    good = tmp_path / "good.md"
    good.write_text(f"sources = `{_source_hash()}`\n\ndram bytes per PCG iteration: 123456\n")
    monkeypatch.setitem(bench.PROFILES, 1, (str(good), bench.PCG_SOURCES))
    assert bench.profiled_pcg_traffic(1) == 123456.0
    stale = tmp_path / "stale.md"
    stale.write_text("sources = `0123456789abcdef`\n\ndram bytes per PCG iteration: 123456\n")
    monkeypatch.setitem(bench.PROFILES, 1, (str(stale), bench.PCG_SOURCES))
    assert bench.profiled_pcg_traffic(1) is None
    monkeypatch.setitem(bench.PROFILES, 1, (str(tmp_path / "missing.md"), bench.PCG_SOURCES))
    assert bench.profiled_pcg_traffic(1) is None
    assert bench.profiled_pcg_traffic(0) is None              # no summary for that form
