"""Host-side pieces of bench.py (no GPU): variant tables and algorithmic bytes."""
import math

import bench


def test_gradient_table_is_rounded_exponential_within_p1():
    t = bench.gradient_table(10, 16.0)
    assert t.shape == (256,) and t[0] == 10 and (t >= 0).all() and (t <= 10).all()
    assert all(t[g] == math.floor(10 * math.exp(-g / 16.0) + 0.5) for g in range(256))
    assert (t[1:] <= t[:-1]).all()                     # non-increasing in the gradient


def test_variant_names_keep_the_headline_for_the_plain_matcher():
    assert bench.variant_names("plain") == (bench.METRIC, bench.WORKLOAD)
    m, w = bench.variant_names("paper_gradient")
    assert m.startswith(bench.METRIC[:-1]) and "layered merge" in m and "gradient" in w


def test_algorithmic_bytes():
    alg, nodes = bench.algorithmic_bytes()
    assert nodes == 38_707_200                         # 1280x720, D=128, 3 scales, one view
    px = sum(w * h for (w, h, _, _) in bench.level_geometry())
    assert alg["aggregate"] == 2 * (3 * nodes + 2 * px)
    lay, _ = bench.algorithmic_bytes(variant="paper")
    # 8 paths = 4 layers: 6 B/node for the first, 12 B/node for each later one
    assert lay["aggregate"] == 2 * 42 * nodes
    assert lay["wta"] - alg["wta"] == 2 * 2 * nodes   # the last pair is read, not one S


def test_counters_are_reported_only_for_the_captured_code(tmp_path, monkeypatch):
    src = tmp_path / "k.cu"
    src.write_text("// what it does\nint k() { return 1; }  // one\n")
    h = bench.code_hash(str(src))
    (tmp_path / "profiles").mkdir()
    (tmp_path / "profiles" / "k_counters.txt").write_text(
        f"# comment\nsource=k.cu code_sha256_16={h}\n"
        "level=0 us=10 dram_bytes=100 alu_pct=40 issue_pct=50\n"
        "level=1 us=30 dram_bytes=300 alu_pct=80 issue_pct=70\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    c = bench.measured_counters("k")
    # device-time weighted: (10*40 + 30*80) / 40 = 70 %, (10*50 + 30*70) / 40 = 65 %
    assert c["alu_pipe_active"] == 0.7 and c["issue_active"] == 0.65
    assert c["dram_bytes_per_step"] == 400 and c["launches"] == 2
    # comments and blank lines edited: the same code, the same counters
    src.write_text("/* what\n   it does */\n\nint k() { return 1; }\n// the end\n")
    assert bench.measured_counters("k")["dram_bytes_per_step"] == 400
    src.write_text("int k() { return 2; }\n")         # the code changed: nothing reported
    assert bench.measured_counters("k") is None
    assert bench.measured_counters("absent") is None


def test_survey_bytes_add_one_byte_per_node_read_and_written():
    a1, nodes = bench.algorithmic_bytes()
    a2, _ = bench.algorithmic_bytes(cost_bytes=2)
    assert a2["aggregate"] - a1["aggregate"] == 2 * nodes      # the cost read, both views
    assert a2["cost"] - a1["cost"] == 2 * nodes                # the cost write
