"""Host logic of bench.py on CPU: the per-draw operation counts and the
min-over-pipes bound, the traffic record and the clock summary."""
import hashlib

import pytest

import bench


def test_class_counts_d3():
    f = bench.class_counts(3, False)
    # Philox: 3/4 call per draw, 19 wide multiplies and 20 ALU ops per call;
    # Box-Muller: 3/2 pairs, 4 ALU + 6 FP32 + 4 MUFU each; L z: 6 FP32;
    # indicator: 3 compares + 1 count add
    assert f["mul_wide"] == pytest.approx(14.25)
    assert f["alu"] == pytest.approx(15 + 6 + 4)
    assert f["ffma"] == pytest.approx(9 + 6)
    for k in ("lg2", "sqrt", "sin", "cos"):
        assert f[k] == pytest.approx(1.5)
    assert f["ex2"] == f["rcp"] == f["lds128"] == 0
    g = bench.class_counts(3, True)
    # adjoint FP32 (packed form, d odd): A and B packed on half the draws
    # (1 packed + 1 scalar) and scalar on the other half (3 each); the four
    # sigmoid terms 1 packed + 1 scalar each; the running product 3
    assert g["ffma"] == pytest.approx(15 + 2 * (0.5 + 1.5) + 4 + 3)
    assert g["ffma2"] == pytest.approx(2 * 0.5 + 4)
    assert g["ex2"] == g["rcp"] == 3
    assert g["alu"] == pytest.approx(26)
    assert sum(g.values()) == pytest.approx(83.25)
    assert bench.ops_per_draw(3, True) == pytest.approx(81)


@pytest.mark.parametrize("d,scalar,packed", [
    (3, 11, 5),
    (4, 4, 2 * 2 + 4 * 2),       # even d: A and B packed on every draw
    (10, 10, 2 * 5 + 4 * 5),
    (16, 7 * 16, 0),             # the scalar form at d = 16, 18, 20
    (20, 7 * 20, 0),
])
def test_adjoint_fp32_ops(d, scalar, packed):
    sc, pk = bench.adjoint_fp32_ops(d)
    assert sc == pytest.approx(scalar) and pk == pytest.approx(packed)
    assert sc + 2 * pk == pytest.approx(7 * d)   # a packed instruction does two coordinates' work


@pytest.mark.parametrize("d,grad,lds", [
    (10, False, 18 / 2),        # factor chunks shared by the 2 draws of a group
    (10, True, 18 + 2 * 10),    # volatile reloads: every chunk and both thresholds
    (13, True, 28 / 4 + 13),    # plain loads, groups of 4 draws, scaled thresholds
    (20, False, 60),
    (20, True, 60 + 20),
    (6, True, 0),               # factor in registers
])
def test_class_counts_shared_loads(d, grad, lds):
    assert bench.class_counts(d, grad)["lds128"] == pytest.approx(lds)


def test_pipe_bound_picks_the_busiest_pipe():
    rates = {"mul_wide": 25.0, "philox": 30.0, "mad_lo": 64.0, "lop3": 64.0, "ffma": 128.0,
             "lg2": 16.0, "sqrt": 16.0, "sin": 16.0, "cos": 16.0, "ex2": 32.0, "rcp": 16.0,
             "mixed": 124.0, "lds128": 16.0}
    b = bench.pipe_bound(rates, 3, True, 152, mhz=2000.0)
    n = bench.class_counts(3, True)
    issue = sum(n.values()) / 128.0
    mufu = sum(n[k] / rates[k] for k in bench.MUFU)
    assert b["sm_clk_per_draw"]["issue"] == pytest.approx(issue)
    assert b["sm_clk_per_draw"]["mufu"] == pytest.approx(mufu)
    # the wide multiplies take the faster of the two measured rates
    assert b["sm_clk_per_draw"]["int_multiply"] == pytest.approx(n["mul_wide"] / 30.0)
    # the busiest pipe binds; with the adjoint's packed FP32 work, MUFU (9
    # ops at 16 per clock, 3 at 32) is within 1 % of issue at d=3
    clk = b["sm_clk_per_draw"]
    assert b["binding"] == max(clk, key=clk.get) == "mufu"
    assert b["bound_draw_evals_per_s"] == pytest.approx(152 * 2000e6 / mufu)
    fast = dict(rates, lg2=64.0, sqrt=64.0, sin=64.0, cos=64.0, rcp=64.0, ex2=64.0)
    bf = bench.pipe_bound(fast, 3, True, 152, mhz=2000.0)
    assert bf["binding"] == "issue"
    assert bf["bound_draw_evals_per_s"] == pytest.approx(152 * 2000e6 / issue)
    slow = dict(rates, sin=2.0)
    b2 = bench.pipe_bound(slow, 3, True, 152, mhz=2000.0)
    assert b2["binding"] == "mufu"
    assert b2["bound_draw_evals_per_s"] < b["bound_draw_evals_per_s"]


def test_traffic_record_scales_per_tile_and_checks_the_sources(tmp_path, monkeypatch):
    h = hashlib.sha256()
    for p in bench.KERNEL_SOURCES:
        with open(p, "rb") as f:
            h.update(f.read())
    rec = tmp_path / "traffic.txt"
    rec.write_text("# comment: with a colon\nsrc_sha256: %s\ndram_bytes_read_small: 1500\n"
                   "dram_bytes_write_small: 500\ntiles_small: 100\n" % h.hexdigest())
    monkeypatch.setattr(bench, "TRAFFIC_FILE", str(rec))
    assert bench.traffic_record(1000) == pytest.approx(20000.0)
    rec.write_text("src_sha256: %s\ndram_bytes_read_small: 1500\ndram_bytes_write_small: 500\n"
                   "tiles_small: 100\n" % ("0" * 64))
    assert bench.traffic_record(1000) is None
    monkeypatch.setattr(bench, "TRAFFIC_FILE", str(tmp_path / "missing.txt"))
    assert bench.traffic_record(1000) is None


def test_committed_traffic_record_matches_the_sources():
    assert bench.traffic_record(1024) is not None


def test_clock_summary():
    lines = ["0, 2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active",
             "0, 2040, 2070, 1100.0, 0x4, Not Active, Not Active, Not Active, Active",
             "0, 2070, 2070, 1000.0, 0x0, Not Active, Not Active, Not Active, Not Active",
             "garbage",
             "0, [N/A], 2070, 1.0, 0x0, Not Active, Not Active, Not Active, Not Active"]
    c = bench.ClockSampler.summarise(lines)
    assert c["sm_mhz"] == 2070.0
    assert c["sm_max_mhz"] == 2070.0
    assert c["reasons"] == ["sw_power_cap"]
    assert c["samples"] == 3
    assert bench.ClockSampler.summarise([])["sm_mhz"] is None


def test_hbm_peak_reads_the_measured_figure_or_falls_back(tmp_path):
    f = tmp_path / "peaks.json"
    f.write_text('{"hbm_gbs": 6790.0, "bf16_tflops": 1979.2}')
    assert bench.hbm_peak(str(f)) == (6790.0, "measured (MEASURED_PEAKS.json hbm_gbs)")
    f.write_text("not json")
    assert bench.hbm_peak(str(f))[0] == 6800.0
    f.write_text('{"bf16_tflops": 1979.2}')
    assert bench.hbm_peak(str(f))[0] == 6800.0
    assert bench.hbm_peak(str(tmp_path / "missing.json"))[0] == 6800.0


def test_shared_class_counts_and_bound():
    """The shared-draw kernel's per-draw-evaluation counts: forward, packed
    differences and their sign; adjoint, packed differences and sums, the
    minimum and the skip test, and the sigmoid's work in the active
    fraction of warp-draws only."""
    f = bench.shared_class_counts(3, False, 4)
    assert f["ffma2"] == 1 and f["ffma"] == 1 and f["alu"] == 2 and f["lds128"] == pytest.approx(0.25)
    assert f["ex2"] == f["rcp"] == f["mul_wide"] == 0
    g = bench.shared_class_counts(3, True, 4, active=0.5)
    # packed: 1 difference pair + 2 sum pairs, and 4 pairs of sigmoid work
    # in half the warp-draws; scalar: the odd difference, and the odd
    # coordinate's 4 plus the 3 products of the running product
    assert g["ffma2"] == pytest.approx(3 + 0.5 * 4) and g["alu"] == 4
    assert g["ex2"] == g["rcp"] == pytest.approx(1.5)
    assert g["ffma"] == pytest.approx(1 + 0.5 * 7)
    assert g["lds128"] == pytest.approx(0.5)
    e = bench.shared_class_counts(10, True, 1, active=0.0)
    assert e["ffma2"] == 10 and e["ffma"] == 0 and e["alu"] == 5 + 5
    o = bench.shared_class_counts(5, True, 2, active=0.0)
    assert o["ffma2"] == 2 + 3 and o["ffma"] == 1 and o["alu"] == 2 + 3
    rates = {"lop3": 64.0, "ffma": 128.0, "ffma2": 64.0, "lg2": 16.0, "sqrt": 16.0, "sin": 16.0, "cos": 16.0,
             "ex2": 32.0, "rcp": 16.0, "lds128": 16.0}
    b = bench.shared_pipe_bound(rates, 3, True, 4, 1.0, 152, mhz=2000.0)
    assert b["sm_clk_per_draw"]["mufu"] == pytest.approx(3 / 32 + 3 / 16)
    assert b["sm_clk_per_draw"]["fp32"] == pytest.approx((1 + 7) / 128 + (3 + 4) / 64)
    full = bench.shared_class_counts(3, True, 4, active=1.0)
    assert b["sm_clk_per_draw"]["issue"] == pytest.approx(sum(full.values()) / 128)
    slow = dict(rates, ex2=4.0, rcp=4.0)
    assert bench.shared_pipe_bound(slow, 3, True, 4, 1.0, 152, mhz=2000.0)["binding"] == "mufu"
    b0 = bench.shared_pipe_bound(rates, 3, True, 4, 0.0, 152, mhz=2000.0)
    assert b0["sm_clk_per_draw"]["mufu"] == 0.0
    assert b0["sm_clk_per_draw"]["alu"] == pytest.approx(4 / 64.0)
    assert b0["bound_draw_evals_per_s"] > b["bound_draw_evals_per_s"]
    assert bench.shared_fp32_flops(3, False) == 3
    assert bench.shared_fp32_flops(3, True, 0.5) == pytest.approx(3 + 3 + 9)


def test_shared_active_fraction_limits():
    import numpy as np

    import workloads
    S = workloads.equicorrelated(3, 0.5)
    J = 64
    far = workloads.Problem("far", [S], [0] * J, [np.zeros(3)] * J, [np.full(3, 50.0)] * J, [100] * J, [0] * J)
    assert bench.shared_active_fraction(far, 0.01, draws=64) == 0.0
    wide = workloads.Problem("wide", [S], [0] * J, [np.zeros(3)] * J, [np.full(3, 1.0)] * J, [100] * J, [0] * J)
    assert bench.shared_active_fraction(wide, 100.0, draws=64) == 1.0
    mid = bench.shared_active_fraction(workloads.c2(n_scen=1, g1=8, g2=8, n_draws=10), 0.01, draws=256)
    assert 0.0 < mid < 1.0


def test_committed_shared_traffic_record_matches_the_sources():
    assert bench.shared_traffic_record() is not None
