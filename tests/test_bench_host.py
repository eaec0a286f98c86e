"""Host-side logic of bench.py (no GPU): the quartet sampler used by the oracle
legs returns only significant canonical quartets, and the sampled class mix
follows the list."""
import numpy as np

import bench
import oracle
import workloads as W


def test_sampled_quartets_are_significant_and_canonical():
    basis, _ = W.workload(0)
    lists = bench._lists_without_gpu(basis)
    Q = lists["Q"]
    q = bench.sample_quartets(lists, basis, 500, seed=3)
    pidx = lambda a, b: a * (a + 1) // 2 + b
    for a, b, c, d in q:
        assert a >= b and c >= d
        assert float(Q[pidx(a, b)]) * float(Q[pidx(c, d)]) >= bench.THRESH
    o = oracle.Oracle(basis)
    assert o.quartet_batch(q[:20]) > 0.0


def test_class_rows_rates_and_fractions():
    """Per-class rows: FLOPs per step over ms per step, against the tier's peak."""
    prof = [{"bra_class": 7, "ket_class": 1, "tier": 1, "ms": 500.0, "flops": 1e12, "launches": 5},
            {"bra_class": 2, "ket_class": 2, "tier": 0, "ms": 2000.0, "flops": 2.5e11, "launches": 5}]
    rows = bench.class_rows(prof, steps=5)
    assert rows[0][:2] == ["(pp|pp)", "fp64"] and rows[1][:2] == ["(fp|ps)", "fp32"]
    # (pp|pp): 2.5e11 FLOP per step in 400 ms -> 0.625 TFLOP/s = half of 1.25
    assert abs(rows[0][3] - 0.625) < 1e-9 and abs(rows[0][4] - 0.5) < 1e-9
    # (fp|ps): 1e12 FLOP in 100 ms -> 10 TFLOP/s of 80.5
    assert abs(rows[1][3] - 10.0) < 1e-9 and abs(rows[1][4] - round(10.0 / 80.5, 5)) < 1e-12


def test_class_rows_gradient_and_jengine_tiers_use_fp64_peak():
    """Profile tiers 2 (gradient) and 3 (J-engine) run in FP64: their fraction is
    taken against the FP64 peak, nominal or the measured one when given."""
    prof = [{"bra_class": 9, "ket_class": 9, "tier": 2, "ms": 100.0, "flops": 5e10, "launches": 1},
            {"bra_class": 0, "ket_class": 0, "tier": 3, "ms": 50.0, "flops": 1e10, "launches": 1}]
    rows = bench.class_rows(prof, steps=1)
    assert rows[0][:2] == ["(ff|ff)", "grad-fp64"] and rows[1][:2] == ["(ss|ss)", "jengine-fp64"]
    assert abs(rows[0][3] - 0.5) < 1e-9 and abs(rows[0][4] - 0.4) < 1e-9
    rows_m = bench.class_rows(prof, steps=1, peaks={0: 1.0, 1: 80.0})
    assert abs(rows_m[1][4] - 0.2) < 1e-9


def test_traffic_reader(tmp_path):
    """roofline.traffic comes from the committed ncu summary only while the J/K
    kernel sources hash to the value recorded in it."""
    import bench
    h = bench.source_hash()
    p = tmp_path / "t.md"
    p.write_text(f"source_hash: {h}\n\n| kernel | tier | dram bytes per launch |\n|---|---|---:|\n"
                 "| (fp\\|dp) | fp32 | 2500000.0 |\n| (ss\\|ss) | fp64 | 10 |\n")
    assert bench.traffic_for(7, 4, 1, path=str(p)) == 2500000.0
    assert bench.traffic_for(0, 0, 0, path=str(p)) == 10.0
    assert bench.traffic_for(7, 4, 0, path=str(p)) is None
    p.write_text("source_hash: 0000000000000000\n| (fp\\|dp) | fp32 | 2500000.0 |\n")
    assert bench.traffic_for(7, 4, 1, path=str(p)) is None


def test_tier_peaks_and_names():
    """FP32 tiers (J/K FP32, gradient FP32, J-engine FP32) take the FP32 ALU
    peak, the others the FP64 one; every profile tier has a name."""
    import bench
    peaks = {0: 1.0, 1: 64.0}
    assert [bench.tier_peak(t, peaks) for t in range(6)] == [1.0, 64.0, 1.0, 1.0, 64.0, 64.0]
    assert set(bench.TIER_NAMES) == set(range(6))
