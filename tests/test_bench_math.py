"""bench.py's roofline arithmetic and the oracle sample's multipliers, on the CPU."""
import os
import sys

import numpy as np
import pytest

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402


def test_pcg_roofline_is_algorithmic_bytes_over_launch_time():
    # the float32 PCG apply on the 80 x 44 x 43 chain: n = 1,175,805, 32,817,315 stored entries,
    # block width 24, 80 launches in 42.788 ms
    n, nnz, w = 1175805, 32817315, 24.0
    prof = {"pcg_spmm": {"ms": 42.788, "launches": 80}, "poisson": {"ms": 99.0, "launches": 1}}
    r = bench.roofline(prof, n, 41, nnz, 908160, 6756.8, "measured", elem=4, pcg_w=w)
    per = 42.788e-3 / 80
    alg = 12 * nnz + 20 * n * w                       # (4 + 2 s) nnz + 5 s n w at s = 4
    assert r["kernel"] == "pcg_spmm" and r["bound"] == "hbm"   # the Hartree total is not a candidate
    assert r["achieved"] == pytest.approx(alg / per / 1e9, abs=0.05)
    assert r["frac"] == pytest.approx(r["achieved"] / 6756.8, abs=1e-4)
    assert r["traffic"] == int(alg * bench.PCG_F32_DRAM_PER_ALG)
    assert 0.9 < bench.PCG_F32_DRAM_PER_ALG < 1.1    # the mid-size capture moved 0.96x its algorithmic bytes


def test_float64_pcg_roofline_is_against_the_fp64_rate():
    bench.ALU_PEAKS.update({"fp64": 1.25, "fp32": 78.0, "kind": "test"})
    prof = {"pcg_spmm": {"ms": 243.0, "launches": 80}}
    r = bench.roofline(prof, 1175805, 41, 32817315, 908160, 6756.8, "measured", elem=8, pcg_w=24.0)
    flops = 4 * 32817315 * 24.0 + 6 * 1175805 * 24.0
    assert r["bound"] == "alu" and r["unit"] == "TFLOP/s (fp64)" and r["traffic"] is None
    assert r["achieved"] == pytest.approx(flops / (243e-3 / 80) / 1e12, abs=1e-4)
    assert r["frac"] == pytest.approx(r["achieved"] / 1.25, abs=1e-4)


@pytest.mark.parametrize("p,active", [(41, 23), (41, 41), (41, 1), (2, 1)])
def test_oracle_sample_has_the_requested_active_columns(p, active):
    sh = bench.shifts_with_active(p, active)
    assert sh.shape == (p,) and int(np.sum(sh < 0)) == active and np.all(sh != 0)


def test_multi_kernel_families_are_not_the_dominant_kernel():
    # the Hartree preconditioner's scope (gather, six contractions, scatter) outweighs every
    # single kernel here, but the roofline names the largest one-launch family, the SpMM of B
    prof = {"poisson_pc": {"ms": 9.0, "launches": 76}, "spmm_b": {"ms": 8.6, "launches": 10},
            "spmm_h": {"ms": 7.3, "launches": 10}, "pcg_sep": {"ms": 5.7, "launches": 10},
            "gcn": {"ms": 35.0, "launches": 2}, "judge": {"ms": 9.9, "launches": 2},
            "poisson": {"ms": 20.0, "launches": 10}}
    r = bench.roofline(prof, 1175805, 41, 32817315, 908160, 6756.8, "measured", elem=4)
    assert r["kernel"] == "spmm_b"
    alg = (4 + 4) * 32817315 + 3 * 4 * 1175805 * 41
    assert r["achieved"] == pytest.approx(alg / (8.6e-3 / 10) / 1e9, abs=0.05)


def test_float32_hartree_spmv_is_against_hbm():
    # in the float32 forms the Hartree CG's SpMV runs in float-float on the FP32 pipes: its
    # algorithmic flops are far below the FP32 rate, so its roofline is the HBM one
    bench.ALU_PEAKS.update({"fp64": 1.25, "fp32": 78.0, "kind": "test"})
    prof = {"poisson_spmv": {"ms": 6.3, "launches": 57}, "spmm_b": {"ms": 6.0, "launches": 10}}
    model = (8 * 18648214 + 24 * 1175805, 2 * 35120623)
    r = bench.roofline(prof, 1175805, 41, 32817315, 908160, 6756.8, "measured", model, elem=4)
    assert r["kernel"] == "poisson_spmv" and r["bound"] == "hbm"
    assert r["achieved"] == pytest.approx(model[0] / (6.3e-3 / 57) / 1e9, abs=0.05)
    r64 = bench.roofline(prof, 1175805, 41, 32817315, 908160, 6756.8, "measured", model, elem=8)
    assert r64["bound"] == "alu" and r64["unit"] == "TFLOP/s (fp64)"


def test_time_to_target_needs_both_energy_and_feasibility():
    # history rows (k, seconds, E, kkt, fea, eta): the target is the first row with |E - E*| <=
    # 1e-6 Ha AND fea <= 1e-7; an energy that passes through E* while still infeasible, or a
    # feasible row still 2e-6 Ha away, does not count
    E = -276.85
    hist = [(0, 0.0, E + 1.0, 1.0, 1e-2, 1.0),
            (1, 0.5, E + 5e-7, 1e-3, 1e-5, 1.0),      # close in energy, infeasible
            (2, 1.0, E - 2e-6, 1e-4, 1e-8, 1.0),      # feasible, 2e-6 Ha away
            (3, 1.25, E + 9e-7, 1e-5, 5e-8, 1.0),     # the first hit
            (4, 1.5, E, 1e-6, 1e-9, 1.0)]
    assert bench.first_hit(hist, E) == (1.25, 3)
    assert bench.first_hit(hist[:3], E) == (None, None)
    assert bench.first_hit(hist, E, target=1e-5, fea_max=1e-4) == (0.5, 1)
