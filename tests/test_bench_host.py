"""Host-side arithmetic of bench.py (no GPU): the roofline fractions, the
launch count claimed per timed step, the units of one step and the replica
helpers."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402

PEAKS = {"hbm_gbs": 6762.3, "sm_max_mhz": 2070.0}
CLK = {"sm_mhz": 2070.0}


def test_alu_roofline_uses_minimal_alu_instructions_and_measured_lanes():
    """Minimal ALU-pipe instructions: 11 per Hybrid Taus draw, 8 per Ran2 draw,
    four draws an oscillator-step; the regenerating adjoint draws twice."""
    assert bench.INT_OPS_PER_OSC_STEP == {"taus": 44, "ran2": 32}
    units = bench.N_OSC * bench.LD_STEPS
    r = bench.roofline("ld_taus", 61.7, units, PEAKS, "measured", CLK)
    assert r["bound"] == "alu" and r["unit"] == "Tops/s"
    assert r["achieved"] == pytest.approx(44 * units / 0.0617 / 1e12)
    assert r["peak"] == pytest.approx(152 * 64 * 2070e6 / 1e12)
    assert r["frac"] == pytest.approx(r["achieved"] / r["peak"])
    assert r["ncu_alu_pipe_pct"] == bench.NCU_ALU_PIPE_PCT["ld_taus"]
    big = bench.roofline("ld_ran2_1e8", 700.0, 10**11, PEAKS, "measured", CLK)
    assert big["achieved"] == pytest.approx(32 * 10**11 / 0.7 / 1e12)
    adj = bench.roofline("adjoint_ran2", 20.0, 10**9, PEAKS, "measured", CLK)
    assert adj["achieved"] == pytest.approx(2 * 32 * 10**9 / 0.02 / 1e12)
    # the Taus uniform fill as fast as measured (2^30 numbers in 0.908 ms) stays below 1
    f = bench.roofline("fill_uniform_taus", 0.908, 0, PEAKS, "measured", CLK)
    assert f["alt"]["bound"] == "alu" and f["alt"]["frac"] < 1.0


def test_fill_and_lagfib_rooflines():
    f = bench.roofline("fill_uniform_taus", 0.9, 0, PEAKS, "measured", CLK)
    assert f["bound"] == "hbm" and f["achieved"] == pytest.approx(4 * 2**30 / 0.0009 / 1e9)
    assert f["frac"] == pytest.approx(f["achieved"] / 6762.3)
    assert f["alt"]["achieved"] == pytest.approx(11 * 2**30 / 0.0009 / 1e12)
    lf = bench.roofline("fill_uniform_lagfib", 2.4, 0, PEAKS, "measured", CLK, l2_gbs=7900.0)
    assert lf["bound"] == "l2" and lf["achieved"] == pytest.approx(16 * 2**30 / 0.0024 / 1e9)
    assert lf["frac"] == pytest.approx(lf["achieved"] / 7900.0)
    assert lf["alt"]["bound"] == "hbm"
    assert lf["alt"]["achieved"] == pytest.approx(4 * 2**30 / 0.0024 / 1e9)
    l2 = bench.roofline("ld_lagfib", 117.0, 10**10, PEAKS, "measured", CLK, l2_gbs=7900.0)
    assert l2["bound"] == "l2" and l2["achieved"] == pytest.approx(48 * 1e10 / 0.117 / 1e9)
    assert bench.roofline("ld_lagfib", 117.0, 10**10, PEAKS, "m", CLK)["frac"] is None
    big = bench.roofline("ld_lagfib_1e8", 2000.0, 10**11, PEAKS, "measured", CLK, l2_gbs=7900.0)
    assert big["bound"] == "hbm" and big["achieved"] == pytest.approx(48 * 1e11 / 2.0 / 1e9)
    assert big["frac"] == pytest.approx(big["achieved"] / 6762.3)
    assert big["alt"]["bound"] == "l2"


def test_launch_count_per_step():
    parts = [(n, 0, None) for n in ("ld_taus", "ld_ran2", "ld_lagfib", "fill_uniform_taus",
                                    "fill_normal_taus", "batched_taus", "adjoint_taus")]
    # 3 fused x 2 + 2 fills + batched (1 launch + reduce) + adjoint x 2
    assert bench.gpu_launches(parts, 1, (256, 1, 0)) == 6 + 2 + 2 + 2
    # steps per launch L = 715 -> ceil(5000 / 715) = 7 launches + reduce
    assert bench.gpu_launches(parts, 3, (128, 1, 715)) == 3 * (6 + 2 + 8 + 2)


def test_step_units_and_replica_helpers():
    u = bench._step_units()
    assert u["ld_taus"] == 10**10 and u["fill_normal_lagfib"] == 2**30
    assert u["adjoint_taus"] == u["adjoint_ran2"] == 10**9
    assert bench._step_osc_steps(u) == 3 * 10**10 + u["batched_taus"] + 2 * 10**9
    assert bench.rank_seed(0) != bench.rank_seed(1)
    assert bench.max_over_ranks(3.5, None, "cpu") == 3.5
    assert bench.whole_job_rate(4, 1e9, 500.0) == pytest.approx(8e9)


def test_headline_keys_per_generator():
    pp = {"ld_taus": {"osc_steps_per_s": 1.0, "roofline": {"frac": 0.5, "bound": "alu",
                                                            "ncu_alu_pipe_pct": 70.0}},
          "ld_lagfib_1e8": {"osc_steps_per_s": 2.0, "roofline": {"frac": 0.4, "bound": "hbm"}},
          "fill_normal_taus": {"numbers_per_s": 3.0, "roofline": {"frac": 0.3}}}
    h = bench.headline(pp)
    assert h["ld_taus.osc_steps_per_s"] == 1.0 and h["ld_taus.ncu_alu_pipe_pct"] == 70.0
    assert h["ld_lagfib_1e8.bound"] == "hbm" and not any(k.startswith("fill") for k in h)
    assert bench.part_kind("ld_lagfib_1e8") == "lagfib"
    assert bench.part_kind("adjoint_ran2") == "ran2"


def test_host_cpu_names_the_architecture():
    import platform
    assert bench.host_cpu().startswith(platform.machine())
