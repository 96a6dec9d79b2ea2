"""bench.py's roofline accounting on the CPU: the algorithmic FP64 flops per particle-turn that
the roofline's `achieved` divides by the kernel's duration, spelled out term by term, and the
executed-flop figure taken from the ncu capture of the Ruth4 kernel."""
import bench


def test_algorithmic_flops_of_the_paper_scale_workload():
    # drift = 1 FMA (2 flops); kick = phase FMA (2) + sine (20) + subtract (1) + FMA (2) = 25;
    # transverse = 2 planes x (2 MUL + 2 FMA) = 12
    assert bench.KICK_FLOPS == 25
    assert bench.alg_flops("euler_cromer", True, True) == 2 + 25 + 12
    assert bench.alg_flops("leapfrog", True, True) == 2 * 2 + 25 + 12
    assert bench.alg_flops("ruth4", True, True) == 4 * 2 + 3 * 25 + 12
    assert bench.alg_flops("ruth4", False, False) == 4 * 2 + 3 * 25


def test_algorithmic_flops_of_the_extensions():
    ring = {"eta1": 0.05, "eta2": 2.0, "xi_x": 5.0, "xi_y": -3.0}
    # widened drift 3 FMA (6 flops) per drift; a chromatic plane 41 flops
    assert bench.alg_flops("ruth4", True, True, ring) == 4 * 6 + 3 * 25 + 2 * 41
    dual = {"voltage2_V": 1.35e6}
    # the second RF system adds a phase FMA, sine, subtract and FMA per kick; with eta1 =
    # eta2 = 0 the drifts stay linear in the count (the kernel's expansion FMAs on zeros are
    # not the method's work)
    assert bench.alg_flops("ruth4", True, True, dual) == 4 * 2 + 3 * 25 + 3 * 25 + 12
    # classic RK4: four right-hand sides of slippage (1 MUL, or 2 FMA + 1 MUL with the
    # expansion), phase FMA, sine, subtract and multiply; stage arguments 10; weighted sums 12
    assert bench.alg_flops("rk4", True, True) == 4 * (1 + 2 + 20 + 1 + 1) + 10 + 12 + 12
    assert bench.alg_flops("rk4", True, True, dual) == 4 * (1 + 2 + 20 + 1 + 1) + 10 + 12 + 4 * 25 + 12
    assert bench.alg_flops("rk4", False, False, {"eta1": 0.1}) == 4 * (5 + 2 + 20 + 1 + 1) + 10 + 12
    # collective step: the slice index (subtract, multiply) and the kick's add
    assert bench.COLLECTIVE_FLOPS == 3
    assert bench.alg_flops("leapfrog", True, True) + bench.COLLECTIVE_FLOPS == 44


def test_executed_flops_only_where_the_capture_applies():
    wl = {"transverse": True, "stride": 1}
    e = bench.executed_flops("f64", "ruth4", wl, 1e10)
    assert abs(e["executed_flops_per_particle_turn_ncu"] - 86.09) < 0.02
    assert abs(e["executed_tflops"] - 0.8608) < 1e-3
    assert bench.executed_flops("f64", "leapfrog", wl, 1e10) == {}
    assert bench.executed_flops("f64", "ruth4", dict(wl, wake={"nslices": 512}), 1e10) == {}
    assert bench.executed_flops("f64", "ruth4", dict(wl, perturn=True), 1e10) == {}
    assert bench.executed_flops("f32cd", "ruth4", wl, 1e10) == {}
    # each map variant takes its own capture: the widened map's per-plane phase sine and
    # cosine, the double-RF kick's second sine
    for name, scheme, lo, hi in (("widened_map_1e6x1e4_f64", "ruth4", 150, 200),
                                 ("double_rf_1e6x1e4_ec_lf_ruth4_f64", "ruth4", 150, 200),
                                 ("rk4_double_rf_1e6x1e4_f64", "rk4", 200, 260),
                                 ("ramp_1e6x1e4_ec_lf_ruth4_f64", "ruth4", 90, 110)):
        w = bench.WORKLOADS[name]
        f = bench.executed_flops("f64", scheme, w, 1e10)["executed_flops_per_particle_turn_ncu"]
        assert lo < f < hi, (name, f)
        assert f > bench.NCU_EXEC_FLOPS_PER_PARTICLE_TURN[("f64", "ruth4", True, True, "plain")]
    assert bench.executed_flops("f64", "leapfrog", bench.WORKLOADS["ramp_1e6x1e4_ec_lf_ruth4_f64"],
                                1e10) == {}
    assert bench.map_variant(bench.WORKLOADS["ramp_1e6x1e4_ec_lf_ruth4_f64"]) == "ramp"
    assert bench.map_variant(bench.WORKLOADS[bench.DEFAULT_WORKLOAD]) == "plain"


def test_fp64_roofline_leads_with_the_executed_count():
    wl = dict(bench.WORKLOADS[bench.DEFAULT_WORKLOAD])
    n, tpl, dur = 1_000_000, 264, 0.023
    alg = bench.alg_flops("ruth4", True, True) * n * tpl / dur / 1e12
    r = bench.fp64_roofline("k", "f64", "ruth4", wl, n, tpl, dur, bench.alg_flops("ruth4", True, True), alg)
    assert r["frac"] == r["executed_frac"] and r["achieved"] == r["executed_tflops"]
    assert abs(r["executed_tflops"] - 86.09 * n * tpl / dur / 1e12) < 2e-3
    assert r["alg_frac"] == alg / bench.FP64_PEAK_TFLOPS
    # the sine-free count: 4 drifts (2 each), 3 kicks (phase FMA, subtract, FMA), transverse 12
    assert r["alg_flops_per_particle_turn_without_sines"] == 4 * 2 + 3 * 5 + 12
    # a variant without a stored ncu count falls back to the algorithmic count
    w2 = dict(bench.WORKLOADS["widened_map_1e6x1e4_f64"])
    f2 = bench.alg_flops("leapfrog", True, True, w2["ring"])
    r2 = bench.fp64_roofline("k", "f64", "leapfrog", w2, n, tpl, dur, f2, 0.9)
    assert r2["frac"] == r2["alg_frac"] == 0.9 / bench.FP64_PEAK_TFLOPS
    assert "executed_frac" not in r2


def test_issue_roofline_uses_the_stored_instruction_count():
    key = ("f32cd", "leapfrog", True, True, False)
    saved = dict(bench.NCU_WARP_INST_PER_PARTICLE_TURN)
    try:
        bench.NCU_WARP_INST_PER_PARTICLE_TURN[key] = 10.0
        r = bench.issue_roofline("k", key, 5e10, 2000.0)
        assert abs(r["achieved"] - 500.0) < 1e-9
        assert abs(r["peak"] - 152 * 4 * 2.0) < 1e-9
        assert abs(r["frac"] - 500.0 / (152 * 4 * 2.0)) < 1e-12
        r = bench.issue_roofline("k", ("f32cd", "euler_cromer", False, False, False), 5e10, 2000.0)
        assert r["frac"] is None
    finally:
        bench.NCU_WARP_INST_PER_PARTICLE_TURN.clear()
        bench.NCU_WARP_INST_PER_PARTICLE_TURN.update(saved)


def test_batched_lines_have_a_roofline():
    # FP64 batch: the FP64-pipe roofline from the batched kernel's own ncu count
    wl = dict(bench.WORKLOADS["batched_64_bunches_f64_lf"], transverse=False)
    fpt = bench.alg_flops("leapfrog", False, True)
    pts, t = 2.6e10, 0.7  # particle-turns per run, seconds
    r = bench.fp64_roofline("k", "f64", "leapfrog", wl, pts, 1, t, fpt, fpt * pts / t / 1e12)
    assert abs(r["executed_flops_per_particle_turn_ncu"] - 26.10) < 0.01
    assert r["frac"] == r["executed_frac"]
    assert abs(r["achieved"] - 26.10 * pts / t / 1e12) < 1e-3
    # FP32CD batch: an issue roofline
    r2 = bench.issue_roofline("k", ("f32cd", "leapfrog", False, True, True), 1.4e11, 2070.0)
    assert abs(r2["warp_inst_per_particle_turn_ncu"] - 6.826) < 1e-3
    assert 0.7 < r2["frac"] < 0.9


def test_collective_and_variant_keys():
    wl = dict(bench.WORKLOADS["collective_wake_1e6x1e4_lf_f64"])
    assert bench.map_variant(wl) == "collective"
    e = bench.executed_flops("f64", "leapfrog", wl, 1.7e10)
    # 18 DFMA, 3 DMUL, 2.06 DADD per particle-turn: the leap-frog map, the three-shear planes,
    # the slice index and the kick's add
    assert abs(e["executed_flops_per_particle_turn_ncu"] - 41.06) < 0.01
    assert bench.map_variant(dict(wl, perturn=True)) is None


def test_general_fp32_kernels_have_issue_counts():
    for dt in ("f32c", "f32cd", "f32cs"):
        for scheme, variant in (("leapfrog", "widened"), ("ruth4", "widened"), ("rk4", "double_rf")):
            per = bench.NCU_WARP_INST_PER_PARTICLE_TURN[(dt, scheme, True, True, variant)]
            plain = bench.NCU_WARP_INST_PER_PARTICLE_TURN.get((dt, "leapfrog", True, True, False))
            assert per > plain  # the general map does more than the linear one
    r = bench.issue_roofline("k", ("f32cd", "rk4", True, True, "double_rf"), 1.2e10, 2070.0)
    assert abs(r["warp_inst_per_particle_turn_ncu"] - 56.75) < 0.01 and 0.4 < r["frac"] < 0.7
