"""Host logic of bench.py (no GPU): the spectral grid sizes, the traffic entries' source check, and the
per-stage roofline figures."""
import json

import bench


def _smooth(m):
    for p in (2, 3, 5, 7):
        while m % p == 0:
            m //= p
    return m == 1


def test_fft_size_is_the_smallest_smooth_size():
    for n in list(range(1, 300)) + [1000, 4099]:
        m = bench.fft_size(n)
        assert m >= n and _smooth(m)
        assert not any(_smooth(k) for k in range(n, m))


def test_traffic_entries_follow_their_sources(tmp_path, monkeypatch):
    # an entry recorded for the sources as they are is returned; one recorded for other sources, or a
    # workload without an entry, gives None (the bench then reports no traffic)
    t = {"shell": {"channel512": {"fp32": {"bytes_per_launch": 123.0,
                                           "source_hash": bench.source_hash(bench.KERNEL_SOURCES["shell"])}}},
         "collide": {"channel512": {"fp32": {"bytes_per_launch": 456.0, "source_hash": "0" * 16}}}}
    p = tmp_path / "traffic.txt"
    p.write_text(json.dumps(t))
    monkeypatch.setattr(bench, "TRAFFIC_FILE", str(p))
    assert bench.traffic_for("shell", "channel512", "fp32") == 123.0
    assert bench.traffic_for("collide", "channel512", "fp32") is None
    assert bench.traffic_for("shell", "well256", "fp32") is None
    assert bench.traffic_for("density", "channel512", "fp32") is None


def test_kernel_rooflines_use_the_algorithmic_bytes():
    N, M = 1000, 2
    stages = {"density": (2.0, 4), "collide": (8.0, 4), "contact": (1.0, 4)}
    w = {"sigma": [4.0, 6.0], "shape": (10, 10, 10), "periodic": (1, 0, 0)}
    out = bench.kernel_rooflines(stages, w, "fp32", N, M, 4, 1000.0, None, 152, 2070.0, "direct")
    assert out["collide"]["algorithmic_bytes_per_launch"] == N * M * 4 * 19 * 4
    assert out["collide"]["bound"] == "hbm"
    assert out["density"]["algorithmic_bytes_per_launch"] == N * M * (19 * 4 + 4)
    # 2 ms over 4 launches: 0.5 ms per launch
    assert abs(out["density"]["avg_launch_ms"] - 0.5) < 1e-12
    assert abs(out["collide"]["achieved_gbs"] - N * M * 304 / 2e-3 / 1e9) < 1e-9
    assert "shell" not in out
    # the stencil contact kernel: one shared load per ball point (33 for sigma 4, 123 for sigma 6) against
    # the shared-memory bandwidth of the device's multiprocessors
    c = out["contact"]
    assert c["bound"] == "smem"
    assert c["algorithmic_smem_bytes_per_launch"] == N * (33 + 123) * 4
    assert abs(c["peak_gbs"] - 152 * 128 * 2070e6 / 1e9) < 1e-6
    assert abs(c["frac"] - c["achieved_gbs"] / c["peak_gbs"]) < 1e-12


def test_fp64_collide_is_reported_against_the_fp64_rate():
    N, M = 1000, 2
    stages = {"collide": (8.0, 4)}
    w = {"sigma": [4.0, 6.0], "shape": (10, 10, 10), "periodic": (1, 1, 1)}
    out = bench.kernel_rooflines(stages, w, "fp64", N, M, 8, 1000.0, None, 152, 2070.0, "spectral")
    c = out["collide"]
    assert c["bound"] == "alu"
    assert c["algorithmic_flops_per_launch"] == N * M * bench.K4_FLOPS_PER_NODE_SPECIES
    assert abs(c["frac"] - c["achieved_tflops"] / bench.FP64_NOMINAL_TFLOPS) < 1e-12
    assert c["algorithmic_bytes_per_launch"] == N * M * 4 * 19 * 8


def test_ball_counts_match_the_contact_balls():
    # the oracle's ball lists, counted independently
    assert [bench.ball_count(r) for r in (0.0, 1.5, 2.0, 2.5, 3.0)] == [1, 19, 33, 81, 123]


def test_step_roofline_totals_and_stage_sum():
    """The step's bytes and flops from their per-node counts, the max-roof against the two peaks, and
    the sum of the stages' own bounds (stage time x fraction)."""
    N, M = 1000, 2
    w = {"sigma": [4.0, 6.0], "shape": (10, 10, 10), "periodic": (1, 0, 0)}
    stage_ms = {"density": 0.2, "contact": 0.25, "shell": 1.5, "collide": 0.9, "flux": 0.02}
    kernels = {"density": {"frac": 0.8}, "contact": {"frac": 0.5}, "shell": {"frac": 0.6},
               "collide": {"frac": 0.85}}
    r = bench.step_roofline(w, "fp32", N, M, 4, 3.0, stage_ms, kernels, 1000.0, 80.0, "direct")
    assert r["population_bytes_per_step"] == N * M * 4 * 19 * 4
    assert r["full_bytes_per_step"] == N * M * (304 + 7 * 4) + N * 4
    S_list = [4, 5, 5, 6]
    flops = N * (sum(bench.shell_flops_per_node(S) for S in S_list) + M * bench.K4_FLOPS_PER_NODE_SPECIES
                 + 33 + 123)
    assert r["flops_per_step"] == flops
    t_b = r["full_bytes_per_step"] / 1000e9 * 1e3
    t_f = flops / 80e12 * 1e3
    assert abs(r["roof_max_ms"] - max(t_b, t_f)) < 1e-15
    assert abs(r["frac_of_roof_max"] - max(t_b, t_f) / 3.0) < 1e-15
    want = 0.2 * 0.8 + 0.25 * 0.5 + 1.5 * 0.6 + 0.9 * 0.85
    assert abs(r["stage_roof_sum_ms"] - want) < 1e-12
    assert "flux" not in r["stage_roof_ms"]
    # the spectral form: no flops roof, the stage sum still
    r2 = bench.step_roofline(w, "fp32", N, M, 4, 3.0, stage_ms, kernels, 1000.0, 80.0, "spectral")
    assert "roof_max_ms" not in r2 and abs(r2["stage_roof_sum_ms"] - want) < 1e-12


def test_shell_roofline_in_both_forms_and_its_kernels_entry():
    """K3's roofline comes from the shell stage's own time: the stencil against the FP32 FMA peak, the
    spectral form against the copy bandwidth (FP32), and the kernels table carries it either way."""
    N, M = 1000, 2
    w = {"sigma": [4.0, 6.0], "shape": (10, 10, 10), "periodic": (1, 0, 0)}
    peaks = {"hbm_gbs": 1000.0, "sm_max_mhz": 2070.0}
    r = bench.shell_roofline(w, "fp32", N, M, (8.0, 16), peaks, "measured", 152, "x", "direct")
    flops = sum(bench.shell_flops_per_node(S) for S in (4, 5, 5, 6)) * N / 4
    assert r["bound"] == "alu" and abs(r["avg_launch_ms"] - 0.5) < 1e-12
    assert abs(r["achieved"] - flops / 0.5e-3 / 1e12) < 1e-12
    assert abs(r["peak"] - 152 * 128 * 2 * 2070e6 / 1e12) < 1e-9
    rs = bench.shell_roofline(w, "fp32", N, M, (8.0, 4), peaks, "measured", 152, "x", "spectral")
    assert rs["bound"] == "hbm" and rs["unit"] == "GB/s"
    for roof, key in ((r, "achieved_tflops"), (rs, "achieved_gbs")):
        out = bench.kernel_rooflines({"shell": (8.0, 16)}, w, "fp32", N, M, 4, 1000.0, roof, 152, 2070.0, "direct")
        assert out["shell"]["frac"] == roof["frac"] and key in out["shell"]
    c = bench.collide_roofline(N, M, 4, (4.0, 4), peaks, "measured", "x", "fp32")
    assert c["algorithmic_bytes_per_launch"] == N * M * 304 and abs(c["avg_launch_ms"] - 1.0) < 1e-12
