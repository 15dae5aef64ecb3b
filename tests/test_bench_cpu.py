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
    out = bench.kernel_rooflines(stages, w, "fp32", N, M, 4, 1000.0, {"bound": "hbm"}, 152, 2070.0, "direct")
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
    out = bench.kernel_rooflines(stages, w, "fp64", N, M, 8, 1000.0, {"bound": "alu"}, 152, 2070.0, "spectral")
    c = out["collide"]
    assert c["bound"] == "alu"
    assert c["algorithmic_flops_per_launch"] == N * M * bench.K4_FLOPS_PER_NODE_SPECIES
    assert abs(c["frac"] - c["achieved_tflops"] / bench.FP64_NOMINAL_TFLOPS) < 1e-12
    assert c["algorithmic_bytes_per_launch"] == N * M * 4 * 19 * 8


def test_ball_counts_match_the_contact_balls():
    # the oracle's ball lists, counted independently
    assert [bench.ball_count(r) for r in (0.0, 1.5, 2.0, 2.5, 3.0)] == [1, 19, 33, 81, 123]
