"""bench.py's accounting on the host: algorithmic bytes against the
workload definitions' closed forms, the whole-job value, the image shards,
and the guard that drops ncu counters taken on other kernel sources."""
import json

import pytest

import bench


def test_step_bytes_of_the_fp32_workload():
    # forward reads I_h, p_l, I_l and writes O_h; backward reads dO_h, I_h, p_l, I_l and
    # writes dI_h, dp_l, dI_l: 1082.1 MB for FP32 4 x 3 x 512^2 -> 2048^2
    N, C, hl, wl, h, w, e = 4, 3, 512, 512, 2048, 2048, 4
    hi, lo = N * C * h * w * e, N * C * hl * wl * e
    step = (2 * hi + 2 * lo) + (3 * hi + 4 * lo)
    assert abs(step / 1e6 - 1082.1) < 0.1
    shape = (N, C, hl, wl, h, w)
    fused = bench.algorithmic_bytes("k12_fused_forward", shape, e) + \
        bench.algorithmic_bytes("k13_fused_backward", shape, e)
    # the fused kernels move every high-res byte of the step; K4 the low-res gradients
    assert fused == 2 * hi + 2 * lo + 3 * hi + 2 * lo
    assert bench.algorithmic_bytes("k4_lowres_bwd", shape, e) == lo * 2 + N * C * hl * wl * 8 + lo * 2


def test_kernel_bytes_per_unit():
    shape = (2, 3, 540, 960, 2160, 3840)
    hi, lo = 2 * 3 * 2160 * 3840, 2 * 3 * 540 * 960
    assert bench.algorithmic_bytes("k2_hires_apply", shape, 2) == hi * 4
    assert bench.algorithmic_bytes("k3_hires_bwd", shape, 2) == hi * 6
    assert bench.algorithmic_bytes("k1_lowres_coef", shape, 2) == lo * 12
    assert bench.algorithmic_bytes("nonexistent", shape, 2) is None


@pytest.mark.parametrize("n,world", [(12, 1), (12, 5), (7, 8), (0, 3)])
def test_shards_cover_every_image_once(n, world):
    parts = [bench.shard(n, r, world) for r in range(world)]
    assert parts[0][0] == 0 and parts[-1][1] == n
    for (a0, a1), (b0, b1) in zip(parts, parts[1:]):
        assert a1 == b0
    sizes = [b - a for a, b in parts]
    assert max(sizes) - min(sizes) <= 1


def test_job_value_is_all_ranks_pixels_over_the_slowest_time():
    assert bench.job_value(16.777216e6, 1, 0.2317) == pytest.approx(72409.2, rel=1e-4)
    assert bench.job_value(1e6, 4, 2.0) == pytest.approx(2000.0)


def test_ncu_counters_follow_the_kernel_sources(tmp_path, monkeypatch):
    data = {"wl": {"k": {"dram_bytes_per_launch": 123, "source_hash": "abcdabcdabcdabcd"},
                   "old": {"dram_bytes_per_launch": 456, "source_hash": "0000000000000000"}}}
    (tmp_path / "profiles").mkdir()
    (tmp_path / "profiles" / "ncu_traffic.json").write_text(json.dumps(data))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: "abcdabcdabcdabcd")
    assert bench.ncu_traffic("k", "wl") == 123
    assert bench.ncu_traffic("old", "wl") is None      # taken on other kernel sources
    assert bench.ncu_traffic("missing", "wl") is None
