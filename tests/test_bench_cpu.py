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


def test_accuracy_leg_reports_the_oracle_errors(tmp_path):
    """The oracle half of bench.py's accuracy leg on tiny cases whose 'GPU'
    outputs are the oracle's own plus a known perturbation."""
    import numpy as np

    import oracle
    import synth
    d = {k: v.numpy() for k, v in synth.photo_like(3, 1, 1, 8, 10, 4).items()}
    R = synth.upstream_grad(4, d["I_h"].shape).numpy()
    o = oracle.forward(d["p_l"], d["I_l"], d["I_h"], 1, 1e-3)
    dp, dil, dih = oracle.backward(R, d["p_l"], d["I_l"], d["I_h"], 1, 1e-3)
    o2 = o.copy()
    o2[0, 0, 3, 5] += 1e-3
    f = tmp_path / "plain.npz"
    np.savez(f, p_l=d["p_l"], I_l=d["I_l"], I_h=d["I_h"], R=R, O_h=o2, dp_l=dp, dI_l=dil, dI_h=2 * dih)
    dg = {k: v.numpy() for k, v in synth.photo_like(5, 1, 3, 4, 4, 4).items()}
    w = {k: v.numpy() for k, v in synth.guide_weights(6).items()}
    Rg = synth.upstream_grad(7, dg["I_h"].shape).numpy()
    og = oracle.forward_guided(dg["p_l"], dg["I_h"], w["w1"], w["w2"], w["b2"], 2, 1e-3)
    gp, gih, gw1, gw2, gb2 = oracle.backward_guided(Rg, dg["p_l"], dg["I_h"], w["w1"], w["w2"], w["b2"], 2, 1e-3)
    fg = tmp_path / "guided.npz"
    np.savez(fg, p_l=dg["p_l"], I_h=dg["I_h"], R=Rg, O_h=og, dp_l=gp, dI_h=gih, w1=w["w1"], w2=w["w2"],
             b2=w["b2"], dw1=gw1, dw2=gw2, db2=gb2)
    man = [{"name": "p", "kind": "plain", "file": str(f), "r": 1, "eps": 1e-3, "dtype": "f32", "sample": "all"},
           {"name": "g", "kind": "guided", "file": str(fg), "r": 2, "eps": 1e-3, "dtype": "f32", "sample": "all"}]
    res = bench.accuracy_oracle(man, str(tmp_path))
    assert "error" not in res, res
    assert res["p"]["O_h"]["max_abs"] == pytest.approx(1e-3, rel=1e-6)
    assert res["p"]["dp_l"]["max_abs"] == 0.0 and res["p"]["dI_l"]["rel_l2"] == 0.0
    assert res["p"]["dI_h"]["rel_l2"] == pytest.approx(1.0)
    for k in ("O_h", "dp_l", "dI_h", "dW"):
        assert res["g"][k]["max_abs"] < 1e-12
