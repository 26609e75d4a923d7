"""Full-size workloads on the GPU, checked against the FP64 oracle on sampled
planes or images (the oracle computes those completely), with the tile
shapes chosen by the autotuner as in the benchmark.

* plain FP32 forward + backward, 4 x 3 x 512^2 -> 2048^2, r = 1, eps = 1e-4
* BF16 4K batch, 2 x 3 x 540x960 -> 2160x3840, r = 2, eps = 1e-3
* 64 uneven BF16 images through the batched graph path (long side 512..4096,
  factor 4 or 8, r in {1, 2, 4}) and the batched backward; every image bitwise
  equal to its single call
* the training step with the guidance transform, 8 x 3 x 256^2 -> 2048^2,
  r = 8, eps = 1e-4, BF16, weight gradients included
* the plain FP32 step from pinned host memory (dgf_host_step, six plane
  groups as in the end-to-end benchmark): every output bitwise equal to the
  device calls
"""
import numpy as np
import pytest
import torch

import oracle as O
import synth
from paper_1803_05619_gb300 import _lib as L
from paper_1803_05619_gb300.layer import (gf_backward, gf_backward_batched, gf_forward, gf_forward_batched,
                                          gf_step_host)
from tests.helpers import assert_fwd, assert_grad, f64, rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def autotuned():
    L.dgf_autotune(True)
    yield
    L.dgf_autotune(False)


def _planes_equal_oracle(st, R, r, eps, dtype, planes):
    p_l, I_l, I_h = (st[k] for k in ("p_l", "I_l", "I_h"))
    ref = O.forward(f64(p_l), f64(I_l), f64(I_h), r, eps, planes=planes)
    dp, dIl, dIh = O.backward(f64(R), f64(p_l), f64(I_l), f64(I_h), r, eps, planes=planes)
    return ref, dp, dIl, dIh


def test_fp32_plain_fullsize():
    N, C, hl, wl, f, r, eps = 4, 3, 512, 512, 4, 1, 1e-4
    d = synth.blobs_tone_curve(0, N, C, hl, wl, f, device="cuda")
    st = {k: v.float() for k, v in d.items()}
    R = synth.upstream_grad(1, st["I_h"].shape).float()
    g = {k: v.cuda() for k, v in st.items()}
    out = gf_forward(g["p_l"], g["I_l"], g["I_h"], r, eps)
    dp, dIl, dIh, _ = gf_backward(R.cuda(), g["p_l"], g["I_l"], g["I_h"], r, eps)
    torch.cuda.synchronize()
    planes = [(0, 0), (3, 2)]
    ref, rp, rIl, rIh = _planes_equal_oracle(st, R, r, eps, torch.float32, planes)
    for n, c in planes:
        assert_fwd(f64(out[n, c]), ref[n, c], torch.float32, eps)
        assert_grad(f64(dp[n, c]), rp[n, c], torch.float32, "dp_l")
        assert_grad(f64(dIl[n, c]), rIl[n, c], torch.float32, "dI_l")
        assert_grad(f64(dIh[n, c]), rIh[n, c], torch.float32, "dI_h")


def test_host_step_fullsize():
    N, C, hl, wl, f, r, eps = 4, 3, 512, 512, 4, 1, 1e-4
    d = synth.blobs_tone_curve(0, N, C, hl, wl, f, device="cuda")
    g = {k: v.float().cuda() for k, v in d.items()}
    R = synth.upstream_grad(1, g["I_h"].shape).float().cuda()
    out = gf_forward(g["p_l"], g["I_l"], g["I_h"], r, eps)
    dp, dIl, dIh, _ = gf_backward(R, g["p_l"], g["I_l"], g["I_h"], r, eps)
    torch.cuda.synchronize()
    h = {k: v.cpu().pin_memory() for k, v in g.items()}
    res = gf_step_host(h["p_l"], h["I_l"], h["I_h"], R.cpu().pin_memory(), r, eps, groups=6)
    for a, b in zip(res, (out, dp, dIl, dIh)):
        assert torch.equal(a, b.cpu())


def test_bf16_4k_fullsize():
    N, C, hl, wl, f, r, eps = 2, 3, 540, 960, 4, 2, 1e-3
    st = {k: v.to(torch.bfloat16) for k, v in synth.photo_like(7, N, C, hl, wl, f).items()}
    R = synth.upstream_grad(8, st["I_h"].shape).to(torch.bfloat16)
    g = {k: v.cuda() for k, v in st.items()}
    out = gf_forward(g["p_l"], g["I_l"], g["I_h"], r, eps)
    dp, dIl, dIh, _ = gf_backward(R.cuda(), g["p_l"], g["I_l"], g["I_h"], r, eps)
    torch.cuda.synchronize()
    planes = [(1, 1)]
    ref, rp, rIl, rIh = _planes_equal_oracle(st, R, r, eps, torch.bfloat16, planes)
    n, c = planes[0]
    assert_fwd(f64(out[n, c]), ref[n, c], torch.bfloat16, eps)
    assert_grad(f64(dp[n, c]), rp[n, c], torch.bfloat16, "dp_l")
    assert_grad(f64(dIl[n, c]), rIl[n, c], torch.bfloat16, "dI_l")
    assert_grad(f64(dIh[n, c]), rIh[n, c], torch.bfloat16, "dI_h")
    # batched entry on the same two images: bitwise equal to the single call
    images = [{"p_l": g["p_l"][i], "I_l": g["I_l"][i], "I_h": g["I_h"][i], "r": r, "eps": eps}
              for i in range(N)]
    outs = gf_forward_batched(images)
    torch.cuda.synchronize()
    for i in range(N):
        assert torch.equal(outs[i], out[i])


def test_batched_64_uneven_fullsize():
    specs = synth.mixed_sizes(seed=0, n=64)
    eps = 1e-3
    images, host = [], []
    for i, s in enumerate(specs):
        d = synth.photo_like(1000 + i, 1, 3, s.h_l, s.w_l, s.f)
        st = {k: v.to(torch.bfloat16) for k, v in d.items()}
        host.append(st)
        images.append({"p_l": st["p_l"][0].cuda(), "I_l": st["I_l"][0].cuda(), "I_h": st["I_h"][0].cuda(),
                       "r": s.r, "eps": eps})
    mpix = sum(s.h * s.w for s in specs) / 1e6
    assert 150 < mpix < 450
    # single calls first: any shape the autotuner picks on them is then used by the batch too
    singles = [gf_forward(im["p_l"][None], im["I_l"][None], im["I_h"][None], im["r"], im["eps"])[0]
               for im in images]
    outs = gf_forward_batched(images)
    torch.cuda.synchronize()
    for o, single in zip(outs, singles):
        assert torch.equal(o, single)
    # oracle on three images: the two smallest and one mid-size
    order = sorted(range(len(specs)), key=lambda i: specs[i].h * specs[i].w)
    for i in (order[0], order[1], order[len(order) // 2]):
        ref = O.forward(f64(host[i]["p_l"]), f64(host[i]["I_l"]), f64(host[i]["I_h"]), specs[i].r, eps)
        assert_fwd(f64(outs[i])[None], ref, torch.bfloat16, eps, what=f"image {i}")
    # batched backward: every image bitwise equal to its single call (single
    # calls first, so any shape the autotuner picks is the batch's too); the
    # smallest image against the oracle
    grads = [synth.upstream_grad(2000 + i, im["I_h"].shape).to(torch.bfloat16).cuda() for i, im in enumerate(images)]
    singles = [gf_backward(R[None], im["p_l"][None], im["I_l"][None], im["I_h"][None], im["r"], im["eps"])
               for im, R in zip(images, grads)]
    gouts = gf_backward_batched(images, grads)
    torch.cuda.synchronize()
    for go, single in zip(gouts, singles):
        for a, b in zip(go, single[:3]):
            assert torch.equal(a, b[0])
    i = order[0]
    R = grads[i].cpu()[None]
    rp, rIl, rIh = O.backward(f64(R), f64(host[i]["p_l"]), f64(host[i]["I_l"]), f64(host[i]["I_h"]), specs[i].r, eps)
    assert_grad(f64(gouts[i][0])[None], rp, torch.bfloat16, "dp_l")
    assert_grad(f64(gouts[i][1])[None], rIl, torch.bfloat16, "dI_l")
    assert_grad(f64(gouts[i][2])[None], rIh, torch.bfloat16, "dI_h")


def test_guided_training_step_fullsize():
    N, C, hl, wl, f, r, eps = 8, 3, 256, 256, 8, 8, 1e-4
    st = {k: v.to(torch.bfloat16) for k, v in synth.photo_like(21, N, C, hl, wl, f).items()}
    w = {k: v.float() for k, v in synth.guide_weights(22).items()}
    R = synth.upstream_grad(23, st["I_h"].shape).to(torch.bfloat16)
    g = {k: v.cuda() for k, v in st.items()}
    wc = {k: v.cuda() for k, v in w.items()}
    out = gf_forward(g["p_l"], None, g["I_h"], r, eps, wc["w1"], wc["w2"], wc["b2"], 0.2)
    dp, _, dIh, dws = gf_backward(R.cuda(), g["p_l"], None, g["I_h"], r, eps, wc["w1"], wc["w2"], wc["b2"],
                                  0.2)
    torch.cuda.synchronize()
    w64 = {k: v.double().numpy() for k, v in w.items()}
    img = [0]
    ref = O.forward_guided(f64(st["p_l"]), f64(st["I_h"]), w64["w1"], w64["w2"], w64["b2"], r, eps,
                           images=img)
    assert_fwd(f64(out[0]), ref[0], torch.bfloat16, eps)
    rp, rI, _, _, _ = O.backward_guided(f64(R), f64(st["p_l"]), f64(st["I_h"]), w64["w1"], w64["w2"],
                                        w64["b2"], r, eps, images=img)
    assert_grad(f64(dp[0]), rp[0], torch.bfloat16, "dp_l")
    assert_grad(f64(dIh[0]), rI[0], torch.bfloat16, "dI_h")
    # the weight gradients sum over all 8 images: compare with the oracle over all of them
    _, _, rw1, rw2, _ = O.backward_guided(f64(R), f64(st["p_l"]), f64(st["I_h"]), w64["w1"], w64["w2"],
                                          w64["b2"], r, eps)
    assert rel_l2(f64(dws[0]), rw1) <= 2e-2
    assert rel_l2(f64(dws[1]), rw2) <= 2e-2
    assert np.all(np.isfinite(f64(dws[2])))
