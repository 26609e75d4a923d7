"""CUDA path vs the FP64 oracle, element by element (needs a GPU).

Sizes span several tiles of every kernel and end in ragged tails; the
cases cover integer factors 2, 4, 8, non-integer ratios, odd widths (scalar
path), r from 0 to 16, FP32/BF16/FP16 storage.
"""
import ctypes

import numpy as np
import pytest
import torch

import oracle as O
import synth
from paper_1803_05619_gb300 import _lib as L
from paper_1803_05619_gb300.layer import gf_backward, gf_backward_batched, gf_forward, gf_forward_batched
from tests.helpers import (assert_fwd, assert_grad, f64, make_case, oracle_backward, oracle_forward,
                           rel_l2, to_storage, TOL_F32_REL_L2)

pytestmark = pytest.mark.gpu

F32, BF16, F16 = torch.float32, torch.bfloat16, torch.float16

# kind, N, C, h_l, w_l, h, w, r, eps
FWD_CASES = [
    ("photo", 1, 1, 64, 64, 256, 256, 1, 1e-2),     # configuration-1 shape
    ("photo", 2, 3, 70, 90, 280, 360, 1, 1e-3),     # several tiles + ragged tails, f = 4
    ("photo", 1, 2, 40, 44, 320, 352, 2, 1e-3),     # f = 8
    ("photo", 1, 1, 33, 47, 66, 94, 4, 1e-3),       # f = 2
    ("ragged", 1, 2, 37, 53, 150, 211, 1, 1e-3),    # non-integer ratio, odd width
    ("ragged", 2, 1, 19, 23, 61, 92, 2, 1e-3),      # non-integer, even width
    ("photo", 1, 1, 48, 40, 192, 160, 8, 1e-3),     # r = 8
    ("photo", 1, 1, 20, 24, 80, 96, 16, 1e-2),      # r = 16 > image half-size
    ("photo", 1, 1, 30, 36, 120, 144, 0, 1e-2),     # r = 0
    ("photo", 1, 2, 50, 70, 200, 280, 3, 1e-3),     # r = 3 (generic-radius tile kernels)
    ("photo", 2, 1, 36, 300, 144, 1200, 4, 1e-3),   # r = 4, wide: several column-walking tiles
    ("photo", 1, 1, 70, 40, 560, 320, 8, 1e-4),     # r = 8 over several tiles, eps = 1e-4
    ("blobs", 1, 3, 64, 72, 256, 288, 1, 1e-4),     # configuration-2 recipe, eps = 1e-4
    ("ragged", 1, 1, 1, 1, 7, 5, 1, 1e-3),          # single low-res pixel
    ("ragged", 1, 1, 3, 1, 9, 4, 1, 1e-3),          # one column
    ("ragged", 1, 1, 5, 6, 5, 6, 1, 1e-3),          # f = 1 (plain guided filter)
]


def _ids(cases):
    return ["-".join(str(v) for v in c) for c in cases]


@pytest.mark.parametrize("dtype", [F32, BF16, F16], ids=["f32", "bf16", "f16"])
@pytest.mark.parametrize("case", FWD_CASES, ids=_ids(FWD_CASES))
def test_forward_parity(case, dtype):
    kind, N, C, hl, wl, h, w, r, eps = case
    st = to_storage(make_case(kind, 100 + r, N, C, hl, wl, h, w), dtype)
    g = {k: v.cuda() for k, v in st.items()}
    out = gf_forward(g["p_l"], g["I_l"], g["I_h"], r, eps)
    torch.cuda.synchronize()
    ref = oracle_forward(st, r, eps)
    assert_fwd(f64(out), ref, dtype, eps)
    assert L.dgf_device_status() == 0


BWD_CASES = [c for c in FWD_CASES if c[0] != "ragged" or c[3] > 1] + [
    ("photo", 1, 1, 48, 64, 384, 512, 2, 1e-3),     # f = 8 with an even low-res width
    ("blobs", 1, 1, 256, 256, 1024, 1024, 1, 1e-4),  # large flat regions: gamma ~ 1/eps
    ("blobs", 1, 1, 200, 240, 800, 960, 2, 1e-4),
]


@pytest.mark.parametrize("dtype", [F32, BF16, F16], ids=["f32", "bf16", "f16"])
@pytest.mark.parametrize("case", BWD_CASES, ids=_ids(BWD_CASES))
def test_backward_parity(case, dtype):
    kind, N, C, hl, wl, h, w, r, eps = case
    st = to_storage(make_case(kind, 200 + r, N, C, hl, wl, h, w), dtype)
    R = synth.upstream_grad(7, st["I_h"].shape).to(dtype)
    g = {k: v.cuda() for k, v in st.items()}
    dp, dIl, dIh, _ = gf_backward(R.cuda(), g["p_l"], g["I_l"], g["I_h"], r, eps)
    torch.cuda.synchronize()
    rp, rIl, rIh = oracle_backward(R, st, r, eps)
    if dtype == F32 and eps < 1e-3:
        pass  # same gate: relative L2 <= 1e-4
    assert_grad(f64(dp), rp, dtype, "dp_l")
    assert_grad(f64(dIl), rIl, dtype, "dI_l")
    assert_grad(f64(dIh), rIh, dtype, "dI_h")


def test_autograd_function_matches_oracle():
    from paper_1803_05619_gb300 import GuidedFilter
    st = to_storage(make_case("photo", 5, 2, 3, 24, 40, 96, 160), F32)
    R = synth.upstream_grad(9, st["I_h"].shape).float()
    p = st["p_l"].cuda().requires_grad_(True)
    il = st["I_l"].cuda().requires_grad_(True)
    ih = st["I_h"].cuda().requires_grad_(True)
    out = GuidedFilter(r=2, eps=1e-3)(p, il, ih)
    (out * R.cuda()).sum().backward()
    rp, rIl, rIh = oracle_backward(R, st, 2, 1e-3)
    assert_grad(f64(p.grad), rp, F32, "dp_l")
    assert_grad(f64(il.grad), rIl, F32, "dI_l")
    assert_grad(f64(ih.grad), rIh, F32, "dI_h")


@pytest.fixture
def pin():
    """Pin autotuner table entries for one test; the table is cleared after."""
    L.dgf_autotune_reset()
    yield lambda *args: L.check(L.dgf_autotune_pin(*args))
    L.dgf_autotune_reset()


# Low-res kernel forms for r <= 2 (kind 1 = K1, 4 = K4): warp strips
# (a = rows per segment, b = 0) and column-walking tiles (a = columns,
# b = rows of the coefficient region)
LOW_FORMS = [(1, 1, 16, 0), (1, 1, 64, 0), (1, 1, 64, 32), (1, 1, 128, 16), (1, 2, 32, 0), (1, 2, 16, 0),
             (1, 2, 64, 32), (1, 2, 128, 64),
             (4, 1, 8, 0), (4, 1, 32, 0), (4, 1, 128, 0), (4, 1, 64, 16), (4, 2, 16, 0), (4, 2, 64, 0),
             (4, 2, 64, 32)]


@pytest.mark.parametrize("dtype", [F32, BF16], ids=["f32", "bf16"])
@pytest.mark.parametrize("form", LOW_FORMS, ids=_ids(LOW_FORMS))
def test_lowres_forms_match_oracle(form, dtype, pin):
    kind, r, a, b = form
    dt = L.DGF_F32 if dtype == F32 else L.DGF_BF16
    pin(kind, dt, r, 0, 0, 0, a, b)
    # ragged against strips of 28 / 24 columns and segments of 16..64 rows
    st = to_storage(make_case("photo", 30 + r, 1, 2, 77, 131, 308, 524), dtype)
    R = synth.upstream_grad(31, st["I_h"].shape).to(dtype)
    g = {k: v.cuda() for k, v in st.items()}
    out = gf_forward(g["p_l"], g["I_l"], g["I_h"], r, 1e-3)
    dp, dIl, dIh, _ = gf_backward(R.cuda(), g["p_l"], g["I_l"], g["I_h"], r, 1e-3)
    torch.cuda.synchronize()
    assert_fwd(f64(out), oracle_forward(st, r, 1e-3), dtype, 1e-3)
    rp, rIl, rIh = oracle_backward(R, st, r, 1e-3)
    assert_grad(f64(dp), rp, dtype, "dp_l")
    assert_grad(f64(dIl), rIl, dtype, "dI_l")
    assert_grad(f64(dIh), rIh, dtype, "dI_h")
    assert L.dgf_device_status() == 0


# Sliding-sum low-res strips (16-bit storage): (r, rows per segment, dtype,
# kind, N, C, h_l, w_l, h, w, eps).  Widths that are not a multiple of the
# lane's columns take the masked scalar loads; "blobs" has flat, clipped
# regions where var << eps = 1e-4.
SLIDE_CASES = [(1, 8, BF16, "photo", 1, 2, 77, 131, 308, 524, 1e-3),
               (1, 64, F16, "photo", 2, 1, 64, 240, 256, 960, 1e-3),
               (2, 12, BF16, "photo", 1, 3, 135, 240, 540, 960, 1e-3),
               (2, 32, F16, "ragged", 1, 2, 37, 53, 150, 211, 1e-3),
               (2, 16, BF16, "blobs", 1, 2, 128, 128, 512, 512, 1e-4),
               (4, 16, BF16, "photo", 1, 2, 70, 233, 280, 932, 1e-3),
               (4, 48, F16, "photo", 1, 1, 100, 96, 400, 384, 1e-3),
               (8, 16, BF16, "photo", 2, 1, 64, 100, 512, 800, 1e-4),
               (8, 32, F16, "photo", 1, 2, 29, 35, 232, 280, 1e-3),
               (8, 64, BF16, "blobs", 1, 1, 96, 96, 384, 384, 1e-4)]


@pytest.mark.parametrize("case", SLIDE_CASES, ids=_ids(SLIDE_CASES))
def test_sliding_lowres_matches_oracle(case, pin):
    r, seg, dtype, kind, N, C, hl, wl, h, w, eps = case
    dt = L.DGF_BF16 if dtype == BF16 else L.DGF_F16
    st = to_storage(make_case(kind, 500 + r, N, C, hl, wl, h, w), dtype)
    R = synth.upstream_grad(501, st["I_h"].shape).to(dtype)
    g = {k: v.cuda() for k, v in st.items()}
    v1, v4 = (8 if r <= 2 else 4), 4
    pin(1, dt, r, 0, 0, 0, seg, -v1)
    pin(4, dt, r, 0, 0, 0, seg, -v4)
    n0 = L.dgf_launch_count()
    L.dgf_profile_reset()
    L.dgf_profile_enable(True)
    try:
        out = gf_forward(g["p_l"], g["I_l"], g["I_h"], r, eps)
        dp, dIl, dIh, _ = gf_backward(R.cuda(), g["p_l"], g["I_l"], g["I_h"], r, eps)
        torch.cuda.synchronize()
        names = list(L.dgf_profile_read().keys())
    finally:
        L.dgf_profile_enable(False)
    assert L.dgf_launch_count() > n0
    assert "k1_lowres_coef" in names and "k4_lowres_bwd" in names
    assert_fwd(f64(out), oracle_forward(st, r, eps), dtype, eps)
    rp, rIl, rIh = oracle_backward(R, st, r, eps)
    assert_grad(f64(dp), rp, dtype, "dp_l")
    assert_grad(f64(dIl), rIl, dtype, "dI_l")
    assert_grad(f64(dIh), rIh, dtype, "dI_h")
    assert L.dgf_device_status() == 0
    # the exactly centred forms agree with it within the same gates
    L.dgf_set_lowres_slide(False)
    try:
        L.dgf_autotune_reset()
        ex = gf_forward(g["p_l"], g["I_l"], g["I_h"], r, eps)
        exb = gf_backward(R.cuda(), g["p_l"], g["I_l"], g["I_h"], r, eps)
        torch.cuda.synchronize()
    finally:
        L.dgf_set_lowres_slide(True)
    assert_fwd(f64(out), f64(ex), dtype, eps)
    for a, b, name in zip((dp, dIl, dIh), exb[:3], ("dp_l", "dI_l", "dI_h")):
        assert_grad(f64(a), f64(b), dtype, name)


@pytest.mark.parametrize("dtype", [BF16, F16], ids=["bf16", "f16"])
def test_sliding_lowres_bits_do_not_depend_on_the_plane_count(dtype):
    # the default segment length is a function of the plane height and r
    # only, so a plane gives the same bits alone or among others
    st = to_storage(make_case("photo", 510, 2, 3, 60, 90, 240, 360), dtype)
    R = synth.upstream_grad(511, st["I_h"].shape).to(dtype).cuda()
    g = {k: v.cuda() for k, v in st.items()}
    full = gf_forward(g["p_l"], g["I_l"], g["I_h"], 2, 1e-3)
    fb = gf_backward(R, g["p_l"], g["I_l"], g["I_h"], 2, 1e-3)[:3]
    sub = {k: v[1:, 2:].contiguous() for k, v in g.items()}
    one = gf_forward(sub["p_l"], sub["I_l"], sub["I_h"], 2, 1e-3)
    ob = gf_backward(R[1:, 2:].contiguous(), sub["p_l"], sub["I_l"], sub["I_h"], 2, 1e-3)[:3]
    torch.cuda.synchronize()
    assert torch.equal(full[1:, 2:], one)
    for a, b in zip(fb, ob):
        assert torch.equal(a[1:, 2:], b)


@pytest.mark.parametrize("r", [1, 2])
@pytest.mark.parametrize("dtype", [F32, BF16], ids=["f32", "bf16"])
def test_k4_saved_statistics_match_recomputed(r, dtype, pin):
    # K1 strips keep each window's statistics for the K4 strips; with K1 in
    # tile form K4 recomputes them.  Same formulas; the compiler may contract
    # a product and a sum into one FMA differently in the two kernels, so the
    # results agree to rounding (dI_h takes Abar from K1, whose forms differ).
    dt = L.DGF_F32 if dtype == F32 else L.DGF_BF16
    st = to_storage(make_case("photo", 40 + r, 2, 2, 75, 133, 300, 532), dtype)
    R = synth.upstream_grad(41, st["I_h"].shape).to(dtype).cuda()
    g = {k: v.cuda() for k, v in st.items()}
    pin(4, dt, r, 0, 0, 0, 32, 0)
    saved = gf_backward(R, g["p_l"], g["I_l"], g["I_h"], r, 1e-3)
    pin(1, dt, r, 0, 0, 0, 64, 32)
    recomputed = gf_backward(R, g["p_l"], g["I_l"], g["I_h"], r, 1e-3)
    torch.cuda.synchronize()
    bound = 1e-6 if dtype == F32 else 2e-3
    for name, a, b in zip(("dp_l", "dI_l"), saved[:2], recomputed[:2]):
        assert rel_l2(f64(a), f64(b)) <= bound, name
    assert_grad(f64(saved[2]), f64(recomputed[2]), dtype, "dI_h")


def test_autotune_pin_rejects_bad_keys():
    with pytest.raises(L.DGFError):
        L.check(L.dgf_autotune_pin(0, L.DGF_F32, 1, 0, 0, 0, 64, 32))
    with pytest.raises(L.DGFError):
        L.check(L.dgf_autotune_pin(1, L.DGF_F32, 1, 0, 0, 0, -4, 32))


def test_unbuilt_pinned_shape_falls_back_to_default(pin):
    st = to_storage(make_case("photo", 5, 1, 1, 40, 52, 160, 208), F32)
    g = {k: v.cuda() for k, v in st.items()}
    ref = gf_forward(g["p_l"], g["I_l"], g["I_h"], 1, 1e-3)
    pin(1, L.DGF_F32, 1, 0, 0, 0, 100, 7)  # not a built shape: ignored at plan time
    out = gf_forward(g["p_l"], g["I_l"], g["I_h"], 1, 1e-3)
    torch.cuda.synchronize()
    assert torch.equal(out, ref)


@pytest.mark.parametrize("dtype,size", [(BF16, (2, 3, 64, 96, 256, 384)), (F32, (1, 2, 70, 90, 280, 360)),
                                        (BF16, (1, 1, 40, 44, 320, 352))], ids=["bf16-f4", "f32-f4", "bf16-f8"])
@pytest.mark.parametrize("k1_form", ["tiles", "strips"])
def test_tma_and_plain_staging_identical(dtype, size, k1_form, pin):
    # every kernel that stages by TMA (K1 tiles or strips, K2, K3, K4 strips)
    # against its plain-load form
    if k1_form == "tiles":
        pin(1, L.DGF_F32 if dtype == F32 else L.DGF_BF16, 2, 0, 0, 0, 64, 32)
    N, C, hl, wl, h, w = size
    st = to_storage(make_case("photo", 3, N, C, hl, wl, h, w), dtype)
    R = synth.upstream_grad(4, st["I_h"].shape).to(dtype).cuda()
    g = {k: v.cuda() for k, v in st.items()}
    res = []
    for on in (True, False):
        L.dgf_set_tma(on)
        out = gf_forward(g["p_l"], g["I_l"], g["I_h"], 2, 1e-3)
        grads = gf_backward(R, g["p_l"], g["I_l"], g["I_h"], 2, 1e-3)[:3]
        res.append((out, *grads))
    L.dgf_set_tma(True)
    torch.cuda.synchronize()
    for a, b in zip(*res):
        assert torch.equal(a, b)


def test_deterministic():
    st = to_storage(make_case("photo", 4, 2, 3, 40, 48, 160, 192), F32)
    g = {k: v.cuda() for k, v in st.items()}
    R = synth.upstream_grad(3, st["I_h"].shape).float().cuda()
    o1 = gf_forward(g["p_l"], g["I_l"], g["I_h"], 1, 1e-3)
    o2 = gf_forward(g["p_l"], g["I_l"], g["I_h"], 1, 1e-3)
    a = gf_backward(R, g["p_l"], g["I_l"], g["I_h"], 1, 1e-3)
    b = gf_backward(R, g["p_l"], g["I_l"], g["I_h"], 1, 1e-3)
    assert torch.equal(o1, o2)
    for x, y in zip(a[:3], b[:3]):
        assert torch.equal(x, y)


@pytest.mark.parametrize("dtype,r,f", [(F32, 1, 4), (BF16, 2, 4), (F16, 4, 8)], ids=["f32-r1", "bf16-r2", "f16-r4"])
def test_graph_captured_step_matches_eager(dtype, r, f):
    """A forward + backward step captured in a CUDA graph (as bench.py times
    it) and replayed gives the eager calls' bits, replay after replay, also
    after the inputs change in place."""
    st = to_storage(make_case("photo", 40 + r, 2, 3, 48, 64, 48 * f, 64 * f), dtype)
    g = {k: v.cuda() for k, v in st.items()}
    R = synth.upstream_grad(41, st["I_h"].shape).to(dtype).cuda()
    outs = {"O": torch.empty_like(g["I_h"]), "dp": torch.empty_like(g["p_l"]),
            "dIl": torch.empty_like(g["I_l"]), "dIh": torch.empty_like(g["I_h"])}
    N, C, h_l, w_l = g["p_l"].shape
    h, w = g["I_h"].shape[2:]
    dt = {F32: L.DGF_F32, BF16: L.DGF_BF16, F16: L.DGF_F16}[dtype]
    lib = L.lib()
    nb = L.dgf_workspace_size(N, C, h_l, w_l, h, w, r, dt, None)
    ws = torch.empty(nb, dtype=torch.uint8, device="cuda")
    P = lambda t: ctypes.c_void_p(t.data_ptr())  # noqa: E731
    cap = torch.cuda.Stream()

    def step():
        s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
        L.check(lib.dgf_forward(P(g["p_l"]), P(g["I_l"]), P(g["I_h"]), P(outs["O"]), N, C, h_l, w_l, h, w, r,
                                ctypes.c_float(1e-3), dt, None, P(ws), ws.numel(), s))
        L.check(lib.dgf_backward(P(R), P(g["p_l"]), P(g["I_l"]), P(g["I_h"]), P(outs["dp"]), P(outs["dIl"]),
                                 P(outs["dIh"]), None, N, C, h_l, w_l, h, w, r, ctypes.c_float(1e-3), dt, None,
                                 P(ws), ws.numel(), s))

    with torch.cuda.stream(cap):
        step()
    torch.cuda.synchronize()
    eager = {k: v.clone() for k, v in outs.items()}
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=cap):
        step()
    for v in outs.values():
        v.zero_()
    for _ in range(2):
        graph.replay()
        torch.cuda.synchronize()
        for k in outs:
            assert torch.equal(outs[k], eager[k]), k
    # new input values in the same buffers: the replay computes them
    g["p_l"].copy_(g["p_l"].flip(-1))
    with torch.cuda.stream(cap):
        step()
    torch.cuda.synchronize()
    eager2 = {k: v.clone() for k, v in outs.items()}
    graph.replay()
    torch.cuda.synchronize()
    for k in outs:
        assert torch.equal(outs[k], eager2[k]), k
    assert not torch.equal(eager2["O"], eager["O"])


def test_guard_regions_untouched():
    # outputs written into the middle of sentinel-filled buffers
    N, C, hl, wl, h, w = 1, 3, 30, 50, 120, 200
    st = to_storage(make_case("photo", 6, N, C, hl, wl, h, w), F32)
    g = {k: v.cuda() for k, v in st.items()}
    guard = 4096
    big = torch.full((guard * 2 + N * C * h * w,), 12345.0, device="cuda")
    out = big[guard:guard + N * C * h * w].view(N, C, h, w)
    gf_forward(g["p_l"], g["I_l"], g["I_h"], 1, 1e-3, out=out)
    torch.cuda.synchronize()
    assert torch.all(big[:guard] == 12345.0) and torch.all(big[-guard:] == 12345.0)
    assert_fwd(f64(out), oracle_forward(st, 1, 1e-3), F32, 1e-3)


def test_constant_target_gives_constant_output():
    st = to_storage(make_case("photo", 8, 1, 2, 40, 40, 160, 160), F32)
    st["p_l"] = torch.full_like(st["p_l"], 0.5)
    g = {k: v.cuda() for k, v in st.items()}
    out = gf_forward(g["p_l"], g["I_l"], g["I_h"], 2, 1e-3)
    assert torch.all(out == 0.5)


@pytest.mark.parametrize("k1_form", ["default", "tiles"])
@pytest.mark.parametrize("dtype", [F32, BF16], ids=["f32", "bf16"])
def test_batched_matches_single_bitwise(dtype, k1_form, pin):
    if k1_form == "tiles":
        dt = L.DGF_F32 if dtype == F32 else L.DGF_BF16
        pin(1, dt, 1, 0, 0, 0, 64, 32)
        pin(1, dt, 2, 0, 0, 0, 128, 32)
    specs = synth.mixed_sizes(seed=3, n=9, long_lo=96, long_hi=520)
    images = []
    for i, s in enumerate(specs):
        d = to_storage(synth.photo_like(50 + i, 1, 3, s.h_l, s.w_l, s.f), dtype)
        images.append({"p_l": d["p_l"][0].cuda(), "I_l": d["I_l"][0].cuda(), "I_h": d["I_h"][0].cuda(),
                       "r": s.r, "eps": 1e-3, "_st": d})
    for rep in range(2):  # second call replays the updated graph
        outs = gf_forward_batched(images)
        torch.cuda.synchronize()
        for im, o in zip(images, outs):
            single = gf_forward(im["p_l"][None], im["I_l"][None], im["I_h"][None], im["r"], im["eps"])
            assert torch.equal(o, single[0])
    # and against the oracle
    for im, o in zip(images, outs):
        ref = oracle_forward(im["_st"], im["r"], im["eps"])
        assert_fwd(f64(o)[None], ref, dtype, im["eps"])


@pytest.mark.parametrize("dtype", [F32, BF16], ids=["f32", "bf16"])
def test_batched_paper_literal_matches_single_bitwise(dtype):
    # mean_ab = False through the batched calls: each image's outputs are the
    # single calls' with the same option (radii 1, 2, 4 and factors 4, 8)
    specs = synth.mixed_sizes(seed=7, n=6, long_lo=96, long_hi=400)
    images, grads, host = [], [], []
    for i, s in enumerate(specs):
        d = to_storage(synth.photo_like(80 + i, 1, 3, s.h_l, s.w_l, s.f), dtype)
        R = synth.upstream_grad(95 + i, d["I_h"].shape).to(dtype)
        host.append((d, R, s.r))
        images.append({"p_l": d["p_l"][0].cuda(), "I_l": d["I_l"][0].cuda(), "I_h": d["I_h"][0].cuda(),
                       "r": s.r, "eps": 1e-3})
        grads.append(R[0].cuda())
    outs = gf_forward_batched(images, mean_ab=False)
    bouts = gf_backward_batched(images, grads, mean_ab=False)
    torch.cuda.synchronize()
    for im, R, o, b in zip(images, grads, outs, bouts):
        single = gf_forward(im["p_l"][None], im["I_l"][None], im["I_h"][None], im["r"], im["eps"], mean_ab=False)
        assert torch.equal(o, single[0])
        sg = gf_backward(R[None], im["p_l"][None], im["I_l"][None], im["I_h"][None], im["r"], im["eps"],
                         mean_ab=False)
        for a, c in zip(b, sg[:3]):
            assert torch.equal(a, c[0])
    d, R, r = host[0]
    ref = O.forward(f64(d["p_l"]), f64(d["I_l"]), f64(d["I_h"]), r, 1e-3, mean_ab=False)
    assert_fwd(f64(outs[0])[None], ref, dtype, 1e-3)
    rp, rIl, rIh = O.backward(f64(R), f64(d["p_l"]), f64(d["I_l"]), f64(d["I_h"]), r, 1e-3, mean_ab=False)
    for got, want, name in zip(bouts[0], (rp, rIl, rIh), ("dp_l", "dI_l", "dI_h")):
        assert_grad(f64(got)[None], want, dtype, name)
    # the other options are refused
    arr = (L.dgf_image * 1)()
    opt = L.dgf_options(1, 2, 0)
    assert L.dgf_forward_batched_opt(arr, 1, L.DGF_F32, None, 0, None, ctypes.byref(opt)) == 2  # DGF_ERR_UNSUPPORTED
    assert L.dgf_device_status() == 0


@pytest.mark.parametrize("dtype", [F32, BF16], ids=["f32", "bf16"])
def test_batched_backward_matches_single_bitwise(dtype):
    specs = synth.mixed_sizes(seed=5, n=7, long_lo=96, long_hi=520)
    images, grads, host = [], [], []
    for i, s in enumerate(specs):
        d = to_storage(synth.photo_like(70 + i, 1, 3, s.h_l, s.w_l, s.f), dtype)
        R = synth.upstream_grad(90 + i, d["I_h"].shape).to(dtype)
        host.append((d, R))
        images.append({"p_l": d["p_l"][0].cuda(), "I_l": d["I_l"][0].cuda(), "I_h": d["I_h"][0].cuda(),
                       "r": s.r, "eps": 1e-3})
        grads.append(R[0].cuda())
    for rep in range(2):  # the second call replays the updated graph (16-bit storage)
        outs = gf_backward_batched(images, grads)
        torch.cuda.synchronize()
        for im, R, o in zip(images, grads, outs):
            single = gf_backward(R[None], im["p_l"][None], im["I_l"][None], im["I_h"][None], im["r"], im["eps"])
            for a, b in zip(o, single[:3]):
                assert torch.equal(a, b[0])
    # and against the oracle on the two smallest images
    order = sorted(range(len(specs)), key=lambda i: specs[i].h * specs[i].w)
    for i in order[:2]:
        d, R = host[i]
        rp, rIl, rIh = oracle_backward(R, d, specs[i].r, 1e-3)
        assert_grad(f64(outs[i][0])[None], rp, dtype, "dp_l")
        assert_grad(f64(outs[i][1])[None], rIl, dtype, "dI_l")
        assert_grad(f64(outs[i][2])[None], rIh, dtype, "dI_h")


@pytest.mark.parametrize("dtype", [BF16, F16], ids=["bf16", "f16"])
def test_batched_backward_graph_partial_outputs(dtype):
    """The one-graph batched backward against the per-image chains and the
    single calls: every radius of the sliding kernels, factors 2, 4, 8,
    images that want only some of the gradients (K1 runs only for d I_h)."""
    specs = synth.mixed_sizes(seed=11, n=10, long_lo=64, long_hi=420, radii=(1, 2, 4, 8), factors=(2, 4, 8))
    needs = [(True, True, True), (True, False, True), (False, True, False), (False, False, True),
             (True, True, False)]
    images, grads = [], []
    for i, s in enumerate(specs):
        d = to_storage(synth.photo_like(130 + i, 1, 3, s.h_l, s.w_l, s.f), dtype)
        np_, nl, nh = needs[i % len(needs)]
        images.append({"p_l": d["p_l"][0].cuda(), "I_l": d["I_l"][0].cuda(), "I_h": d["I_h"][0].cuda(),
                       "r": s.r, "eps": 1e-3, "need_p": np_, "need_Il": nl, "need_Ih": nh})
        grads.append(synth.upstream_grad(150 + i, d["I_h"].shape).to(dtype)[0].cuda())
    try:
        L.dgf_set_batched_graph_backward(False)
        chains = gf_backward_batched(images, grads)
        torch.cuda.synchronize()
    finally:
        L.dgf_set_batched_graph_backward(True)
    launches = L.dgf_launch_count()
    for rep in range(2):
        outs = gf_backward_batched(images, grads)
        torch.cuda.synchronize()
        for im, R, o, c in zip(images, grads, outs, chains):
            single = gf_backward(R[None], im["p_l"][None], im["I_l"][None], im["I_h"][None], im["r"], im["eps"],
                                 need_p=im["need_p"], need_Il=im["need_Il"], need_Ih=im["need_Ih"])
            for a, b, cc in zip(o, single[:3], c):
                assert (a is None) == (b is None) == (cc is None)
                if a is not None:
                    assert torch.equal(a, b[0]) and torch.equal(a, cc)
    assert L.dgf_launch_count() > launches


# the layer as printed (no box mean of A, b): every low-res kernel form that
# supports it (strips for r in {1, 2}, generic tiles otherwise)
LIT_CASES = [("photo", 1, 2, 70, 90, 280, 360, 1, 1e-3), ("photo", 1, 2, 40, 44, 320, 352, 2, 1e-3),
             ("ragged", 1, 1, 37, 53, 150, 211, 1, 1e-3), ("photo", 1, 2, 50, 70, 200, 280, 3, 1e-3),
             ("photo", 1, 1, 36, 300, 144, 1200, 4, 1e-3), ("photo", 1, 1, 48, 40, 192, 160, 8, 1e-3),
             ("photo", 1, 1, 30, 36, 120, 144, 0, 1e-2)]


@pytest.mark.parametrize("dtype", [F32, BF16], ids=["f32", "bf16"])
@pytest.mark.parametrize("case", LIT_CASES, ids=_ids(LIT_CASES))
def test_paper_literal_variant_parity(case, dtype):
    kind, N, C, hl, wl, h, w, r, eps = case
    st = to_storage(make_case(kind, 300 + r, N, C, hl, wl, h, w), dtype)
    R = synth.upstream_grad(9, st["I_h"].shape).to(dtype)
    g = {k: v.cuda() for k, v in st.items()}
    out = gf_forward(g["p_l"], g["I_l"], g["I_h"], r, eps, mean_ab=False)
    dp, dIl, dIh, _ = gf_backward(R.cuda(), g["p_l"], g["I_l"], g["I_h"], r, eps, mean_ab=False)
    torch.cuda.synchronize()
    ref = O.forward(f64(st["p_l"]), f64(st["I_l"]), f64(st["I_h"]), r, eps, mean_ab=False)
    assert_fwd(f64(out), ref, dtype, eps)
    rp, rIl, rIh = O.backward(f64(R), f64(st["p_l"]), f64(st["I_l"]), f64(st["I_h"]), r, eps, mean_ab=False)
    assert_grad(f64(dp), rp, dtype, "dp_l")
    if r > 0:
        assert_grad(f64(dIl), rIl, dtype, "dI_l")
    assert_grad(f64(dIh), rIh, dtype, "dI_h")
    if r > 0:  # and it is not the default form
        assert not torch.equal(out, gf_forward(g["p_l"], g["I_l"], g["I_h"], r, eps))


# grey guide (Sec. 4.2, DGF_b with differing channel counts): kind, N, guide
# channels, output channels, h_l, w_l, h, w, r, eps, mean_ab
GREY_CASES = [("photo", 2, 3, 1, 40, 50, 160, 200, 1, 1e-3, True),     # RGB guide, one output channel
              ("photo", 1, 3, 1, 45, 70, 360, 560, 2, 1e-3, True),     # f = 8, r = 2
              ("photo", 2, 1, 3, 30, 33, 120, 132, 1, 1e-2, True),     # one guide channel, three outputs
              ("ragged", 1, 3, 2, 37, 53, 150, 211, 1, 1e-3, True),    # non-integer ratio, odd width
              ("photo", 1, 3, 1, 20, 24, 80, 96, 1, 1e-3, False)]      # the layer as printed


@pytest.mark.parametrize("dtype", [F32, BF16, F16], ids=["f32", "bf16", "f16"])
@pytest.mark.parametrize("case", GREY_CASES, ids=_ids(GREY_CASES))
def test_grey_guide_parity(case, dtype):
    kind, N, n_in, C, hl, wl, h, w, r, eps, mean_ab = case
    gsrc = to_storage(make_case(kind, 400 + r, N, n_in, hl, wl, h, w), dtype)
    psrc = to_storage(make_case(kind, 410 + r, N, C, hl, wl, h, w), dtype)
    p_l, I_l, I_h = psrc["p_l"], gsrc["I_l"], gsrc["I_h"]
    R = synth.upstream_grad(11, (N, C, h, w)).to(dtype)
    out = gf_forward(p_l.cuda(), I_l.cuda(), I_h.cuda(), r, eps, mean_ab=mean_ab)
    dp, dIl, dIh, _ = gf_backward(R.cuda(), p_l.cuda(), I_l.cuda(), I_h.cuda(), r, eps, mean_ab=mean_ab)
    torch.cuda.synchronize()
    assert out.shape == (N, C, h, w) and dIl.shape == I_l.shape and dIh.shape == I_h.shape
    ref = O.forward_grey(f64(p_l), f64(I_l), f64(I_h), r, eps, mean_ab=mean_ab)
    assert_fwd(f64(out), ref, dtype, eps)
    rp, rIl, rIh = O.backward_grey(f64(R), f64(p_l), f64(I_l), f64(I_h), r, eps, mean_ab=mean_ab)
    assert_grad(f64(dp), rp, dtype, "dp_l")
    assert_grad(f64(dIl), rIl, dtype, "dI_l")
    assert_grad(f64(dIh), rIh, dtype, "dI_h")
    # every guide channel receives the same gradient
    for k in range(1, n_in):
        assert torch.equal(dIh[:, k], dIh[:, 0]) and torch.equal(dIl[:, k], dIl[:, 0])
    assert L.dgf_device_status() == 0


# grey cases of the folded high-resolution kernels (integer factor 2, 4, 8;
# partial tiles in both directions): kind, N, guide channels, output
# channels, h_l, w_l, h, w, r, eps
GREY_FOLD_CASES = [("photo", 2, 3, 1, 37, 62, 148, 248, 1, 1e-3),   # f = 4, RGB guide -> one channel
                   ("photo", 1, 3, 1, 45, 70, 360, 560, 2, 1e-3),   # f = 8 (FP32: the streaming form)
                   ("photo", 1, 2, 3, 33, 50, 66, 100, 1, 1e-3),    # f = 2, two guide channels -> three
                   ("photo", 2, 4, 2, 20, 64, 80, 256, 4, 1e-3)]    # f = 4, r = 4, four -> two


def _grey_run(p_l, I_l, I_h, R, r, eps):
    L.dgf_profile_reset()
    L.dgf_profile_enable(True)
    try:
        out = gf_forward(p_l, I_l, I_h, r, eps)
        dp, dIl, dIh, _ = gf_backward(R, p_l, I_l, I_h, r, eps)
        torch.cuda.synchronize()
        names = set(L.dgf_profile_read().keys())
    finally:
        L.dgf_profile_enable(False)
    return (out, dp, dIl, dIh), names


@pytest.mark.parametrize("dtype", [F32, BF16, F16], ids=["f32", "bf16", "f16"])
@pytest.mark.parametrize("case", GREY_FOLD_CASES, ids=_ids(GREY_FOLD_CASES))
def test_grey_fold_matches_oracle_and_streaming_form(case, dtype):
    kind, N, n_in, C, hl, wl, h, w, r, eps = case
    gsrc = to_storage(make_case(kind, 420 + r, N, n_in, hl, wl, h, w), dtype)
    psrc = to_storage(make_case(kind, 430 + r, N, C, hl, wl, h, w), dtype)
    p_l, I_l, I_h = (t.cuda() for t in (psrc["p_l"], gsrc["I_l"], gsrc["I_h"]))
    R = synth.upstream_grad(13, (N, C, h, w)).to(dtype)
    folded = not (dtype == F32 and h // hl == 8)
    res, names = _grey_run(p_l, I_l, I_h, R.cuda(), r, eps)
    assert ({"k2_grey_apply", "k3_grey_bwd"} <= names) == folded, names
    out, dp, dIl, dIh = res
    ref = O.forward_grey(f64(p_l), f64(I_l), f64(I_h), r, eps)
    assert_fwd(f64(out), ref, dtype, eps)
    rp, rIl, rIh = O.backward_grey(f64(R), f64(p_l), f64(I_l), f64(I_h), r, eps)
    assert_grad(f64(dp), rp, dtype, "dp_l")
    assert_grad(f64(dIl), rIl, dtype, "dI_l")
    assert_grad(f64(dIh), rIh, dtype, "dI_h")
    for k in range(1, n_in):
        assert torch.equal(dIh[:, k], dIh[:, 0]) and torch.equal(dIl[:, k], dIl[:, 0])
    assert L.dgf_device_status() == 0
    # the streaming form (grey guide formed in the workspace) meets the same
    # gates, and the two forms agree within them
    L.dgf_set_grey_fold(False)
    try:
        res2, names2 = _grey_run(p_l, I_l, I_h, R.cuda(), r, eps)
    finally:
        L.dgf_set_grey_fold(True)
    assert "k2_grey_apply" not in names2 and "k3_grey_bwd" not in names2
    assert_fwd(f64(res2[0]), ref, dtype, eps)
    assert_fwd(f64(out), f64(res2[0]), dtype, eps)
    for a, b, ro, name in zip(res[1:], res2[1:], (rp, rIl, rIh), ("dp_l", "dI_l", "dI_h")):
        assert_grad(f64(b), ro, dtype, name)
    assert L.dgf_device_status() == 0


def test_paper_literal_guided_parity():
    N, C, hl, wl, f, r, eps = 1, 3, 24, 32, 4, 2, 1e-3
    st = {k: v.to(BF16) for k, v in synth.photo_like(61, N, C, hl, wl, f).items()}
    w = {k: v.float() for k, v in synth.guide_weights(62).items()}
    R = synth.upstream_grad(63, st["I_h"].shape).to(BF16)
    g = {k: v.cuda() for k, v in st.items()}
    wc = {k: v.cuda() for k, v in w.items()}
    out = gf_forward(g["p_l"], None, g["I_h"], r, eps, wc["w1"], wc["w2"], wc["b2"], 0.2, mean_ab=False)
    dp, _, dIh, dws = gf_backward(R.cuda(), g["p_l"], None, g["I_h"], r, eps, wc["w1"], wc["w2"], wc["b2"], 0.2,
                                  mean_ab=False)
    torch.cuda.synchronize()
    w64 = {k: v.double().numpy() for k, v in w.items()}
    ref = O.forward_guided(f64(st["p_l"]), f64(st["I_h"]), w64["w1"], w64["w2"], w64["b2"], r, eps, mean_ab=False)
    assert_fwd(f64(out), ref, BF16, eps)
    rp, rI, rw1, rw2, _ = O.backward_guided(f64(R), f64(st["p_l"]), f64(st["I_h"]), w64["w1"], w64["w2"],
                                            w64["b2"], r, eps, mean_ab=False)
    assert_grad(f64(dp), rp, BF16, "dp_l")
    assert_grad(f64(dIh), rI, BF16, "dI_h")
    assert rel_l2(f64(dws[0]), rw1) <= 2e-2
    assert rel_l2(f64(dws[1]), rw2) <= 2e-2


def test_forced_wait_timeout_is_reported_and_sticky():
    # Every first wait of a kernel on one of its TMA copies gives up at once
    # (0 polls): the kernels record a timeout, wait for the copies they have
    # in flight (that wait keeps its full limit, so every copy lands) and
    # stop.  Nothing is starved and nothing faults; the call's results are
    # invalid, and the next call on the device fails with DGF_ERR_TIMEOUT
    # until the status is cleared.
    st = to_storage(make_case("photo", 12, 1, 3, 64, 96, 256, 384), F32)
    R = synth.upstream_grad(13, st["I_h"].shape).float().cuda()
    g = {k: v.cuda() for k, v in st.items()}
    ref = gf_forward(g["p_l"], g["I_l"], g["I_h"], 1, 1e-3)
    refb = gf_backward(R, g["p_l"], g["I_l"], g["I_h"], 1, 1e-3)[:3]
    torch.cuda.synchronize()
    assert L.dgf_device_status() == 0
    try:
        L.check(L.dgf_set_wait_polls(0))
        gf_backward(R, g["p_l"], g["I_l"], g["I_h"], 1, 1e-3)  # K13 and K4 stage rows by TMA
        torch.cuda.synchronize()
        assert L.dgf_device_status() & 1
        with pytest.raises(L.DGFError) as e:
            gf_forward(g["p_l"], g["I_l"], g["I_h"], 1, 1e-3)
        assert e.value.status == 4 and "wait" in str(e.value)
        with pytest.raises(L.DGFError) as e:  # sticky: every later call
            gf_backward(R, g["p_l"], g["I_l"], g["I_h"], 1, 1e-3)
        assert e.value.status == 4
    finally:
        L.check(L.dgf_set_wait_polls(1 << 22))
        L.check(L.dgf_clear_device_status())
    out = gf_forward(g["p_l"], g["I_l"], g["I_h"], 1, 1e-3)
    outb = gf_backward(R, g["p_l"], g["I_l"], g["I_h"], 1, 1e-3)[:3]
    torch.cuda.synchronize()
    assert L.dgf_device_status() == 0
    assert torch.equal(out, ref)
    for a, b in zip(outb, refb):
        assert torch.equal(a, b)
    assert_fwd(f64(out), oracle_forward(st, 1, 1e-3), F32, 1e-3)
    with pytest.raises(L.DGFError):
        L.check(L.dgf_set_wait_polls(-1))


def test_invalid_arguments_report_status():
    st = to_storage(make_case("photo", 9, 1, 1, 8, 8, 32, 32), F32)
    g = {k: v.cuda() for k, v in st.items()}
    with pytest.raises(L.DGFError) as e:
        gf_forward(g["p_l"], g["I_l"], g["I_h"], -1, 1e-3)
    assert e.value.status == 1
    with pytest.raises(L.DGFError) as e:
        gf_forward(g["p_l"], g["I_l"], g["I_h"], 1, 0.0)
    assert e.value.status == 1
    with pytest.raises(L.DGFError) as e:
        gf_forward(g["p_l"], g["I_l"], g["I_h"], 17, 1e-3)
    assert e.value.status == 2


# ------------------------------------------------------ guidance transform
GUIDED_CASES = [  # N, h_l, w_l, f, r, eps, dtype
    (2, 24, 20, 4, 1, 1e-3, F32),
    (1, 20, 30, 8, 2, 1e-4, BF16),
    (2, 16, 29, 8, 8, 1e-4, BF16),   # r = 8 as in the training configuration; ragged K3 tile
    (1, 26, 18, 4, 1, 1e-3, F16),
    (1, 22, 26, 2, 1, 1e-3, F32),    # f = 2
    (2, 18, 30, 2, 2, 1e-3, BF16),   # f = 2, 8-byte vectors
    (2, 16, 29, 4, 8, 1e-4, F32),    # r = 8 as in the training configuration, FP32 (f = 4: FP32 vectors hold 4 pixels); ragged
]


@pytest.mark.parametrize("case", GUIDED_CASES, ids=_ids(GUIDED_CASES))
def test_guided_forward_backward_parity(case):
    N, hl, wl, f, r, eps, dtype = case
    d = synth.photo_like(60 + r, N, 3, hl, wl, f)
    st = to_storage(d, dtype)
    gw = synth.guide_weights(11)
    w = {k: v.float() for k, v in gw.items()}
    R = synth.upstream_grad(12, st["I_h"].shape).to(dtype)
    g = {k: v.cuda() for k, v in st.items()}
    wc = {k: v.cuda() for k, v in w.items()}
    out = gf_forward(g["p_l"], None, g["I_h"], r, eps, wc["w1"], wc["w2"], wc["b2"], 0.2)
    dp, _, dIh, dws = gf_backward(R.cuda(), g["p_l"], None, g["I_h"], r, eps, wc["w1"], wc["w2"],
                                  wc["b2"], 0.2)
    torch.cuda.synchronize()
    w64 = {k: v.double().numpy() for k, v in w.items()}
    ref = O.forward_guided(f64(st["p_l"]), f64(st["I_h"]), w64["w1"], w64["w2"], w64["b2"], r, eps)
    assert_fwd(f64(out), ref, dtype, eps if dtype != F32 else max(eps, 1e-3))
    rp, rI, rw1, rw2, rb2 = O.backward_guided(f64(R), f64(st["p_l"]), f64(st["I_h"]), w64["w1"],
                                              w64["w2"], w64["b2"], r, eps)
    assert_grad(f64(dp), rp, dtype, "dp_l")
    assert_grad(f64(dIh), rI, dtype, "dI_h")
    wtol = TOL_F32_REL_L2 if dtype == F32 else 2e-2
    for got, refw, name in ((dws[0], rw1, "dw1"), (dws[1], rw2, "dw2")):
        err = float(np.linalg.norm(f64(got) - refw) / np.linalg.norm(refw))
        assert err <= wtol, f"{name}: rel L2 {err:.3e}"
    # the guide-shift invariance makes db2 vanish; compare on the scale of dw2
    assert float(np.max(np.abs(f64(dws[2])))) <= 1e-3 * float(np.max(np.abs(rw2)))


# the transform applied to each guide on its own (G_l = F(I_l), guide_low)
GUIDED_LOW_CASES = [  # N, h_l, w_l, f, r, eps, dtype, mean_ab
    (2, 24, 20, 4, 1, 1e-3, F32, True),
    (1, 20, 30, 8, 2, 1e-4, BF16, True),
    (1, 26, 18, 4, 1, 1e-3, F16, True),
    (1, 16, 22, 4, 1, 1e-3, F32, False),
]


@pytest.mark.parametrize("case", GUIDED_LOW_CASES, ids=_ids(GUIDED_LOW_CASES))
def test_guided_low_guide_parity(case):
    N, hl, wl, f, r, eps, dtype, mean_ab = case
    st = to_storage(synth.photo_like(70 + r, N, 3, hl, wl, f), dtype)
    w = {k: v.float() for k, v in synth.guide_weights(13).items()}
    R = synth.upstream_grad(14, st["I_h"].shape).to(dtype)
    g = {k: v.cuda() for k, v in st.items()}
    wc = {k: v.cuda() for k, v in w.items()}
    args = (wc["w1"], wc["w2"], wc["b2"], 0.2)
    out = gf_forward(g["p_l"], g["I_l"], g["I_h"], r, eps, *args, mean_ab=mean_ab, guide_low=True)
    dp, dIl, dIh, dws = gf_backward(R.cuda(), g["p_l"], g["I_l"], g["I_h"], r, eps, *args, mean_ab=mean_ab,
                                    guide_low=True)
    # d I_l alone (the low-res chain without K6) and d W alone give the same values
    only_il = gf_backward(R.cuda(), g["p_l"], g["I_l"], g["I_h"], r, eps, *args, need_p=False, need_Ih=False,
                          need_w=False, mean_ab=mean_ab, guide_low=True)[1]
    only_w = gf_backward(R.cuda(), g["p_l"], g["I_l"], g["I_h"], r, eps, *args, need_p=False, need_Il=False,
                         need_Ih=False, mean_ab=mean_ab, guide_low=True)[3]
    torch.cuda.synchronize()
    assert torch.equal(only_il, dIl)
    for a, b in zip(only_w, dws):
        assert torch.equal(a, b)
    w64 = {k: v.double().numpy() for k, v in w.items()}
    ref = O.forward_guided_separate(f64(st["p_l"]), f64(st["I_l"]), f64(st["I_h"]), w64["w1"], w64["w2"],
                                    w64["b2"], r, eps, mean_ab=mean_ab)
    assert_fwd(f64(out), ref, dtype, eps if dtype != F32 else max(eps, 1e-3))
    rp, rIl, rIh, rw1, rw2, rb2 = O.backward_guided_separate(f64(R), f64(st["p_l"]), f64(st["I_l"]),
                                                             f64(st["I_h"]), w64["w1"], w64["w2"], w64["b2"],
                                                             r, eps, mean_ab=mean_ab)
    assert_grad(f64(dp), rp, dtype, "dp_l")
    assert_grad(f64(dIl), rIl, dtype, "dI_l")
    assert_grad(f64(dIh), rIh, dtype, "dI_h")
    wtol = TOL_F32_REL_L2 if dtype == F32 else 2e-2
    for got, refw, name in ((dws[0], rw1, "dw1"), (dws[1], rw2, "dw2")):
        err = float(np.linalg.norm(f64(got) - refw) / np.linalg.norm(refw))
        assert err <= wtol, f"{name}: rel L2 {err:.3e}"
    assert float(np.max(np.abs(f64(dws[2])))) <= 1e-3 * float(np.max(np.abs(rw2)))
    # and it is not the block-mean form
    assert not torch.equal(out, gf_forward(g["p_l"], None, g["I_h"], r, eps, *args, mean_ab=mean_ab))
    assert L.dgf_device_status() == 0


# ------------------------------------------------------------ shape invariance
# The K1 strips sum their register rings oldest row first and do their pair
# arithmetic through non-contracting intrinsics, so every segment length the
# autotuner may pick gives the same bits; the column-walking tiles compute the
# same formula with other rounding, so across tile shapes only the last place
# or two may move.
K1_SHAPES = {"strips": [(8, 0), (24, 0), (32, 0), (64, 0)], "tiles": [(64, 32), (128, 16), (64, 64)]}


def _close_bits(a, b, dtype):
    """Same values up to a few ulp of FP32 arithmetic (stored in dtype)."""
    d = (a.float() - b.float()).abs().max().item()
    tol = 2e-6 if dtype == F32 else (2 ** -7 if dtype == BF16 else 2 ** -10)
    assert d <= tol, (d, tol)


@pytest.mark.parametrize("form", ["strips", "tiles"])
@pytest.mark.parametrize("dtype,r,eps", [(F32, 1, 1e-4), (BF16, 2, 1e-3)], ids=["f32-r1", "bf16-r2"])
def test_forward_does_not_depend_on_k1_shape(form, dtype, r, eps, pin):
    dt = L.DGF_F32 if dtype == F32 else L.DGF_BF16
    st = to_storage(make_case("photo", 41, 2, 2, 77, 150, 308, 600), dtype)
    g = {k: v.cuda() for k, v in st.items()}
    L.dgf_set_fused(False)  # the two-kernel form, whose K1 shape is under test
    try:
        outs = []
        for a, b in K1_SHAPES[form]:
            L.dgf_autotune_reset()
            pin(1, dt, r, 0, 0, 0, a, b)
            outs.append(gf_forward(g["p_l"], g["I_l"], g["I_h"], r, eps))
        torch.cuda.synchronize()
    finally:
        L.dgf_set_fused(True)
    for o in outs[1:]:
        if form == "strips":
            assert torch.equal(o, outs[0])
        else:
            _close_bits(o, outs[0], dtype)
    assert_fwd(f64(outs[0]), oracle_forward(st, r, eps), dtype, eps)


# --------------------------------------------------------------- fused forward
# (dtype, N, C, h_l, w_l, F, r, eps): every factor / radius / dtype the fused
# kernel serves, ragged against its 32-column strips and its segments
K12_CASES = [(F32, 2, 3, 70, 90, 4, 1, 1e-4), (F32, 1, 2, 77, 131, 2, 2, 1e-3), (BF16, 2, 2, 45, 70, 8, 1, 1e-3),
             (BF16, 1, 3, 54, 96, 4, 2, 1e-3), (F16, 2, 1, 33, 40, 4, 2, 1e-2), (F32, 1, 1, 5, 3, 4, 1, 1e-2)]


@pytest.mark.parametrize("ls", [8, 32])
@pytest.mark.parametrize("case", K12_CASES, ids=_ids(K12_CASES))
def test_fused_forward_equals_two_kernel_forward(case, ls, pin):
    dtype, N, C, hl, wl, f, r, eps = case
    dt = {F32: L.DGF_F32, BF16: L.DGF_BF16, F16: L.DGF_F16}[dtype]
    st = to_storage(make_case("photo", 60 + r, N, C, hl, wl, hl * f, wl * f), dtype)
    g = {k: v.cuda() for k, v in st.items()}
    pin(1, dt, r, 0, 0, 0, 32, 0)        # the two-kernel form with K1 strips
    pin(5, dt, r, f, 0, 0, ls, 0)        # K12 segment length
    L.dgf_set_fused(False)
    try:
        ref = gf_forward(g["p_l"], g["I_l"], g["I_h"], r, eps)
    finally:
        L.dgf_set_fused(True)
    out = gf_forward(g["p_l"], g["I_l"], g["I_h"], r, eps)
    torch.cuda.synchronize()
    assert torch.equal(out, ref)
    assert_fwd(f64(out), oracle_forward(st, r, eps), dtype, eps)
    assert L.dgf_device_status() == 0


# ------------------------------------------------------- plane-group pipeline
@pytest.mark.parametrize("dtype,r,planes", [(F32, 1, (2, 3)), (BF16, 2, (1, 2)), (F32, 2, (1, 7))],
                         ids=["f32-r1-6", "bf16-r2-2", "f32-r2-7"])
def test_plane_group_pipeline_gives_the_same_bits(dtype, r, planes):
    N, C = planes
    st = to_storage(make_case("photo", 70 + r, N, C, 45, 70, 180, 280), dtype)
    R = synth.upstream_grad(71, st["I_h"].shape).to(dtype).cuda()
    g = {k: v.cuda() for k, v in st.items()}
    res = []
    for on in (False, True, True):  # the first pipelined call may tune on one stream
        L.dgf_set_pipeline(on)
        try:
            out = gf_forward(g["p_l"], g["I_l"], g["I_h"], r, 1e-3)
            grads = gf_backward(R, g["p_l"], g["I_l"], g["I_h"], r, 1e-3)[:3]
            torch.cuda.synchronize()
        finally:
            L.dgf_set_pipeline(False)
        res.append((out, *grads))
    for a, b in zip(res[0], res[2]):
        assert torch.equal(a, b)
    assert L.dgf_device_status() == 0


# -------------------------------------------------------------- fused backward
# (dtype, N, C, h_l, w_l, F, r, eps): the K3 strips the fused backward serves
# (16-byte vectors, one low-res cell per lane), ragged against its 30-cell
# strips and its segments
K13_CASES = [(F32, 2, 3, 70, 90, 4, 1, 1e-4), (F32, 1, 2, 77, 131, 4, 2, 1e-3), (BF16, 2, 2, 45, 70, 8, 1, 1e-3),
             (BF16, 1, 3, 54, 96, 8, 2, 1e-3), (F16, 1, 2, 33, 40, 8, 1, 1e-2), (F32, 1, 1, 5, 3, 4, 1, 1e-2)]


@pytest.mark.parametrize("k4_form", ["strips", "tiles"])
@pytest.mark.parametrize("ls", [8, 24])
@pytest.mark.parametrize("case", K13_CASES, ids=_ids(K13_CASES))
def test_fused_backward_equals_two_kernel_backward(case, ls, k4_form, pin):
    dtype, N, C, hl, wl, f, r, eps = case
    dt = {F32: L.DGF_F32, BF16: L.DGF_BF16, F16: L.DGF_F16}[dtype]
    vec = 16 // (4 if dtype == F32 else 2)
    st = to_storage(make_case("photo", 80 + r, N, C, hl, wl, hl * f, wl * f), dtype)
    R = synth.upstream_grad(81, st["I_h"].shape).to(dtype)
    g = {k: v.cuda() for k, v in st.items()}
    pin(1, dt, r, 0, 0, 0, 32, 0)                 # K1 strips
    if k4_form == "tiles":
        pin(4, dt, r, 0, 0, 0, 64, 16)            # K4 recomputing its statistics: none saved
    pin(6, dt, r, f, vec, 0, ls, 0)               # K13 segment length
    L.dgf_set_fused(False)
    try:
        ref = gf_backward(R.cuda(), g["p_l"], g["I_l"], g["I_h"], r, eps)[:3]
    finally:
        L.dgf_set_fused(True)
    out = gf_backward(R.cuda(), g["p_l"], g["I_l"], g["I_h"], r, eps)[:3]
    torch.cuda.synchronize()
    for a, b in zip(out, ref):
        assert torch.equal(a, b)
    rp, rIl, rIh = oracle_backward(R, st, r, eps)
    assert_grad(f64(out[0]), rp, dtype, "dp_l")
    assert_grad(f64(out[1]), rIl, dtype, "dI_l")
    assert_grad(f64(out[2]), rIh, dtype, "dI_h")
    assert L.dgf_device_status() == 0


# the forward's coefficients kept for the backward (dgf_options.coef): kind,
# N, C (output), guide channels, h_l, w_l, h, w, r, eps, dtype, mean_ab, reuses
KEEP_CASES = [
    ("photo", 2, 3, 3, 45, 70, 180, 280, 2, 1e-3, BF16, True, True),    # sliding K1/K4
    ("photo", 1, 2, 2, 40, 36, 320, 288, 8, 1e-3, F16, True, True),     # f = 8, r = 8
    ("photo", 1, 1, 1, 64, 64, 256, 256, 1, 1e-2, BF16, True, True),
    ("photo", 2, 3, 3, 40, 50, 160, 200, 1, 1e-3, F32, True, False),    # FP32 r = 1: K13, statistics
    ("photo", 1, 2, 2, 36, 60, 144, 240, 4, 1e-3, F32, True, True),     # FP32 tiles at r = 4
    ("photo", 1, 2, 2, 30, 40, 120, 160, 2, 1e-3, BF16, False, False),  # the layer as printed: strips, statistics
    ("ragged", 1, 2, 2, 37, 53, 150, 211, 1, 1e-3, BF16, True, True),   # non-integer ratio
    ("photo", 2, 1, 3, 37, 62, 148, 248, 1, 1e-3, BF16, True, True),    # grey guide, folded
    ("ragged", 1, 2, 3, 37, 53, 150, 211, 1, 1e-3, F16, True, True),    # grey guide, streaming form
]


@pytest.mark.parametrize("case", KEEP_CASES, ids=_ids(KEEP_CASES))
@pytest.mark.parametrize("pipeline", [False, True], ids=["onestream", "pipeline"])
def test_kept_coefficients_give_the_same_bits(case, pipeline):
    kind, N, C, n_in, hl, wl, h, w, r, eps, dtype, mean_ab, reuses = case
    gsrc = to_storage(make_case(kind, 440 + r, N, n_in, hl, wl, h, w), dtype)
    psrc = to_storage(make_case(kind, 450 + r, N, C, hl, wl, h, w), dtype)
    p_l, I_l, I_h = (t.cuda() for t in (psrc["p_l"], gsrc["I_l"], gsrc["I_h"]))
    R = synth.upstream_grad(15, (N, C, h, w)).to(dtype).cuda()
    from paper_1803_05619_gb300.layer import backward_reuses_coef, coef_buffer
    assert backward_reuses_coef(p_l, I_h, r, mean_ab=mean_ab) == reuses
    L.dgf_set_pipeline(pipeline)
    try:
        out = gf_forward(p_l, I_l, I_h, r, eps, mean_ab=mean_ab)
        ref = gf_backward(R, p_l, I_l, I_h, r, eps, mean_ab=mean_ab)[:3]
        cf = coef_buffer(p_l, I_h)
        out_k = gf_forward(p_l, I_l, I_h, r, eps, mean_ab=mean_ab, coef=cf)
        got = gf_backward(R, p_l, I_l, I_h, r, eps, mean_ab=mean_ab, coef=cf)[:3]
        only_ih = gf_backward(R, p_l, I_l, I_h, r, eps, mean_ab=mean_ab, coef=cf, need_p=False,
                              need_Il=False)[2]
        torch.cuda.synchronize()
    finally:
        L.dgf_set_pipeline(False)
    assert torch.equal(out_k, out)
    for a, b in zip(got, ref):
        assert torch.equal(a, b)
    assert torch.equal(only_ih, ref[2])
    assert L.dgf_device_status() == 0


@pytest.mark.parametrize("guide_low", [False, True], ids=["blockmean", "guide_low"])
@pytest.mark.parametrize("dtype", [F32, BF16], ids=["f32", "bf16"])
def test_kept_coefficients_guided(dtype, guide_low):
    # the guided backward takes Abar (for K6) and G_l (for K4) from the
    # forward: no K1 and no guide pass
    N, hl, wl, f, r, eps = 2, 20, 30, 4, 2, 1e-4
    st = {k: v.to(dtype).cuda() for k, v in synth.photo_like(73, N, 3, hl, wl, f).items()}
    wc = {k: v.float().cuda() for k, v in synth.guide_weights(17).items()}
    R = synth.upstream_grad(18, st["I_h"].shape).to(dtype).cuda()
    args = (wc["w1"], wc["w2"], wc["b2"], 0.2)
    I_l = st["I_l"] if guide_low else None
    from paper_1803_05619_gb300.layer import coef_buffer
    out = gf_forward(st["p_l"], I_l, st["I_h"], r, eps, *args, guide_low=guide_low)
    ref = gf_backward(R, st["p_l"], I_l, st["I_h"], r, eps, *args, guide_low=guide_low)
    cf = coef_buffer(st["p_l"], st["I_h"], guided=True)
    out_k = gf_forward(st["p_l"], I_l, st["I_h"], r, eps, *args, guide_low=guide_low, coef=cf)
    L.dgf_profile_reset()
    L.dgf_profile_enable(True)
    try:
        got = gf_backward(R, st["p_l"], I_l, st["I_h"], r, eps, *args, guide_low=guide_low, coef=cf)
        torch.cuda.synchronize()
        names = set(L.dgf_profile_read().keys())
    finally:
        L.dgf_profile_enable(False)
    assert not names & {"k1_lowres_coef", "k5_guide_down", "k5_guide_low"}, names
    assert torch.equal(out_k, out)
    for k in (0, 1, 2):
        assert (got[k] is None and ref[k] is None) or torch.equal(got[k], ref[k])
    for a, b in zip(got[3], ref[3]):
        assert torch.equal(a, b)


@pytest.mark.parametrize("dtype", [F32, BF16], ids=["f32", "bf16"])
def test_kept_coefficients_batched(dtype):
    # the batched forward writes each image's coefficients to its buffer and
    # the batched backward takes them (the one-graph form skips those images'
    # K1 work items): the bits of the calls without them
    from paper_1803_05619_gb300.layer import coef_buffer
    specs = synth.mixed_sizes(seed=9, n=5, long_lo=96, long_hi=400)
    images, grads = [], []
    for i, s in enumerate(specs):
        d = to_storage(synth.photo_like(110 + i, 1, 3, s.h_l, s.w_l, s.f), dtype)
        images.append({"p_l": d["p_l"][0].cuda(), "I_l": d["I_l"][0].cuda(), "I_h": d["I_h"][0].cuda(),
                       "r": s.r, "eps": 1e-3})
        grads.append(synth.upstream_grad(120 + i, d["I_h"].shape).to(dtype)[0].cuda())
    outs = gf_forward_batched(images)
    ref = gf_backward_batched(images, grads)
    kept = [dict(im, coef=coef_buffer(im["p_l"][None], im["I_h"][None])) for im in images]
    kept[1]["coef"] = None  # one image recomputes them
    outs_k = gf_forward_batched(kept)
    got = gf_backward_batched(kept, grads)
    torch.cuda.synchronize()
    for a, b in zip(outs_k, outs):
        assert torch.equal(a, b)
    for ga, gb in zip(got, ref):
        for a, b in zip(ga, gb):
            assert torch.equal(a, b)
    assert L.dgf_device_status() == 0

