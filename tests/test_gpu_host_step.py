"""dgf_host_step: forward + backward of a batch in host memory, pipelined over
plane groups, against the device-memory calls (bitwise) and the oracle."""
import pytest
import torch

import synth
from paper_1803_05619_gb300 import _lib as L
from paper_1803_05619_gb300.layer import gf_backward, gf_forward, gf_step_host, workspace
from tests.helpers import assert_fwd, assert_grad, f64, make_case, oracle_backward, oracle_forward, to_storage

pytestmark = pytest.mark.gpu

F32, BF16, F16 = torch.float32, torch.bfloat16, torch.float16

# dtype, N, C, h_l, w_l, f, r, eps, groups
CASES = [
    (F32, 2, 3, 40, 50, 4, 1, 1e-3, 0),     # default groups (6 planes -> 6)
    (F32, 2, 3, 40, 50, 4, 1, 1e-3, 4),     # groups of 1 and 2 planes
    (F32, 1, 2, 37, 45, 4, 2, 1e-3, 16),    # more groups than planes; odd low-res plane bytes
    (BF16, 1, 3, 37, 45, 4, 2, 1e-3, 2),    # ragged: groups of 1 and 2 planes
    (BF16, 2, 2, 20, 24, 8, 1, 1e-3, 3),    # f = 8
    (F16, 3, 1, 21, 33, 4, 1, 1e-2, 1),     # one group: no overlap
]


def _ids(cases):
    return [f"{str(c[0]).split('.')[-1]}-{c[1]}x{c[2]}x{c[3]}x{c[4]}-f{c[5]}-r{c[6]}-g{c[8]}" for c in cases]


def _host(t, pinned):
    return t.contiguous().pin_memory() if pinned else t.contiguous().clone()


@pytest.mark.parametrize("pinned", [True, False], ids=["pinned", "pageable"])
@pytest.mark.parametrize("case", CASES, ids=_ids(CASES))
def test_host_step_equals_device_calls(case, pinned):
    dtype, N, C, hl, wl, f, r, eps, groups = case
    st = to_storage(make_case("photo", 60 + r, N, C, hl, wl, hl * f, wl * f), dtype)
    R = synth.upstream_grad(61, st["I_h"].shape).to(dtype)
    g = {k: v.cuda() for k, v in st.items()}
    ref_O = gf_forward(g["p_l"], g["I_l"], g["I_h"], r, eps)
    ref = gf_backward(R.cuda(), g["p_l"], g["I_l"], g["I_h"], r, eps)[:3]
    torch.cuda.synchronize()
    h = {k: _host(v, pinned) for k, v in st.items()}
    out = gf_step_host(h["p_l"], h["I_l"], h["I_h"], _host(R, pinned), r, eps, groups=groups)
    assert all(not t.is_cuda for t in out)
    assert torch.equal(out[0], ref_O.cpu())
    for a, b in zip(out[1:], ref):
        assert torch.equal(a, b.cpu())
    # and against the oracle
    assert_fwd(f64(out[0]), oracle_forward(st, r, eps), dtype, eps)
    rp, rIl, rIh = oracle_backward(R, st, r, eps)
    assert_grad(f64(out[1]), rp, dtype, "dp_l")
    assert_grad(f64(out[2]), rIl, dtype, "dI_l")
    assert_grad(f64(out[3]), rIh, dtype, "dI_h")
    assert L.dgf_device_status() == 0


def test_host_step_partial_outputs_and_buffer_reuse():
    dtype, N, C, hl, wl, f, r, eps = F32, 1, 3, 33, 41, 4, 1, 1e-3
    st = to_storage(make_case("photo", 70, N, C, hl, wl, hl * f, wl * f), dtype)
    R = synth.upstream_grad(71, st["I_h"].shape).to(dtype)
    g = {k: v.cuda() for k, v in st.items()}
    ref_O = gf_forward(g["p_l"], g["I_l"], g["I_h"], r, eps).cpu()
    ref = [x.cpu() for x in gf_backward(R.cuda(), g["p_l"], g["I_l"], g["I_h"], r, eps)[:3]]
    h = {k: v.pin_memory() for k, v in st.items()}
    Rh = R.pin_memory()
    nb = L.dgf_host_step_device_bytes(N, C, hl, wl, hl * f, wl * f, r, L.DGF_F32, 2)
    buf = workspace(nb, torch.device("cuda"))
    # forward only: the gradient outputs stay untouched
    sentinel = torch.full(st["p_l"].shape, 7.0)
    O = torch.empty(st["I_h"].shape).pin_memory()
    gf_step_host(h["p_l"], h["I_l"], h["I_h"], Rh, r, eps, out=(O, None, None, None), groups=2, buf=buf)
    assert torch.equal(O, ref_O)
    # backward only (dI_l alone), into the same device buffer
    dIl = sentinel.clone().pin_memory()
    gf_step_host(h["p_l"], h["I_l"], h["I_h"], Rh, r, eps, out=(None, None, dIl, None), groups=2, buf=buf)
    assert torch.equal(dIl, ref[1])
    # the full step twice on one buffer, the second call overwriting the first's outputs
    outs = (torch.empty_like(O).pin_memory(), torch.empty(st["p_l"].shape).pin_memory(),
            torch.empty(st["p_l"].shape).pin_memory(), torch.empty_like(O).pin_memory())
    for _ in range(2):
        gf_step_host(h["p_l"], h["I_l"], h["I_h"], Rh, r, eps, out=outs, groups=2, buf=buf, sync=False)
    torch.cuda.synchronize()
    assert torch.equal(outs[0], ref_O)
    for a, b in zip(outs[1:], ref):
        assert torch.equal(a, b)
    assert L.dgf_device_status() == 0


@pytest.mark.parametrize("dtype", [F32, BF16], ids=["f32", "bf16"])
def test_host_step_paper_literal_equals_device_calls(dtype):
    # mean_ab = False (the layer as Sec. 3.2 prints it): every plane's outputs
    # are those of the device calls with the same option
    N, C, hl, wl, f, r, eps = 2, 2, 37, 45, 4, 2, 1e-3
    st = to_storage(make_case("photo", 66, N, C, hl, wl, hl * f, wl * f), dtype)
    R = synth.upstream_grad(67, st["I_h"].shape).to(dtype)
    g = {k: v.cuda() for k, v in st.items()}
    ref_O = gf_forward(g["p_l"], g["I_l"], g["I_h"], r, eps, mean_ab=False)
    ref = gf_backward(R.cuda(), g["p_l"], g["I_l"], g["I_h"], r, eps, mean_ab=False)[:3]
    torch.cuda.synchronize()
    h = {k: _host(v, True) for k, v in st.items()}
    out = gf_step_host(h["p_l"], h["I_l"], h["I_h"], _host(R, True), r, eps, groups=3, mean_ab=False)
    assert torch.equal(out[0], ref_O.cpu())
    for a, b in zip(out[1:], ref):
        assert torch.equal(a, b.cpu())
    assert not torch.equal(out[0], gf_forward(g["p_l"], g["I_l"], g["I_h"], r, eps).cpu())
    assert L.dgf_device_status() == 0
