"""The allocation-free forward entry point (collected last on purpose).

dgf_forward_noalloc serves callers that cannot allocate device memory at
call time (cudaMalloc may synchronise the device or fail under memory
pressure, so real-time loops and frameworks that own all device memory
forbid it).  It keeps its scratch in a fixed array inside the library.
These tests call it through the C ABI and compare it bit for bit with
dgf_forward (the workspace entry point, which runs the same kernels) on two
calls in a row with different inputs, so the second call also shows that
the scratch's leftover contents do not leak into the result; one case fills
the scratch exactly, and every result is also checked against the FP64
oracle at the parity gates.
"""
import ctypes

import pytest
import torch

from paper_1803_05619_gb300 import _lib as L
from paper_1803_05619_gb300.layer import dtype_code, gf_forward
from tests.helpers import assert_fwd, f64, make_case, oracle_forward, to_storage

pytestmark = pytest.mark.gpu


def _noalloc(g, r, eps):
    out = torch.empty_like(g["I_h"])
    N, C, h, w = g["I_h"].shape
    h_l, w_l = g["p_l"].shape[2:]
    P = lambda t: ctypes.c_void_p(t.data_ptr())  # noqa: E731
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    st = L.dgf_forward_noalloc(P(g["p_l"]), P(g["I_l"]), P(g["I_h"]), P(out), N, C, h_l, w_l, h, w, r,
                               ctypes.c_float(eps), dtype_code(g["I_h"]), stream)
    return st, out


def _check_two_calls(dtype, r, eps, cases):
    for call, (kind, seed, shape) in enumerate(cases):
        N, C, hl, wl, h, w = shape
        st_in = to_storage(make_case(kind, seed, N, C, hl, wl, h, w), dtype)
        g = {k: v.cuda() for k, v in st_in.items()}
        ref = gf_forward(g["p_l"], g["I_l"], g["I_h"], r, eps)
        torch.cuda.synchronize()
        assert L.dgf_device_status() == 0
        st, out = _noalloc(g, r, eps)
        torch.cuda.synchronize()
        assert st == 0, L.dgf_last_error()
        assert L.dgf_device_status() == 0
        assert torch.equal(out, ref), f"call {call}: differs from dgf_forward"
        assert_fwd(f64(out), oracle_forward(st_in, r, eps), dtype, eps)


@pytest.mark.parametrize("dtype", [torch.float32, torch.bfloat16], ids=["f32", "bf16"])
@pytest.mark.parametrize("r", [0, 1, 2, 4, 8])
def test_noalloc_matches_workspace_entry_point_twice(dtype, r):
    eps = 1e-3
    _check_two_calls(dtype, r, eps, [("photo", 71 + r, (2, 3, 60, 90, 240, 360)),
                                     ("photo", 72 + r, (1, 3, 77, 40, 308, 160))])


def test_noalloc_non_integer_ratio_twice():
    _check_two_calls(torch.float32, 2, 1e-3, [("ragged", 73, (1, 2, 37, 53, 150, 211)),
                                              ("ragged", 74, (2, 1, 41, 29, 100, 97))])


@pytest.mark.parametrize("shape", [(1, 1, 1024, 1024, 4096, 4096),    # exactly the scratch
                                   (1, 1, 1023, 1025, 4092, 4100)],  # just below, odd width
                         ids=["full", "odd"])
def test_noalloc_at_the_scratch_limit(shape):
    assert shape[0] * shape[1] * shape[2] * shape[3] <= L.dgf_noalloc_max_pairs()
    # the bitwise comparison with dgf_forward covers every pixel here; the
    # smaller cases above tie both entry points to the oracle
    N, C, hl, wl, h, w = shape
    st_in = to_storage(make_case("photo", 75, N, C, hl, wl, h, w), torch.bfloat16)
    g = {k: v.cuda() for k, v in st_in.items()}
    for _ in range(2):
        ref = gf_forward(g["p_l"], g["I_l"], g["I_h"], 1, 1e-3)
        st, out = _noalloc(g, 1, 1e-3)
        torch.cuda.synchronize()
        assert st == 0, L.dgf_last_error()
        assert L.dgf_device_status() == 0
        assert torch.equal(out, ref)


def test_noalloc_rejects_sizes_beyond_its_scratch():
    cap = L.dgf_noalloc_max_pairs()
    assert cap == 1 << 20
    # 1 x 1 x 1025 x 1024 low-res pixels: one row more than the scratch holds.
    # The buffers are real and sized for the call, so nothing reads outside
    # them even if the size check were ever bypassed.
    hl, wl = 1025, 1024
    p = torch.zeros(1, 1, hl, wl, device="cuda")
    il = torch.zeros_like(p)
    ih = torch.zeros(1, 1, 4 * hl, 4 * wl, device="cuda")
    out = torch.empty_like(ih)
    P = lambda t: ctypes.c_void_p(t.data_ptr())  # noqa: E731
    st = L.dgf_forward_noalloc(P(p), P(il), P(ih), P(out), 1, 1, hl, wl, 4 * hl, 4 * wl, 1,
                               ctypes.c_float(1e-3), L.DGF_F32, None)
    assert st == 2 and "exceeds" in L.dgf_last_error()
    torch.cuda.synchronize()
    assert L.dgf_device_status() == 0
