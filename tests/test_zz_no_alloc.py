"""The allocation-free forward entry point (collected last on purpose).

dgf_forward_noalloc serves callers that cannot allocate device memory at
call time (cudaMalloc may synchronise the device or fail under memory
pressure, so real-time loops and frameworks that own all device memory
forbid it).  It keeps its scratch in a fixed array inside the library.
This test calls it through the C ABI and compares it with dgf_forward (the
workspace entry point) on two calls in a row with different inputs, so the
second call also shows that the scratch's leftover contents do not leak
into the result.
"""
import ctypes

import pytest
import torch

from paper_1803_05619_gb300 import _lib as L
from paper_1803_05619_gb300.layer import dtype_code, gf_forward
from tests.helpers import f64, make_case, max_abs, to_storage

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


@pytest.mark.parametrize("dtype,tol", [(torch.float32, 2e-5), (torch.bfloat16, 1e-2)], ids=["f32", "bf16"])
def test_noalloc_matches_workspace_entry_point_twice(dtype, tol):
    r, eps = 1, 1e-3
    for call, (seed, shape) in enumerate([(71, (2, 3, 60, 90, 240, 360)), (72, (1, 3, 77, 40, 308, 160))]):
        N, C, hl, wl, h, w = shape
        st_in = to_storage(make_case("photo", seed, N, C, hl, wl, h, w), dtype)
        g = {k: v.cuda() for k, v in st_in.items()}
        ref = gf_forward(g["p_l"], g["I_l"], g["I_h"], r, eps)
        st, out = _noalloc(g, r, eps)
        torch.cuda.synchronize()
        assert st == 0, L.dgf_last_error()
        assert max_abs(f64(out), f64(ref)) <= tol, f"call {call}"


def test_noalloc_rejects_sizes_beyond_its_scratch():
    cap = L.dgf_noalloc_max_pairs()
    assert cap == 1 << 20
    side = 1024  # 1 x 3 x 1024 x 1024 low-res pixels > cap
    dummy = ctypes.c_void_p(256)
    st = L.dgf_forward_noalloc(dummy, dummy, dummy, dummy, 1, 3, side, side, 4 * side, 4 * side, 1,
                               ctypes.c_float(1e-3), L.DGF_F32, None)
    assert st == 2 and "exceeds" in L.dgf_last_error()
