"""The C-ABI library without a GPU: it builds, loads, exports every symbol
include/dgf.h declares, and its host-side validation rejects bad arguments
before anything touches CUDA."""
import ctypes
import os
import re

import pytest

from paper_1803_05619_gb300 import _lib as L
from paper_1803_05619_gb300 import build as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "dgf.h")


@pytest.fixture(scope="module")
def lib():
    B.build()
    return L.lib()


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"\b(dgf_[a-z_]+)\s*\(", src)
    return sorted(set(names))


def test_header_declares_the_abi():
    names = declared_functions()
    for n in ("dgf_forward", "dgf_backward", "dgf_forward_batched", "dgf_workspace_size"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_binding_names_match_header():
    for name in declared_functions():
        assert hasattr(L, name), name


def test_workspace_size_is_host_only(lib):
    n = L.dgf_workspace_size(4, 3, 512, 512, 2048, 2048, 1, L.DGF_F32, None)
    lo = 4 * 3 * 512 * 512
    assert n >= 2 * lo * 8
    assert L.dgf_workspace_size(1, 1, 8, 8, 4, 4, 1, L.DGF_F32, None) == 0  # h_l > h
    assert L.dgf_workspace_size(1, 1, 8, 8, 32, 32, -1, L.DGF_F32, None) == 0


def _fwd(**kw):
    a = dict(p_l=1024, I_l=2048, I_h=4096, O_h=8192, N=1, C=1, h_l=8, w_l=8, h=32, w=32, r=1,
             eps=1e-3, dt=L.DGF_F32, g=None, ws=None, ws_bytes=0, stream=None)
    a.update(kw)
    return L.dgf_forward(*(ctypes.c_void_p(a[k]) if k in ("p_l", "I_l", "I_h", "O_h", "ws") and a[k]
                           else a[k] for k in a))


@pytest.mark.parametrize("bad,status", [
    (dict(r=-1), 1), (dict(eps=0.0), 1), (dict(eps=float("nan")), 1), (dict(eps=float("inf")), 1),
    (dict(h_l=64), 1), (dict(C=0), 1), (dict(N=-1), 1), (dict(dt=7), 1), (dict(r=17), 2),
    (dict(p_l=0), 1), (dict(O_h=0), 1), (dict(ws=None), 5), (dict(ws=4096 + 8, ws_bytes=1 << 20), 5),
    (dict(ws=4096, ws_bytes=16), 5),
])
def test_forward_rejects_bad_arguments_on_host(lib, bad, status):
    assert _fwd(**bad) == status
    assert L.dgf_last_error() != ""


def test_empty_batch_is_ok(lib):
    assert _fwd(N=0) == 0


def test_guide_validation(lib):
    g = L.dgf_guide(16, 32, 48, 0, 0.2)  # hidden = 0
    assert _fwd(C=3, g=ctypes.byref(g)) == 1
    g = L.dgf_guide(16, 32, 48, 15, 0.2)
    assert _fwd(C=1, g=ctypes.byref(g)) == 2  # needs C = 3
    assert _fwd(C=3, h=33, g=ctypes.byref(g)) == 1  # needs an integer factor


def test_backward_validation(lib):
    z = ctypes.c_void_p(4096)
    st = L.dgf_backward(z, z, z, z, z, z, z, None, 1, 1, 8, 8, 32, 32, 1, -1.0, L.DGF_F32, None, None,
                        0, None)
    assert st == 1
    # dW without a guidance transform
    st = L.dgf_backward(z, z, z, z, z, z, z, ctypes.c_void_p(8192), 1, 1, 8, 8, 32, 32, 1, 1e-3,
                        L.DGF_F32, None, None, 0, None)
    assert st == 1


def test_batched_validation(lib):
    arr = (L.dgf_image * 2)()
    arr[0] = L.dgf_image(16, 32, 48, 64, 3, 8, 8, 32, 32, 1, 1e-3)
    arr[1] = L.dgf_image(16, 32, 48, 64, 3, 8, 8, 32, 32, -2, 1e-3)
    assert L.dgf_workspace_size_batched(arr, 2, L.DGF_BF16) == 0
    assert L.dgf_workspace_size_batched(arr, 1, L.DGF_BF16) > 0
    assert L.dgf_forward_batched(arr, 1, L.DGF_BF16, None, 0, None) == 5
    assert L.dgf_forward_batched(arr, 200, L.DGF_BF16, None, 0, None) == 1


def test_batched_backward_validation(lib):
    arr = (L.dgf_image_grad * 3)()
    arr[0] = L.dgf_image_grad(16, 32, 48, 64, 80, 96, 112, 3, 8, 8, 32, 32, 1, 1e-3)
    arr[1] = L.dgf_image_grad(16, 32, 48, 64, None, None, 112, 1, 12, 10, 48, 40, 2, 1e-3)
    arr[2] = L.dgf_image_grad(16, None, 48, 64, 80, 96, 112, 3, 8, 8, 32, 32, 1, 1e-3)  # NULL p_l
    one = L.dgf_workspace_size_batched_backward(arr, 1, L.DGF_F32)
    two = L.dgf_workspace_size_batched_backward(arr, 2, L.DGF_F32)
    assert one > 0 and two > one and one % 256 == 0
    assert L.dgf_workspace_size_batched_backward(arr, 3, L.DGF_F32) == 0
    assert "image 2" in L.dgf_last_error()
    assert L.dgf_workspace_size_batched_backward(arr, 200, L.DGF_F32) == 0
    assert L.dgf_backward_batched(arr, 3, L.DGF_F32, None, 0, None) == 1
    assert L.dgf_backward_batched(arr, 2, L.DGF_F32, None, 0, None) == 5  # workspace too small
    assert L.dgf_backward_batched(arr, 0, L.DGF_F32, None, 0, None) == 0


def test_host_step_validation(lib):
    """dgf_host_step's size query and argument checks run on the host, before any CUDA call."""
    nb = L.dgf_host_step_device_bytes(2, 3, 16, 20, 64, 80, 1, L.DGF_F32, 0)
    assert nb > 0 and nb % 256 == 0
    # eight full-size device tensors at least
    assert nb >= 4 * (2 * 3 * 64 * 80 * 4) + 4 * (2 * 3 * 16 * 20 * 4)
    # more groups: a smaller per-group workspace
    assert L.dgf_host_step_device_bytes(2, 3, 16, 20, 64, 80, 1, L.DGF_F32, 6) <= \
        L.dgf_host_step_device_bytes(2, 3, 16, 20, 64, 80, 1, L.DGF_F32, 1)
    assert L.dgf_host_step_device_bytes(2, 3, 16, 20, 64, 80, 1, L.DGF_F32, 17) == 0
    assert L.dgf_host_step_device_bytes(2, 3, 16, 20, 64, 80, -1, L.DGF_F32, 0) == 0
    io = L.dgf_host_step_io(16, 32, 48, 64, 80, 96, 112, 128)
    assert L.dgf_host_step(None, 2, 3, 16, 20, 64, 80, 1, 1e-3, L.DGF_F32, 0, None, 0, None) == 1
    assert L.dgf_host_step(ctypes.byref(io), 2, 3, 16, 20, 64, 80, 1, 1e-3, L.DGF_F32, 99, None, 0, None) == 1
    assert L.dgf_host_step(ctypes.byref(io), 2, 3, 16, 20, 64, 80, 1, 1e-3, L.DGF_F32, 0, None, 0, None) == 5
    no_dO = L.dgf_host_step_io(16, 32, 48, None, 80, 96, 112, 128)  # gradients wanted, no dO_h
    assert L.dgf_host_step(ctypes.byref(no_dO), 2, 3, 16, 20, 64, 80, 1, 1e-3, L.DGF_F32, 0, None, 0, None) == 1
    fwd_only = L.dgf_host_step_io(16, 32, 48, None, 80, None, None, None)
    assert L.dgf_host_step(ctypes.byref(fwd_only), 2, 3, 16, 20, 64, 80, 1, 1e-3, L.DGF_F32, 0, None, 0,
                           None) == 5
    nothing = L.dgf_host_step_io(16, 32, 48, None, None, None, None, None)
    assert L.dgf_host_step(ctypes.byref(nothing), 2, 3, 16, 20, 64, 80, 1, 1e-3, L.DGF_F32, 0, None, 0, None) == 0
    assert L.dgf_host_step(ctypes.byref(io), 0, 3, 16, 20, 64, 80, 1, 1e-3, L.DGF_F32, 0, None, 0, None) == 0


def test_batched_and_host_step_options_on_host(lib):
    """The batched and host-memory calls take mean_ab only; their checks run on the host."""
    arr = (L.dgf_image * 1)()
    arr[0] = L.dgf_image(16, 32, 48, 64, 3, 8, 8, 32, 32, 1, 1e-3)
    grads = (L.dgf_image_grad * 1)()
    grads[0] = L.dgf_image_grad(16, 32, 48, 64, 80, 96, 112, 3, 8, 8, 32, 32, 1, 1e-3)
    io = L.dgf_host_step_io(16, 32, 48, 64, 80, 96, 112, 128)
    literal, grey, low = L.dgf_options(0, 0, 0), L.dgf_options(1, 1, 0), L.dgf_options(1, 0, 1)
    for opt in (grey, low):
        assert L.dgf_forward_batched_opt(arr, 1, L.DGF_F32, None, 0, None, ctypes.byref(opt)) == 2
        assert L.dgf_backward_batched_opt(grads, 1, L.DGF_F32, None, 0, None, ctypes.byref(opt)) == 2
        assert L.dgf_host_step_opt(ctypes.byref(io), 1, 3, 8, 8, 32, 32, 1, 1e-3, L.DGF_F32, 0, None, 0, None,
                                   ctypes.byref(opt)) == 2
    # mean_ab = 0 or no options: the size and workspace checks of the plain calls
    for opt in (ctypes.byref(literal), None):
        assert L.dgf_forward_batched_opt(arr, 1, L.DGF_F32, None, 0, None, opt) == 5
        assert L.dgf_backward_batched_opt(grads, 1, L.DGF_F32, None, 0, None, opt) == 5
        assert L.dgf_host_step_opt(ctypes.byref(io), 1, 3, 8, 8, 32, 32, 1, 1e-3, L.DGF_F32, 0, None, 0, None,
                                   opt) == 5
        assert L.dgf_forward_batched_opt(arr, 0, L.DGF_F32, None, 0, None, opt) == 0


def test_coefficient_reuse_query_on_host(lib):
    """dgf_backward_reuses_coef: where the backward's K1 pass computes the coefficients alone."""
    q = L.dgf_backward_reuses_coef
    # FP32 r = 1: the K1 strips also write the window statistics K4 reads
    assert q(4, 3, 512, 512, 2048, 2048, 1, L.DGF_F32, None, None) == 0
    # 16-bit storage, sliding sums: K1 computes the coefficients alone
    assert q(2, 3, 540, 960, 2160, 3840, 2, L.DGF_BF16, None, None) == 1
    assert q(1, 1, 64, 64, 256, 256, 8, L.DGF_F16, None, None) == 1
    # with a guidance transform: always
    g = L.dgf_guide(16, 32, 48, 15, 0.2)
    assert q(8, 3, 256, 256, 2048, 2048, 8, L.DGF_BF16, ctypes.byref(g), None) == 1
    # a folded grey guide: always
    grey = L.dgf_options(1, 3, 0)
    assert q(4, 1, 512, 512, 2048, 2048, 1, L.DGF_F32, None, ctypes.byref(grey)) == 1
    # invalid sizes
    assert q(1, 1, 64, 64, 256, 256, -1, L.DGF_F32, None, None) == 0
    # a misaligned coefficient buffer is refused before anything runs
    bad = L.dgf_options(1, 0, 0, 4)
    assert L.dgf_forward_opt(16, 32, 48, 64, 1, 1, 8, 8, 32, 32, 1, 1e-3, L.DGF_F32, None, None, 0, None,
                             ctypes.byref(bad)) == 1
    assert "aligned" in L.dgf_last_error()
    # the kept values: the pairs, and with a guidance transform the low-res guide after them
    assert L.dgf_coef_bytes(2, 3, 10, 13, 40, 52, None) == 2 * 3 * 10 * 13 * 8
    # with a guidance transform: G_l and F(I_h) after the pairs, each from a 256-byte boundary
    assert L.dgf_coef_bytes(2, 3, 10, 13, 40, 52, ctypes.byref(g)) == 6400 + 3328 + 2 * 3 * 40 * 52 * 4
    assert L.dgf_coef_bytes(2, 0, 10, 13, 40, 52, None) == 0
    assert L.dgf_backward_opt(16, 32, 48, 64, 80, 96, 112, None, 1, 1, 8, 8, 32, 32, 1, 1e-3, L.DGF_F32, None,
                              None, 0, None, ctypes.byref(bad)) == 1
    img = (L.dgf_image * 1)()
    img[0] = L.dgf_image(16, 32, 48, 64, 3, 8, 8, 32, 32, 1, 1e-3, 4)
    assert L.dgf_workspace_size_batched(img, 1, L.DGF_F32) == 0


def test_grey_guide_options_on_host(lib):
    """Grey-guide options: workspace sizes and argument checks run on the host."""
    plain = L.dgf_workspace_size(2, 1, 16, 20, 64, 80, 1, L.DGF_BF16, None)
    same = L.dgf_options(1, 1)  # guide_channels == C: the plain layer
    assert L.dgf_workspace_size_opt(2, 1, 16, 20, 64, 80, 1, L.DGF_BF16, None, ctypes.byref(same)) == plain
    assert L.dgf_workspace_size_opt(2, 1, 16, 20, 64, 80, 1, L.DGF_BF16, None, None) == plain
    grey = L.dgf_options(1, 3)
    nb = L.dgf_workspace_size_opt(2, 1, 16, 20, 64, 80, 1, L.DGF_BF16, None, ctypes.byref(grey))
    # the FP32 grey guide at both resolutions, its FP32 low-res and BF16 high-res
    # gradients, each repeated over C = 1 output channel
    assert nb >= plain + 2 * 64 * 80 * 4 + 2 * 16 * 20 * 4 * 2 + 2 * 64 * 80 * 2 and nb % 256 == 0
    assert L.dgf_workspace_size_opt(2, 1, 16, 20, 64, 80, 1, L.DGF_BF16, None,
                                    ctypes.byref(L.dgf_options(1, -2))) == 0
    gd = L.dgf_guide(16, 32, 48, 16, 0.2)
    assert L.dgf_workspace_size_opt(2, 1, 16, 20, 64, 80, 1, L.DGF_BF16, ctypes.byref(gd),
                                    ctypes.byref(grey)) == 0
    ptr = ctypes.c_void_p(256)
    st = L.dgf_forward_opt(ptr, ptr, ptr, ptr, 2, 1, 16, 20, 64, 80, 1, 1e-3, L.DGF_BF16, ctypes.byref(gd),
                           None, 0, None, ctypes.byref(grey))
    assert st == 1 and "exclude" in L.dgf_last_error()
    st = L.dgf_forward_opt(ptr, ptr, ptr, ptr, 2, 1, 16, 20, 64, 80, 1, 1e-3, L.DGF_BF16, None,
                           None, 0, None, ctypes.byref(grey))
    assert st == 5  # workspace missing
    dW = ctypes.c_void_p(512)
    st = L.dgf_backward_opt(ptr, ptr, ptr, ptr, ptr, ptr, ptr, ctypes.cast(dW, ctypes.POINTER(ctypes.c_float)),
                            2, 1, 16, 20, 64, 80, 1, 1e-3, L.DGF_BF16, None, None, 0, None, ctypes.byref(grey))
    assert st == 1 and "dW" in L.dgf_last_error()


def test_guide_low_option_on_host(lib):
    """guide_low needs a guidance transform and I_l; it admits dI_l with a transform."""
    ptr = ctypes.c_void_p(256)
    low = L.dgf_options(1, 0, 1)
    st = L.dgf_forward_opt(ptr, ptr, ptr, ptr, 1, 3, 16, 16, 64, 64, 1, 1e-3, L.DGF_F32, None,
                           None, 0, None, ctypes.byref(low))
    assert st == 1 and "guide_low" in L.dgf_last_error()
    gd = L.dgf_guide(16, 32, 48, 16, 0.2)
    st = L.dgf_forward_opt(ptr, None, ptr, ptr, 1, 3, 16, 16, 64, 64, 1, 1e-3, L.DGF_F32, ctypes.byref(gd),
                           None, 0, None, ctypes.byref(low))
    assert st == 1  # I_l is read
    # dI_l is rejected with a transform unless guide_low; with it the call gets as far as the workspace
    st = L.dgf_backward(ptr, ptr, ptr, ptr, None, ptr, None, None, 1, 3, 16, 16, 64, 64, 1, 1e-3, L.DGF_F32,
                        ctypes.byref(gd), None, 0, None)
    assert st == 1 and "dI_l" in L.dgf_last_error()
    st = L.dgf_backward_opt(ptr, ptr, ptr, ptr, None, ptr, None, None, 1, 3, 16, 16, 64, 64, 1, 1e-3, L.DGF_F32,
                            ctypes.byref(gd), None, 0, None, ctypes.byref(low))
    assert st == 5


def test_autotune_cache_skips_corrupt_and_foreign_lines(lib, tmp_path):
    """A corrupted or foreign cache file is ignored line by line (those keys
    are re-tuned); valid lines of this library version and device are used,
    and pinning a shape rewrites the file keeping the other lines."""
    import subprocess
    import sys
    cache = tmp_path / "tune.txt"
    me = "dgf3/unknown"  # no device in the subprocess: the device name is "unknown"
    cache.write_text(
        f"{me} 1 1 2 0 0 0 0 16 -4\n"        # sliding K1 strips, BF16, r = 2, large planes: used
        "garbage that is not an entry\n"
        f"{me} 2 0 0 4 4 0 1 12 0\n"         # K2 strip segments, small planes: used
        f"{me} 3 0 0 4 4 0 0 99999 0\n"      # out of range: skipped
        f"{me} 1 1 2 0 0 0 0 16\n"           # truncated: skipped
        f"{me} 4 1 2 0 0 0 0 16 -9\n"        # no such column width: skipped
        f"{me} 4 1 2 0 0 0 2 16 -4\n"        # no such size class: skipped
        "dgf2/unknown 1 1 1 0 0 0 32 0\n"    # the previous line format: skipped
        "dgf1/unknown 1 1 1 0 0 0 0 32 0\n"  # another library version: kept, never used
        f"{me} 5 0 1 4 0 0 0 8 0 extra\n"    # trailing junk: skipped
        "\x00\xff\n")
    code = ("import ctypes, sys; L = ctypes.CDLL(sys.argv[1]); n = L.dgf_autotune_entries(); "
            "pin = int(sys.argv[2]); st = L.dgf_autotune_pin(6, 1, 1, 8, 8, 0, 16, 0) if pin else 0; "
            "print(n, st, L.dgf_autotune_entries())")
    env = dict(os.environ, DGF_TUNE_CACHE=str(cache), CUDA_VISIBLE_DEVICES="")
    out = subprocess.run([sys.executable, "-c", code, B.OUT, "1"], capture_output=True, text=True, env=env,
                         timeout=120)
    assert out.returncode == 0, out.stderr
    # a pin serves both size classes: two entries
    assert out.stdout.split() == ["2", "0", "4"]
    text = cache.read_text()
    assert "dgf1/unknown 1 1 1 0 0 0 0 32 0" in text and "dgf2/unknown" not in text
    assert f"{me} 6 1 1 8 8 0 0 16 0" in text and f"{me} 6 1 1 8 8 0 1 16 0" in text
    out = subprocess.run([sys.executable, "-c", code, B.OUT, "0"], capture_output=True, text=True, env=env,
                         timeout=120)
    assert out.stdout.split() == ["4", "0", "4"]
