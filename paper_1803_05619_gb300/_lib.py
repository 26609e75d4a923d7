"""ctypes binding of libdgf.so: the C ABI of include/dgf.h, same names.

Argument marshalling only.  Every entry point takes raw pointers and sizes
exactly as the C functions do; the torch-facing helpers live in layer.py.
There is no fallback: if the library is missing or fails to load, the
first call raises.
"""
from __future__ import annotations

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libdgf.so")

DGF_F32, DGF_BF16, DGF_F16 = 0, 1, 2
STATUS = {0: "DGF_OK", 1: "DGF_ERR_INVALID", 2: "DGF_ERR_UNSUPPORTED", 3: "DGF_ERR_CUDA",
          4: "DGF_ERR_TIMEOUT", 5: "DGF_ERR_WORKSPACE"}
MAX_BATCH = 128


class dgf_guide(ctypes.Structure):
    _fields_ = [("w1", ctypes.c_void_p), ("w2", ctypes.c_void_p), ("b2", ctypes.c_void_p),
                ("hidden", ctypes.c_int), ("slope", ctypes.c_float)]


class dgf_image(ctypes.Structure):
    _fields_ = [("p_l", ctypes.c_void_p), ("I_l", ctypes.c_void_p), ("I_h", ctypes.c_void_p),
                ("O_h", ctypes.c_void_p), ("C", ctypes.c_int), ("h_l", ctypes.c_int),
                ("w_l", ctypes.c_int), ("h", ctypes.c_int), ("w", ctypes.c_int), ("r", ctypes.c_int),
                ("eps", ctypes.c_float), ("coef", ctypes.c_void_p)]


class dgf_options(ctypes.Structure):
    _fields_ = [("mean_ab", ctypes.c_int), ("guide_channels", ctypes.c_int), ("guide_low", ctypes.c_int),
                ("coef", ctypes.c_void_p)]


class dgf_image_grad(ctypes.Structure):
    _fields_ = [("dO_h", ctypes.c_void_p), ("p_l", ctypes.c_void_p), ("I_l", ctypes.c_void_p),
                ("I_h", ctypes.c_void_p), ("dp_l", ctypes.c_void_p), ("dI_l", ctypes.c_void_p),
                ("dI_h", ctypes.c_void_p), ("C", ctypes.c_int), ("h_l", ctypes.c_int), ("w_l", ctypes.c_int),
                ("h", ctypes.c_int), ("w", ctypes.c_int), ("r", ctypes.c_int), ("eps", ctypes.c_float),
                ("coef", ctypes.c_void_p)]


class dgf_host_step_io(ctypes.Structure):
    _fields_ = [("p_l", ctypes.c_void_p), ("I_l", ctypes.c_void_p), ("I_h", ctypes.c_void_p),
                ("dO_h", ctypes.c_void_p), ("O_h", ctypes.c_void_p), ("dp_l", ctypes.c_void_p),
                ("dI_l", ctypes.c_void_p), ("dI_h", ctypes.c_void_p)]


class DGFError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS.get(status, status)}: {message}")
        self.status = status


_lib = None

_I, _F, _P, _S = ctypes.c_int, ctypes.c_float, ctypes.c_void_p, ctypes.c_size_t
_SIGS = {
    "dgf_workspace_size": (_S, [_I, _I, _I, _I, _I, _I, _I, _I, ctypes.POINTER(dgf_guide)]),
    "dgf_forward": (_I, [_P, _P, _P, _P, _I, _I, _I, _I, _I, _I, _I, _F, _I,
                         ctypes.POINTER(dgf_guide), _P, _S, _P]),
    "dgf_backward": (_I, [_P, _P, _P, _P, _P, _P, _P, _P, _I, _I, _I, _I, _I, _I, _I, _F, _I,
                          ctypes.POINTER(dgf_guide), _P, _S, _P]),
    "dgf_forward_opt": (_I, [_P, _P, _P, _P, _I, _I, _I, _I, _I, _I, _I, _F, _I,
                             ctypes.POINTER(dgf_guide), _P, _S, _P, ctypes.POINTER(dgf_options)]),
    "dgf_backward_opt": (_I, [_P, _P, _P, _P, _P, _P, _P, _P, _I, _I, _I, _I, _I, _I, _I, _F, _I,
                              ctypes.POINTER(dgf_guide), _P, _S, _P, ctypes.POINTER(dgf_options)]),
    "dgf_workspace_size_opt": (_S, [_I, _I, _I, _I, _I, _I, _I, _I, ctypes.POINTER(dgf_guide),
                                    ctypes.POINTER(dgf_options)]),
    "dgf_backward_reuses_coef": (_I, [_I, _I, _I, _I, _I, _I, _I, _I, ctypes.POINTER(dgf_guide),
                                      ctypes.POINTER(dgf_options)]),
    "dgf_coef_bytes": (_S, [_I, _I, _I, _I, _I, _I, ctypes.POINTER(dgf_guide)]),
    "dgf_workspace_size_batched": (_S, [ctypes.POINTER(dgf_image), _I, _I]),
    "dgf_forward_batched": (_I, [ctypes.POINTER(dgf_image), _I, _I, _P, _S, _P]),
    "dgf_workspace_size_batched_backward": (_S, [ctypes.POINTER(dgf_image_grad), _I, _I]),
    "dgf_backward_batched": (_I, [ctypes.POINTER(dgf_image_grad), _I, _I, _P, _S, _P]),
    "dgf_forward_batched_opt": (_I, [ctypes.POINTER(dgf_image), _I, _I, _P, _S, _P, ctypes.POINTER(dgf_options)]),
    "dgf_backward_batched_opt": (_I, [ctypes.POINTER(dgf_image_grad), _I, _I, _P, _S, _P,
                                      ctypes.POINTER(dgf_options)]),
    "dgf_last_error": (ctypes.c_char_p, []),
    "dgf_profile_enable": (None, [_I]),
    "dgf_profile_reset": (None, []),
    "dgf_profile_read": (_I, [ctypes.POINTER(ctypes.c_char_p), ctypes.POINTER(ctypes.c_double),
                              ctypes.POINTER(ctypes.c_longlong), _I]),
    "dgf_launch_count": (ctypes.c_longlong, []),
    "dgf_device_status": (_I, []),
    "dgf_clear_device_status": (_I, []),
    "dgf_set_wait_polls": (_I, [ctypes.c_longlong]),
    "dgf_set_tma": (None, [_I]),
    "dgf_set_fused": (None, [_I]),
    "dgf_set_lowres_slide": (None, [_I]),
    "dgf_set_grey_fold": (None, [_I]),
    "dgf_set_batched_graph_backward": (None, [_I]),
    "dgf_set_pipeline": (None, [_I]),
    "dgf_shutdown": (None, []),
    "dgf_autotune": (None, [_I]),
    "dgf_autotune_entries": (_I, []),
    "dgf_autotune_reset": (None, []),
    "dgf_autotune_pin": (_I, [_I, _I, _I, _I, _I, _I, _I, _I]),
    "dgf_forward_noalloc": (_I, [_P, _P, _P, _P, _I, _I, _I, _I, _I, _I, _I, _F, _I, _P]),
    "dgf_noalloc_max_pairs": (_S, []),
    "dgf_host_step_device_bytes": (_S, [_I, _I, _I, _I, _I, _I, _I, _I, _I]),
    "dgf_host_step": (_I, [ctypes.POINTER(dgf_host_step_io), _I, _I, _I, _I, _I, _I, _I, _F, _I, _I, _P, _S,
                           _P]),
    "dgf_host_step_opt": (_I, [ctypes.POINTER(dgf_host_step_io), _I, _I, _I, _I, _I, _I, _I, _F, _I, _I, _P,
                               _S, _P, ctypes.POINTER(dgf_options)]),
}


def lib() -> ctypes.CDLL:
    """Load libdgf.so (built by build.py); raise if it is missing."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(
                f"{LIB_PATH} is missing: build it with paper_1803_05619_gb300.build.build() "
                "(the CUDA path has no fallback)")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def check(status: int) -> None:
    if status != 0:
        raise DGFError(status, lib().dgf_last_error().decode())


# Same names as the C ABI (thin pass-throughs).
def dgf_workspace_size(N, C, h_l, w_l, h, w, r, dt, g=None) -> int:
    return lib().dgf_workspace_size(N, C, h_l, w_l, h, w, r, dt, g)


def dgf_forward(p_l, I_l, I_h, O_h, N, C, h_l, w_l, h, w, r, eps, dt, g, ws, ws_bytes, stream) -> int:
    return lib().dgf_forward(p_l, I_l, I_h, O_h, N, C, h_l, w_l, h, w, r, eps, dt, g, ws, ws_bytes,
                             stream)


def dgf_backward(dO_h, p_l, I_l, I_h, dp_l, dI_l, dI_h, dW, N, C, h_l, w_l, h, w, r, eps, dt, g, ws,
                 ws_bytes, stream) -> int:
    return lib().dgf_backward(dO_h, p_l, I_l, I_h, dp_l, dI_l, dI_h, dW, N, C, h_l, w_l, h, w, r, eps,
                              dt, g, ws, ws_bytes, stream)


def dgf_forward_opt(p_l, I_l, I_h, O_h, N, C, h_l, w_l, h, w, r, eps, dt, g, ws, ws_bytes, stream, opt) -> int:
    return lib().dgf_forward_opt(p_l, I_l, I_h, O_h, N, C, h_l, w_l, h, w, r, eps, dt, g, ws, ws_bytes,
                                 stream, opt)


def dgf_backward_opt(dO_h, p_l, I_l, I_h, dp_l, dI_l, dI_h, dW, N, C, h_l, w_l, h, w, r, eps, dt, g, ws,
                     ws_bytes, stream, opt) -> int:
    return lib().dgf_backward_opt(dO_h, p_l, I_l, I_h, dp_l, dI_l, dI_h, dW, N, C, h_l, w_l, h, w, r, eps,
                                  dt, g, ws, ws_bytes, stream, opt)


def dgf_workspace_size_opt(N, C, h_l, w_l, h, w, r, dt, g, opt) -> int:
    return lib().dgf_workspace_size_opt(N, C, h_l, w_l, h, w, r, dt, g, opt)


def dgf_backward_reuses_coef(N, C, h_l, w_l, h, w, r, dt, g, opt) -> int:
    return lib().dgf_backward_reuses_coef(N, C, h_l, w_l, h, w, r, dt, g, opt)


def dgf_coef_bytes(N, C, h_l, w_l, h, w, g) -> int:
    return lib().dgf_coef_bytes(N, C, h_l, w_l, h, w, g)


def dgf_workspace_size_batched(imgs, n, dt) -> int:
    return lib().dgf_workspace_size_batched(imgs, n, dt)


def dgf_forward_batched(imgs, n, dt, ws, ws_bytes, stream) -> int:
    return lib().dgf_forward_batched(imgs, n, dt, ws, ws_bytes, stream)


def dgf_workspace_size_batched_backward(imgs, n, dt) -> int:
    return lib().dgf_workspace_size_batched_backward(imgs, n, dt)


def dgf_backward_batched(imgs, n, dt, ws, ws_bytes, stream) -> int:
    return lib().dgf_backward_batched(imgs, n, dt, ws, ws_bytes, stream)


def dgf_forward_batched_opt(imgs, n, dt, ws, ws_bytes, stream, opt) -> int:
    return lib().dgf_forward_batched_opt(imgs, n, dt, ws, ws_bytes, stream, opt)


def dgf_backward_batched_opt(imgs, n, dt, ws, ws_bytes, stream, opt) -> int:
    return lib().dgf_backward_batched_opt(imgs, n, dt, ws, ws_bytes, stream, opt)


def dgf_last_error() -> str:
    return lib().dgf_last_error().decode()


def dgf_profile_enable(on: bool) -> None:
    lib().dgf_profile_enable(1 if on else 0)


def dgf_profile_reset() -> None:
    lib().dgf_profile_reset()


def dgf_profile_read() -> dict:
    L = lib()
    n = L.dgf_profile_read(None, None, None, 0)
    names = (ctypes.c_char_p * max(n, 1))()
    ms = (ctypes.c_double * max(n, 1))()
    cnt = (ctypes.c_longlong * max(n, 1))()
    n = L.dgf_profile_read(names, ms, cnt, n)
    return {names[i].decode(): (ms[i], cnt[i]) for i in range(n)}


def dgf_launch_count() -> int:
    return lib().dgf_launch_count()


def dgf_device_status() -> int:
    return lib().dgf_device_status()


def dgf_clear_device_status() -> int:
    return lib().dgf_clear_device_status()


def dgf_set_wait_polls(polls: int) -> int:
    return lib().dgf_set_wait_polls(int(polls))


def dgf_set_tma(on: bool) -> None:
    lib().dgf_set_tma(1 if on else 0)


def dgf_set_fused(on: bool) -> None:
    lib().dgf_set_fused(1 if on else 0)


def dgf_set_lowres_slide(on: bool) -> None:
    lib().dgf_set_lowres_slide(1 if on else 0)


def dgf_set_grey_fold(on: bool) -> None:
    lib().dgf_set_grey_fold(1 if on else 0)


def dgf_set_batched_graph_backward(on: bool) -> None:
    lib().dgf_set_batched_graph_backward(1 if on else 0)


def dgf_set_pipeline(on: bool) -> None:
    lib().dgf_set_pipeline(1 if on else 0)


def dgf_shutdown() -> None:
    lib().dgf_shutdown()


def dgf_autotune(on: bool) -> None:
    lib().dgf_autotune(1 if on else 0)


def dgf_autotune_entries() -> int:
    return lib().dgf_autotune_entries()


def dgf_autotune_reset() -> None:
    lib().dgf_autotune_reset()


def dgf_autotune_pin(kind, dt, r, F, vec, guide_f32, a, b) -> int:
    return lib().dgf_autotune_pin(kind, dt, r, F, vec, guide_f32, a, b)


def dgf_forward_noalloc(p_l, I_l, I_h, O_h, N, C, h_l, w_l, h, w, r, eps, dt, stream) -> int:
    return lib().dgf_forward_noalloc(p_l, I_l, I_h, O_h, N, C, h_l, w_l, h, w, r, eps, dt, stream)


def dgf_noalloc_max_pairs() -> int:
    return lib().dgf_noalloc_max_pairs()


def dgf_host_step_device_bytes(N, C, h_l, w_l, h, w, r, dt, groups) -> int:
    return lib().dgf_host_step_device_bytes(N, C, h_l, w_l, h, w, r, dt, groups)


def dgf_host_step(io, N, C, h_l, w_l, h, w, r, eps, dt, groups, device, device_bytes, stream) -> int:
    return lib().dgf_host_step(io, N, C, h_l, w_l, h, w, r, eps, dt, groups, device, device_bytes, stream)


def dgf_host_step_opt(io, N, C, h_l, w_l, h, w, r, eps, dt, groups, device, device_bytes, stream, opt) -> int:
    return lib().dgf_host_step_opt(io, N, C, h_l, w_l, h, w, r, eps, dt, groups, device, device_bytes, stream, opt)
