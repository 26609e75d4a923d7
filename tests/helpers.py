"""Shared helpers of the GPU tests: input preparation, oracle calls, metrics."""
import numpy as np
import torch

import oracle as O
import synth

TOL_FWD_F32_ABS = 2e-5     # FP32 path, eps >= 1e-3, inputs in [0, 1]
TOL_F32_REL_L2 = 1e-4      # FP32 path: forward at eps < 1e-3 and every gradient
TOL_FWD_BF16_ABS = 1e-2    # BF16 storage: half an ulp of BF16 at 1 is 2^-8 ~ 3.9e-3
TOL_FWD_F16_ABS = 1e-3     # FP16 storage: half an ulp at 1 is 2^-11 ~ 4.9e-4
TOL_GRAD_BF16_REL_L2 = 1e-2  # gradient stores round to BF16 (2^-9 relative)
TOL_GRAD_F16_REL_L2 = 2e-3   # gradient stores round to FP16 (2^-12 relative)


def rel_l2(got, ref):
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    return float(np.linalg.norm(got - ref) / max(np.linalg.norm(ref), 1e-300))


def max_abs(got, ref):
    return float(np.max(np.abs(np.asarray(got, np.float64) - np.asarray(ref, np.float64))))


def to_storage(d: dict, dtype) -> dict:
    """Round the FP64 inputs to the storage dtype (the oracle then sees the
    rounded values, upcast, so the comparison measures the kernels)."""
    return {k: v.to(dtype) for k, v in d.items()}


def f64(t) -> np.ndarray:
    return t.detach().cpu().double().numpy()


def make_case(kind, seed, N, C, h_l, w_l, h, w):
    if kind == "photo":
        f = h // h_l
        return synth.photo_like(seed, N, C, h_l, w_l, f)
    if kind == "blobs":
        f = h // h_l
        return synth.blobs_tone_curve(seed, N, C, h_l, w_l, f)
    return synth.ragged_case(seed, N, C, h_l, w_l, h, w)


def oracle_forward(st, r, eps, planes=None):
    return O.forward(f64(st["p_l"]), f64(st["I_l"]), f64(st["I_h"]), r, eps, planes=planes)


def oracle_backward(R, st, r, eps, planes=None):
    return O.backward(f64(R), f64(st["p_l"]), f64(st["I_l"]), f64(st["I_h"]), r, eps, planes=planes)


def fwd_tol(dtype, eps):
    """(kind, bound) of the forward gate for this storage type."""
    if dtype == torch.float32:
        return ("abs", TOL_FWD_F32_ABS) if eps >= 1e-3 else ("rel", TOL_F32_REL_L2)
    if dtype == torch.bfloat16:
        return ("abs", TOL_FWD_BF16_ABS)
    return ("abs", TOL_FWD_F16_ABS)


def grad_tol(dtype):
    if dtype == torch.float32:
        return TOL_F32_REL_L2
    if dtype == torch.bfloat16:
        return TOL_GRAD_BF16_REL_L2
    return TOL_GRAD_F16_REL_L2


def assert_fwd(got, ref, dtype, eps, what="O_h"):
    kind, bound = fwd_tol(dtype, eps)
    err = max_abs(got, ref) if kind == "abs" else rel_l2(got, ref)
    assert err <= bound, f"{what}: {kind} error {err:.3e} > {bound:.1e}"
    return err


def assert_grad(got, ref, dtype, what):
    if not np.any(ref):
        # the gradient is identically zero (e.g. r = 0: single-pixel windows
        # have zero variance, so A = 0 and O_h does not depend on I_l)
        err = float(np.max(np.abs(got)))
        assert err <= 1e-5, f"{what}: expected zero gradient, max abs {err:.3e}"
        return err
    err = rel_l2(got, ref)
    assert err <= grad_tol(dtype), f"{what}: rel L2 {err:.3e} > {grad_tol(dtype):.1e}"
    return err
