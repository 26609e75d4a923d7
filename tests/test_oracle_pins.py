"""Pins of the FP64 oracle against things other than itself (CPU only).

The paper prints no worked numerical example of the layer, so the oracle is
pinned by: brute force on tiny inputs (plain Python loops), closed forms and
invariants that the definition fixes (constant output, the linear-target
identity, the eps limits, the global window), special cases that reduce to
library routines (torch's clipped average pool and bilinear interpolate in
FP64, He's textbook guided filter written with uncentred moments), torch
autograd on that independent composition, adjoint dot-product identities and
FP64 central finite differences.
"""
import itertools
import math

import numpy as np
import pytest
import torch

import oracle as O
import synth
from tests import torch_composition as TC

pytestmark = pytest.mark.filterwarnings("ignore::UserWarning")


def rng(seed=0):
    return np.random.default_rng(seed)


# ---------------------------------------------------------------- box filter

@pytest.mark.parametrize("h,w,r", [(1, 1, 0), (1, 7, 2), (5, 7, 1), (6, 4, 3), (9, 13, 2)])
def test_window_count_closed_form(h, w, r):
    N = O.window_count(h, w, r)
    for i in range(h):
        for j in range(w):
            cy = min(i + r, h - 1) - max(i - r, 0) + 1
            cx = min(j + r, w - 1) - max(j - r, 0) + 1
            assert N[i, j] == cy * cx


@pytest.mark.parametrize("h,w,r", [(5, 7, 1), (4, 9, 2), (3, 3, 4)])
def test_window_sum_brute_force(h, w, r):
    x = rng(1).normal(size=(h, w))
    S = O.window_sum(x, r)
    for i in range(h):
        for j in range(w):
            ref = 0.0
            for a in range(h):
                for b in range(w):
                    if abs(a - i) <= r and abs(b - j) <= r:
                        ref += x[a, b]
            assert abs(S[i, j] - ref) < 1e-12


@pytest.mark.parametrize("h,w,r", [(8, 11, 1), (16, 9, 2), (7, 7, 3), (5, 12, 5)])
def test_box_mean_matches_avg_pool(h, w, r):
    x = rng(2).uniform(size=(h, w))
    ref = TC.box(torch.from_numpy(x), r).numpy()
    np.testing.assert_allclose(O.box_mean(x, r), ref, rtol=0, atol=1e-14)


def test_box_mean_global_window():
    x = rng(3).uniform(size=(6, 9))
    M = O.box_mean(x, 9)
    np.testing.assert_allclose(M, np.full_like(x, x.mean()), rtol=0, atol=1e-14)


@pytest.mark.parametrize("h,w,r", [(6, 9, 1), (10, 7, 2), (4, 4, 5)])
def test_box_mean_transpose_identity(h, w, r):
    R = rng(4)
    x, y = R.normal(size=(h, w)), R.normal(size=(h, w))
    lhs = np.sum(O.box_mean(x, r) * y)
    rhs = np.sum(x * O.box_mean_T(y, r))
    assert abs(lhs - rhs) <= 1e-13 * max(1.0, abs(lhs))


# ------------------------------------------------------------ window stats

@pytest.mark.parametrize("h,w,r", [(5, 6, 1), (7, 5, 2), (3, 4, 3)])
def test_window_stats_against_numpy_var_cov(h, w, r):
    R = rng(5)
    G, P = R.uniform(size=(h, w)), R.uniform(size=(h, w))
    mu, nu, var, cov = O.window_stats(G, P, r)
    for i in range(h):
        for j in range(w):
            gs = G[max(i - r, 0):i + r + 1, max(j - r, 0):j + r + 1].ravel()
            ps = P[max(i - r, 0):i + r + 1, max(j - r, 0):j + r + 1].ravel()
            assert abs(mu[i, j] - gs.mean()) < 1e-14
            assert abs(nu[i, j] - ps.mean()) < 1e-14
            assert abs(var[i, j] - np.var(gs)) < 1e-14
            c = np.cov(np.stack([gs, ps]), bias=True) if gs.size > 1 else np.zeros((2, 2))
            assert abs(cov[i, j] - c[0, 1]) < 1e-14


# --------------------------------------------------------------- upsampler

@pytest.mark.parametrize("hl,wl,h,w", [(4, 4, 16, 16), (5, 3, 16, 13), (1, 2, 4, 9),
                                       (7, 7, 7, 7), (3, 8, 24, 64)])
def test_upsample_matches_torch_interpolate(hl, wl, h, w):
    X = rng(6).normal(size=(hl, wl))
    ref = TC.up(torch.from_numpy(X), h, w).numpy()
    np.testing.assert_allclose(O.upsample(X, h, w), ref, rtol=0, atol=1e-14)


def test_upsample_constant_and_ramp():
    # constants are reproduced exactly; a ramp exactly away from the clamped border
    X = np.full((5, 6), 0.375)
    assert np.all(O.upsample(X, 20, 24) == 0.375)
    f = 4
    ramp = np.tile(np.arange(6, dtype=float), (5, 1))  # value = column index j
    U = O.upsample(ramp, 20, 24)
    for x in range(24):
        t = (x + 0.5) / f - 0.5
        if 0.0 <= t <= 5.0:
            assert abs(U[3, x] - t) < 1e-14


@pytest.mark.parametrize("f", [2, 4, 8])
def test_bilinear_weights_f_periodic(f):
    n_in = 6
    W = O.bilinear_matrix(n_in * f, n_in)
    for k in range(f, (n_in - 1) * f):
        t = (k + 0.5) / f - 0.5
        i0 = math.floor(t)
        lam = t - i0
        assert abs(W[k, i0] - (1 - lam)) < 1e-15 and abs(W[k, i0 + 1] - lam) < 1e-15
        assert abs(W[k].sum() - 1.0) < 1e-15


@pytest.mark.parametrize("hl,wl,h,w", [(4, 5, 16, 20), (5, 3, 17, 11)])
def test_upsample_transpose_identity(hl, wl, h, w):
    R = rng(7)
    X, Z = R.normal(size=(hl, wl)), R.normal(size=(h, w))
    lhs = np.sum(O.upsample(X, h, w) * Z)
    rhs = np.sum(X * O.upsample_T(Z, hl, wl))
    assert abs(lhs - rhs) <= 1e-13 * max(1.0, abs(lhs))


# ----------------------------------------------------------- whole forward

CASES = [  # N, C, h_l, w_l, h, w, r, eps
    (1, 1, 8, 8, 32, 32, 1, 1e-2),
    (2, 3, 6, 9, 24, 36, 2, 1e-3),
    (1, 2, 5, 7, 17, 23, 1, 1e-4),
    (1, 1, 4, 4, 32, 32, 8, 1e-4),
]


@pytest.mark.parametrize("case", CASES)
def test_forward_matches_torch_composition(case):
    N, C, hl, wl, h, w, r, eps = case
    d = synth.ragged_case(11, N, C, hl, wl, h, w)
    out = O.forward(d["p_l"], d["I_l"], d["I_h"], r, eps)
    ref = TC.gf(d["p_l"], d["I_l"], d["I_h"], r, eps).numpy()
    np.testing.assert_allclose(out, ref, rtol=0, atol=1e-10)


def test_f1_reduces_to_textbook_guided_filter():
    # With h = h_l the layer is He's guided filter with q = mean(a) I + mean(b).
    d = synth.ragged_case(12, 1, 1, 12, 10, 12, 10)
    G, P = d["I_l"][0, 0].numpy(), d["p_l"][0, 0].numpy()
    r, eps = 2, 1e-3
    Gt, Pt = torch.from_numpy(G), torch.from_numpy(P)
    mean_I = TC.box(Gt, r)
    mean_p = TC.box(Pt, r)
    a = (TC.box(Gt * Pt, r) - mean_I * mean_p) / (TC.box(Gt * Gt, r) - mean_I ** 2 + eps)
    b = mean_p - a * mean_I
    q = TC.box(a, r) * Gt + TC.box(b, r)
    out = O.forward_plane(P, G, G, r, eps)
    np.testing.assert_allclose(out, q.numpy(), rtol=0, atol=1e-12)


def test_constant_target_is_reproduced_exactly():
    d = synth.ragged_case(13, 1, 2, 9, 7, 36, 28)
    p = np.full((1, 2, 9, 7), 0.5)
    out = O.forward(p, d["I_l"], d["I_h"], 2, 1e-3)
    assert np.all(out == 0.5)


def test_linear_target_closed_form():
    # p = alpha G + beta  =>  A = alpha var/(var+eps), b = beta + alpha mu eps/(var+eps)
    d = synth.ragged_case(14, 1, 1, 10, 12, 40, 48)
    G = d["I_l"][0, 0].numpy()
    alpha, beta, eps, r = 0.7, 0.1, 1e-3, 1
    P = alpha * G + beta
    mu, _, var, _ = O.window_stats(G, P, r)
    A, b = O.coefficients(G, P, r, eps)
    np.testing.assert_allclose(A, alpha * var / (var + eps), rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(b, beta + alpha * mu * eps / (var + eps), rtol=1e-12, atol=1e-14)
    # eps -> 0: the layer reproduces alpha G_h + beta
    Gh = d["I_h"][0, 0].numpy()
    out = O.forward_plane(P, G, Gh, r, 1e-14)
    np.testing.assert_allclose(out, alpha * Gh + beta, rtol=0, atol=1e-9)


def test_large_eps_limit():
    # eps -> inf: A -> 0, so O_h -> f_up(f_mu(f_mu(p)))
    d = synth.ragged_case(15, 1, 1, 8, 9, 32, 27)
    G, P, Gh = d["I_l"][0, 0].numpy(), d["p_l"][0, 0].numpy(), d["I_h"][0, 0].numpy()
    r = 1
    out = O.forward_plane(P, G, Gh, r, 1e12)
    ref = O.upsample(O.box_mean(O.box_mean(P, r), r), 32, 27)
    np.testing.assert_allclose(out, ref, rtol=0, atol=1e-11)


def test_global_window_is_one_ridge_regression():
    # r >= image size: a single scalar A (1-D ridge regression) for the whole image
    d = synth.ragged_case(16, 1, 1, 5, 6, 20, 24)
    G, P = d["I_l"][0, 0].numpy(), d["p_l"][0, 0].numpy()
    eps = 1e-3
    A, b = O.coefficients(G, P, 10, eps)
    g, p = G.ravel(), P.ravel()
    A_ref = np.mean((g - g.mean()) * (p - p.mean())) / (np.var(g) + eps)
    b_ref = p.mean() - A_ref * g.mean()
    np.testing.assert_allclose(A, A_ref, rtol=1e-12)
    np.testing.assert_allclose(b, b_ref, rtol=1e-12)


# ---------------------------------------------------------------- adjoint

@pytest.mark.parametrize("case", CASES)
def test_backward_matches_torch_autograd(case):
    N, C, hl, wl, h, w, r, eps = case
    d = synth.ragged_case(21, N, C, hl, wl, h, w)
    R = synth.upstream_grad(1, d["I_h"].shape)
    p = d["p_l"].clone().requires_grad_(True)
    gl = d["I_l"].clone().requires_grad_(True)
    gh = d["I_h"].clone().requires_grad_(True)
    (TC.gf(p, gl, gh, r, eps) * R).sum().backward()
    dp, dIl, dIh = O.backward(R, d["p_l"], d["I_l"], d["I_h"], r, eps)
    for got, ref in ((dp, p.grad), (dIl, gl.grad), (dIh, gh.grad)):
        ref = ref.numpy()
        err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
        assert err < 1e-10, err


def _fd_check(fun, x, grad, n_probe=None, seed=0):
    """Central differences of the scalar fun at x against grad (norm-wise)."""
    idx = list(np.ndindex(*x.shape))
    if n_probe is not None and n_probe < len(idx):
        sel = np.random.default_rng(seed).choice(len(idx), n_probe, replace=False)
        idx = [idx[i] for i in sel]
    fd = np.empty(len(idx))
    an = np.empty(len(idx))
    for k, i in enumerate(idx):
        # step ~ cube root of FP64 epsilon balances truncation and rounding error
        hstep = 5e-6 * max(1.0, abs(x[i]))
        x0 = x[i]
        x[i] = x0 + hstep
        fp = fun()
        x[i] = x0 - hstep
        fm = fun()
        x[i] = x0
        fd[k] = (fp - fm) / (2 * hstep)
        an[k] = grad[i]
    return np.linalg.norm(fd - an) / np.linalg.norm(an)


@pytest.mark.parametrize("hl,wl,h,w,r,eps", [(4, 4, 16, 16, 1, 1e-2), (8, 8, 16, 16, 2, 1e-3),
                                             (5, 6, 16, 16, 1, 1e-2)])
def test_backward_finite_differences(hl, wl, h, w, r, eps):
    d = synth.ragged_case(31, 1, 1, hl, wl, h, w)
    P = d["p_l"][0, 0].numpy().copy()
    Gl = d["I_l"][0, 0].numpy().copy()
    Gh = d["I_h"][0, 0].numpy().copy()
    R = synth.upstream_grad(2, (h, w)).numpy()
    dP, dGl, dGh = O.backward_plane(R, P, Gl, Gh, r, eps)

    def loss():
        return float(np.sum(O.forward_plane(P, Gl, Gh, r, eps) * R))

    assert _fd_check(loss, P, dP) < 1e-6
    assert _fd_check(loss, Gl, dGl) < 1e-6
    assert _fd_check(loss, Gh, dGh, n_probe=64) < 1e-6


# ------------------------------------------------------- guidance transform

def test_guided_forward_and_backward_match_torch():
    N, C, f, hl, wl, r, eps = 2, 3, 4, 4, 5, 1, 1e-3
    d = synth.photo_like(41, N, C, hl, wl, f)
    g = synth.guide_weights(3)
    R = synth.upstream_grad(4, d["I_h"].shape)
    out = O.forward_guided(d["p_l"], d["I_h"], g["w1"], g["w2"], g["b2"], r, eps)
    p = d["p_l"].clone().requires_grad_(True)
    ih = d["I_h"].clone().requires_grad_(True)
    w1 = g["w1"].clone().requires_grad_(True)
    w2 = g["w2"].clone().requires_grad_(True)
    b2 = g["b2"].clone().requires_grad_(True)
    ref = TC.gf_guided(p, ih, w1, w2, b2, r, eps)
    np.testing.assert_allclose(out, ref.detach().numpy(), rtol=0, atol=1e-12)
    (ref * R).sum().backward()
    got = O.backward_guided(R, d["p_l"], d["I_h"], g["w1"], g["w2"], g["b2"], r, eps)
    for a, b in zip(got[:4], (p.grad, ih.grad, w1.grad, w2.grad)):
        b = b.numpy()
        assert np.linalg.norm(a - b) / np.linalg.norm(b) < 1e-10
    # Adding a constant to the guide leaves the layer unchanged (b absorbs it:
    # b -> b - A c, so Abar_h c - f_up(f_mu(A c)) = 0), hence dL/db2 = 0.
    assert np.max(np.abs(got[4])) < 1e-12 and np.max(np.abs(b2.grad.numpy())) < 1e-12


def test_guided_backward_finite_differences():
    C, f, hl, wl, r, eps = 3, 4, 4, 4, 1, 1e-2
    d = synth.photo_like(42, 1, C, hl, wl, f)
    Ih = d["I_h"].numpy().copy()
    # keep away from the leaky-ReLU kink so central differences are valid:
    # draw weight seeds until no hidden pre-activation is within 1e-4 of 0
    for seed in range(5, 200):
        g = {k: v.numpy().copy() for k, v in synth.guide_weights(seed).items()}
        _, Z = O.guide_apply(Ih[0], g["w1"], g["w2"], g["b2"])
        if np.min(np.abs(Z)) > 1e-4:
            break
    assert np.min(np.abs(Z)) > 1e-4
    P = d["p_l"].numpy().copy()
    R = synth.upstream_grad(6, Ih.shape).numpy()
    dP, dI, dw1, dw2, db2 = O.backward_guided(R, P, Ih, g["w1"], g["w2"], g["b2"], r, eps)

    def loss():
        return float(np.sum(O.forward_guided(P, Ih, g["w1"], g["w2"], g["b2"], r, eps) * R))

    assert _fd_check(loss, P, dP) < 1e-6
    assert _fd_check(loss, Ih, dI, n_probe=48) < 1e-6
    assert _fd_check(loss, g["w1"], dw1) < 1e-6
    assert _fd_check(loss, g["w2"], dw2) < 1e-6
    assert np.max(np.abs(db2)) < 1e-12  # guide-shift invariance


# ------------------------------- the transform applied to each guide (F(I_l))

@pytest.mark.parametrize("mean_ab", [True, False])
def test_guided_separate_matches_torch(mean_ab):
    N, C, f, hl, wl, r, eps = 2, 3, 4, 5, 4, 1, 1e-3
    d = synth.photo_like(45, N, C, hl, wl, f)
    g = synth.guide_weights(7)
    R = synth.upstream_grad(8, d["I_h"].shape)
    out = O.forward_guided_separate(d["p_l"], d["I_l"], d["I_h"], g["w1"], g["w2"], g["b2"], r, eps,
                                    mean_ab=mean_ab)
    ts = {k: v.clone().requires_grad_(True) for k, v in (("p", d["p_l"]), ("il", d["I_l"]), ("ih", d["I_h"]),
                                                         ("w1", g["w1"]), ("w2", g["w2"]), ("b2", g["b2"]))}
    ref = TC.gf_guided_separate(ts["p"], ts["il"], ts["ih"], ts["w1"], ts["w2"], ts["b2"], r, eps,
                                mean_ab=mean_ab)
    np.testing.assert_allclose(out, ref.detach().numpy(), rtol=0, atol=1e-12)
    (ref * R).sum().backward()
    got = O.backward_guided_separate(R, d["p_l"], d["I_l"], d["I_h"], g["w1"], g["w2"], g["b2"], r, eps,
                                     mean_ab=mean_ab)
    for a, k in zip(got[:5], ("p", "il", "ih", "w1", "w2")):
        b = ts[k].grad.numpy()
        assert np.linalg.norm(a - b) / np.linalg.norm(b) < 1e-10, k
    # a constant added to both guides is absorbed by b, so d b2 vanishes here too
    assert np.max(np.abs(got[5])) < 1e-12 and np.max(np.abs(ts["b2"].grad.numpy())) < 1e-12


def test_guided_separate_equals_block_mean_form_on_blocky_guides():
    """With I_h constant on every f x f block and I_l its block values, F(I_l) is the block mean of F(I_h)."""
    N, C, f, hl, wl, r, eps = 1, 3, 4, 6, 5, 1, 1e-3
    d = synth.photo_like(46, N, C, hl, wl, f)
    I_l = d["I_l"]
    I_h = I_l.repeat_interleave(f, dim=2).repeat_interleave(f, dim=3)
    g = synth.guide_weights(9)
    a = O.forward_guided_separate(d["p_l"], I_l, I_h, g["w1"], g["w2"], g["b2"], r, eps)
    b = O.forward_guided(d["p_l"], I_h, g["w1"], g["w2"], g["b2"], r, eps)
    assert np.max(np.abs(a - b)) < 1e-12


def test_guided_separate_finite_differences():
    C, f, hl, wl, r, eps = 3, 4, 4, 4, 1, 1e-2
    d = synth.photo_like(47, 1, C, hl, wl, f)
    Il, Ih = d["I_l"].numpy().copy(), d["I_h"].numpy().copy()
    for seed in range(5, 200):  # away from the leaky-ReLU kink at both resolutions
        g = {k: v.numpy().copy() for k, v in synth.guide_weights(seed).items()}
        zh = O.guide_apply(Ih[0], g["w1"], g["w2"], g["b2"])[1]
        zl = O.guide_apply(Il[0], g["w1"], g["w2"], g["b2"])[1]
        if min(np.min(np.abs(zh)), np.min(np.abs(zl))) > 1e-4:
            break
    P = d["p_l"].numpy().copy()
    R = synth.upstream_grad(10, Ih.shape).numpy()
    _, dIl, dIh, dw1, dw2, _ = O.backward_guided_separate(R, P, Il, Ih, g["w1"], g["w2"], g["b2"], r, eps)

    def loss():
        return float(np.sum(O.forward_guided_separate(P, Il, Ih, g["w1"], g["w2"], g["b2"], r, eps) * R))

    assert _fd_check(loss, Il, dIl) < 1e-6
    assert _fd_check(loss, Ih, dIh, n_probe=32) < 1e-6
    assert _fd_check(loss, g["w1"], dw1) < 1e-6
    assert _fd_check(loss, g["w2"], dw2) < 1e-6


# ---------------------------------- the layer as printed (no mean of A, b)

@pytest.mark.parametrize("case", CASES)
def test_paper_literal_forward_and_backward_match_torch(case):
    # Sec. 3.2 / Algorithm 1 as printed: A_l, b_l upsampled directly
    N, C, hl, wl, h, w, r, eps = case
    d = synth.ragged_case(51, N, C, hl, wl, h, w)
    R = synth.upstream_grad(5, d["I_h"].shape)
    out = O.forward(d["p_l"], d["I_l"], d["I_h"], r, eps, mean_ab=False)
    p = d["p_l"].clone().requires_grad_(True)
    gl = d["I_l"].clone().requires_grad_(True)
    gh = d["I_h"].clone().requires_grad_(True)
    ref = TC.gf(p, gl, gh, r, eps, mean_ab=False)
    np.testing.assert_allclose(out, ref.detach().numpy(), rtol=0, atol=1e-10)
    (ref * R).sum().backward()
    got = O.backward(R, d["p_l"], d["I_l"], d["I_h"], r, eps, mean_ab=False)
    for a, b in zip(got, (p.grad, gl.grad, gh.grad)):
        b = b.numpy()
        assert np.linalg.norm(a - b) / np.linalg.norm(b) < 1e-10


def test_paper_literal_differs_from_mean_form_and_agrees_where_it_must():
    d = synth.ragged_case(52, 1, 1, 9, 11, 36, 44)
    lit = O.forward(d["p_l"], d["I_l"], d["I_h"], 1, 1e-3, mean_ab=False)
    mean = O.forward(d["p_l"], d["I_l"], d["I_h"], 1, 1e-3)
    assert np.max(np.abs(lit - mean)) > 1e-3  # the variants are distinct
    # r = 0: the box mean is the identity, so the two forms coincide
    lit0 = O.forward(d["p_l"], d["I_l"], d["I_h"], 0, 1e-3, mean_ab=False)
    np.testing.assert_allclose(lit0, O.forward(d["p_l"], d["I_l"], d["I_h"], 0, 1e-3), rtol=0, atol=1e-15)
    # a linear target p = a G + b with eps -> 0: A = a and b exactly per window, both forms
    G = d["I_l"][0, 0].numpy()
    P = 0.6 * G + 0.25
    Gh = d["I_h"][0, 0].numpy()
    lit_lin = O.forward_plane(P, G, Gh, 1, 1e-14, mean_ab=False)
    np.testing.assert_allclose(lit_lin, 0.6 * Gh + 0.25, rtol=0, atol=1e-7)


def test_paper_literal_finite_differences():
    d = synth.ragged_case(53, 1, 1, 6, 7, 24, 28)
    P = d["p_l"][0, 0].numpy().copy()
    Gl = d["I_l"][0, 0].numpy().copy()
    Gh = d["I_h"][0, 0].numpy().copy()
    R = synth.upstream_grad(3, (24, 28)).numpy()
    dP, dGl, dGh = O.backward_plane(R, P, Gl, Gh, 2, 1e-3, mean_ab=False)

    def loss():
        return float(np.sum(O.forward_plane(P, Gl, Gh, 2, 1e-3, mean_ab=False) * R))

    assert _fd_check(loss, P, dP) < 1e-6
    assert _fd_check(loss, Gl, dGl) < 1e-6
    assert _fd_check(loss, Gh, dGh, n_probe=48) < 1e-6


def test_paper_literal_guided_matches_torch():
    N, C, f, hl, wl, r, eps = 1, 3, 4, 5, 4, 1, 1e-3
    d = synth.photo_like(54, N, C, hl, wl, f)
    g = synth.guide_weights(7)
    R = synth.upstream_grad(8, d["I_h"].shape)
    out = O.forward_guided(d["p_l"], d["I_h"], g["w1"], g["w2"], g["b2"], r, eps, mean_ab=False)
    p = d["p_l"].clone().requires_grad_(True)
    ih = d["I_h"].clone().requires_grad_(True)
    w1 = g["w1"].clone().requires_grad_(True)
    w2 = g["w2"].clone().requires_grad_(True)
    ref = TC.gf_guided(p, ih, w1, w2, g["b2"], r, eps, mean_ab=False)
    np.testing.assert_allclose(out, ref.detach().numpy(), rtol=0, atol=1e-12)
    (ref * R).sum().backward()
    got = O.backward_guided(R, d["p_l"], d["I_h"], g["w1"], g["w2"], g["b2"], r, eps, mean_ab=False)
    for a, b in zip(got[:4], (p.grad, ih.grad, w1.grad, w2.grad)):
        b = b.numpy()
        assert np.linalg.norm(a - b) / np.linalg.norm(b) < 1e-10


# ------------------------------------------------------------- grey guide

def _grey_case(seed, N, n_in, C, hl, wl, h, w):
    """Guide with n_in channels, target with C channels (independent draws)."""
    g = synth.ragged_case(seed, N, n_in, hl, wl, h, w)
    p = synth.ragged_case(seed + 1, N, C, hl, wl, h, w)["p_l"]
    return p, g["I_l"], g["I_h"]


def test_grey_guide_with_one_channel_is_the_plain_filter():
    p, il, ih = _grey_case(40, 2, 1, 1, 6, 7, 18, 20)
    assert np.array_equal(O.forward_grey(p, il, ih, 1, 1e-2), O.forward(p, il, ih, 1, 1e-2))
    R = synth.upstream_grad(3, ih.shape)
    for a, b in zip(O.backward_grey(R, p, il, ih, 1, 1e-2), O.backward(R, p, il, ih, 1, 1e-2)):
        assert np.array_equal(a, b)


def test_grey_guide_of_equal_channels_is_that_channel():
    p, il, ih = _grey_case(41, 1, 1, 2, 5, 6, 20, 24)
    il3, ih3 = il.repeat(1, 3, 1, 1), ih.repeat(1, 3, 1, 1)
    got = O.forward_grey(p, il3, ih3, 2, 1e-3)
    ref = O.forward(p, il.repeat(1, 2, 1, 1), ih.repeat(1, 2, 1, 1), 2, 1e-3)
    assert np.max(np.abs(got - ref)) < 1e-14


@pytest.mark.parametrize("n_in,C", [(3, 1), (1, 3), (3, 2)])
def test_grey_forward_and_backward_match_torch(n_in, C):
    p, il, ih = _grey_case(42, 2, n_in, C, 5, 6, 15, 17)
    R = synth.upstream_grad(4, (2, C, 15, 17))
    pt = p.clone().requires_grad_(True)
    ilt = il.clone().requires_grad_(True)
    iht = ih.clone().requires_grad_(True)
    # the channel mean and its broadcast written with torch; autograd gives the adjoint
    Gl = ilt.mean(dim=1, keepdim=True).expand(-1, C, -1, -1)
    Gh = iht.mean(dim=1, keepdim=True).expand(-1, C, -1, -1)
    out = TC.gf(pt, Gl, Gh, 1, 1e-2)
    (out * R).sum().backward()
    assert np.max(np.abs(O.forward_grey(p, il, ih, 1, 1e-2) - out.detach().numpy())) < 1e-12
    got = O.backward_grey(R, p, il, ih, 1, 1e-2)
    for a, b in zip(got, (pt.grad, ilt.grad, iht.grad)):
        b = b.numpy()
        assert np.linalg.norm(a - b) / np.linalg.norm(b) < 1e-10
    if n_in != C:  # an adjoint that divides by the output channels instead is caught
        wrong = got[2] * n_in / C
        assert np.linalg.norm(wrong - iht.grad.numpy()) / np.linalg.norm(iht.grad.numpy()) > 0.1


def test_grey_backward_finite_differences():
    p, il, ih = _grey_case(43, 1, 3, 2, 4, 4, 12, 12)
    p, il, ih = p.numpy().copy(), il.numpy().copy(), ih.numpy().copy()
    R = synth.upstream_grad(5, (1, 2, 12, 12)).numpy()
    _, dil, dih = O.backward_grey(R, p, il, ih, 1, 1e-2)

    def loss():
        return float((O.forward_grey(p, il, ih, 1, 1e-2) * R).sum())
    assert _fd_check(loss, il, dil, n_probe=12) < 1e-6
    assert _fd_check(loss, ih, dih, n_probe=12, seed=1) < 1e-6


def test_grey_guide_is_the_exact_channel_mean():
    """Sec. 4.2: the grey guide is the average along the channel axis; brute
    force over the channels, in exact rational arithmetic on dyadic inputs."""
    from fractions import Fraction
    x = rng(44).integers(0, 2 ** 20, size=(2, 3, 5, 6)) / 2.0 ** 20
    G = O.grey_guide(x)
    assert G.shape == (2, 1, 5, 6)
    for n in range(2):
        for y in range(5):
            for xx in range(6):
                exact = sum(Fraction(float(x[n, k, y, xx])) for k in range(3)) / 3
                assert abs(Fraction(float(G[n, 0, y, xx])) - exact) <= Fraction(1, 2 ** 53)


# ------------------------------------------------ planted mistakes (pins bite)

def test_pins_catch_a_dropped_mean_of_coefficients(monkeypatch):
    # Planting the paper-literal variant (no box mean of A, b) must fail the
    # torch-composition pin, which proves that pin sees that step.
    case = CASES[1]
    N, C, hl, wl, h, w, r, eps = case
    d = synth.ragged_case(11, N, C, hl, wl, h, w)
    monkeypatch.setattr(O.dgf_oracle, "mean_coefficients",
                        lambda G, P, r, eps: O.dgf_oracle.coefficients(G, P, r, eps))
    out = O.forward(d["p_l"], d["I_l"], d["I_h"], r, eps)
    ref = TC.gf(d["p_l"], d["I_l"], d["I_h"], r, eps).numpy()
    assert np.max(np.abs(out - ref)) > 1e-4


def test_pins_catch_a_sign_error_in_the_adjoint(monkeypatch):
    d = synth.ragged_case(31, 1, 1, 4, 4, 16, 16)
    P = d["p_l"][0, 0].numpy().copy()
    Gl = d["I_l"][0, 0].numpy().copy()
    Gh = d["I_h"][0, 0].numpy().copy()
    R = synth.upstream_grad(2, (16, 16)).numpy()
    good = O.backward_plane(R, P, Gl, Gh, 1, 1e-2)[1]
    real_T = O.dgf_oracle.box_mean_T
    calls = {"n": 0}

    def flipped(y, r):
        calls["n"] += 1
        out = real_T(y, r)
        return -out if calls["n"] == 6 else out  # the f_mu^T of d Sigma_G
    monkeypatch.setattr(O.dgf_oracle, "box_mean_T", flipped)
    bad = O.backward_plane(R, P, Gl, Gh, 1, 1e-2)[1]
    assert np.linalg.norm(bad - good) / np.linalg.norm(good) > 1e-3
