"""FP64 CPU oracle of the fast guided filtering layer.

TEST INFRASTRUCTURE.  This module is the correctness reference that the
CUDA path is checked against; only the tests, ``__graft_entry__.smoke()``
and the CPU-baseline / reference legs of ``bench.py`` may import it.  It
shares no code with the CUDA path and never calls it.

What it computes (Wu et al., "Fast End-to-End Trainable Guided Filter"):

* Sec. 3.2, Eq. 1 - the local linear model O_l ~ A_l * I_l + b_l inside
  every (2r+1)^2 window w_k of the low-resolution guide, fitted by least
  squares: A = cov_k(G, P) / (var_k(G) + eps), b = mean_k(P) - A mean_k(G).
* Sec. 3.3 - the mean filter f_mu is a box filter of radius r; A and b are
  box-averaged once more at low resolution (He et al.'s fast guided filter,
  which the paper builds on), then upsampled bilinearly (f_up) and applied
  to the high-resolution guide: O_h = A_h * G_h + b_h (Eq. 2).
* Algorithm 1 - the gradients of O_h with respect to O_l (= p_l), I_l and
  I_h, extended with the transpose of the extra box mean of A and b.
* Sec. 3.4 - the guidance transform F: 1x1 conv, leaky ReLU (slope 0.2),
  1x1 conv, applied per pixel; with it the low-resolution guide is the
  f x f block mean of F(I_h).
* Sec. 3.4, read literally - F applied to each resolution on its own:
  G_l = F(I_l), G_h = F(I_h) (``forward_guided_separate``).
* Sec. 4.2 (DGF_b) - when the guide and the output differ in channel count,
  F is the mean over the guide's channels (a grey guide), used for every
  output channel.

Readings of points the paper leaves open (each is also listed in the design
notes): windows are clipped to the image and divided by the number of
in-image pixels N_k; variances are population variances (divide by N_k);
bilinear upsampling uses half-pixel centres (align_corners=False) with the
source coordinate clamped at 0 and the index clamped at the last sample.

Everything is plain FP64 numpy: window sums are direct sums over the
(2r+1)^2 offsets (vectorised over the window centre), the statistics are
formed in two passes (means first, then centred sums), and bilinear
interpolation is the product with explicit interpolation matrices.
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "window_count",
    "window_sum",
    "box_mean",
    "box_mean_T",
    "window_stats",
    "coefficients",
    "mean_coefficients",
    "bilinear_matrix",
    "upsample",
    "upsample_T",
    "forward_plane",
    "backward_plane",
    "forward",
    "backward",
    "guide_apply",
    "block_mean",
    "forward_guided",
    "backward_guided",
    "forward_guided_separate",
    "backward_guided_separate",
    "grey_guide",
    "forward_grey",
    "backward_grey",
]


# --------------------------------------------------------------------------
# Box (mean) filter f_mu over clipped windows - Sec. 3.3
# --------------------------------------------------------------------------

def _overlap(n: int, d: int):
    """Slices (dst, src) with dst index k and src index k + d, both in [0, n)."""
    if abs(d) >= n:
        return slice(0, 0), slice(0, 0)
    if d >= 0:
        return slice(0, n - d), slice(d, n)
    return slice(-d, n), slice(0, n + d)


def window_count(h: int, w: int, r: int) -> np.ndarray:
    """N_k: number of in-image pixels of the window of radius r centred at k."""
    n = np.zeros((h, w))
    for dy in range(-r, r + 1):
        yd, _ = _overlap(h, dy)
        for dx in range(-r, r + 1):
            xd, _ = _overlap(w, dx)
            n[yd, xd] += 1.0
    return n


def window_sum(x: np.ndarray, r: int) -> np.ndarray:
    """S_k = sum of x_i over the in-image pixels i of window k (direct sum)."""
    h, w = x.shape
    s = np.zeros((h, w))
    for dy in range(-r, r + 1):
        yd, ys = _overlap(h, dy)
        for dx in range(-r, r + 1):
            xd, xs = _overlap(w, dx)
            s[yd, xd] += x[ys, xs]
    return s


def box_mean(x: np.ndarray, r: int) -> np.ndarray:
    """f_mu(x)_k = S_k / N_k."""
    h, w = x.shape
    return window_sum(x, r) / window_count(h, w, r)


def box_mean_T(y: np.ndarray, r: int) -> np.ndarray:
    """Transpose of f_mu: (f_mu^T y)_i = sum over windows m containing i of y_m / N_m.

    Window membership is symmetric (i in w_m iff m in w_i, both clipped to
    the image), so this is the window sum of y / N.
    """
    h, w = y.shape
    return window_sum(y / window_count(h, w, r), r)


def window_stats(G: np.ndarray, P: np.ndarray, r: int):
    """Per-window mean_G, mean_P, var_G, cov_GP (two-pass, centred).

    Returns (mu, nu, var, cov) with var and cov population moments over the
    clipped window (Sec. 3.2; Algorithm 1's \\bar G_l, \\bar O_l, Sigma_G,
    Sigma_GO).
    """
    h, w = G.shape
    N = window_count(h, w, r)
    mu = window_sum(G, r) / N
    nu = window_sum(P, r) / N
    var = np.zeros((h, w))
    cov = np.zeros((h, w))
    for dy in range(-r, r + 1):
        yd, ys = _overlap(h, dy)
        for dx in range(-r, r + 1):
            xd, xs = _overlap(w, dx)
            dg = G[ys, xs] - mu[yd, xd]
            dp = P[ys, xs] - nu[yd, xd]
            var[yd, xd] += dg * dg
            cov[yd, xd] += dg * dp
    return mu, nu, var / N, cov / N


def coefficients(G: np.ndarray, P: np.ndarray, r: int, eps: float):
    """A_l, b_l of the local linear model (Eq. 1, least squares with ridge eps)."""
    mu, nu, var, cov = window_stats(G, P, r)
    A = cov / (var + eps)
    b = nu - A * mu
    return A, b


def mean_coefficients(G: np.ndarray, P: np.ndarray, r: int, eps: float):
    """Abar = f_mu(A), bbar = f_mu(b) (the second box mean at low resolution)."""
    A, b = coefficients(G, P, r, eps)
    return box_mean(A, r), box_mean(b, r)


# --------------------------------------------------------------------------
# Bilinear upsampler f_up - Sec. 3.3
# --------------------------------------------------------------------------

def bilinear_matrix(n_out: int, n_in: int) -> np.ndarray:
    """(n_out, n_in) matrix of linear-interpolation weights.

    Output sample y sits at source coordinate t = (y + 0.5) n_in / n_out - 0.5,
    clamped below at 0; it blends samples i0 = floor(t) and i1 = i0 + 1
    (clamped to n_in - 1) with weights 1 - lam and lam, lam = t - i0.
    """
    W = np.zeros((n_out, n_in))
    scale = n_in / n_out
    for y in range(n_out):
        t = max((y + 0.5) * scale - 0.5, 0.0)
        i0 = min(int(np.floor(t)), n_in - 1)
        i1 = min(i0 + 1, n_in - 1)
        lam = t - i0
        W[y, i0] += 1.0 - lam
        W[y, i1] += lam
    return W


def upsample(X: np.ndarray, h: int, w: int) -> np.ndarray:
    """f_up: (h_l, w_l) -> (h, w), separable bilinear."""
    h_l, w_l = X.shape
    return bilinear_matrix(h, h_l) @ X @ bilinear_matrix(w, w_l).T


def upsample_T(Z: np.ndarray, h_l: int, w_l: int) -> np.ndarray:
    """Transpose of f_up: (h, w) -> (h_l, w_l)."""
    h, w = Z.shape
    return bilinear_matrix(h, h_l).T @ Z @ bilinear_matrix(w, w_l)


# --------------------------------------------------------------------------
# One plane (one image, one channel) of the layer
# --------------------------------------------------------------------------

def forward_plane(P: np.ndarray, G_l: np.ndarray, G_h: np.ndarray, r: int,
                  eps: float, mean_ab: bool = True) -> np.ndarray:
    """O_h = f_up(Abar) * G_h + f_up(bbar) (Eq. 2 with the mean of A, b).

    mean_ab=False is the layer as Sec. 3.2 prints it: A_l, b_l upsampled
    directly, O_h = f_up(A_l) * G_h + f_up(b_l).
    """
    h, w = G_h.shape
    if mean_ab:
        Abar, bbar = mean_coefficients(G_l, P, r, eps)
    else:
        Abar, bbar = coefficients(G_l, P, r, eps)
    return upsample(Abar, h, w) * G_h + upsample(bbar, h, w)


def backward_plane(R: np.ndarray, P: np.ndarray, G_l: np.ndarray, G_h: np.ndarray,
                   r: int, eps: float, mean_ab: bool = True):
    """Gradients of sum(O_h * R) for one plane, following Algorithm 1.

    Returns (dP, dG_l, dG_h).  The steps and names follow Algorithm 1
    (d b_l, d A_l, d Sigma_GO, d Sigma_G, d Obar_l, d O_l, d Gbar_l, d G_l,
    d I_h), with two extensions: f_up acts on the box-averaged Abar, bbar,
    so its transpose is followed by f_mu^T; and each ".grad f_mu" of the
    algorithm is the transpose box_mean_T of the clipped mean filter.
    With mean_ab=False there is no f_mu^T after f_up^T: Algorithm 1 as printed.
    """
    h, w = G_h.shape
    h_l, w_l = P.shape
    mu, nu, var, cov = window_stats(G_l, P, r)        # \bar G_l, \bar O_l, Sigma_G, Sigma_GO
    A = cov / (var + eps)
    Abar = box_mean(A, r) if mean_ab else A
    # d b_l = dO_h . grad_{b_l} f_up  (through bbar = f_mu(b))
    d_bbar = upsample_T(R, h_l, w_l)
    d_b = box_mean_T(d_bbar, r) if mean_ab else d_bbar
    # d A_l = dO_h * G_h . grad_{A_l} f_up - d b_l * \bar G_l
    d_Abar = upsample_T(R * G_h, h_l, w_l)
    d_A = (box_mean_T(d_Abar, r) if mean_ab else d_Abar) - d_b * mu
    # d Sigma_GO = d A_l / (Sigma_G + eps);  d Sigma_G = -d A_l Sigma_GO / (Sigma_G + eps)^2
    d_cov = d_A / (var + eps)
    d_var = -d_A * cov / (var + eps) ** 2
    # d \bar O_l = d b_l - d Sigma_GO * \bar G_l
    d_nu = d_b - d_cov * mu
    # d O_l = d Sigma_GO . grad_{G_l O_l} f_mu * G_l + d \bar O_l . grad_{O_l} f_mu
    dP = box_mean_T(d_cov, r) * G_l + box_mean_T(d_nu, r)
    # d \bar G_l = -d b_l * A_l - d Sigma_GO * \bar O_l - 2 d Sigma_G * \bar G_l
    d_mu = -d_b * A - d_cov * nu - 2.0 * d_var * mu
    # d G_l = d Sigma_GO . grad f_mu * O_l + 2 d Sigma_G . grad f_mu * G_l + d \bar G_l . grad f_mu
    dG_l = (box_mean_T(d_cov, r) * P + 2.0 * box_mean_T(d_var, r) * G_l
            + box_mean_T(d_mu, r))
    # d I_h = dO_h * A_h (identity F)
    dG_h = R * upsample(Abar, h, w)
    return dP, dG_l, dG_h


# --------------------------------------------------------------------------
# Batched NCHW wrappers, per-channel guide (F = identity)
# --------------------------------------------------------------------------

def _f64(x) -> np.ndarray:
    if hasattr(x, "detach"):
        x = x.detach().cpu().double().numpy()
    return np.asarray(x, dtype=np.float64)


def forward(p_l, I_l, I_h, r: int, eps: float, planes=None, mean_ab: bool = True) -> np.ndarray:
    """O_h for NCHW inputs; ``planes`` optionally restricts to [(n, c), ...]."""
    p_l, I_l, I_h = _f64(p_l), _f64(I_l), _f64(I_h)
    N, C = I_h.shape[:2]
    out = np.full(I_h.shape, np.nan)
    for n in range(N):
        for c in range(C):
            if planes is not None and (n, c) not in planes:
                continue
            out[n, c] = forward_plane(p_l[n, c], I_l[n, c], I_h[n, c], r, eps, mean_ab)
    return out


def backward(R, p_l, I_l, I_h, r: int, eps: float, planes=None, mean_ab: bool = True):
    """(dp_l, dI_l, dI_h) of sum(O_h * R) for NCHW inputs."""
    R, p_l, I_l, I_h = _f64(R), _f64(p_l), _f64(I_l), _f64(I_h)
    N, C = I_h.shape[:2]
    dp = np.full(p_l.shape, np.nan)
    dIl = np.full(I_l.shape, np.nan)
    dIh = np.full(I_h.shape, np.nan)
    for n in range(N):
        for c in range(C):
            if planes is not None and (n, c) not in planes:
                continue
            dp[n, c], dIl[n, c], dIh[n, c] = backward_plane(
                R[n, c], p_l[n, c], I_l[n, c], I_h[n, c], r, eps, mean_ab)
    return dp, dIl, dIh


# --------------------------------------------------------------------------
# Guidance transform F (Sec. 3.4) and the layer with it
# --------------------------------------------------------------------------

def guide_apply(I: np.ndarray, w1: np.ndarray, w2: np.ndarray, b2: np.ndarray,
                slope: float = 0.2):
    """G = w2 . lrelu(w1 . I) + b2 per pixel for a (C_in, h, w) image.

    Returns (G, Z) with Z the pre-activation of the hidden layer.
    """
    Z = np.einsum("kc,chw->khw", w1, I)
    H = np.where(Z > 0.0, Z, slope * Z)
    G = np.einsum("ck,khw->chw", w2, H) + b2[:, None, None]
    return G, Z


def block_mean(X: np.ndarray, f: int) -> np.ndarray:
    """Mean over each f x f block of a (C, h, w) array (h, w divisible by f)."""
    C, h, w = X.shape
    out = np.zeros((C, h // f, w // f))
    for qy in range(f):
        for qx in range(f):
            out += X[:, qy::f, qx::f]
    return out / (f * f)


def forward_guided(p_l, I_h, w1, w2, b2, r: int, eps: float, slope: float = 0.2,
                   images=None, mean_ab: bool = True) -> np.ndarray:
    """O_h with G_h = F(I_h) and G_l = block_mean(G_h, f), per channel c."""
    p_l, I_h = _f64(p_l), _f64(I_h)
    w1, w2, b2 = _f64(w1), _f64(w2), _f64(b2)
    N, C, h, w = I_h.shape
    f = h // p_l.shape[2]
    out = np.full(I_h.shape, np.nan)
    for n in range(N):
        if images is not None and n not in images:
            continue
        G_h, _ = guide_apply(I_h[n], w1, w2, b2, slope)
        G_l = block_mean(G_h, f)
        for c in range(C):
            out[n, c] = forward_plane(p_l[n, c], G_l[c], G_h[c], r, eps, mean_ab)
    return out


def backward_guided(R, p_l, I_h, w1, w2, b2, r: int, eps: float, slope: float = 0.2,
                    images=None, mean_ab: bool = True):
    """(dp_l, dI_h, dw1, dw2, db2) of sum(O_h * R) with the guidance transform.

    dG_h collects dO_h * A_h and, through the block mean, dG_l / f^2 on every
    pixel of its block; it is then chained through the 1x1 convolutions and
    the leaky ReLU (Algorithm 1's last two lines, d I = d G . grad F).
    Weight gradients are summed over the images processed.
    """
    R, p_l, I_h = _f64(R), _f64(p_l), _f64(I_h)
    w1, w2, b2 = _f64(w1), _f64(w2), _f64(b2)
    N, C, h, w = I_h.shape
    f = h // p_l.shape[2]
    dp = np.full(p_l.shape, np.nan)
    dI = np.full(I_h.shape, np.nan)
    dw1 = np.zeros_like(w1)
    dw2 = np.zeros_like(w2)
    db2 = np.zeros_like(b2)
    for n in range(N):
        if images is not None and n not in images:
            continue
        G_h, Z = guide_apply(I_h[n], w1, w2, b2, slope)
        H = np.where(Z > 0.0, Z, slope * Z)
        G_l = block_mean(G_h, f)
        dG_h = np.zeros_like(G_h)
        for c in range(C):
            dp[n, c], dG_l, dG_h[c] = backward_plane(R[n, c], p_l[n, c], G_l[c],
                                                     G_h[c], r, eps, mean_ab)
            dG_h[c] += np.repeat(np.repeat(dG_l, f, axis=0), f, axis=1) / (f * f)
        dw2 += np.einsum("chw,khw->ck", dG_h, H)
        db2 += dG_h.sum(axis=(1, 2))
        dH = np.einsum("ck,chw->khw", w2, dG_h)
        dZ = dH * np.where(Z > 0.0, 1.0, slope)
        dw1 += np.einsum("khw,chw->kc", dZ, I_h[n])
        dI[n] = np.einsum("kc,khw->chw", w1, dZ)
    return dp, dI, dw1, dw2, db2


def forward_guided_separate(p_l, I_l, I_h, w1, w2, b2, r: int, eps: float, slope: float = 0.2,
                            mean_ab: bool = True) -> np.ndarray:
    """O_h with the transform applied to each guide: G_l = F(I_l), G_h = F(I_h)."""
    p_l, I_l, I_h = _f64(p_l), _f64(I_l), _f64(I_h)
    w1, w2, b2 = _f64(w1), _f64(w2), _f64(b2)
    N, C = I_h.shape[:2]
    out = np.full(I_h.shape, np.nan)
    for n in range(N):
        G_h, _ = guide_apply(I_h[n], w1, w2, b2, slope)
        G_l, _ = guide_apply(I_l[n], w1, w2, b2, slope)
        for c in range(C):
            out[n, c] = forward_plane(p_l[n, c], G_l[c], G_h[c], r, eps, mean_ab)
    return out


def _guide_adjoint(I, Z, dG, w1, w2, slope):
    """d I, d w1, d w2, d b2 of a loss through G = F(I), given d G (C, h, w)."""
    H = np.where(Z > 0.0, Z, slope * Z)
    dw2 = np.einsum("chw,khw->ck", dG, H)
    db2 = dG.sum(axis=(1, 2))
    dH = np.einsum("ck,chw->khw", w2, dG)
    dZ = dH * np.where(Z > 0.0, 1.0, slope)
    dw1 = np.einsum("khw,chw->kc", dZ, I)
    dI = np.einsum("kc,khw->chw", w1, dZ)
    return dI, dw1, dw2, db2


def backward_guided_separate(R, p_l, I_l, I_h, w1, w2, b2, r: int, eps: float, slope: float = 0.2,
                             mean_ab: bool = True):
    """(dp_l, dI_l, dI_h, dw1, dw2, db2) of sum(O_h * R) with G_l = F(I_l), G_h = F(I_h).

    Algorithm 1 per channel gives d G_l and d G_h; each goes back through the
    transform of its own resolution (the last line, d I = d G . grad F), and
    the weight gradients add the two resolutions' terms.
    """
    R, p_l, I_l, I_h = _f64(R), _f64(p_l), _f64(I_l), _f64(I_h)
    w1, w2, b2 = _f64(w1), _f64(w2), _f64(b2)
    N, C = I_h.shape[:2]
    dp = np.full(p_l.shape, np.nan)
    dIl = np.full(I_l.shape, np.nan)
    dIh = np.full(I_h.shape, np.nan)
    dw1, dw2, db2 = np.zeros_like(w1), np.zeros_like(w2), np.zeros_like(b2)
    for n in range(N):
        G_h, Z_h = guide_apply(I_h[n], w1, w2, b2, slope)
        G_l, Z_l = guide_apply(I_l[n], w1, w2, b2, slope)
        dG_l = np.zeros_like(G_l)
        dG_h = np.zeros_like(G_h)
        for c in range(C):
            dp[n, c], dG_l[c], dG_h[c] = backward_plane(R[n, c], p_l[n, c], G_l[c], G_h[c], r, eps, mean_ab)
        for I, Z, dG, dI in ((I_h[n], Z_h, dG_h, dIh), (I_l[n], Z_l, dG_l, dIl)):
            gI, g1, g2, gb = _guide_adjoint(I, Z, dG, w1, w2, slope)
            dI[n] = gI
            dw1 += g1
            dw2 += g2
            db2 += gb
    return dp, dIl, dIh, dw1, dw2, db2


# --------------------------------------------------------------------------
# Grey guide (DGF_b with differing channel counts, Sec. 4.2)
# --------------------------------------------------------------------------

def grey_guide(I) -> np.ndarray:
    """(N, 1, h, w): the mean of an (N, n_I, h, w) guide along its channel axis.

    Sec. 4.2 (DGF_b): when the guide and the output differ in channel count,
    F turns the guide into a grey image by averaging along the channel axis.
    The mean is exact (FP64); nothing about its storage or summation order
    is part of the definition.
    """
    return _f64(I).mean(axis=1, keepdims=True)


def forward_grey(p_l, I_l, I_h, r: int, eps: float, mean_ab: bool = True) -> np.ndarray:
    """O_h (N, C, h, w) with the grey guide of I_l, I_h (N, n_I, ...) for every output channel."""
    p_l = _f64(p_l)
    C = p_l.shape[1]
    G_l = np.repeat(grey_guide(I_l), C, axis=1)
    G_h = np.repeat(grey_guide(I_h), C, axis=1)
    return forward(p_l, G_l, G_h, r, eps, mean_ab=mean_ab)


def backward_grey(R, p_l, I_l, I_h, r: int, eps: float, mean_ab: bool = True):
    """(dp_l, dI_l, dI_h) of sum(O_h * R) with the grey guide.

    The grey guide feeds every output channel, so its gradient is the sum of
    the channels' guide gradients (Algorithm 1 per channel); the channel mean
    hands 1 / n_I of it to each guide channel.
    """
    p_l, I_l, I_h = _f64(p_l), _f64(I_l), _f64(I_h)
    C, n_in = p_l.shape[1], I_l.shape[1]
    G_l = np.repeat(grey_guide(I_l), C, axis=1)
    G_h = np.repeat(grey_guide(I_h), C, axis=1)
    dp, dG_l, dG_h = backward(R, p_l, G_l, G_h, r, eps, mean_ab=mean_ab)
    dI_l = np.repeat(dG_l.sum(axis=1, keepdims=True) / n_in, n_in, axis=1)
    dI_h = np.repeat(dG_h.sum(axis=1, keepdims=True) / n_in, n_in, axis=1)
    return dp, dI_l, dI_h
