"""An independent FP64 torch formulation of the fast guided filtering layer.

Used only by the oracle's pin tests.  It is He et al.'s textbook fast
guided filter written with library routines (``avg_pool2d`` with
``count_include_pad=False`` for the clipped box mean, ``interpolate`` in
bilinear mode with ``align_corners=False`` for the upsampler) and the
uncentred moments E[x y] - E[x] E[y]; autograd supplies its gradients.  It
shares no code with the oracle, so agreement pins the oracle's window
clipping, counts, centred sums, interpolation convention and hand-derived
adjoint.
"""
import torch
import torch.nn.functional as F


def box(x: torch.Tensor, r: int) -> torch.Tensor:
    """Clipped-window mean of an (h, w) tensor."""
    return F.avg_pool2d(x[None, None], 2 * r + 1, stride=1, padding=r,
                        count_include_pad=False)[0, 0]


def up(x: torch.Tensor, h: int, w: int) -> torch.Tensor:
    return F.interpolate(x[None, None], size=(h, w), mode="bilinear",
                         align_corners=False)[0, 0]


def gf_plane(P, G_l, G_h, r: int, eps: float, mean_ab: bool = True):
    mu = box(G_l, r)
    nu = box(P, r)
    var = box(G_l * G_l, r) - mu * mu
    cov = box(G_l * P, r) - mu * nu
    A = cov / (var + eps)
    b = nu - A * mu
    h, w = G_h.shape
    if not mean_ab:  # the layer as printed: A_l, b_l upsampled directly
        return up(A, h, w) * G_h + up(b, h, w)
    return up(box(A, r), h, w) * G_h + up(box(b, r), h, w)


def gf(p_l, I_l, I_h, r: int, eps: float, mean_ab: bool = True):
    N, C = I_h.shape[:2]
    rows = []
    for n in range(N):
        rows.append(torch.stack([gf_plane(p_l[n, c], I_l[n, c], I_h[n, c], r, eps, mean_ab)
                                 for c in range(C)]))
    return torch.stack(rows)


def guide(I, w1, w2, b2, slope=0.2):
    """1x1 conv (no bias) -> leaky ReLU -> 1x1 conv (bias) on (N, C, h, w)."""
    z = F.conv2d(I, w1[:, :, None, None])
    hdn = F.leaky_relu(z, slope)
    return F.conv2d(hdn, w2[:, :, None, None], b2)


def gf_guided(p_l, I_h, w1, w2, b2, r: int, eps: float, slope=0.2, mean_ab: bool = True):
    f = I_h.shape[2] // p_l.shape[2]
    G_h = guide(I_h, w1, w2, b2, slope)
    G_l = F.avg_pool2d(G_h, f, stride=f)
    return gf(p_l, G_l, G_h, r, eps, mean_ab)


def gf_guided_separate(p_l, I_l, I_h, w1, w2, b2, r: int, eps: float, slope=0.2, mean_ab: bool = True):
    """The transform applied to each guide on its own: G_l = F(I_l), G_h = F(I_h)."""
    return gf(p_l, guide(I_l, w1, w2, b2, slope), guide(I_h, w1, w2, b2, slope), r, eps, mean_ab)
