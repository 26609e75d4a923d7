"""Seeded synthetic inputs for the guided filtering layer.

This module is shared by the tests, the benchmark and the FP64 oracle's
checks.  It holds none of the layer's own arithmetic: it only draws images
shaped like the paper's photo workloads (MIT-Adobe FiveK photos resized to
512s..2048s with a 64s low-resolution input, Sec. 5.3), which are not
available here and are replaced by the recipes below.

Every random number comes from numpy's PCG64 (``np.random.default_rng``);
image ``i`` of a batch uses seed ``base + i``.  Arrays are returned as FP64
``torch`` tensors on the CPU, laid out NCHW; callers cast them to the
storage dtype they test (FP32, BF16 or FP16).

Recipes
-------
* ``photo_like`` (configurations 1, 3, 4 and the p_l of configuration 5):
  I_h is U[0,1] noise plus 3 axis-aligned step edges (amplitude
  U[-0.5, 0.5] added on one side of a uniform position), clipped to [0,1];
  I_l is the f x f area mean of I_h (the "downsample" that feeds the
  low-resolution network in Sec. 4); p_l = clip(0.7 I_l + 0.1 + N(0, 0.05^2)).
* ``blobs_tone_curve`` (configuration 2): I_h = 0.5 + 40 anisotropic
  Gaussian blobs + 8 step edges + N(0, 0.02^2), clipped; I_l its 4x area
  mean; p_l a random monotone cubic tone curve of I_l per channel.
* ``mixed_sizes`` (configuration 4): 64 images, long side U[512, 4096],
  aspect U[0.5, 2], factor 4 or 8, radius in {1, 2, 4}; sizes rounded down
  to multiples of the factor.
* ``ragged_case``: arbitrary (h_l, w_l, h, w), including non-integer ratios,
  for edge-case tests; I_l is drawn independently of I_h.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np
import torch

__all__ = [
    "area_mean",
    "photo_like",
    "blobs_tone_curve",
    "ragged_case",
    "mixed_sizes",
    "guide_weights",
    "upstream_grad",
    "ImageSpec",
]


def area_mean(x: torch.Tensor, f: int) -> torch.Tensor:
    """f x f block average of an (..., h, w) tensor with h, w divisible by f.

    Input preparation only (the low-resolution input I_l of configurations
    1-4 is a downsampled photo); the layer itself never calls this.
    """
    *lead, h, w = x.shape
    assert h % f == 0 and w % f == 0, (h, w, f)
    y = x.reshape(*lead, h // f, f, w // f, f)
    return y.mean(dim=(-3, -1))


def _step_edges(rng: np.random.Generator, img: np.ndarray, n_edges: int) -> None:
    """Add n_edges axis-aligned steps in place to an (h, w) plane."""
    h, w = img.shape
    for _ in range(n_edges):
        axis = int(rng.integers(0, 2))
        amp = rng.uniform(-0.5, 0.5)
        if axis == 0:
            pos = int(rng.integers(0, h))
            img[pos:, :] += amp
        else:
            pos = int(rng.integers(0, w))
            img[:, pos:] += amp


def photo_like(seed: int, N: int, C: int, h_l: int, w_l: int, f: int,
               n_edges: int = 3) -> dict:
    """Noise-plus-edges photo stand-in (configurations 1, 3, 4)."""
    h, w = h_l * f, w_l * f
    I_h = np.empty((N, C, h, w))
    p_noise = np.empty((N, C, h_l, w_l))
    for n in range(N):
        rng = np.random.default_rng(seed + n)
        for c in range(C):
            plane = rng.uniform(0.0, 1.0, size=(h, w))
            _step_edges(rng, plane, n_edges)
            np.clip(plane, 0.0, 1.0, out=plane)
            I_h[n, c] = plane
            p_noise[n, c] = rng.normal(0.0, 0.05, size=(h_l, w_l))
    I_h_t = torch.from_numpy(I_h)
    I_l_t = area_mean(I_h_t, f)
    p_l_t = torch.clamp(0.7 * I_l_t + 0.1 + torch.from_numpy(p_noise), 0.0, 1.0)
    return {"I_h": I_h_t, "I_l": I_l_t, "p_l": p_l_t}


def _blob_field(rng: np.random.Generator, h: int, w: int, n_blobs: int,
                device: str) -> torch.Tensor:
    """0.5 + sum of anisotropic rotated Gaussian blobs on an h x w grid."""
    side = float(max(h, w))
    cy = rng.uniform(0, h, n_blobs)
    cx = rng.uniform(0, w, n_blobs)
    sy = rng.uniform(0.01, 0.2, n_blobs) * side
    sx = rng.uniform(0.01, 0.2, n_blobs) * side
    th = rng.uniform(0.0, math.pi, n_blobs)
    amp = rng.uniform(-0.5, 0.5, n_blobs)
    yy = torch.arange(h, dtype=torch.float64, device=device).view(h, 1)
    xx = torch.arange(w, dtype=torch.float64, device=device).view(1, w)
    field = torch.full((h, w), 0.5, dtype=torch.float64, device=device)
    for k in range(n_blobs):
        dy = yy - cy[k]
        dx = xx - cx[k]
        c, s = math.cos(th[k]), math.sin(th[k])
        u = (c * dx + s * dy) / sx[k]
        v = (-s * dx + c * dy) / sy[k]
        field += amp[k] * torch.exp(-0.5 * (u * u + v * v))
    return field


def blobs_tone_curve(seed: int, N: int, C: int, h_l: int, w_l: int, f: int,
                     device: str = "cpu") -> dict:
    """Smooth-blob photo stand-in with a tone-curve target (configuration 2).

    The blob field is evaluated with torch on ``device`` (the CPU for tests;
    the GPU may be used to speed up full-size benchmark inputs) from
    parameters drawn on the host, so the recipe is the same everywhere.
    """
    h, w = h_l * f, w_l * f
    I_h = torch.empty((N, C, h, w), dtype=torch.float64, device=device)
    coeffs = np.empty((N, C, 3))
    for n in range(N):
        rng = np.random.default_rng(seed + n)
        for c in range(C):
            plane = _blob_field(rng, h, w, 40, device)
            edges = np.zeros((h, w))
            _step_edges(rng, edges, 8)
            noise = rng.normal(0.0, 0.02, size=(h, w))
            plane += torch.from_numpy(edges + noise).to(device)
            I_h[n, c] = plane.clamp_(0.0, 1.0)
            a = rng.uniform(0.0, 1.0, 3)
            coeffs[n, c] = a / a.sum()
    I_l = area_mean(I_h, f)
    a = torch.from_numpy(coeffs).to(device)
    x = I_l
    p_l = (a[..., 0, None, None] * x + a[..., 1, None, None] * x * x
           + a[..., 2, None, None] * x * x * x)
    return {"I_h": I_h.cpu(), "I_l": I_l.cpu(), "p_l": p_l.cpu()}


def ragged_case(seed: int, N: int, C: int, h_l: int, w_l: int, h: int, w: int) -> dict:
    """Arbitrary-size case (any h_l <= h, w_l <= w) for edge-case tests."""
    rng = np.random.default_rng(seed)
    I_h = rng.uniform(0.0, 1.0, size=(N, C, h, w))
    I_l = rng.uniform(0.0, 1.0, size=(N, C, h_l, w_l))
    for n in range(N):
        for c in range(C):
            _step_edges(rng, I_h[n, c], 2)
            _step_edges(rng, I_l[n, c], 2)
    I_h = np.clip(I_h, 0.0, 1.0)
    I_l = np.clip(I_l, 0.0, 1.0)
    p_l = np.clip(0.7 * I_l + 0.1 + rng.normal(0.0, 0.05, size=I_l.shape), 0.0, 1.0)
    return {"I_h": torch.from_numpy(I_h), "I_l": torch.from_numpy(I_l),
            "p_l": torch.from_numpy(p_l)}


@dataclass
class ImageSpec:
    """One image of the mixed-size batch."""
    h: int
    w: int
    f: int
    r: int

    @property
    def h_l(self) -> int:
        return self.h // self.f

    @property
    def w_l(self) -> int:
        return self.w // self.f


def mixed_sizes(seed: int = 0, n: int = 64, long_lo: int = 512, long_hi: int = 4096,
                radii=(1, 2, 4), factors=(4, 8)) -> list:
    """Uneven image sizes for the batched path (configuration 4)."""
    rng = np.random.default_rng(seed)
    specs = []
    for _ in range(n):
        long_side = rng.uniform(long_lo, long_hi)
        aspect = rng.uniform(0.5, 2.0)
        f = int(factors[int(rng.integers(0, len(factors)))])
        r = int(radii[int(rng.integers(0, len(radii)))])
        if aspect >= 1.0:
            w, h = long_side, long_side / aspect
        else:
            h, w = long_side, long_side * aspect
        h = max(f, int(h) // f * f)
        w = max(f, int(w) // f * f)
        specs.append(ImageSpec(h=h, w=w, f=f, r=r))
    return specs


def guide_weights(seed: int, c_in: int = 3, hidden: int = 15, c_out: int = 3) -> dict:
    """N(0, 0.1^2) weights of the 1x1 -> LReLU -> 1x1 guidance transform.

    conv1 has no bias and conv2 has one (Table 1's bias row).
    """
    rng = np.random.default_rng(seed)
    w1 = rng.normal(0.0, 0.1, size=(hidden, c_in))
    w2 = rng.normal(0.0, 0.1, size=(c_out, hidden))
    b2 = rng.normal(0.0, 0.1, size=(c_out,))
    return {"w1": torch.from_numpy(w1), "w2": torch.from_numpy(w2),
            "b2": torch.from_numpy(b2)}


def upstream_grad(seed: int, shape, device: str = "cpu") -> torch.Tensor:
    """R ~ N(0, 1): the loss is sum(O_h * R), so dL/dO_h = R."""
    rng = np.random.default_rng(seed)
    return torch.from_numpy(rng.normal(0.0, 1.0, size=tuple(shape))).to(device)
