"""Torch-facing side of the guided filtering layer: tensor checks and
marshalling onto the C ABI, a ``torch.autograd.Function`` whose backward is
the library's hand-written adjoint (Algorithm 1), and ``nn.Module`` wrappers.

PyTorch provides device memory and the current stream only; every step of
the layer runs in libdgf.so's kernels.
"""
from __future__ import annotations

import ctypes

import torch

from . import _lib as L

_DT = {torch.float32: L.DGF_F32, torch.bfloat16: L.DGF_BF16, torch.float16: L.DGF_F16}


def dtype_code(t: torch.Tensor) -> int:
    if t.dtype not in _DT:
        raise TypeError(f"unsupported dtype {t.dtype}; use float32, bfloat16 or float16")
    return _DT[t.dtype]


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream(device) -> ctypes.c_void_p:
    return ctypes.c_void_p(torch.cuda.current_stream(device).cuda_stream)


def _check(*ts):
    dev = None
    for t in ts:
        if t is None:
            continue
        if not t.is_cuda:
            raise ValueError("tensors must be CUDA tensors (the layer has no CPU path)")
        if not t.is_contiguous():
            raise ValueError("tensors must be contiguous NCHW")
        if dev is None:
            dev = t.device
        elif t.device != dev:
            raise ValueError("tensors on different devices")
    return dev


def workspace(nbytes: int, device) -> torch.Tensor:
    ws = torch.empty(max(int(nbytes), 256) + 256, dtype=torch.uint8, device=device)
    off = (-ws.data_ptr()) % 256
    return ws[off:off + max(int(nbytes), 256)]


def _guide_struct(w1, w2, b2, slope):
    if w1 is None:
        return None
    for t in (w1, w2, b2):
        if t.dtype != torch.float32 or not t.is_contiguous() or not t.is_cuda:
            raise ValueError("guide weights must be contiguous float32 CUDA tensors")
    hidden = w1.shape[0]
    if tuple(w1.shape) != (hidden, 3) or tuple(w2.shape) != (3, hidden) or tuple(b2.shape) != (3,):
        raise ValueError("guide weights: w1 (hidden, 3), w2 (3, hidden), b2 (3,)")
    return L.dgf_guide(w1.data_ptr(), w2.data_ptr(), b2.data_ptr(), hidden, float(slope))


def _sizes(p_l, I_h, grey_ok=False):
    """(N, C, h_l, w_l, h, w) with C the output's channels; with grey_ok the
    guide may have another channel count (its channel mean is the guide)."""
    N, n_I, h, w = I_h.shape
    h_l, w_l = p_l.shape[2], p_l.shape[3]
    C = p_l.shape[1]
    if p_l.shape[0] != N or (C != n_I and not grey_ok):
        raise ValueError("p_l and I_h disagree on N or C")
    return N, C, h_l, w_l, h, w


def _options(mean_ab, C, I_h, g, guide_low=False, coef=None):
    """dgf_options for the call, or None for the defaults."""
    n_I = I_h.shape[1]
    if n_I != C and g is not None:
        raise ValueError("a grey guide (guide channels != output channels) excludes the guidance transform")
    if guide_low and g is None:
        raise ValueError("guide_low applies the guidance transform to I_l: it needs the transform's weights")
    if mean_ab and n_I == C and not guide_low and coef is None:
        return None
    return L.dgf_options(1 if mean_ab else 0, n_I if n_I != C else 0, 1 if guide_low else 0,
                         None if coef is None else coef.data_ptr())


def _coef_bytes(p_l, I_h, guided):
    N, C, h_l, w_l = p_l.shape
    h, w = I_h.shape[-2:]
    g = L.dgf_guide(None, None, None, 1, 0.2) if guided else None
    return L.dgf_coef_bytes(N, C, h_l, w_l, h, w, ctypes.byref(g) if g is not None else None)


def coef_buffer(p_l, I_h, guided=False):
    """A buffer for the values a forward call keeps for its backward: the
    coefficients (Abar, bbar) and, with the guidance transform (guided=True),
    the low-res and high-res guides (dgf_options.coef, dgf_coef_bytes)."""
    nb = _coef_bytes(p_l, I_h, guided)
    return torch.empty((nb + 3) // 4, dtype=torch.float32, device=p_l.device)


def backward_reuses_coef(p_l, I_h, r, w1=None, mean_ab=True, guide_low=False) -> bool:
    """Whether the backward skips work given the forward's coefficients
    (dgf_backward_reuses_coef): the forward then keeps them."""
    N, C, h_l, w_l, h, w = _sizes(p_l, I_h, grey_ok=True)
    g = L.dgf_guide(None, None, None, w1.shape[0], 0.2) if w1 is not None else None
    opt = _options(mean_ab, C, I_h, g, guide_low)
    return bool(L.dgf_backward_reuses_coef(N, C, h_l, w_l, h, w, int(r), dtype_code(I_h),
                                           ctypes.byref(g) if g is not None else None,
                                           ctypes.byref(opt) if opt is not None else None))


def _check_coef(coef, p_l, I_h, guided=False):
    if coef is None:
        return
    nb = _coef_bytes(p_l, I_h, guided)
    if (coef.dtype != torch.float32 or not coef.is_cuda or not coef.is_contiguous()
            or 4 * coef.numel() < nb or coef.device != p_l.device or coef.data_ptr() % 256 != 0):
        raise ValueError("coef must be a contiguous, 256-byte aligned float32 CUDA tensor of "
                         "dgf_coef_bytes bytes (coef_buffer)")


def gf_forward(p_l, I_l, I_h, r: int, eps: float, w1=None, w2=None, b2=None, slope=0.2, out=None,
               mean_ab=True, guide_low=False, coef=None):
    """O_h of the fast guided filtering layer (Eq. 1-2, box mean of A and b;
    mean_ab=False: A_l, b_l upsampled directly, the layer as printed; a guide
    with another channel count than p_l: its channel mean guides every
    channel; guide_low=True with the transform's weights: G_l = F(I_l)
    instead of the block mean of F(I_h); coef (coef_buffer): the call's
    coefficients are written there for a backward that takes them)."""
    dev = _check(p_l, I_l, I_h, w1, w2, b2)
    N, C, h_l, w_l, h, w = _sizes(p_l, I_h, grey_ok=True)
    dt = dtype_code(I_h)
    if p_l.dtype != I_h.dtype or (I_l is not None and I_l.dtype != I_h.dtype):
        raise TypeError("p_l, I_l and I_h must share one dtype")
    g = _guide_struct(w1, w2, b2, slope)
    gp = ctypes.byref(g) if g is not None else None
    _check_coef(coef, p_l, I_h, g is not None)
    opt = _options(mean_ab, C, I_h, g, guide_low, coef)
    if out is None:
        out = torch.empty((N, C, h, w), dtype=I_h.dtype, device=I_h.device)
    with torch.cuda.device(dev):
        if opt is None:
            ws = workspace(L.dgf_workspace_size(N, C, h_l, w_l, h, w, r, dt, gp), dev)
            L.check(L.dgf_forward(_ptr(p_l), _ptr(I_l), _ptr(I_h), _ptr(out), N, C, h_l, w_l, h, w, r,
                                  float(eps), dt, gp, _ptr(ws), ws.numel(), _stream(dev)))
        else:
            ws = workspace(L.dgf_workspace_size_opt(N, C, h_l, w_l, h, w, r, dt, gp, ctypes.byref(opt)), dev)
            L.check(L.dgf_forward_opt(_ptr(p_l), _ptr(I_l), _ptr(I_h), _ptr(out), N, C, h_l, w_l, h, w, r,
                                      float(eps), dt, gp, _ptr(ws), ws.numel(), _stream(dev), ctypes.byref(opt)))
    return out


def gf_backward(dO_h, p_l, I_l, I_h, r: int, eps: float, w1=None, w2=None, b2=None, slope=0.2,
                need_p=True, need_Il=True, need_Ih=True, need_w=True, mean_ab=True, guide_low=False, coef=None):
    """(dp_l, dI_l, dI_h, (dw1, dw2, db2)) by the library's adjoint kernels;
    coef: the coefficients gf_forward kept for the same inputs and options."""
    dev = _check(dO_h, p_l, I_l, I_h, w1, w2, b2)
    N, C, h_l, w_l, h, w = _sizes(p_l, I_h, grey_ok=True)
    dt = dtype_code(I_h)
    g = _guide_struct(w1, w2, b2, slope)
    gp = ctypes.byref(g) if g is not None else None
    _check_coef(coef, p_l, I_h, g is not None)
    opt = _options(mean_ab, C, I_h, g, guide_low, coef)
    dO_h = dO_h.to(I_h.dtype).contiguous()
    dp = torch.empty_like(p_l) if need_p else None
    dIl = torch.empty_like(I_l) if (need_Il and (g is None or guide_low)) else None
    dIh = torch.empty_like(I_h) if need_Ih else None
    dW = None
    if g is not None and need_w:
        dW = torch.empty(6 * g.hidden + 3, dtype=torch.float32, device=dev)
    with torch.cuda.device(dev):
        if opt is None:
            ws = workspace(L.dgf_workspace_size(N, C, h_l, w_l, h, w, r, dt, gp), dev)
            L.check(L.dgf_backward(_ptr(dO_h), _ptr(p_l), _ptr(I_l), _ptr(I_h), _ptr(dp), _ptr(dIl),
                                   _ptr(dIh), _ptr(dW), N, C, h_l, w_l, h, w, r, float(eps), dt, gp,
                                   _ptr(ws), ws.numel(), _stream(dev)))
        else:
            ws = workspace(L.dgf_workspace_size_opt(N, C, h_l, w_l, h, w, r, dt, gp, ctypes.byref(opt)), dev)
            L.check(L.dgf_backward_opt(_ptr(dO_h), _ptr(p_l), _ptr(I_l), _ptr(I_h), _ptr(dp), _ptr(dIl),
                                       _ptr(dIh), _ptr(dW), N, C, h_l, w_l, h, w, r, float(eps), dt, gp,
                                       _ptr(ws), ws.numel(), _stream(dev), ctypes.byref(opt)))
    dws = None
    if dW is not None:
        hid = g.hidden
        dws = (dW[:3 * hid].view(hid, 3), dW[3 * hid:6 * hid].view(3, hid), dW[6 * hid:])
    return dp, dIl, dIh, dws


def gf_step_host(p_l, I_l, I_h, dO_h, r: int, eps: float, out=None, groups: int = 0, device=None, buf=None,
                 sync: bool = True, mean_ab: bool = True):
    """Forward and backward of a batch held in host memory (dgf_host_step;
    mean_ab=False: the layer as printed, dgf_host_step_opt).

    p_l, I_l, I_h, dO_h: contiguous CPU tensors of one dtype (pinned memory
    lets the copies overlap the kernels).  Returns host tensors
    (O_h, dp_l, dI_l, dI_h), written into ``out`` when given (entries may
    be None: not wanted).  ``buf``: a device byte tensor of at least
    dgf_host_step_device_bytes bytes, 256-byte aligned, reused across calls
    (allocated here when None).  With sync=False the outputs are complete
    once the device's current stream has reached the end of the call, and
    the inputs must stay alive until then.
    """
    for t in (p_l, I_l, I_h, dO_h):
        if t is None or t.is_cuda or not t.is_contiguous():
            raise ValueError("gf_step_host takes contiguous CPU tensors")
        if t.dtype != I_h.dtype:
            raise TypeError("p_l, I_l, I_h and dO_h must share one dtype")
    dev = torch.device(device if device is not None else "cuda")
    N, C, h_l, w_l, h, w = _sizes(p_l, I_h)
    dt = dtype_code(I_h)
    pin = I_h.is_pinned()
    if out is None:
        out = (torch.empty(I_h.shape, dtype=I_h.dtype, pin_memory=pin),
               torch.empty(p_l.shape, dtype=p_l.dtype, pin_memory=pin),
               torch.empty(p_l.shape, dtype=p_l.dtype, pin_memory=pin),
               torch.empty(I_h.shape, dtype=I_h.dtype, pin_memory=pin))
    nb = L.dgf_host_step_device_bytes(N, C, h_l, w_l, h, w, r, dt, groups)
    if nb == 0:
        raise ValueError("invalid sizes or groups for dgf_host_step")
    if buf is None or buf.numel() < nb:
        buf = workspace(nb, dev)
    io = L.dgf_host_step_io(*(None if x is None else x.data_ptr() for x in (p_l, I_l, I_h, dO_h, *out)))
    with torch.cuda.device(dev):
        if mean_ab:
            L.check(L.dgf_host_step(ctypes.byref(io), N, C, h_l, w_l, h, w, r, float(eps), dt, groups, _ptr(buf),
                                    buf.numel(), _stream(dev)))
        else:
            opt = L.dgf_options(0, 0, 0)
            L.check(L.dgf_host_step_opt(ctypes.byref(io), N, C, h_l, w_l, h, w, r, float(eps), dt, groups,
                                        _ptr(buf), buf.numel(), _stream(dev), ctypes.byref(opt)))
        if sync:
            torch.cuda.current_stream(dev).synchronize()
    return out


def gf_forward_batched(images, out=None, mean_ab=True):
    """Uneven batch in one graph-replayed persistent launch per stage.

    ``images``: list of dicts with p_l, I_l, I_h (C x h x w tensors, one
    dtype), r, eps, and optionally coef (coef_buffer(p_l[None], I_h[None]): the
    image's coefficients are written there).  Returns the list of O_h.
    mean_ab=False: the layer as printed (dgf_forward_batched_opt; every
    image's kernels on library streams).
    """
    n = len(images)
    if n == 0:
        return []
    dt = dtype_code(images[0]["I_h"])
    dev = images[0]["I_h"].device
    arr = (L.dgf_image * n)()
    outs = []
    for i, im in enumerate(images):
        _check(im["p_l"], im["I_l"], im["I_h"])
        o = out[i] if out is not None else torch.empty_like(im["I_h"])
        outs.append(o)
        C, h, w = im["I_h"].shape
        h_l, w_l = im["p_l"].shape[1:]
        cf = im.get("coef")
        _check_coef(cf, im["p_l"][None], im["I_h"][None])
        arr[i] = L.dgf_image(im["p_l"].data_ptr(), im["I_l"].data_ptr(), im["I_h"].data_ptr(),
                             o.data_ptr(), C, h_l, w_l, h, w, int(im["r"]), float(im["eps"]),
                             None if cf is None else cf.data_ptr())
    nb = L.dgf_workspace_size_batched(arr, n, dt)
    if nb == 0:
        raise L.DGFError(1, L.dgf_last_error())
    ws = workspace(nb, dev)
    with torch.cuda.device(dev):
        if mean_ab:
            L.check(L.dgf_forward_batched(arr, n, dt, _ptr(ws), ws.numel(), _stream(dev)))
        else:
            opt = L.dgf_options(0, 0, 0)
            L.check(L.dgf_forward_batched_opt(arr, n, dt, _ptr(ws), ws.numel(), _stream(dev), ctypes.byref(opt)))
    return outs


def gf_backward_batched(images, grads, mean_ab=True):
    """Batched backward (Algorithm 1 per image, one graph or concurrent chains).

    ``images``: list of dicts with p_l, I_l, I_h (C x h x w tensors, one
    dtype), r, eps, and optionally need_p / need_Il / need_Ih (default
    True) and coef (the coefficients the batched forward kept);
    ``grads``: the matching list of d O_h.  Returns a list of
    (dp_l, dI_l, dI_h) per image, None where not wanted.  mean_ab=False:
    Algorithm 1 as printed (dgf_backward_batched_opt).
    """
    n = len(images)
    if n == 0:
        return []
    dt = dtype_code(images[0]["I_h"])
    dev = images[0]["I_h"].device
    arr = (L.dgf_image_grad * n)()
    outs = []
    for i, (im, R) in enumerate(zip(images, grads)):
        _check(im["p_l"], im["I_l"], im["I_h"])
        if R.dtype != im["I_h"].dtype or R.shape != im["I_h"].shape or not R.is_contiguous():
            raise ValueError("d O_h must match I_h in shape, dtype and layout")
        dp = torch.empty_like(im["p_l"]) if im.get("need_p", True) else None
        dIl = torch.empty_like(im["I_l"]) if im.get("need_Il", True) else None
        dIh = torch.empty_like(im["I_h"]) if im.get("need_Ih", True) else None
        outs.append((dp, dIl, dIh))
        C, h, w = im["I_h"].shape
        h_l, w_l = im["p_l"].shape[1:]
        cf = im.get("coef")
        _check_coef(cf, im["p_l"][None], im["I_h"][None])
        arr[i] = L.dgf_image_grad(R.data_ptr(), im["p_l"].data_ptr(), im["I_l"].data_ptr(), im["I_h"].data_ptr(),
                                  *(None if t is None else t.data_ptr() for t in (dp, dIl, dIh)),
                                  C, h_l, w_l, h, w, int(im["r"]),
                                  float(im["eps"]), None if cf is None else cf.data_ptr())
    nb = L.dgf_workspace_size_batched_backward(arr, n, dt)
    if nb == 0:
        raise L.DGFError(1, L.dgf_last_error())
    ws = workspace(nb, dev)
    with torch.cuda.device(dev):
        if mean_ab:
            L.check(L.dgf_backward_batched(arr, n, dt, _ptr(ws), ws.numel(), _stream(dev)))
        else:
            opt = L.dgf_options(0, 0, 0)
            L.check(L.dgf_backward_batched_opt(arr, n, dt, _ptr(ws), ws.numel(), _stream(dev), ctypes.byref(opt)))
    return outs


class GuidedFilterFn(torch.autograd.Function):
    """O_h = GF(p_l, I_l, I_h); backward = Algorithm 1 in libdgf.so."""

    @staticmethod
    def forward(ctx, p_l, I_l, I_h, r, eps):
        p_l, I_l, I_h = p_l.contiguous(), I_l.contiguous(), I_h.contiguous()
        # the coefficients are kept for the backward where it then skips work
        coef = coef_buffer(p_l, I_h) if backward_reuses_coef(p_l, I_h, r) else None
        ctx.save_for_backward(p_l, I_l, I_h, coef)
        ctx.r, ctx.eps = r, eps
        return gf_forward(p_l, I_l, I_h, r, eps, coef=coef)

    @staticmethod
    def backward(ctx, dO_h):
        p_l, I_l, I_h, coef = ctx.saved_tensors
        dp, dIl, dIh, _ = gf_backward(dO_h.contiguous(), p_l, I_l, I_h, ctx.r, ctx.eps,
                                      need_p=ctx.needs_input_grad[0],
                                      need_Il=ctx.needs_input_grad[1],
                                      need_Ih=ctx.needs_input_grad[2], coef=coef)
        return dp, dIl, dIh, None, None


class GuidedFilterTransformFn(torch.autograd.Function):
    """O_h with the trainable guidance transform F (Sec. 3.4)."""

    @staticmethod
    def forward(ctx, p_l, I_h, w1, w2, b2, r, eps, slope):
        p_l, I_h = p_l.contiguous(), I_h.contiguous()
        w1, w2, b2 = w1.contiguous(), w2.contiguous(), b2.contiguous()
        coef = coef_buffer(p_l, I_h, guided=True)  # the guided backward always reuses them
        ctx.save_for_backward(p_l, I_h, w1, w2, b2, coef)
        ctx.r, ctx.eps, ctx.slope = r, eps, slope
        return gf_forward(p_l, None, I_h, r, eps, w1, w2, b2, slope, coef=coef)

    @staticmethod
    def backward(ctx, dO_h):
        p_l, I_h, w1, w2, b2, coef = ctx.saved_tensors
        need_w = any(ctx.needs_input_grad[2:5])
        dp, _, dIh, dws = gf_backward(dO_h.contiguous(), p_l, None, I_h, ctx.r, ctx.eps, w1, w2, b2,
                                      ctx.slope, need_p=ctx.needs_input_grad[0], need_Il=False,
                                      need_Ih=ctx.needs_input_grad[1], need_w=need_w, coef=coef)
        dw1, dw2, db2 = dws if dws is not None else (None, None, None)
        return dp, dIh, dw1, dw2, db2, None, None, None


class GuidedFilter(torch.nn.Module):
    """Fast guided filtering layer without a learned transform (DGF_b): the
    guide itself when it has the output's channels, else its channel mean."""

    def __init__(self, r: int = 1, eps: float = 1e-8):
        super().__init__()
        self.r, self.eps = int(r), float(eps)

    def forward(self, p_l, I_l, I_h):
        return GuidedFilterFn.apply(p_l, I_l, I_h, self.r, self.eps)


class GuidedFilterWithTransform(torch.nn.Module):
    """Guided filtering layer with the learnable guidance map F(I) (Sec. 3.4)."""

    def __init__(self, r: int = 1, eps: float = 1e-8, hidden: int = 16, slope: float = 0.2):
        super().__init__()
        self.r, self.eps, self.slope = int(r), float(eps), float(slope)
        self.w1 = torch.nn.Parameter(torch.randn(hidden, 3) * 0.1)
        self.w2 = torch.nn.Parameter(torch.randn(3, hidden) * 0.1)
        self.b2 = torch.nn.Parameter(torch.zeros(3))

    def forward(self, p_l, I_h):
        return GuidedFilterTransformFn.apply(p_l, I_h, self.w1, self.w2, self.b2, self.r, self.eps,
                                             self.slope)
