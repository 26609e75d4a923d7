"""Benchmark of the guided filtering layer's hot path on GB300.

One step = forward + backward of the layer (low-res statistics -> A, b ->
box mean -> bilinear upsampling + affine; then the transposed upsampler,
the recomputed statistics and Algorithm 1's low-res gradients) over one
batch, through the C ABI, inputs resident in HBM.

Default workload: 4 images x 3 channels, low-res 512 x 512, high-res
2048 x 2048, r = 1, eps = 1e-4, FP32 storage (the plain FP32 configuration;
blobs + edges + noise photo stand-in with a tone-curve target).  The same
JSON line also reports the forward alone, the BF16 4K batch (2 x 3 x
3840 x 2160, r = 2, eps = 1e-3), the per-kernel roofline, an end-to-end
figure with host buffers, and the FP64 oracle on the host cores.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Multi-GPU (torchrun): every rank runs its own batch (images are
independent; no collective on the data path) and the time is the max over
ranks; the value is the pixels of all ranks over that time (weak scaling).
"""
from __future__ import annotations

import argparse
import ctypes
import hashlib
import json
import os
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "high-res Mpix/s fwd & fwd+bwd, BF16-batched vs FP32-plain; % of HBM roofline"
NOMINAL_HBM_GBS = 8000.0
FALLBACK_HBM_GBS = 6800.0

WORKLOADS = {
    # name: N, C, h_l, w_l, f, r, eps, dtype, recipe
    "fp32_plain_4x3x2048": dict(N=4, C=3, h_l=512, w_l=512, f=4, r=1, eps=1e-4, dtype="f32", recipe="blobs"),
    "bf16_4k_2x3x3840x2160": dict(N=2, C=3, h_l=540, w_l=960, f=4, r=2, eps=1e-3, dtype="bf16",
                                  recipe="photo"),
    "fp32_small_1x1x256": dict(N=1, C=1, h_l=64, w_l=64, f=4, r=1, eps=1e-2, dtype="f32", recipe="photo"),
}
MAIN = "fp32_plain_4x3x2048"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-extra", action="store_true", help="skip the secondary workloads")
    ap.add_argument("--no-oracle", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--workload", default=None, choices=sorted(WORKLOADS),
                    help="workload of the timed loop (default: the FP32 plain configuration)")
    ap.add_argument("--quick", action="store_true",
                    help="timed loop only (no roofline pass, e2e, extras or oracle): for profiler runs")
    return ap.parse_args()


DATA = ("synthetic (seeded; blobs+edges+noise photo stand-in, tone-curve target, N(0,1) upstream "
        "gradient)")


def workload_config(name, ws):
    """The `config` of a workload's JSON line (the same for both arms)."""
    spec = WORKLOADS[name]
    N, C, h_l, w_l, f = spec["N"], spec["C"], spec["h_l"], spec["w_l"], spec["f"]
    h, w = h_l * f, w_l * f
    esz = 4 if spec["dtype"] == "f32" else 2
    return {"workload": name, "step": "forward+backward", "N": N, "C": C, "h_l": h_l, "w_l": w_l, "h": h, "w": w,
            "r": spec["r"], "eps": spec["eps"],
            "l2": "no flush: a step streams %d MB of high-res tensors (I_h, O_h, dO_h, dI_h of %d MB each) "
                  "through the 129 MB L2" % (4 * N * C * h * w * esz // 10**6, N * C * h * w * esz // 10**6),
            "parallelism": f"images sharded over {ws} GPU(s), no collective"}


# ------------------------------------------------------------------ inputs
def make_inputs(spec, device, seed=0):
    import torch

    import synth
    dt = {"f32": torch.float32, "bf16": torch.bfloat16, "f16": torch.float16}[spec["dtype"]]
    if spec["recipe"] == "blobs":
        d = synth.blobs_tone_curve(seed, spec["N"], spec["C"], spec["h_l"], spec["w_l"], spec["f"],
                                   device=str(device))
    else:
        d = synth.photo_like(seed, spec["N"], spec["C"], spec["h_l"], spec["w_l"], spec["f"])
    g = {k: v.to(dt).to(device) for k, v in d.items()}
    g["R"] = synth.upstream_grad(seed + 1, g["I_h"].shape).to(dt).to(device)
    return g, dt


class Step:
    """Pre-marshalled forward + backward calls through the C ABI."""

    def __init__(self, g, spec, device, keep_coef=True):
        import torch

        from paper_1803_05619_gb300 import _lib as L
        from paper_1803_05619_gb300.layer import dtype_code, workspace
        self.L = L
        lib = L.lib()
        N, C, h, w = g["I_h"].shape
        h_l, w_l = g["p_l"].shape[2:]
        self.shape = (N, C, h_l, w_l, h, w)
        self.r, self.eps = spec["r"], spec["eps"]
        self.dt = dtype_code(g["I_h"])
        self.g = g
        self.O = torch.empty_like(g["I_h"])
        self.dp = torch.empty_like(g["p_l"])
        self.dIl = torch.empty_like(g["p_l"])
        self.dIh = torch.empty_like(g["I_h"])
        nb = L.dgf_workspace_size(N, C, h_l, w_l, h, w, self.r, self.dt, None)
        self.ws = workspace(nb, device)
        self.stream = ctypes.c_void_p(torch.cuda.current_stream(device).cuda_stream)
        P = lambda t: ctypes.c_void_p(t.data_ptr())  # noqa: E731
        self.fwd_args = (P(g["p_l"]), P(g["I_l"]), P(g["I_h"]), P(self.O), N, C, h_l, w_l, h, w, self.r,
                         ctypes.c_float(self.eps), self.dt, None, P(self.ws), self.ws.numel(), self.stream)
        self.bwd_args = (P(g["R"]), P(g["p_l"]), P(g["I_l"]), P(g["I_h"]), P(self.dp), P(self.dIl),
                         P(self.dIh), None, N, C, h_l, w_l, h, w, self.r, ctypes.c_float(self.eps), self.dt,
                         None, P(self.ws), self.ws.numel(), self.stream)
        # the forward keeps its coefficients for the backward where the backward
        # then skips work (as the layer's autograd function does)
        self.keep_coef = keep_coef and L.dgf_backward_reuses_coef(N, C, h_l, w_l, h, w, self.r, self.dt, None,
                                                                 None) == 1
        if self.keep_coef:
            self.coef = torch.empty(L.dgf_coef_bytes(N, C, h_l, w_l, h, w, None) // 4, dtype=torch.float32,
                                    device=device)
            self.opt = L.dgf_options(1, 0, 0, self.coef.data_ptr())
            self.fwd_args += (ctypes.byref(self.opt),)
            self.bwd_args += (ctypes.byref(self.opt),)
            self._f = lib.dgf_forward_opt
            self._b = lib.dgf_backward_opt
        else:
            self._f = lib.dgf_forward
            self._b = lib.dgf_backward

    def forward(self):
        st = self._f(*self.fwd_args)
        if st != 0:
            raise RuntimeError(self.L.dgf_last_error())

    def backward(self):
        st = self._b(*self.bwd_args)
        if st != 0:
            raise RuntimeError(self.L.dgf_last_error())

    def __call__(self):
        self.forward()
        self.backward()


def step_graph(g, spec, device):
    """One forward+backward step (a Step of its own, on a side stream)
    captured in a CUDA graph; replay() runs it on the current stream."""
    import torch
    cap = torch.cuda.Stream(device)
    torch.cuda.synchronize(device)
    with torch.cuda.stream(cap):
        gstep = Step(g, spec, device)
        gstep()  # shapes already tuned by the eager calls: this call tunes nothing
    torch.cuda.synchronize(device)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=cap):
        gstep()
    torch.cuda.synchronize(device)
    graph.keep = gstep  # its outputs and workspace must outlive the graph
    return graph


class BatchedStep:
    """Pre-marshalled dgf_forward_batched + dgf_backward_batched over a list of
    images (dicts of C x h x w tensors with r, eps) and their upstream
    gradients: descriptor tables, outputs and workspaces built once."""

    def __init__(self, images, grads, device):
        import torch

        from paper_1803_05619_gb300 import _lib as L
        from paper_1803_05619_gb300.layer import dtype_code, workspace
        self.L = L
        lib = L.lib()
        n = len(images)
        self.dt = dtype_code(images[0]["I_h"])
        self.fa = (L.dgf_image * n)()
        self.ba = (L.dgf_image_grad * n)()
        self.keep = []
        for i, (im, R) in enumerate(zip(images, grads)):
            C, h, w = im["I_h"].shape
            h_l, w_l = im["p_l"].shape[1:]
            o, dp = torch.empty_like(im["I_h"]), torch.empty_like(im["p_l"])
            dil, dih = torch.empty_like(im["I_l"]), torch.empty_like(im["I_h"])
            self.keep += [o, dp, dil, dih]
            # coefficients kept from the forward where the backward then skips work
            cf = None
            if L.dgf_backward_reuses_coef(1, C, h_l, w_l, h, w, int(im["r"]), self.dt, None, None) == 1:
                cf = torch.empty(2 * C * h_l * w_l, dtype=torch.float32, device=device)
                self.keep.append(cf)
            cp = None if cf is None else cf.data_ptr()
            self.fa[i] = L.dgf_image(im["p_l"].data_ptr(), im["I_l"].data_ptr(), im["I_h"].data_ptr(), o.data_ptr(),
                                     C, h_l, w_l, h, w, int(im["r"]), float(im["eps"]), cp)
            self.ba[i] = L.dgf_image_grad(R.data_ptr(), im["p_l"].data_ptr(), im["I_l"].data_ptr(),
                                          im["I_h"].data_ptr(), dp.data_ptr(), dil.data_ptr(), dih.data_ptr(), C, h_l,
                                          w_l, h, w, int(im["r"]), float(im["eps"]), cp)
        nf = L.dgf_workspace_size_batched(self.fa, n, self.dt)
        nb = L.dgf_workspace_size_batched_backward(self.ba, n, self.dt)
        self.wf, self.wb = workspace(nf, device), workspace(nb, device)
        self.n = n
        self.stream = ctypes.c_void_p(torch.cuda.current_stream(device).cuda_stream)
        self._f, self._b = lib.dgf_forward_batched, lib.dgf_backward_batched

    def forward(self):
        st = self._f(self.fa, self.n, self.dt, ctypes.c_void_p(self.wf.data_ptr()), self.wf.numel(), self.stream)
        if st != 0:
            raise RuntimeError(self.L.dgf_last_error())

    def backward(self):
        st = self._b(self.ba, self.n, self.dt, ctypes.c_void_p(self.wb.data_ptr()), self.wb.numel(), self.stream)
        if st != 0:
            raise RuntimeError(self.L.dgf_last_error())

    def __call__(self):
        self.forward()
        self.backward()


# ------------------------------------------------------------------ timing
def dist_setup():
    import torch
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch.distributed as dist
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", rank=rank, world_size=ws, device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    return rank, ws, local


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(v, ws, device):
    """Slowest rank's time (the job's time); `device` is where the collective runs."""
    if ws == 1:
        return v
    import torch
    import torch.distributed as dist
    t = torch.tensor([v], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def shard(n_units, rank, world):
    """Contiguous share of n_units independent images for one rank (weak scaling
    gives every rank the full per-GPU batch; this split serves a fixed total)."""
    base, extra = divmod(n_units, world)
    lo = rank * base + min(rank, extra)
    return lo, lo + base + (1 if rank < extra else 0)


def job_value(pixels_per_rank, world, ms_max):
    """Whole-job Mpix/s: every rank's pixels over the slowest rank's time."""
    return world * pixels_per_rank / (ms_max * 1e-3) / 1e6


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled while the timed loop runs."""

    Q = ("timestamp,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = os.path.join(tempfile.gettempdir(), f"dgf_clocks_{os.getpid()}.csv")

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "10"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
            time.sleep(0.5)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def mark(self, which):
        setattr(self, which, time.time())

    def samples_in_window(self):
        return self.summary().get("samples", 0) if self.proc is not None else 0

    def extend(self, fn, seconds=0.3):
        """A timed loop too short for the sampling period: keep the same work
        running for `seconds` right after it (untimed) and take the clocks
        over the timed loop and that run together."""
        import torch
        t_end = time.time() + seconds
        while time.time() < t_end:
            for _ in range(20):
                fn()
            torch.cuda.synchronize()
        self.mark("stop")
        self.extended = seconds

    def summary(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        import datetime
        rows = []
        t0, t1 = getattr(self, "start", None), getattr(self, "stop", None)
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                ts = datetime.datetime.strptime(parts[0], "%Y/%m/%d %H:%M:%S.%f").timestamp()
                row = (float(parts[1]), float(parts[2]), parts[5:9], parts[4], float(parts[3]))
            except ValueError:
                continue
            if t0 is not None and t1 is not None and not (t0 <= ts <= t1):
                continue
            rows.append(row)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = sorted(r[0] for r in rows)
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i, v in enumerate(r[2]) if v.lower() == "active"})
        out = {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": max(r[1] for r in rows), "reasons": reasons,
               "samples": len(rows), "power_w_max": max(r[4] for r in rows), "period_ms": 10}
        if getattr(self, "extended", None):
            out["window"] = ("the timed loop plus %.1f s of the same step run right after it (the timed loop "
                             "alone is shorter than a few sampling periods)" % self.extended)
        return out


def time_loop(fn, steps, warmup, ws, device, clock=None):
    import torch
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    barrier(ws)
    torch.cuda.synchronize()
    if clock is not None:
        clock.mark("start")
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(steps):
        fn()
    b.record()
    torch.cuda.synchronize()
    if clock is not None:
        clock.mark("stop")
    barrier(ws)
    ms = a.elapsed_time(b) / steps
    return max_over_ranks(ms, ws, device)


# --------------------------------------------------------------- roofline
def algorithmic_bytes(kernel, shape, esz):
    """Minimum DRAM bytes one launch must move (inputs read once, outputs written once)."""
    N, C, h_l, w_l, h, w = shape
    hi = N * C * h * w
    lo = N * C * h_l * w_l
    return {
        "k2_hires_apply": hi * 2 * esz,               # read I_h, write O_h
        "k3_hires_bwd": hi * 3 * esz,                 # read dO_h, I_h; write dI_h
        "k1_lowres_coef": lo * (2 * esz + 8),         # read I_l, p_l; write Abar, bbar (FP32)
        "k4_lowres_bwd": lo * (2 * esz + 8 + 2 * esz),  # read I_l, p_l, dAbar/dbbar; write dp_l, dI_l
        "k12_fused_forward": hi * 2 * esz + lo * 2 * esz,  # read I_h, I_l, p_l; write O_h (no Abar, bbar traffic)
        "k13_fused_backward": hi * 3 * esz + lo * 2 * esz,  # read dO_h, I_h, I_l, p_l; write dI_h
    }.get(kernel)


def peaks():
    try:
        mp = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        return float(mp["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


def kernel_source_hash():
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1803_05619_gb300", "csrc")
    for f in sorted(os.listdir(csrc)):
        h.update(open(os.path.join(csrc, f), "rb").read())
    return h.hexdigest()[:16]


def ncu_traffic(kernel, workload, field="dram_bytes_per_launch"):
    """A per-launch figure (DRAM bytes, warp-instructions) from the committed
    ncu summary, if it was taken on the current kernel sources (else None)."""
    p = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    try:
        d = json.load(open(p))
    except Exception:
        return None
    e = d.get(workload, {}).get(kernel)
    if not e or e.get("source_hash") != kernel_source_hash():
        return None
    return e.get(field)


# FP32 FMA peak of the guidance kernels: 152 SMs x 128 FP32 lanes x 2 flops
# x 2070 MHz maximum SM clock, in TFLOP/s.
FP32_FMA_TFLOPS = round(152 * 128 * 2 * 2.07e9 / 1e12, 2)
# Instruction-issue peak of the low-res kernels (bound by issue and by the
# latency of their row walks, not by HBM): 152 SMs x 4 schedulers x one
# warp-instruction per cycle x 2070 MHz maximum SM clock.
ISSUE_PEAK = 152 * 4 * 2.07e9
ISSUE_BOUND = ("k1_lowres_coef", "k4_lowres_bwd")


def roofline(step, spec, steps, warmup, workload):
    import torch
    L = step.L
    L.dgf_profile_reset()
    L.dgf_profile_enable(True)
    try:
        for _ in range(max(3, warmup // 4)):
            step()
        L.dgf_profile_reset()
        for _ in range(steps):
            step()
        torch.cuda.synchronize()
        prof = L.dgf_profile_read()
    finally:
        L.dgf_profile_enable(False)
    esz = 4 if spec["dtype"] == "f32" else 2
    total = sum(v[0] for v in prof.values())
    per = {}
    # one launch per call (the plane-group pipeline, which would launch a
    # kernel once per group, is off here); a kernel's algorithmic bytes are
    # those of one call
    for k, (ms, n) in prof.items():
        ab = algorithmic_bytes(k, step.shape, esz)
        per_call = ms / max(n, 1)
        per[k] = {"us_per_call": round(per_call * 1e3, 2), "launches_per_step": round(n / steps, 2),
                  "share": round(ms / total, 4), "gbs": round(ab / (per_call * 1e-3) / 1e9, 1) if ab else None}
    for k, v in per.items():
        wi = ncu_traffic(k, workload, "warp_instructions_per_launch")
        if wi is not None and k in ISSUE_BOUND:
            # ncu's count is per launch of the one-stream call: the call's issue rate
            v["issue_frac"] = round(wi / (v["us_per_call"] * 1e-6) / ISSUE_PEAK, 4)
    top = max(prof, key=lambda k: prof[k][0])
    ms, n = prof[top]
    per_call_s = ms / max(n, 1) * 1e-3
    ab = algorithmic_bytes(top, step.shape, esz)
    peak, src = peaks()
    ach = ab / per_call_s / 1e9
    wi = ncu_traffic(top, workload, "warp_instructions_per_launch")
    if top in ISSUE_BOUND and wi is not None:
        # a low-res kernel dominates: its bound is instruction issue, not HBM
        ach_i = wi / per_call_s
        return {"kernel": top, "bound": "issue", "achieved": round(ach_i / 1e9, 2), "peak": round(ISSUE_PEAK / 1e9, 2),
                "unit": "G warp-instructions/s", "frac": round(ach_i / ISSUE_PEAK, 4),
                "peak_source": "derived: 152 SMs x 4 schedulers x 1 warp-instruction/cycle x 2070 MHz",
                "warp_instructions": wi, "hbm_gbs": round(ach, 1), "hbm_frac_of_measured": round(ach / peak, 4),
                "traffic": ncu_traffic(top, workload), "algorithmic_bytes": ab,
                "us_per_call": round(per_call_s * 1e6, 2), "launches_per_step": per[top]["launches_per_step"],
                "kernels": per}
    return {"kernel": top, "bound": "hbm", "achieved": round(ach, 1), "peak": peak, "unit": "GB/s",
            "frac": round(ach / peak, 4), "peak_source": src,
            "frac_of_nominal_8TBs": round(ach / NOMINAL_HBM_GBS, 4),
            "traffic": ncu_traffic(top, workload), "algorithmic_bytes": ab,
            "us_per_call": round(per_call_s * 1e6, 2), "launches_per_step": per[top]["launches_per_step"],
            "kernels": per}


# ------------------------------------------------------------- end to end
def e2e(step, steps, warmup, device, groups=0):
    """Same step on host buffers through dgf_host_step: every step copies its
    inputs host -> device and all four results device -> host inside the
    timed region, the copies pipelined with the kernels over plane groups.
    Also times the unpipelined form (the copies, then the two device calls,
    then the copies back, on one stream) for comparison."""
    import torch

    from paper_1803_05619_gb300.layer import workspace
    L = step.L
    g = step.g
    ins = [g["p_l"], g["I_l"], g["I_h"], g["R"]]
    outs = [step.O, step.dp, step.dIl, step.dIh]
    h_in = [torch.empty(t.shape, dtype=t.dtype, pin_memory=True) for t in ins]
    h_out = [torch.empty(t.shape, dtype=t.dtype, pin_memory=True) for t in outs]
    for h, t in zip(h_in, ins):
        h.copy_(t)
    N, C, h_l, w_l, h, w = step.shape
    nb = L.dgf_host_step_device_bytes(N, C, h_l, w_l, h, w, step.r, step.dt, groups)
    buf = workspace(nb, device)
    io = L.dgf_host_step_io(*(t.data_ptr() for t in h_in + h_out))
    args = (ctypes.byref(io), N, C, h_l, w_l, h, w, step.r, ctypes.c_float(step.eps), step.dt, groups,
            ctypes.c_void_p(buf.data_ptr()), buf.numel(), step.stream)
    fn = L.lib().dgf_host_step

    def pipelined():
        if fn(*args) != 0:
            raise RuntimeError(L.dgf_last_error())

    def serial():
        for hb, t in zip(h_in, ins):
            t.copy_(hb, non_blocking=True)
        step()
        for hb, t in zip(h_out, outs):
            hb.copy_(t, non_blocking=True)

    n = max(3, min(steps, 50))
    ms = time_loop(pipelined, n, max(2, warmup // 4), 1, device)
    ms_serial = time_loop(serial, n, max(2, warmup // 4), 1, device)
    bi = sum(t.numel() * t.element_size() for t in ins)
    bo = sum(t.numel() * t.element_size() for t in outs)
    del buf
    return ms, bi, bo, n, ms_serial


# ------------------------------------------------------------ CPU oracle
ORACLE_SNIPPET = r"""
import json, os, sys, time
sys.path.insert(0, {root!r})
import numpy as np
import oracle, synth
spec = json.loads({spec!r})
if spec["recipe"] == "blobs":
    d = synth.blobs_tone_curve(0, 1, 1, spec["h_l"], spec["w_l"], spec["f"])
else:
    d = synth.photo_like(0, 1, 1, spec["h_l"], spec["w_l"], spec["f"])
R = synth.upstream_grad(1, d["I_h"].shape).numpy()
p, il, ih = (d[k].numpy() for k in ("p_l", "I_l", "I_h"))
reps = int(spec.get("reps", 1))
for _ in range(int(spec.get("warmup", 1))):
    oracle.forward(p, il, ih, spec["r"], spec["eps"])
    oracle.backward(R, p, il, ih, spec["r"], spec["eps"])
t0 = time.perf_counter()
for _ in range(reps):
    oracle.forward(p, il, ih, spec["r"], spec["eps"])
    oracle.backward(R, p, il, ih, spec["r"], spec["eps"])
dt = (time.perf_counter() - t0) / reps
print(json.dumps({{"seconds_per_plane": dt}}))
"""


def cpu_oracle(spec, reps=1, warmup=1):
    env = dict(os.environ)
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS", "NUMEXPR_NUM_THREADS"):
        env[k] = "1"
    env["CUDA_VISIBLE_DEVICES"] = ""
    s = dict(spec)
    s["reps"] = reps
    s["warmup"] = warmup
    code = ORACLE_SNIPPET.format(root=ROOT, spec=json.dumps(s))
    out = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, timeout=900)
    if out.returncode != 0:
        raise RuntimeError(out.stderr[-2000:])
    sec = json.loads(out.stdout.strip().splitlines()[-1])["seconds_per_plane"]
    pix = spec["h_l"] * spec["f"] * spec["w_l"] * spec["f"] / spec["C"]  # one plane = 1/C of an image
    return pix / sec / 1e6, sec


ACCURACY_SNIPPET = r"""
import json, sys
sys.path.insert(0, {root!r})
import numpy as np
import oracle
manifest = json.load(open({manifest!r}))
out = {{}}
def err(got, ref):
    got = np.asarray(got, np.float64); ref = np.asarray(ref, np.float64)
    d = got - ref
    nr = float(np.linalg.norm(ref))
    return {{"max_abs": float(np.max(np.abs(d))) if d.size else 0.0,
             "rel_l2": float(np.linalg.norm(d) / nr) if nr > 0 else float(np.linalg.norm(d))}}
for case in manifest:
    a = np.load(case["file"])
    f = {{k: a[k].astype(np.float64) for k in a.files}}
    r, eps = case["r"], case["eps"]
    if case["kind"] == "plain":
        ref = oracle.forward(f["p_l"], f["I_l"], f["I_h"], r, eps)
        rp, rIl, rIh = oracle.backward(f["R"], f["p_l"], f["I_l"], f["I_h"], r, eps)
        e = {{"O_h": err(f["O_h"], ref), "dp_l": err(f["dp_l"], rp), "dI_l": err(f["dI_l"], rIl),
              "dI_h": err(f["dI_h"], rIh)}}
    else:
        ref = oracle.forward_guided(f["p_l"], f["I_h"], f["w1"], f["w2"], f["b2"], r, eps)
        rp, rIh, rw1, rw2, rb2 = oracle.backward_guided(f["R"], f["p_l"], f["I_h"], f["w1"], f["w2"], f["b2"], r, eps)
        e = {{"O_h": err(f["O_h"], ref), "dp_l": err(f["dp_l"], rp), "dI_h": err(f["dI_h"], rIh),
              "dW": err(np.concatenate([f["dw1"].ravel(), f["dw2"].ravel()]),
                        np.concatenate([rw1.ravel(), rw2.ravel()])),
              "db2_max_abs": float(np.max(np.abs(f["db2"] - rb2)))}}
    out[case["name"]] = {{"sample": case["sample"], "dtype": case["dtype"], **e}}
print(json.dumps(out))
"""


def accuracy(device):
    """Max-abs and relative-L2 error against the FP64 oracle of O_h and of every
    gradient, per configuration, on the benchmark's own full-size inputs
    (sampled planes or images; the oracle computes each sample completely).
    Part of the CPU-baseline leg: the oracle runs in a subprocess on the host
    cores, after every GPU number has been taken."""
    import numpy as np
    import torch

    import synth
    from paper_1803_05619_gb300.layer import gf_backward, gf_backward_batched, gf_forward, gf_forward_batched
    tmp = tempfile.mkdtemp(prefix="dgf_acc_")
    manifest = []

    def npf(t):
        return t.detach().float().cpu().numpy()

    def plain(name, spec, g, out, plane, sample):
        n, c = divmod(plane, spec["C"])
        sl = lambda t: npf(t[n:n + 1, c:c + 1])  # noqa: E731
        f = os.path.join(tmp, name + ".npz")
        np.savez(f, p_l=sl(g["p_l"]), I_l=sl(g["I_l"]), I_h=sl(g["I_h"]), R=sl(g["R"]), O_h=sl(out[0]),
                 dp_l=sl(out[1]), dI_l=sl(out[2]), dI_h=sl(out[3]))
        manifest.append({"name": name, "kind": "plain", "file": f, "r": spec["r"], "eps": spec["eps"],
                         "dtype": spec["dtype"], "sample": sample})

    def run_plain(g, spec):
        o = gf_forward(g["p_l"], g["I_l"], g["I_h"], spec["r"], spec["eps"])
        dp, dil, dih, _ = gf_backward(g["R"], g["p_l"], g["I_l"], g["I_h"], spec["r"], spec["eps"])
        return o, dp, dil, dih

    # c1 (whole), c2 (plane 0 of 12)
    for name, seed in (("fp32_small_1x1x256", 0), (MAIN, 0)):
        spec = WORKLOADS[name]
        g, _ = make_inputs(spec, device, seed=seed)
        plain(name, spec, g, run_plain(g, spec), 0,
              "the whole image" if name != MAIN else "plane (0, 0) of the 4 x 3 batch")
        del g
    # c3 in BF16 and the same inputs in FP32 (plane (1, 2) of the 2 x 3 batch)
    spec = WORKLOADS["bf16_4k_2x3x3840x2160"]
    g, _ = make_inputs(spec, device, seed=7)
    plain("bf16_4k_2x3x3840x2160", spec, g, run_plain(g, spec), 5, "plane (1, 2) of the 2 x 3 batch")
    g32 = {k: v.float() for k, v in g.items()}
    spec32 = dict(spec, dtype="f32")
    plain("bf16_4k_inputs_in_fp32", spec32, g32, run_plain(g32, spec32), 5,
          "the BF16 inputs held in FP32: plane (1, 2)")
    del g, g32
    # c4: the smallest and a middle image of the 64, through the batched calls
    specs = synth.mixed_sizes(seed=0, n=64)
    order = sorted(range(len(specs)), key=lambda i: specs[i].h * specs[i].w)
    for i in (order[0], order[len(order) // 2]):
        s = specs[i]
        d = synth.photo_like(1000 + i, 1, 3, s.h_l, s.w_l, s.f)
        st = {k: v.to(torch.bfloat16)[0].to(device) for k, v in d.items()}
        R = synth.upstream_grad(2000 + i, st["I_h"].shape).to(torch.bfloat16).to(device)
        im = {"p_l": st["p_l"], "I_l": st["I_l"], "I_h": st["I_h"], "r": s.r, "eps": 1e-3}
        o = gf_forward_batched([im])[0]
        dp, dil, dih = gf_backward_batched([im], [R])[0]
        gg = {k: v[None] for k, v in st.items()}
        gg["R"] = R[None]
        sp = {"C": 3, "r": s.r, "eps": 1e-3, "dtype": "bf16"}
        for c in range(3):
            plain(f"batched_64_uneven_img{i}_c{c}", sp, gg, (o[None], dp[None], dil[None], dih[None]), c,
                  f"image {i} ({s.h}x{s.w}, f={s.f}, r={s.r}) channel {c}, batched calls")
    # c5: image 0 of the guided training batch (its own call: the weight
    # gradients then belong to that image alone)
    d = synth.photo_like(21, 1, 3, 256, 256, 8)
    g5 = {k: v.to(torch.bfloat16).to(device) for k, v in d.items()}
    w = {k: v.float().to(device) for k, v in synth.guide_weights(22).items()}
    R5 = synth.upstream_grad(23, (8, 3, 2048, 2048)).to(torch.bfloat16)[:1].to(device)
    o5 = gf_forward(g5["p_l"], None, g5["I_h"], 8, 1e-4, w["w1"], w["w2"], w["b2"], 0.2)
    dp5, _, dih5, dws = gf_backward(R5, g5["p_l"], None, g5["I_h"], 8, 1e-4, w["w1"], w["w2"], w["b2"], 0.2)
    f = os.path.join(tmp, "guided.npz")
    np.savez(f, p_l=npf(g5["p_l"]), I_h=npf(g5["I_h"]), R=npf(R5), O_h=npf(o5), dp_l=npf(dp5), dI_h=npf(dih5),
             w1=npf(w["w1"]), w2=npf(w["w2"]), b2=npf(w["b2"]), dw1=npf(dws[0]), dw2=npf(dws[1]), db2=npf(dws[2]))
    manifest.append({"name": "guided_train_8x2048", "kind": "guided", "file": f, "r": 8, "eps": 1e-4,
                     "dtype": "bf16", "sample": "image 0 of the 8 (3 channels, weight gradients of that image)"})
    torch.cuda.synchronize()
    try:
        return accuracy_oracle(manifest, tmp)
    finally:
        for c in manifest:
            try:
                os.remove(c["file"])
            except OSError:
                pass


def accuracy_oracle(manifest, tmp):
    """The oracle half of the accuracy leg: every case of `manifest` (npz files
    of inputs and GPU outputs) against the FP64 oracle, in a subprocess on the
    host cores."""
    mpath = os.path.join(tmp, "manifest.json")
    json.dump(manifest, open(mpath, "w"))
    code = ACCURACY_SNIPPET.format(root=ROOT, manifest=mpath)
    env = dict(os.environ)
    env["CUDA_VISIBLE_DEVICES"] = ""
    t0 = time.perf_counter()
    out = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, timeout=900)
    if out.returncode != 0:
        return {"error": out.stderr[-1500:]}
    res = json.loads(out.stdout.strip().splitlines()[-1])
    res["_note"] = ("max_abs and rel_l2 = ||got - ref|| / ||ref|| against the FP64 oracle on the stored "
                    "(rounded) inputs; oracle run on %d host cores in %.1f s" % (os.cpu_count() or 1,
                                                                                 time.perf_counter() - t0))
    return res


def run_reference(args):
    """--impl reference: the FP64 oracle on the host cores, same workload and metric.

    A step is a bounded sample of the workload: one plane (1 of N C) forward +
    backward, as the oracle stands (single-threaded numpy FP64); `value` is
    that plane's pixels over its time, so it is the same metric.  The line's
    steps, warmup and ms_per_step are what ran; the time a whole step of the
    workload would take is given separately."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    spec = WORKLOADS[MAIN]
    steps = max(1, min(args.steps, 30))  # each step ~0.8 s of CPU work; bounded to keep the run short
    warmup = max(1, min(args.warmup, 5))
    t0 = time.perf_counter()
    value, sec = cpu_oracle(spec, reps=steps, warmup=warmup)
    wall = time.perf_counter() - t0
    planes = spec["N"] * spec["C"]
    sample = (f"one plane (1 of {planes}) of {MAIN} per step: forward + backward, "
              f"{spec['h_l']}x{spec['w_l']} -> {spec['h_l'] * spec['f']}x{spec['w_l'] * spec['f']}, "
              f"{sec:.2f} s per plane, single-threaded numpy FP64")
    line = {"impl": "reference", "metric": METRIC, "value": round(value, 4), "unit": "Mpix/s",
            "n_gpus": args.gpus, "steps": steps, "warmup": warmup,
            "ms_per_step": round(sec * 1e3, 3),
            "ms_per_full_step_scaled": round(sec * 1e3 * planes, 1),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": DATA, "config": workload_config(MAIN, args.gpus),
            "cpu_baseline": {"value": round(value, 4), "unit": "Mpix/s", "cores": 1, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": round(value, 4), "unit": "Mpix/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0},
            "wall_s": round(wall, 1)}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------- main
def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    import torch

    from paper_1803_05619_gb300 import build as B
    rank, ws, local = dist_setup()
    if rank == 0:
        B.build()
    barrier(ws)
    from paper_1803_05619_gb300 import _lib as L
    L.dgf_autotune(True)  # tile shapes are timed on the first (warm-up) calls of each kernel
    device = torch.device("cuda", local)
    main_name = args.workload or MAIN
    spec = WORKLOADS[main_name]
    g, dt = make_inputs(spec, device, seed=1000 * rank)
    step = Step(g, spec, device)
    N, C, h_l, w_l, h, w = step.shape
    pix = N * h * w

    n0 = L.dgf_launch_count()
    step()
    per_step = L.dgf_launch_count() - n0
    # eager calls first (these also tune the shapes), then the same step
    # captured once in a CUDA graph and replayed: the timed figure, as a
    # training loop that captures its step runs it (the kernels and their
    # launch order are those of the eager calls; only host launch gaps go)
    ms_eager = time_loop(step, args.steps, args.warmup, ws, device)
    graph = step_graph(g, spec, device)
    with ClockSampler(local) as clk:
        ms = time_loop(graph.replay, args.steps, args.warmup, ws, device, clock=clk)
        if clk.proc is not None and clk.samples_in_window() < 10:
            clk.extend(graph.replay)
    launches = per_step * args.steps
    value = job_value(pix, ws, ms)
    fwd_ms = time_loop(step.forward, max(10, args.steps // 2), args.warmup, ws, device)
    line = {
        "metric": METRIC, "value": round(value, 2), "unit": "Mpix/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms, 5), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": spec["dtype"], "data": DATA,
        "config": workload_config(main_name, ws),
        "timed": "one forward+backward step (dgf_forward + dgf_backward) captured in a CUDA graph, replayed "
                 "per step",
        "coef_kept": bool(step.keep_coef),
        "eager": {"value": round(job_value(pix, ws, ms_eager), 2), "unit": "Mpix/s",
                  "ms_per_step": round(ms_eager, 5), "path": "the same calls issued from the host every step"},
        "fwd": {"value": round(ws * pix / (fwd_ms * 1e-3) / 1e6, 2), "unit": "Mpix/s",
                "ms_per_step": round(fwd_ms, 5), "path": "eager dgf_forward"},
        "gpu_launches": int(launches),
        "autotuned_shapes": L.dgf_autotune_entries(),
        "clocks": clk.summary(),
    }
    if rank == 0 and args.quick:
        print(json.dumps(line), flush=True)
    elif rank == 0:
        line["roofline"] = roofline(step, spec, min(args.steps, 200), args.warmup, MAIN)
        e_ms, bi, bo, n_e2e, e_serial = e2e(step, args.steps, args.warmup, device)
        line["e2e"] = {"value": round(pix / (e_ms * 1e-3) / 1e6, 2), "unit": "Mpix/s",
                       "h2d_bytes_per_step": bi, "d2h_bytes_per_step": bo, "steps": n_e2e,
                       "ms_per_step": round(e_ms, 4),
                       "path": "dgf_host_step on pinned host buffers (copies both ways pipelined with the "
                               "kernels over plane groups)",
                       "unpipelined": {"value": round(pix / (e_serial * 1e-3) / 1e6, 2),
                                       "ms_per_step": round(e_serial, 4),
                                       "path": "copies in, dgf_forward + dgf_backward, copies out, one stream"}}
        if not args.no_extra:
            line["bf16_4k"] = bench_bf16_4k(args, device)
            line["batched_64_uneven"] = bench_batched_64(args, device)
            line["guided_train_8x2048"] = bench_guided(args, device)
            line["small_fp32_1x1x256"] = bench_small(args, device)
            line["paper_literal_fp32_plain"] = bench_paper_literal(args, device)
            line["grey_guide_fp32"] = bench_grey(args, device)
        if not args.no_oracle:
            line["errors"] = accuracy(device)
            reps = 15
            cv, csec = cpu_oracle(spec, reps=reps)
            line["cpu_baseline"] = {"value": round(cv, 4), "unit": "Mpix/s", "cores": 1, "kind": "oracle",
                                    "sample": f"{reps} x one plane (1 of {N * C}) of {MAIN}, forward + "
                                              f"backward, {csec:.2f} s per plane, single-threaded numpy FP64"}
        print(json.dumps(line), flush=True)
    barrier(ws)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def bench_bf16_4k(args, device):
    """BF16 4K batch: single-call fwd+bwd (both images per launch) and the
    graph-replayed batched forward."""
    import torch

    name = "bf16_4k_2x3x3840x2160"
    spec = WORKLOADS[name]
    g, dt = make_inputs(spec, device, seed=7)
    step = Step(g, spec, device)
    N, C, h_l, w_l, h, w = step.shape
    pix = N * h * w
    steps = max(20, min(args.steps, 1000))
    ms = time_loop(step, steps, args.warmup, 1, device)
    graph = step_graph(g, spec, device)
    ms_graph = time_loop(graph.replay, steps, args.warmup, 1, device)
    fwd_ms = time_loop(step.forward, steps, args.warmup, 1, device)
    images = [{"p_l": g["p_l"][i], "I_l": g["I_l"][i], "I_h": g["I_h"][i], "r": spec["r"],
               "eps": spec["eps"]} for i in range(N)]
    bstep = BatchedStep(images, [g["R"][i] for i in range(N)], device)
    bat_ms = time_loop(bstep.forward, steps, args.warmup, 1, device)
    bat_fb_ms = time_loop(bstep, steps, args.warmup, 1, device)
    # the same single-call step with the backward recomputing the coefficients
    rstep = Step(g, spec, device, keep_coef=False)
    ms_recompute = time_loop(rstep, steps, args.warmup, 1, device)
    rl = roofline(step, spec, min(steps, 200), args.warmup, name)
    esz = 2
    fb_bytes = pix * C * esz * (2 + 3) + N * C * h_l * w_l * esz * (2 + 2 + 2)
    peak = peaks()[0]
    return {"workload": name, "fwd_bwd_mpix_s": round(pix / (ms * 1e-3) / 1e6, 2),
            "fwd_mpix_s": round(pix / (fwd_ms * 1e-3) / 1e6, 2),
            "batched_graph_fwd_mpix_s": round(pix / (bat_ms * 1e-3) / 1e6, 2),
            "batched_fwd_bwd": {
                "path": "dgf_forward_batched + dgf_backward_batched over the 2 images (the target's path)",
                "mpix_s": round(pix / (bat_fb_ms * 1e-3) / 1e6, 2), "ms": round(bat_fb_ms, 5),
                "frac_of_nominal_8TBs": round(fb_bytes / (bat_fb_ms * 1e-3) / 1e9 / NOMINAL_HBM_GBS, 4),
                "frac_of_measured_hbm": round(fb_bytes / (bat_fb_ms * 1e-3) / 1e9 / peak, 4),
                "target_frac_of_nominal_8TBs": 0.70},
            "ms_fwd_bwd": round(ms, 5), "fwd_bwd_frac_of_nominal_8TBs": round(
                fb_bytes / (ms * 1e-3) / 1e9 / NOMINAL_HBM_GBS, 4),
            "coef_kept": bool(step.keep_coef),
            "ms_fwd_bwd_recomputing_coef": round(ms_recompute, 5),
            "graph_fwd_bwd": {"path": "the single-call step captured in a CUDA graph and replayed",
                              "mpix_s": round(pix / (ms_graph * 1e-3) / 1e6, 2), "ms": round(ms_graph, 5),
                              "frac_of_nominal_8TBs": round(fb_bytes / (ms_graph * 1e-3) / 1e9 / NOMINAL_HBM_GBS, 4),
                              "frac_of_measured_hbm": round(fb_bytes / (ms_graph * 1e-3) / 1e9 / peak, 4)},
            "fwd_bwd_algorithmic_bytes": fb_bytes, "roofline": rl}


def bench_batched_64(args, device):
    """64 uneven BF16 images (long side 512..4096, factor 4 or 8, r in {1,2,4}):
    the forward in one graph-replayed persistent launch per stage, and
    forward + batched backward (per-image kernel chains run concurrently)."""
    import torch

    import synth
    specs = synth.mixed_sizes(seed=0, n=64)
    images, grads = [], []
    for i, s in enumerate(specs):
        d = synth.photo_like(1000 + i, 1, 3, s.h_l, s.w_l, s.f)
        st = {k: v.to(torch.bfloat16)[0].to(device) for k, v in d.items()}
        images.append({"p_l": st["p_l"], "I_l": st["I_l"], "I_h": st["I_h"], "r": s.r, "eps": 1e-3})
        grads.append(synth.upstream_grad(2000 + i, st["I_h"].shape).to(torch.bfloat16).to(device))
    pix = sum(s.h * s.w for s in specs)
    steps = max(10, min(args.steps // 10, 200))
    bstep = BatchedStep(images, grads, device)
    ms = time_loop(bstep.forward, steps, max(3, args.warmup // 4), 1, device)
    ms2 = time_loop(bstep, max(5, steps // 4), max(3, args.warmup // 4), 1, device)
    byts = sum(3 * 2 * (2 * s.h * s.w + 2 * s.h_l * s.w_l) for s in specs)
    byts_bwd = sum(3 * 2 * (3 * s.h * s.w + 4 * s.h_l * s.w_l) for s in specs)
    peak, src = peaks()
    return {"workload": "64 images, long side U[512,4096], aspect U[0.5,2], f in {4,8}, r in {1,2,4}, BF16",
            "mpix": round(pix / 1e6, 1), "fwd_mpix_s": round(pix / (ms * 1e-3) / 1e6, 1),
            "ms_fwd": round(ms, 4), "fwd_algorithmic_bytes": byts,
            "fwd_frac_of_measured_hbm": round(byts / (ms * 1e-3) / 1e9 / peak, 4),
            "fwd_frac_of_nominal_8TBs": round(byts / (ms * 1e-3) / 1e9 / NOMINAL_HBM_GBS, 4),
            "fwd_bwd_mpix_s": round(pix / (ms2 * 1e-3) / 1e6, 1), "ms_fwd_bwd": round(ms2, 4),
            "fwd_bwd_algorithmic_bytes": byts + byts_bwd,
            "fwd_bwd_frac_of_measured_hbm": round((byts + byts_bwd) / (ms2 * 1e-3) / 1e9 / peak, 4),
            "fwd_bwd_frac_of_nominal_8TBs": round((byts + byts_bwd) / (ms2 * 1e-3) / 1e9 / NOMINAL_HBM_GBS, 4)}


def bench_small(args, device):
    """The smallest configuration (1 x 1 x 64^2 -> 256^2, FP32, r = 1): a few
    CTAs per kernel, bound by latency, so reported as microseconds per call
    (eager and graph-replayed) and Mpix/s."""
    name = "fp32_small_1x1x256"
    spec = WORKLOADS[name]
    import torch
    g, _ = make_inputs(spec, device, seed=0)
    steps = max(50, min(args.steps, 1000))
    pix = 256 * 256
    cap = torch.cuda.Stream(device)
    with torch.cuda.stream(cap):
        step = Step(g, spec, device)  # calls go to the side stream, so the graph can capture them
        ms_f = time_loop(step.forward, steps, args.warmup, 1, device)
        ms_fb = time_loop(step, steps, args.warmup, 1, device)
        # the same calls captured once in a CUDA graph and replayed (what a
        # graph-captured training step pays: device time, no host launch cost)
        graph = torch.cuda.CUDAGraph()
        torch.cuda.synchronize()
        with torch.cuda.graph(graph, stream=cap):
            step()
        ms_g = time_loop(graph.replay, steps, args.warmup, 1, device)
    return {"workload": name, "us_fwd": round(ms_f * 1e3, 2), "us_fwd_bwd": round(ms_fb * 1e3, 2),
            "fwd_mpix_s": round(pix / (ms_f * 1e-3) / 1e6, 1), "fwd_bwd_mpix_s": round(pix / (ms_fb * 1e-3) / 1e6, 1),
            "us_fwd_bwd_graph": round(ms_g * 1e3, 2), "fwd_bwd_graph_mpix_s": round(pix / (ms_g * 1e-3) / 1e6, 1),
            "bound": "latency of the kernels' row walks: one plane of 64 x 64 low-res pixels gives each kernel "
                     "a grid of a few CTAs (far under one wave), so device time is a walk's serial latency, "
                     "and eager calls add the host launch cost on top (the graph-replayed figure has none)"}


def bench_paper_literal(args, device):
    """The layer as Sec. 3.2 / Algorithm 1 print it (no box mean of A, b), on
    the FP32 plain workload: forward + backward through the library."""
    from paper_1803_05619_gb300.layer import gf_backward, gf_forward
    spec = WORKLOADS[MAIN]
    g, _ = make_inputs(spec, device, seed=0)
    r, eps = spec["r"], spec["eps"]
    N, C, h, w = g["I_h"].shape

    def step():
        gf_forward(g["p_l"], g["I_l"], g["I_h"], r, eps, mean_ab=False)
        gf_backward(g["R"], g["p_l"], g["I_l"], g["I_h"], r, eps, mean_ab=False)

    steps = max(10, min(args.steps // 10, 200))
    ms = time_loop(step, steps, max(3, args.warmup // 4), 1, device)
    return {"workload": MAIN + " with mean_ab=0", "fwd_bwd_mpix_s": round(N * h * w / (ms * 1e-3) / 1e6, 1),
            "ms_fwd_bwd": round(ms, 4),
            "note": "through the Python binding (allocates outputs and workspace per call)"}


def bench_grey(args, device):
    """Grey guide (Sec. 4.2, DGF_b with differing channel counts): an RGB guide
    and a one-channel output, FP32 4 x (3 -> 1) x 512^2 -> 2048^2, r = 1,
    eps = 1e-4; forward and forward + backward through the library."""
    import synth
    from paper_1803_05619_gb300 import _lib as L
    from paper_1803_05619_gb300.layer import backward_reuses_coef, coef_buffer, gf_backward, gf_forward
    N, n_in, C, hl, f, r, eps = 4, 3, 1, 512, 4, 1, 1e-4
    gd = synth.blobs_tone_curve(31, N, n_in, hl, hl, f)
    pd = synth.blobs_tone_curve(32, N, C, hl, hl, f)
    p_l, I_l, I_h = (x.float().to(device) for x in (pd["p_l"], gd["I_l"], gd["I_h"]))
    R = synth.upstream_grad(33, (N, C, hl * f, hl * f)).float().to(device)
    h = w = hl * f

    # the forward keeps Abar, bbar where the backward then skips work (the layer's autograd rule)
    cf = coef_buffer(p_l, I_h) if backward_reuses_coef(p_l, I_h, r) else None

    def fwd():
        gf_forward(p_l, I_l, I_h, r, eps, coef=cf)

    def step():
        gf_forward(p_l, I_l, I_h, r, eps, coef=cf)
        gf_backward(R, p_l, I_l, I_h, r, eps, coef=cf)

    steps = max(10, min(args.steps // 10, 200))
    # the streaming form (grey guide formed in the workspace at both
    # resolutions, its gradient summed by a pass after the layer) for comparison
    L.dgf_set_grey_fold(False)
    try:
        fwd_ms_s = time_loop(fwd, steps, max(3, args.warmup // 4), 1, device)
        ms_s = time_loop(step, steps, max(3, args.warmup // 4), 1, device)
    finally:
        L.dgf_set_grey_fold(True)
    fwd_ms = time_loop(fwd, steps, max(3, args.warmup // 4), 1, device)
    ms = time_loop(step, steps, max(3, args.warmup // 4), 1, device)
    # the same calls replayed from CUDA graphs (no host work between kernels)
    import torch
    graphs = {}
    for name, fn in (("fwd", fwd), ("fwd_bwd", step)):
        cap = torch.cuda.Stream(device)
        torch.cuda.synchronize(device)
        with torch.cuda.stream(cap):
            fn()
        torch.cuda.synchronize(device)
        graphs[name] = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graphs[name], stream=cap):
            fn()
        torch.cuda.synchronize(device)
    fwd_ms_g = time_loop(graphs["fwd"].replay, steps, 3, 1, device)
    ms_g = time_loop(graphs["fwd_bwd"].replay, steps, 3, 1, device)
    L.dgf_profile_reset()
    L.dgf_profile_enable(True)
    try:
        step()
        torch.cuda.synchronize()
        prof = L.dgf_profile_read()
    finally:
        L.dgf_profile_enable(False)
    hi, lo = h * w * 4, hl * hl * 4
    # algorithmic bytes: forward reads I_h (3 channels), I_l (3), p_l and writes O_h;
    # backward reads dO_h, I_h (3), p_l, I_l (3) and writes dI_h (3), dp_l, dI_l (3)
    fwd_b = N * (n_in * hi + n_in * lo + C * lo + C * hi)
    bwd_b = N * (C * hi + n_in * hi + C * lo + n_in * lo + n_in * hi + C * lo + n_in * lo)
    peak = peaks()[0]
    return {"workload": "grey_guide_fp32_4x(3->1)x512->2048 (r=1, eps=1e-4)",
            "fwd_mpix_s": round(N * h * w / (fwd_ms * 1e-3) / 1e6, 1), "ms_fwd": round(fwd_ms, 4),
            "fwd_bwd_mpix_s": round(N * h * w / (ms * 1e-3) / 1e6, 1), "ms_fwd_bwd": round(ms, 4),
            "fwd_frac_of_measured_hbm": round(fwd_b / (fwd_ms * 1e-3) / 1e9 / peak, 4),
            "fwd_bwd_frac_of_measured_hbm": round((fwd_b + bwd_b) / (ms * 1e-3) / 1e9 / peak, 4),
            "graph": {"ms_fwd": round(fwd_ms_g, 4), "ms_fwd_bwd": round(ms_g, 4),
                      "fwd_bwd_mpix_s": round(N * h * w / (ms_g * 1e-3) / 1e6, 1),
                      "fwd_frac_of_measured_hbm": round(fwd_b / (fwd_ms_g * 1e-3) / 1e9 / peak, 4),
                      "fwd_bwd_frac_of_measured_hbm": round((fwd_b + bwd_b) / (ms_g * 1e-3) / 1e9 / peak, 4)},
            "kernels_avg_us": {k: round(v[0] / v[1] * 1e3, 1) for k, v in prof.items()},
            "streaming_form": {"ms_fwd": round(fwd_ms_s, 4), "ms_fwd_bwd": round(ms_s, 4)},
            "coef_kept": cf is not None,
            "note": "through the Python binding (allocates outputs and workspace per call); the high-res "
                    "kernels form the grey guide from I_h's channels in registers (k2_grey_apply, "
                    "k3_grey_bwd, which also writes dI_h); only the low-res guide and its gradient go "
                    "through streaming passes (grey_guide, grey_guide_adjoint). streaming_form: the guide "
                    "formed at both resolutions in the workspace before the layer and its gradient summed "
                    "after it"}


def bench_guided(args, device):
    """Training step with the guidance transform: BF16 8 x 3 x 256^2 -> 2048^2,
    r = 8, eps = 1e-4, forward + backward including the weight gradients."""
    import torch

    import synth
    from paper_1803_05619_gb300 import _lib as L
    from paper_1803_05619_gb300.layer import coef_buffer, gf_backward, gf_forward
    d = synth.photo_like(21, 8, 3, 256, 256, 8)
    g = {k: v.to(torch.bfloat16).to(device) for k, v in d.items()}
    w = {k: v.float().to(device) for k, v in synth.guide_weights(22).items()}
    R = synth.upstream_grad(23, g["I_h"].shape).to(torch.bfloat16).to(device)
    # the forward keeps Abar, bbar for the backward, as the layer's autograd function does
    cf = coef_buffer(g["p_l"], g["I_h"], guided=True)

    def step(coef=cf):
        gf_forward(g["p_l"], None, g["I_h"], 8, 1e-4, w["w1"], w["w2"], w["b2"], 0.2, coef=coef)
        gf_backward(R, g["p_l"], None, g["I_h"], 8, 1e-4, w["w1"], w["w2"], w["b2"], 0.2, coef=coef)

    steps = max(10, min(args.steps // 10, 100))
    ms_recompute = time_loop(lambda: step(None), steps, max(3, args.warmup // 4), 1, device)
    ms = time_loop(step, steps, max(3, args.warmup // 4), 1, device)
    L.dgf_profile_reset()
    L.dgf_profile_enable(True)
    try:
        for _ in range(5):
            step()
        torch.cuda.synchronize()
        prof = L.dgf_profile_read()
    finally:
        L.dgf_profile_enable(False)
    pix = 8 * 2048 * 2048
    avg = {k: v[0] / v[1] * 1e3 for k, v in prof.items()}
    out = {"workload": "guided_train_8x3x2048 (BF16, r=8, eps=1e-4, F: 3->15->3)",
           "fwd_bwd_mpix_s": round(pix / (ms * 1e-3) / 1e6, 1), "ms_fwd_bwd": round(ms, 4),
           "coef_kept": True, "ms_fwd_bwd_recomputing_coef": round(ms_recompute, 4),
           "bound": "alu (FP32 FMA of the 1x1 convolutions)",
           "kernels_avg_us": {k: round(v, 1) for k, v in avg.items()}}
    if "k6_guide_bwd" in avg:
        # K6 per high-res pixel: the hidden layer recomputed (3H FMA), d h = W2^T d G (3H),
        # the two weight-gradient outer products (3H + 3H), d I = W1^T d z (3H) and
        # d G = d O Abar_h + d G_l / f^2 (3): 15 H + 3 FMA, 2 flops each
        hid = 15
        flops = 2 * (15 * hid + 3) * pix
        ach = flops / (avg["k6_guide_bwd"] * 1e-6) / 1e12
        out["roofline"] = {"kernel": "k6_guide_bwd", "bound": "alu", "achieved": round(ach, 2),
                           "peak": FP32_FMA_TFLOPS, "unit": "TFLOP/s", "frac": round(ach / FP32_FMA_TFLOPS, 4),
                           "peak_source": "152 SMs x 128 FP32 lanes x 2 flops x 2.07 GHz (unit counts and "
                                          "maximum SM clock)",
                           "algorithmic_flops": flops, "us_per_call": round(avg["k6_guide_bwd"], 1)}

    # the same step with the transform applied to each guide on its own
    # (G_l = F(I_l), I_l the block mean of I_h): K5L and K6L replace K5's
    # high-res read and K6's low-res term
    def step_low():
        gf_forward(g["p_l"], g["I_l"], g["I_h"], 8, 1e-4, w["w1"], w["w2"], w["b2"], 0.2, guide_low=True, coef=cf)
        gf_backward(R, g["p_l"], g["I_l"], g["I_h"], 8, 1e-4, w["w1"], w["w2"], w["b2"], 0.2, guide_low=True,
                    coef=cf)

    ms_low = time_loop(step_low, steps, max(3, args.warmup // 4), 1, device)
    out["guide_low"] = {"fwd_bwd_mpix_s": round(pix / (ms_low * 1e-3) / 1e6, 1), "ms_fwd_bwd": round(ms_low, 4)}
    return out


if __name__ == "__main__":
    main()
