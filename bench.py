"""Benchmark of the hybrid denoiser (nonlocal BM3D stage + residual CNN).

One step = one pass of the whole hot path over one batch: colour handling
(grey here), BM3D pass 1 (matching, hard-threshold filtering, aggregation),
BM3D pass 2 (matching on the basic estimate, Wiener filtering,
aggregation), the 10-layer residual CNN of Eq. 2-3 and the FP64 error
reduction, on 16 synthetic 1024 x 1024 grey images at sigma = 25 that are
resident in HBM when the timed region starts.

Prints one JSON line (see the keys below).  `--impl reference` times the
FP64 oracle on the host cores instead (a bounded sample per step).
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

H = W = 1024
B = 16
SIGMA = 25.0
SEEDS0 = 100
FL_PREC = "fp32"  # contractions of the flexible network (--fl)
HIGH_PATCHES = False  # --bm3d-patches high: 12 x 12 / 11 x 11 patches above sigma 40
METRIC = "MPix/s BM3D+CNN at <=0.05 dB PSNR loss vs FP32 plain; served p50/p99 ms"
# the machine the FP32 ALU peak is derived for when the device is not queried
# (host-only use of the work counts): GB300's SM count and maximum SM clock
DEFAULT_HW = {"sm_count": 152, "sm_mhz": 2070.0, "source": "assumed (GB300: 152 SMs, 2070 MHz)"}


def fp32_peak(hw):
    """FP32 ALU peak in TFLOP/s: SMs x 128 FP32 lanes x 2 FLOP per FMA x SM clock."""
    return hw["sm_count"] * 128 * 2 * hw["sm_mhz"] * 1e6 / 1e12


def fp32_note(hw):
    return ("FP32 ALU peak = %d SM x 128 lanes x 2 FLOP/FMA x %.0f MHz = %.1f TFLOP/s (derived; SM count and clock %s)"
            % (hw["sm_count"], hw["sm_mhz"], fp32_peak(hw), hw["source"]))


def bm3d_params(precision=None):
    """The library's BM3D parameters (with the high-noise patch sides under
    --bm3d-patches high)."""
    from paper_2403_03488_gb300 import api
    return api.default_bm3d_params(precision=api.DN_FP32 if precision is None else precision,
                                   high_noise_patches=HIGH_PATCHES)


def oracle_passes(oracle):
    """The oracle's passes for the workload's sigma, as bm3d_params() selects them."""
    if HIGH_PATCHES and SIGMA > 40.0:
        return (oracle.Pass(patch=12, step=4, n2=16, tau=5000.0, lambda2d=oracle.LAMBDA2D_HIGH),
                oracle.Pass(patch=11, step=6, n2=32, tau=3500.0))
    return oracle.default_passes(SIGMA)


def workload_name(bm3d, cnn, prefilter="bm3d", net="resnet"):
    pre = "BM3D(%s%s)" % (bm3d, ", 12x12/11x11 patches" if HIGH_PATCHES and SIGMA > 40.0 else "") \
        if prefilter == "bm3d" else "NLM(fp32)"
    body = "CNN(10x32, %s)" % cnn if net == "resnet" else "FL-UNet(48-192, %s)" % FL_PREC
    return "hybrid %s+%s denoise, %d grey %dx%d synthetic images, sigma=%g" % (pre, body, B, H, W, SIGMA)


# ---------------------------------------------------------------------------
# clocks
# ---------------------------------------------------------------------------

class ClockSampler:
    FIELDS = ["clocks.sm", "clocks.max.sm", "power.draw", "clocks_event_reasons.hw_slowdown",
              "clocks_event_reasons.hw_thermal_slowdown", "clocks_event_reasons.sw_thermal_slowdown",
              "clocks_event_reasons.sw_power_cap"]

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + ",".join(self.FIELDS),
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) != len(self.FIELDS):
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[3:]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
# algorithmic work of the dominant kernels (per launch)
# ---------------------------------------------------------------------------

def match_pairs(Hh, Ww, step=3, search=39, k=8):
    """Exact number of (reference, candidate) distance evaluations of one
    matching launch over one image (patches of side k, candidates clipped to
    the image)."""
    from paper_2403_03488_gb300 import api
    hs = search // 2

    def per_axis(L):
        g = np.array(api.grid(L, k, step))
        return (np.minimum(L - k, g + hs) - np.maximum(0, g - hs) + 1).astype(np.int64)

    return int(per_axis(Hh).sum() * per_axis(Ww).sum())


# Collaborative filtering work per patch of a full group (n = n2 patches), in
# FLOP.  "tensor": the 3D transform written as dense contractions, as the
# nominal per-pixel figures of the filtering rows count it: the 2D DCT of a
# patch and its inverse as 64 x 64 matrix-vector products (2 x 8192 each) and
# the group transform as an n x n product per coefficient (2 n per coefficient
# and direction); pass 1 transforms the noisy group forward and back (2 + 2),
# pass 2 the basic and noisy groups forward and the estimate back (3 + 3).
# "alu": the separable form the CUDA-core kernels evaluate: each 2D DCT as 2k
# k-point matrix-vector products (2 k^2 each: 2048 FLOP per 8 x 8 patch), the
# group transform as a fast Walsh-Hadamard transform (log2 n additions per
# coefficient and direction), 2 FLOP per coefficient for shrinkage (pass 2:
# 4, the Wiener gain) and 3 per pixel for the windowed aggregation.  k: the
# patch side (8; 12 and 11 in the high-noise profile's passes).
def filter_flops_per_patch(wiener, n, k=8):
    lg = max(1, int(np.log2(n)))
    nt = 3 if wiener else 2  # 2D transforms per patch
    k2 = k * k
    tensor = nt * 2 * k2 * k2 + nt * 2 * n * k2
    alu = nt * 4 * k ** 3 + nt * k2 * lg + (4 if wiener else 2) * k2 + 3 * k2
    return tensor, alu


def filter_work(wiener, Hh, Ww, batch, step=3, k=8):
    """(tensor FLOP, ALU FLOP) of one filtering launch over `batch` images,
    every group full (n = 16 in pass 1, 32 in pass 2): an upper count, since
    groups below the threshold hold fewer patches."""
    from paper_2403_03488_gb300 import api
    refs = len(api.grid(Hh, k, step)) * len(api.grid(Ww, k, step)) * batch
    n = 32 if wiener else 16
    t, a = filter_flops_per_patch(wiener, n, k)
    return refs * n * t, refs * n * a


# Patch side and grid step of the larger-patch kernels (the high-noise
# profile: 12 x 12 on a step-4 grid in pass 1, 11 x 11 on a step-6 grid in
# pass 2; the pixel matcher runs pass 2 there).
LARGE = {"bm3d_match_pre_large": (12, 4), "bm3d_match_large_fp32": (11, 6),
         "bm3d_filter_hard_large_fp32": (12, 4), "bm3d_filter_wiener_large_fp32": (11, 6)}


def algorithmic(kernel, launches_per_step, batch, hw=None):
    """(bound, unit, work per launch, peak, peak note) for a kernel name."""
    hw = hw or DEFAULT_HW
    peaks = {}
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        peaks = json.load(open(p))
    fpk, fnote = fp32_peak(hw), fp32_note(hw)
    if kernel in LARGE:
        k, step = LARGE[kernel]
        if kernel.startswith("bm3d_match"):
            # 3 FLOP (sub, mul, add) per pixel or prethresholded coefficient of each pair
            return "alu", "TFLOP/s", 3.0 * k * k * match_pairs(H, W, step, 39, k) * min(batch, 64), fpk, fnote
        tensor, alu = filter_work("wiener" in kernel, H, W, batch, step, k)
        return "alu", "TFLOP/s", float(alu), fpk, fnote + " (separable count)"
    if kernel.startswith("bm3d_match"):
        # one launch covers up to 64 images of one pass; 192 FLOP (sub, mul, add over 64 pixels or
        # prethresholded coefficients) per (reference, candidate) pair
        pairs = match_pairs(H, W) * min(batch, 64)
        return "alu", "TFLOP/s", 192.0 * pairs, fpk, fnote
    if kernel.startswith("bm3d_filter_"):
        wiener = "wiener" in kernel
        tensor, alu = filter_work(wiener, H, W, batch)
        if kernel.endswith("bf16"):
            bf = peaks.get("bf16_tflops_sustained", 1700.0)
            return "tensor", "TFLOP/s", float(tensor), bf, "measured bf16_tflops_sustained (dense contractions count)"
        return "alu", "TFLOP/s", float(alu), fpk, fnote + " (separable count)"
    if kernel.startswith("nlm_fp32"):
        # per pixel and search offset: difference + square (2), separable 7 + 7 box sums (12), weight (4:
        # subtract, clamp, scale, exp) and the two weighted accumulations (4)
        flops = 22.0 * 441 * H * W * batch / launches_per_step
        return "alu", "TFLOP/s", flops, fpk, fnote
    if kernel.startswith("conv3x3_fwd_fp32"):
        flops = 2.0 * H * W * batch * (2 * 32 * 9 + 8 * 32 * 32 * 9 + 32 * 9) / launches_per_step
        return "alu", "TFLOP/s", flops, fpk, fnote
    hbm = peaks.get("hbm_gbs", 6800.0)
    px = H * W * batch  # every launch of these kernels covers the whole batch
    hbm_bytes = {
        "conv3x3_tc_bf16": 2 * px * 32 * 2,   # NHWC BF16 activations in and out
        "conv3x3_tc_pair_bf16": 2 * px * 32 * 2,  # two layers per launch: in and out once
        "conv_first_bf16": px * (8 + 64),     # prefilter + noisy FP32 in, 32 BF16 channels out
        "conv_last_bf16": px * (64 + 4 + 4),  # 32 BF16 channels + prefilter in, FP32 out
        "bm3d_normalize": px * (4 * 8 + 4),   # four 64-bit fixed-point planes in, FP32 out
        "error_reduce_fp64": px * 8,          # output and clean image
    }
    if kernel in hbm_bytes:
        return "hbm", "GB/s", float(hbm_bytes[kernel]), hbm, "measured hbm_gbs"
    if kernel.startswith(("fl_pw_fwd", "fl_deconv2x2_fwd", "fl_dw3x3_fwd")):
        from paper_2403_03488_gb300.flnet import work_per_pixel
        wpp, px = work_per_pixel(), H * W * batch / launches_per_step
        if kernel.startswith("fl_dw3x3_fwd"):  # 9 MAC per output: moves bytes, not FLOPs
            return "hbm", "GB/s", wpp["dw_bytes"] * px, hbm, "measured hbm_gbs"
        if kernel.endswith("_tc"):  # tensor-core contractions of FP32 planes: the planes' bytes bound them
            return "hbm", "GB/s", wpp["pw_bytes" if kernel.startswith("fl_pw") else "up_bytes"] * px, hbm, \
                "measured hbm_gbs"
        macs = wpp["pw_macs"] if kernel.startswith("fl_pw_fwd") else wpp["up_macs"]
        return "alu", "TFLOP/s", 2.0 * macs * px, fpk, fnote
    # fall back to bytes: read + write of the image planes
    return "hbm", "GB/s", 8.0 * H * W * batch / launches_per_step, hbm, "measured hbm_gbs"


def kernel_rooflines(res, steps, batch, hw=None):
    """Roofline fraction of every library kernel whose algorithmic work has a
    plain count (see `algorithmic`): the matcher, NLM, the collaborative
    filters and the flexible network's layers in FLOP, the CNN layers, the
    normalisation, the depthwise layers and the error reduction in bytes that
    must cross HBM per launch (activations / planes read and written once,
    halos excluded).  The FP32 filters also carry their dense-contraction
    count against the BF16 tensor peak (`tensor_frac`)."""
    out = {}
    peaks = {}
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        peaks = json.load(open(p))
    for k, (n, ms) in res.items():
        if not k.startswith(("bm3d_match_fp32", "bm3d_match_pre", "bm3d_match_tc", "bm3d_match_large", "bm3d_filter_",
                             "nlm_fp32",
                             "fl_pw_fwd", "fl_deconv2x2_fwd", "fl_dw3x3_fwd", "conv3x3_tc_bf16", "conv3x3_tc_pair",
                             "conv_first_bf16", "conv_last_bf16", "bm3d_normalize", "error_reduce_fp64")):
            continue
        avg = ms / n
        bound, unit, work, peak, _ = algorithmic(k, n / steps, batch, hw)
        ach = work / (avg / 1e3) / (1e12 if unit == "TFLOP/s" else 1e9)
        out[k] = {"bound": bound, "achieved": round(ach, 3 if unit == "TFLOP/s" else 1), "peak": round(peak, 1),
                  "unit": unit, "frac": round(ach / peak, 4), "avg_launch_ms": round(avg, 4),
                  "traffic": load_traffic(k)}
        if k.startswith(("conv3x3_tc_bf16", "conv3x3_tc_pair")):
            nl = 2 if "pair" in k else 1  # hidden 32 -> 32 layers per launch, 2 * 9 * 32 * 32 FLOP per pixel each
            t_ach = nl * 2.0 * 9 * 32 * 32 * H * W * batch / (avg / 1e3) / 1e12
            bf = peaks.get("bf16_tflops_sustained", 1700.0)
            out[k].update({"tensor_achieved": round(t_ach, 3), "tensor_peak": round(bf, 1),
                           "tensor_frac": round(t_ach / bf, 4)})
        if k.startswith("bm3d_filter_") and k.endswith("fp32"):
            ks, st = LARGE.get(k, (8, 3))
            tensor, _ = filter_work("wiener" in k, H, W, batch, st, ks)
            t_ach = tensor / (avg / 1e3) / 1e12
            bf = peaks.get("bf16_tflops_sustained", 1700.0)
            out[k].update({"tensor_achieved": round(t_ach, 3), "tensor_peak": round(bf, 1),
                           "tensor_frac": round(t_ach / bf, 4)})
    return out


# ---------------------------------------------------------------------------
# multi-rank host logic (weak scaling: each rank denoises its own images, no
# data-path collective; only the timing is reduced across ranks)
# ---------------------------------------------------------------------------

def rank_seeds(rank, batch=None):
    """Image seeds of one rank: a batch of its own (B images unless given),
    disjoint from every other rank's."""
    batch = B if batch is None else batch
    return list(range(SEEDS0 + rank * batch, SEEDS0 + (rank + 1) * batch))


def max_over_ranks(x):
    """The largest value of x over all ranks (x itself without a process group)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    dev = torch.device("cuda", torch.cuda.current_device()) if dist.get_backend() == "nccl" else torch.device("cpu")
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_value(mpix_per_rank, world, ms_per_step):
    """Megapixels all ranks processed per second, timed by the slowest rank."""
    return mpix_per_rank * world / (ms_per_step / 1e3)


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------

def run_ours(args):
    import torch
    import torch.distributed as dist

    from paper_2403_03488_gb300 import api, synth
    from paper_2403_03488_gb300.autograd import ResidualNet

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    seeds = rank_seeds(rank)
    clean, noisy = synth.make_batch(seeds, H, W, SIGMA)
    noisy_d = torch.from_numpy(noisy).to(dev)
    clean_d = torch.from_numpy(clean).to(dev)
    out_d = torch.empty_like(noisy_d)
    weights, wsrc = load_weights(dev)
    bprec = bm3d_precision(args)
    prec = api.DN_BF16 if args.cnn == "bf16" else api.DN_FP32
    nlm = args.prefilter == "nlm"
    pf = api.DN_PREFILTER_NLM if nlm else api.DN_PREFILTER_BM3D
    bp = api.default_nlm_params() if nlm else bm3d_params(bprec)
    cnn = api.make_cnn(weights, 10, 32, prec)
    ws = torch.empty(api.hybrid_workspace_bytes(B, 1, H, W, pf, bp, cnn), dtype=torch.uint8, device=dev)
    sse = torch.empty(B, dtype=torch.float64, device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    fl = args.net == "fl"
    if fl:
        flnet, wsrc = load_fl(dev, args.prefilter, api.DN_BF16 if args.fl == "bf16" else api.DN_FP32)
        pre_d = torch.empty_like(noisy_d)
        ws_pre = torch.empty(api.bm3d_workspace_bytes(B, 1, H, W, bp) if not nlm else 1, dtype=torch.uint8,
                             device=dev)

    def denoise(x, out):
        """The hybrid on device tensors: the C-ABI hybrid, or prefilter + the flexible network."""
        if not fl:
            api.denoise_hybrid(x, SIGMA, weights, prefilter=pf, prefilter_params=bp, cnn_precision=prec, out=out,
                               workspace=ws)
            return
        if nlm:
            api.denoise_nlm(x, SIGMA, bp, out=pre_d)
        else:
            api.denoise_bm3d(x, SIGMA, bp, out=pre_d, workspace=ws_pre)
        n = x.shape[0]
        with torch.no_grad():
            flnet(x.view(n, H, W), pre_d.view(n, H, W), [SIGMA] * n, out=out.view(n, H, W))

    def step():
        denoise(noisy_d, out_d)
        api.error_reduce(out_d, clean_d)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()

    clocks = ClockSampler(local)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    time.sleep(0.3)
    total_ms = 0.0
    with api.profile() as prof:
        for _ in range(args.steps):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            step()
            e1.record()
            e1.synchronize()
            total_ms += e0.elapsed_time(e1)
    torch.cuda.synchronize()
    clk = clocks.stop()
    total_ms = max_over_ranks(total_ms)
    if world > 1:
        dist.barrier()

    ms_per_step = total_ms / args.steps
    mpix = B * H * W / 1e6
    value = whole_job_value(mpix, world, ms_per_step)

    # quality of this step's output against the clean images (FP64 reduction)
    sse_d, _ = api.error_reduce(out_d, clean_d)
    mse = float(sse_d.sum().item()) / (B * H * W)
    psnr_out = 10 * np.log10(255.0 ** 2 / mse)
    # the FP32 plain path on the same batch (untimed), for the PSNR-loss criterion
    if fl and args.fl == "fp32":
        plain = out_d.clone()  # the FP32 flexible network is its own plain path
    elif fl:
        fl32, _ = load_fl(dev, args.prefilter, api.DN_FP32)
        plain = torch.empty_like(out_d)
        with torch.no_grad():
            fl32(noisy_d.view(B, H, W), pre_d.view(B, H, W), [SIGMA] * B, out=plain.view(B, H, W))
        del fl32
    else:
        plain = api.denoise_hybrid(noisy_d, SIGMA, weights, prefilter=pf,
                                   prefilter_params=bp if nlm else bm3d_params(),
                                   cnn_precision=api.DN_FP32)
    sse_p, _ = api.error_reduce(plain, clean_d)
    psnr_plain = 10 * np.log10(255.0 ** 2 / (float(sse_p.sum().item()) / (B * H * W)))
    # throughput of the FP32 plain path on the same batch (FP32 BM3D, FP32 SIMT CNN; same L2 flush)
    plain_ms = None
    if not fl:
        plain_out = torch.empty_like(noisy_d)
        pparams = bp if nlm else bm3d_params()
        plain_steps = 2
        plain_ms = 0.0
        for _ in range(plain_steps):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            api.denoise_hybrid(noisy_d, SIGMA, weights, prefilter=pf, prefilter_params=pparams,
                               cnn_precision=api.DN_FP32, out=plain_out)
            api.error_reduce(plain_out, clean_d)
            e1.record()
            e1.synchronize()
            plain_ms += e0.elapsed_time(e1)
        plain_ms = max_over_ranks(plain_ms) / plain_steps
        del plain_out
    out0 = out_d[0].clone()
    plain0 = plain[0].clone()
    bm3d_only = api.denoise_nlm(noisy_d, SIGMA, bp) if nlm else api.denoise_bm3d(noisy_d, SIGMA, bp)
    sse_b, _ = api.error_reduce(bm3d_only, clean_d)
    psnr_bm3d = 10 * np.log10(255.0 ** 2 / (float(sse_b.sum().item()) / (B * H * W)))
    del plain, bm3d_only

    # end to end through the public API with host buffers
    noisy_h = torch.from_numpy(noisy).pin_memory()
    out_h = torch.empty_like(noisy_h).pin_memory()
    for _ in range(2):
        x = noisy_h.to(dev, non_blocking=True)
        denoise(x, out_d)
        out_h.copy_(out_d, non_blocking=True)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    e2e_ms = 0.0
    e2e_steps = max(2, min(args.steps, 5))
    for _ in range(e2e_steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        x = noisy_h.to(dev, non_blocking=True)
        denoise(x, out_d)
        out_h.copy_(out_d, non_blocking=True)
        e1.record()
        e1.synchronize()
        e2e_ms += e0.elapsed_time(e1)
    e2e_ms = max_over_ranks(e2e_ms)
    e2e_value = whole_job_value(mpix, world, e2e_ms / e2e_steps)

    res = prof.result
    launches = sum(c for c, _ in res.values())
    top = max(res.items(), key=lambda kv: kv[1][1])
    kname, (kl, kms) = top
    per_step = kl / args.steps
    props = torch.cuda.get_device_properties(local)
    hw = {"sm_count": int(props.multi_processor_count),
          "sm_mhz": float(clk.get("sm_mhz") or clk.get("sm_max_mhz") or DEFAULT_HW["sm_mhz"]),
          "source": "read: multi_processor_count of the device, median SM clock sampled in the timed region"}
    bound, unit, work, peak, peak_note = algorithmic(kname, per_step, B, hw)
    avg_ms = kms / kl
    achieved = work / (avg_ms / 1e3) / (1e12 if unit == "TFLOP/s" else 1e9)
    traffic = load_traffic(kname)

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return
    line = {
        "metric": (METRIC if args.prefilter == "bm3d" else METRIC.replace("BM3D+CNN", "NLM+CNN")).replace(
            "+CNN", "+CNN" if args.net == "resnet" else "+FL-CNN"),
        "value": round(value, 3),
        "unit": "MPix/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": round(ms_per_step, 3),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "+".join(sorted({"f32" if bprec == api.DN_FP32 else "bf16",
                                  ("f32" if args.fl == "fp32" else "bf16") if args.net == "fl" else
                                  ("f32" if prec == api.DN_FP32 else "bf16")})),
        "data": "synthetic (seeded piecewise-smooth + gratings + repeated tile, AWGN sigma=%g)" % SIGMA,
        "config": {"workload": workload_name(args.bm3d, args.cnn, args.prefilter, args.net), "global_batch": B * world,
                   "image": [H, W],
                   "channels": 1, "sigma": SIGMA,
                   "cnn": ("10 layers x 32 ch, " if args.net == "resnet" else "flexible U-Net (Sec. III), ") + wsrc,
                   "l2": "flushed between timed steps (256 MB write)", "parallelism": "replicas (dp%d)" % world},
        "psnr_db": round(psnr_out, 3),
        "psnr_fp32_plain_db": round(psnr_plain, 3),
        "psnr_loss_vs_fp32_plain_db": round(psnr_plain - psnr_out, 4),
        ("psnr_nlm_only_db" if args.prefilter == "nlm" else "psnr_bm3d_only_db"): round(psnr_bm3d, 3),
        "e2e": {"value": round(e2e_value, 3), "unit": "MPix/s", "h2d_bytes_per_step": int(noisy_h.numel() * 4),
                "d2h_bytes_per_step": int(out_h.numel() * 4)},
        "gpu_launches": int(launches),
        "roofline": {"bound": bound, "kernel": kname, "achieved": round(achieved, 3), "peak": round(peak, 1),
                     "unit": unit, "frac": round(achieved / peak, 4), "traffic": traffic,
                     "avg_launch_ms": round(avg_ms, 4), "peak_source": peak_note},
        "kernels": {k: {"launches": c, "ms": round(t, 3), "share": round(t / sum(x[1] for x in res.values()), 4)}
                    for k, (c, t) in sorted(res.items(), key=lambda kv: -kv[1][1])},
        "kernel_rooflines": kernel_rooflines(res, args.steps, B, hw),
        "fp32_peak": {"tflops": round(fp32_peak(hw), 2), "sm_count": hw["sm_count"], "sm_mhz": hw["sm_mhz"],
                      "source": hw["source"]},
        "clocks": clk,
    }
    if plain_ms is not None:
        line["fp32_plain"] = {"value": round(whole_job_value(mpix, world, plain_ms), 3), "unit": "MPix/s",
                              "ms_per_step": round(plain_ms, 3),
                              "what": "same workload, FP32 BM3D + FP32 CUDA-core CNN, same timing rules"}
    if not args.no_serving:
        line["serving"] = serving_replay(args)
    if world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"], oracle_out = cpu_baseline(args.cpu_side, None if fl else weights)
        if not fl:
            line["vs_fp64_oracle"] = vs_oracle(oracle_out, noisy_d, clean, args.cpu_side, out0, plain0, denoise,
                                               weights, pf, bp, nlm)
    print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()


def bm3d_precision(args):
    from paper_2403_03488_gb300 import api
    return {"fp32": api.DN_FP32, "bf16": api.DN_BF16, "bf16+match": api.DN_BF16 | api.DN_BF16_MATCH}[args.bm3d]


def serving_replay(args):
    """Open-loop Poisson replay through the continuous-batching server (the
    served p50/p99 part of the metric), for the fast path and, on the same
    trace, the FP32 plain path."""
    from paper_2403_03488_gb300 import api, serve
    fast = serve.replay(rate=args.serve_rate, n=args.serve_requests, side=(128, 2048),
                        bm3d_precision=bm3d_precision(args),
                        cnn_precision=api.DN_BF16 if args.cnn == "bf16" else api.DN_FP32)
    # the FP32 plain path serves the first 300 requests of the same trace (at about 36 MPix/s it
    # would need minutes for all of them)
    plain = serve.replay(rate=args.serve_rate, n=min(args.serve_requests, 300), side=(128, 2048),
                         bm3d_precision=api.DN_FP32, cnn_precision=api.DN_FP32, warm=False)
    keys = ("p50_ms", "p99_ms", "served_mpix_s", "served_channel_mpix_s", "makespan_s", "max_inflight", "launches",
            "max_batch")
    out = {k: round(fast[k], 3) for k in keys}
    out.update({"offered_mpix_s": round(fast["offered_mpix_s"], 1), "trace": fast["trace"],
                "budget_gb": 60, "slots": 8,
                "fp32_plain": dict({k: round(plain[k], 3) for k in keys}, trace=plain["trace"])})
    out["saturated"] = bool(fast["served_mpix_s"] < 0.9 * fast["offered_mpix_s"])
    if out["saturated"]:
        # the same trace shape at 60 % of the served rate: latency without a growing queue
        rate = args.serve_rate * 0.6 * fast["served_mpix_s"] / fast["offered_mpix_s"]
        stable = serve.replay(rate=rate, n=args.serve_requests, side=(128, 2048),
                              bm3d_precision=bm3d_precision(args),
                              cnn_precision=api.DN_BF16 if args.cnn == "bf16" else api.DN_FP32, warm=False)
        out["stable_load"] = {k: round(stable[k], 3) for k in keys}
        out["stable_load"].update({"rate_per_s": round(rate, 1), "offered_mpix_s": round(stable["offered_mpix_s"], 1)})
    return out


def load_weights(dev):
    """Trained 10x32 weights when the repository ships them, else He init (seed 0)."""
    import torch
    from paper_2403_03488_gb300.autograd import ResidualNet
    p = os.path.join(ROOT, "paper_2403_03488_gb300", "weights", "resnet10x32_bm3d.npy")
    if os.path.exists(p):
        w = torch.from_numpy(np.load(p).astype(np.float32)).to(dev)
        return w.contiguous(), "trained weights (" + os.path.basename(p) + ")"
    return ResidualNet(10, 32, seed=0).to(dev).flat_weights(), "random init (He, seed 0)"


def load_fl(dev, prefilter="bm3d", precision=None):
    """The flexible network with the shipped weights trained on this prefilter's
    output when present, else He init (seed 0)."""
    from paper_2403_03488_gb300 import api
    from paper_2403_03488_gb300.flnet import FLNet
    import torch
    prec = api.DN_FP32 if precision is None else precision
    p = os.path.join(ROOT, "paper_2403_03488_gb300", "weights", "flnet_%s.npy" % prefilter)
    if os.path.exists(p):
        return FLNet(flat=torch.from_numpy(np.load(p).astype(np.float32)), precision=prec).to(dev), \
            "trained weights (" + os.path.basename(p) + ")"
    return FLNet(seed=0, precision=prec).to(dev), "random init (He, seed 0)"


def load_traffic(kname):
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if os.path.exists(p):
        t = json.load(open(p))
        v = t.get(kname)
        return v
    return None


# ---------------------------------------------------------------------------
# the oracle on host cores
# ---------------------------------------------------------------------------

def oracle_step(side, weights=None):
    """FP64 oracle BM3D (both passes) + residual CNN on one side x side crop of
    image 0 of the workload; returns (seconds, megapixels, output [side, side]).
    weights: the flat FP32 parameters the GPU runs (host or device tensor), else
    He init (seed 0)."""
    import oracle
    from paper_2403_03488_gb300 import synth
    from paper_2403_03488_gb300.synth import he_normal_weights
    clean, noisy = synth.make_batch([SEEDS0], H, W, SIGMA)
    crop = noisy[0, :, :side, :side].astype(np.float64)
    if weights is None:
        params = he_normal_weights(0, 10, 32)
    else:
        from paper_2403_03488_gb300.autograd import ResidualNet
        params = ResidualNet(10, 32, flat=weights.detach().cpu()).numpy_params()
    t0 = time.perf_counter()
    hard, wiener = oracle_passes(oracle)
    _, final = oracle.bm3d(crop, SIGMA, hard=hard, wiener=wiener)
    out = oracle.cnn_forward(crop[:, :, :], final, params)
    dt = time.perf_counter() - t0
    return dt, side * side / 1e6, np.asarray(out)[0]


def cpu_baseline(side, weights=None):
    import oracle
    oracle.build()
    dt, mp, out = oracle_step(side, weights)
    return {"value": round(mp / dt, 5), "unit": "MPix/s", "cores": oracle.num_threads(), "kind": "oracle",
            "sample": "FP64 oracle BM3D (both passes) + 10x32 CNN forward (%s) on one %dx%d crop of image 0 "
                      "(%.1f s)" % ("the bench's weights" if weights is not None else "He init", side, side, dt)}, out


def vs_oracle(ref, noisy_d, clean, side, out0, plain0, denoise, weights, pf, bp, nlm):
    """PSNR delta and max |error| of the GPU results against the FP64 oracle on
    the cpu_baseline crop (image 0; when the crop is the whole image, the
    outputs of the timed step are compared directly)."""
    import torch
    from paper_2403_03488_gb300 import api
    c = clean[0, 0, :side, :side].astype(np.float64)
    if side == H and side == W:
        fast, plain = out0[0].cpu().numpy(), plain0[0].cpu().numpy()
    else:
        x = noisy_d[:1, :, :side, :side].contiguous()
        o = torch.empty_like(x)
        denoise(x, o)
        fast = o[0, 0].cpu().numpy()
        plain = api.denoise_hybrid(x, SIGMA, weights, prefilter=pf,
                                   prefilter_params=bp if nlm else bm3d_params(),
                                   cnn_precision=api.DN_FP32)[0, 0].cpu().numpy()

    def psnr(a):
        return 10 * np.log10(255.0 ** 2 / np.mean((np.clip(a, 0, 255) - c) ** 2))

    out = {"crop": "%dx%d of image 0" % (side, side), "oracle_psnr_db": round(psnr(ref), 4)}
    for name, a in (("fast", fast), ("fp32_plain", plain)):
        e = np.abs(a.astype(np.float64) - ref)
        out[name] = {"psnr_delta_db": round(psnr(a) - psnr(ref), 5), "max_abs_err": round(float(e.max()), 5),
                     "p999_abs_err": round(float(np.quantile(e, 0.999)), 5),
                     "mean_abs_err": round(float(e.mean()), 6)}
    return out


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    oracle.build()
    for _ in range(args.warmup):
        oracle_step(64)
    total, mp = 0.0, 0.0
    for _ in range(args.steps):
        dt, m, _ = oracle_step(args.ref_side)
        total += dt
        mp += m
    value = mp / total
    line = {
        "impl": "reference",
        "metric": METRIC,
        "value": round(value, 5),
        "unit": "MPix/s",
        "n_gpus": int(os.environ.get("WORLD_SIZE", "1")),
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": round(1e3 * total / args.steps, 3),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f64",
        "data": "synthetic (seeded piecewise-smooth + gratings + repeated tile, AWGN sigma=%g)" % SIGMA,
        "config": {"workload": workload_name("fp64 oracle", "fp64 oracle"), "sample_per_step": "%dx%d crop of image 0" % (
            args.ref_side, args.ref_side)},
        "cpu_baseline": {"value": round(value, 5), "unit": "MPix/s", "cores": oracle.num_threads(), "kind": "oracle",
                         "sample": "%dx%d crop per step" % (args.ref_side, args.ref_side)},
        "e2e": {"value": round(value, 5), "unit": "MPix/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--bm3d", default="fp32", choices=["fp32", "bf16", "bf16+match"],
                    help="BM3D precision: fp32 SIMT; bf16 = 2D transforms on the tensor cores; bf16+match = also "
                         "the BF16 tensor-core matching prefilter (exact FP32 re-rank)")
    ap.add_argument("--cnn", default="bf16", choices=["fp32", "bf16"], help="CNN precision")
    ap.add_argument("--net", default="resnet", choices=["resnet", "fl"],
                    help="network after the prefilter: the 10x32 residual CNN, or the flexible U-Net of Sec. III")
    ap.add_argument("--fl", default="fp32", choices=["fp32", "bf16"],
                    help="flexible network: FP32 CUDA-core layers, or its contractions on the tensor cores")
    ap.add_argument("--prefilter", default="bm3d", choices=["bm3d", "nlm"],
                    help="nonlocal prefilter of the hybrid (nlm: the lighter NL-means + CNN variant)")
    ap.add_argument("--cpu-side", type=int, default=1024)
    ap.add_argument("--ref-side", type=int, default=192)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--serve-rate", type=float, default=200.0)
    ap.add_argument("--serve-requests", type=int, default=2000)
    ap.add_argument("--batch", type=int, default=None, help="images per step (profiling runs; default 16)")
    ap.add_argument("--size", type=int, default=None, help="image side (profiling runs; default 1024)")
    ap.add_argument("--sigma", type=float, default=None,
                    help="noise level (default 25; above 40 the first pass matches on prethresholded patches)")
    ap.add_argument("--bm3d-patches", default="8", choices=["8", "high"],
                    help="high: the 12 x 12 / 11 x 11 patches of the high-noise profile above sigma 40")
    args = ap.parse_args()
    global H, W, B, SIGMA, HIGH_PATCHES
    HIGH_PATCHES = args.bm3d_patches == "high"
    if args.sigma:
        SIGMA = args.sigma
    if args.size:
        H = W = args.size
    if args.batch:
        B = args.batch
    args.warmup = max(3, args.warmup) if args.impl == "ours" else args.warmup
    global FL_PREC
    FL_PREC = "bf16 contractions" if args.fl == "bf16" else "fp32"
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
