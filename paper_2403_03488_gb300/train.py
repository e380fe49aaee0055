"""Training of the residual CNN (Sec. II, Eq. 2-3), or of the flexible
lightweight network of Sec. III (--net fl), on the library's kernels.

Pairs: seeded synthetic 512 x 512 scenes, sigma ~ U[5, 50] per image (one
blind model), noisy = clean + AWGN, pre = the GPU BM3D of the noisy image
(denoise_bm3d).  Steps: random 64 x 64 crops, batch 64, L1 loss of Eq. 2,
Adam lr 1e-3, every forward / backward / update in the library's kernels
(ResidualNet.train_step).  Checkpoints hold the master weights, Adam moments,
step and crop-sampler state, so a resumed run is bit-identical.

    python -m paper_2403_03488_gb300.train --steps 20000 --out weights/resnet10x32_bm3d.npy
    python -m paper_2403_03488_gb300.train --net fl --steps 20000 --out weights/flnet_bm3d.npy

The flexible network also receives each crop's noise level (its input plane).
"""
from __future__ import annotations

import argparse
import json
import os
import time

import numpy as np
import torch

from . import api, synth
from .autograd import ResidualNet
from .flnet import FLNet

HERE = os.path.dirname(os.path.abspath(__file__))
DEFAULT_OUT = os.path.join(HERE, "weights", "resnet10x32_bm3d.npy")


def make_pool(n_images=256, H=512, W=512, seed0=10_000, sigma_range=(5.0, 50.0), prefilter="bm3d",
              device="cuda", chunk=16):
    """(clean, noisy, pre, sigma) device tensors [n, H, W] built from seeded scenes."""
    rng = np.random.Generator(np.random.PCG64(seed0))
    sig = rng.uniform(sigma_range[0], sigma_range[1], n_images)
    clean = torch.empty((n_images, H, W), dtype=torch.float32, device=device)
    noisy = torch.empty_like(clean)
    pre = torch.empty_like(clean)
    for c0 in range(0, n_images, chunk):
        c1 = min(n_images, c0 + chunk)
        seeds = list(range(seed0 + c0, seed0 + c1))
        cl, ny = synth.make_batch(seeds, H, W, list(sig[c0:c1]))
        x = torch.from_numpy(ny).to(device)
        if prefilter == "bm3d":
            p = api.denoise_bm3d(x, list(sig[c0:c1]))
        else:
            p = api.denoise_nlm(x, list(sig[c0:c1]))
        clean[c0:c1] = torch.from_numpy(cl[:, 0]).to(device)
        noisy[c0:c1] = x[:, 0]
        pre[c0:c1] = p[:, 0]
    return clean, noisy, pre, sig


class CropSampler:
    """Seeded random crops gathered with one index tensor per batch."""

    def __init__(self, n, H, W, crop, batch, seed, device):
        self.n, self.H, self.W, self.crop, self.batch = n, H, W, crop, batch
        self.rng = np.random.Generator(np.random.PCG64(seed))
        d = torch.arange(crop, device=device)
        self.offs = (d[:, None] * W + d[None, :]).view(1, crop, crop)
        self.device = device

    def next(self, *pools):
        i = self.rng.integers(0, self.n, self.batch)
        y = self.rng.integers(0, self.H - self.crop + 1, self.batch)
        x = self.rng.integers(0, self.W - self.crop + 1, self.batch)
        self.last = i
        base = torch.from_numpy(i * self.H * self.W + y * self.W + x).to(self.device).view(-1, 1, 1)
        idx = base + self.offs
        return [p.view(-1)[idx] for p in pools]


def train(steps=20000, batch=64, crop=64, lr=1e-3, seed=0, n_images=256, prefilter="bm3d", log_every=500,
          checkpoint=None, resume=True, device="cuda", log=print, net_kind="resnet", max_minutes=None,
          precision="fp32"):
    """precision (residual network only): "fp32" = the FP32 CUDA-core layer
    kernels, "bf16" = dn_cnn_grad's tensor-core forward and backward (BF16
    operands, FP32 accumulation and master weights)."""
    t0 = time.time()
    clean, noisy, pre, sig = make_pool(n_images=n_images, prefilter=prefilter, device=device)
    torch.cuda.synchronize()
    log("pool of %d images ready in %.1f s" % (n_images, time.time() - t0))
    fl = net_kind == "fl"
    net = (FLNet(seed=seed) if fl else ResidualNet(10, 32, seed=seed)).to(device)
    sampler = CropSampler(n_images, clean.shape[1], clean.shape[2], crop, batch, seed + 1, device)
    start = 0
    if checkpoint and resume and os.path.exists(checkpoint):
        ck = torch.load(checkpoint, map_location=device)
        net.flat.data.copy_(ck["flat"])
        net.m.copy_(ck["m"])
        net.v.copy_(ck["v"])
        net.t = int(ck["t"])
        sampler.rng.bit_generator.state = ck["rng"]
        start = int(ck["step"])
        log("resumed at step %d" % start)
    history = []
    acc = torch.zeros(1, dtype=torch.float64, device=device)
    t1 = time.time()
    for s in range(start, steps):
        nc, pc, cc = sampler.next(noisy, pre, clean)
        if fl:
            acc += net.train_step(nc, pc, cc, list(sig[sampler.last]), lr=lr, sync=False)
        else:
            acc += net.train_step(nc, pc, cc, lr=lr, sync=False,
                                  precision=api.DN_BF16 if precision == "bf16" else api.DN_FP32)
        # wall-clock cap: stop at a multiple of 50 steps once the budget is spent
        stop = max_minutes is not None and (s + 1) % 50 == 0 and time.time() - t1 > 60.0 * max_minutes
        if (s + 1) % log_every == 0 or s + 1 == steps or stop:
            k = log_every if (s + 1) % log_every == 0 else (s + 1) % log_every
            loss = float(acc.item()) / k
            acc.zero_()
            history.append((s + 1, loss))
            log("step %d  L1 %.4f  (%.2f ms/step)" % (s + 1, loss, 1e3 * (time.time() - t1) / (s + 1 - start)))
            if checkpoint:
                torch.save({"flat": net.flat.data, "m": net.m, "v": net.v, "t": net.t, "step": s + 1,
                            "rng": sampler.rng.bit_generator.state}, checkpoint)
        if stop:
            log("stopped at step %d (wall-clock cap of %.1f min)" % (s + 1, max_minutes))
            break
    return net, history


@torch.no_grad()
def evaluate(weights, sigmas=(15.0, 25.0, 50.0), n_images=32, H=512, W=512, seed0=5000, prefilter="bm3d",
             cnn_precision=api.DN_FP32, device="cuda"):
    """PSNR of the nonlocal filter alone and of the hybrid on held-out scenes."""
    res = {}
    seeds = list(range(seed0, seed0 + n_images))
    for s in sigmas:
        pf, ph, pn = [], [], []
        for c0 in range(0, n_images, 16):
            cl, ny = synth.make_batch(seeds[c0:c0 + 16], H, W, s)
            x = torch.from_numpy(ny).to(device)
            c = torch.from_numpy(cl).to(device)
            pre = api.denoise_bm3d(x, s) if prefilter == "bm3d" else api.denoise_nlm(x, s)
            hyb = api.denoise_hybrid(x, s, weights, prefilter=api.DN_PREFILTER_BM3D if prefilter == "bm3d"
                                     else api.DN_PREFILTER_NLM, cnn_precision=cnn_precision)
            for t, lst in ((pre, pf), (hyb, ph), (x, pn)):
                sse, _ = api.error_reduce(t, c)
                lst += list((10 * torch.log10(255.0 ** 2 / (sse / (H * W)))).cpu().numpy())
        res[s] = {"noisy": float(np.mean(pn)), prefilter: float(np.mean(pf)), "hybrid": float(np.mean(ph)),
                  "gain_db": float(np.mean(ph) - np.mean(pf))}
    return res


@torch.no_grad()
def evaluate_fl(net, sigmas=(15.0, 25.0, 50.0), n_images=32, H=512, W=512, seed0=5000, prefilter="bm3d",
                device="cuda"):
    """PSNR of the nonlocal filter alone and of prefilter + flexible network on held-out scenes."""
    res = {}
    seeds = list(range(seed0, seed0 + n_images))
    for s in sigmas:
        pf, ph, pn = [], [], []
        for c0 in range(0, n_images, 16):
            cl, ny = synth.make_batch(seeds[c0:c0 + 16], H, W, s)
            x = torch.from_numpy(ny).to(device)
            c = torch.from_numpy(cl).to(device)
            pre = api.denoise_bm3d(x, s) if prefilter == "bm3d" else api.denoise_nlm(x, s)
            hyb = net(x[:, 0].contiguous(), pre[:, 0].contiguous(), [s] * x.shape[0]).unsqueeze(1).contiguous()
            for t, lst in ((pre, pf), (hyb, ph), (x, pn)):
                sse, _ = api.error_reduce(t, c)
                lst += list((10 * torch.log10(255.0 ** 2 / (sse / (H * W)))).cpu().numpy())
        res[s] = {"noisy": float(np.mean(pn)), prefilter: float(np.mean(pf)), "hybrid": float(np.mean(ph)),
                  "gain_db": float(np.mean(ph) - np.mean(pf))}
    return res


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--steps", type=int, default=20000)
    ap.add_argument("--batch", type=int, default=64)
    ap.add_argument("--crop", type=int, default=64)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--images", type=int, default=256)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--prefilter", default="bm3d", choices=["bm3d", "nlm"])
    ap.add_argument("--net", default="resnet", choices=["resnet", "fl"],
                    help="resnet: the 10x32 residual CNN of Sec. II; fl: the flexible network of Sec. III")
    ap.add_argument("--max-minutes", type=float, default=None, help="stop training after this wall-clock time")
    ap.add_argument("--precision", default="fp32", choices=["fp32", "bf16"],
                    help="residual network: FP32 CUDA-core kernels or the BF16 tensor-core forward/backward")
    ap.add_argument("--out", default=DEFAULT_OUT)
    ap.add_argument("--checkpoint", default=None)
    ap.add_argument("--eval-images", type=int, default=32)
    ap.add_argument("--report", default=None)
    args = ap.parse_args()
    net, hist = train(args.steps, args.batch, args.crop, args.lr, args.seed, args.images, args.prefilter,
                      checkpoint=args.checkpoint, net_kind=args.net, max_minutes=args.max_minutes,
                      precision=args.precision)
    os.makedirs(os.path.dirname(os.path.abspath(args.out)), exist_ok=True)
    w = net.flat.detach().cpu().numpy().astype(np.float32)
    np.save(args.out, w)
    if args.net == "fl":
        ev = evaluate_fl(net, n_images=args.eval_images, prefilter=args.prefilter)
    else:
        ev = evaluate(net.flat_weights(), n_images=args.eval_images, prefilter=args.prefilter)
    rep = {"net": args.net, "steps": hist[-1][0] if hist else 0, "batch": args.batch, "crop": args.crop,
           "lr": args.lr, "images": args.images, "prefilter": args.prefilter, "loss_history": hist, "eval": ev}
    print(json.dumps(rep["eval"]))
    if args.report:
        json.dump(rep, open(args.report, "w"), indent=1)


if __name__ == "__main__":
    main()
