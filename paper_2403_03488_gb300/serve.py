"""Continuous-batching denoising server on one GPU.

Requests (an image of either colour mode and any size, and its sigma) arrive
over time.  The scheduler admits work as soon as a stream slot is free and
the device-memory footprint of everything in flight plus the new work fits
the HBM budget.  Queued requests of the same shape (C, H, W) are coalesced
into one batched launch (up to max_batch images, each with its own sigma):
the library treats every image of a batch independently and
deterministically, so a request's result is bit for bit the same alone, in
a batch, and beside other requests.  Each launch runs on its own CUDA stream
(host-to-device copy from pinned memory, denoise_hybrid, device-to-host
copy), so work of requests that arrive while others are running overlaps on
the device.  Completion is detected with CUDA events; the buffers are then
released and the next work admitted.  Latency = result ready on the host
minus arrival.  Requests larger than the whole budget are rejected.

    python -m paper_2403_03488_gb300.serve --rate 200 --requests 2000
"""
from __future__ import annotations

import argparse
import collections
import json
import os
import threading
import time
from dataclasses import dataclass, field

import numpy as np
import torch

from . import api, synth

HERE = os.path.dirname(os.path.abspath(__file__))


@dataclass
class Request:
    rid: int
    image: np.ndarray          # [C, H, W] float32, host
    sigma: float
    arrival: float = 0.0       # seconds since the trace start
    done: float = 0.0
    result: np.ndarray = None
    rejected: bool = False
    footprint: int = 0


@dataclass
class ServerStats:
    latencies_ms: list = field(default_factory=list)
    pixels: int = 0
    channel_pixels: int = 0
    max_inflight_bytes: int = 0
    max_inflight: int = 0
    rejected: int = 0
    makespan_s: float = 0.0
    launches: int = 0
    max_batch: int = 0

    def summary(self):
        lat = np.array(self.latencies_ms) if self.latencies_ms else np.zeros(1)
        return {"requests": len(self.latencies_ms), "rejected": self.rejected,
                "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
                "mean_ms": float(lat.mean()), "served_mpix_s": self.pixels / 1e6 / max(self.makespan_s, 1e-9),
                "served_channel_mpix_s": self.channel_pixels / 1e6 / max(self.makespan_s, 1e-9),
                "makespan_s": self.makespan_s, "max_inflight_bytes": self.max_inflight_bytes,
                "max_inflight": self.max_inflight, "launches": self.launches, "max_batch": self.max_batch}


def make_trace(n, rate, seed=0, side=(128, 2048), sigmas=(15.0, 25.0, 50.0), p_rgb=0.5):
    """Open-loop Poisson trace: request k arrives at the k-th event of a
    Poisson process of `rate` per second; sides U{side}, grey or RGB with
    probability p_rgb, sigma uniform over `sigmas`.  Images are built lazily."""
    rng = np.random.Generator(np.random.PCG64(seed))
    gaps = rng.exponential(1.0 / rate, n)
    t = np.cumsum(gaps) - gaps[0]
    Hs = rng.integers(side[0], side[1] + 1, n)
    Ws = rng.integers(side[0], side[1] + 1, n)
    Cs = np.where(rng.random(n) < p_rgb, 3, 1)
    sg = rng.choice(np.asarray(sigmas, float), n)
    return [dict(rid=i, arrival=float(t[i]), H=int(Hs[i]), W=int(Ws[i]), C=int(Cs[i]), sigma=float(sg[i]),
                 seed=1_000_000 + seed * 100_000 + i) for i in range(n)]


def build_request(spec) -> Request:
    clean = synth.make_image(spec["seed"], spec["H"], spec["W"], spec["C"])
    noisy = synth.add_awgn(clean, spec["sigma"], spec["seed"])
    return Request(spec["rid"], noisy, spec["sigma"], spec["arrival"])


class ScenePool:
    """Requests cut from a few pre-built 2048 x 2048 scenes and unit-noise
    fields (seeded offsets), so that long traces are built in milliseconds per
    request instead of generating every scene from scratch."""

    def __init__(self, seed=0, side=2048, n_scenes=3):
        self.side = side
        self.grey = [synth.make_image(50_000 + seed * 10 + i, side, side, 1) for i in range(n_scenes)]
        self.rgb = [synth.make_image(60_000 + seed * 10 + i, side, side, 3) for i in range(n_scenes)]
        rng = np.random.Generator(np.random.PCG64(70_000 + seed))
        self.noise = rng.standard_normal((3, side, side)).astype(np.float32)

    def build(self, spec) -> Request:
        rng = np.random.Generator(np.random.PCG64(spec["seed"]))
        H, W, C = spec["H"], spec["W"], spec["C"]
        scenes = self.rgb if C == 3 else self.grey
        sc = scenes[int(rng.integers(0, len(scenes)))]
        y0, x0 = int(rng.integers(0, self.side - H + 1)), int(rng.integers(0, self.side - W + 1))
        ny, nx = int(rng.integers(0, self.side - H + 1)), int(rng.integers(0, self.side - W + 1))
        clean = sc[:, y0:y0 + H, x0:x0 + W]
        noisy = clean + np.float32(spec["sigma"]) * self.noise[:C, ny:ny + H, nx:nx + W]
        return Request(spec["rid"], np.ascontiguousarray(noisy, dtype=np.float32), spec["sigma"], spec["arrival"])


class Server:
    """Admission-controlled, stream-overlapped execution of denoise requests."""

    def __init__(self, weights: torch.Tensor, budget_bytes=60 << 30, slots=8, bm3d_precision=api.DN_FP32,
                 cnn_precision=api.DN_BF16, prefilter=api.DN_PREFILTER_BM3D, device="cuda", max_batch=8):
        self.dev = torch.device(device)
        self.max_batch = max(1, int(max_batch))
        self.weights = weights
        self.budget = int(budget_bytes)
        self.streams = [torch.cuda.Stream(device=self.dev) for _ in range(slots)]
        self.free_streams = list(range(slots))
        self.prefilter = prefilter
        self.pparams = (api.default_bm3d_params(precision=bm3d_precision) if prefilter == api.DN_PREFILTER_BM3D
                        else api.default_nlm_params())
        self.cnn_precision = cnn_precision
        self.cnn = api.make_cnn(weights, 10, 32, cnn_precision)
        self.inflight = []        # (request, stream index, event, buffers)
        self.inflight_bytes = 0
        self.stats = ServerStats()

    def footprint(self, C, H, W, B=1) -> int:
        img = C * H * W * 4
        ws = api.hybrid_workspace_bytes(B, C, H, W, self.prefilter, self.pparams, self.cnn)
        return 2 * B * img + ws + (1 << 20)

    def _take_batch(self, queue):
        """The head of the queue and up to max_batch - 1 later requests of the
        same shape, if their launch fits the budget (else the largest prefix
        that does); None when not even the head fits right now."""
        head = queue[0]
        same = [head] + [r for r in list(queue)[1:] if r.image.shape == head.image.shape][:self.max_batch - 1]
        C, H, W = head.image.shape
        while same:
            fp = self.footprint(C, H, W, len(same)) if len(same) > 1 else head.footprint
            if self.inflight_bytes + fp <= self.budget:
                for r in same:
                    queue.remove(r)
                return same, fp
            same = same[:-1]
        return None, 0

    def _launch(self, batch, fp, t0: float):
        si = self.free_streams.pop()
        s = self.streams[si]
        host_in = torch.from_numpy(np.stack([r.image for r in batch])).pin_memory()
        host_out = torch.empty_like(host_in).pin_memory()
        with torch.cuda.stream(s):
            x = host_in.to(self.dev, non_blocking=True)
            y = api.denoise_hybrid(x, [r.sigma for r in batch], self.weights, prefilter=self.prefilter,
                                   prefilter_params=self.pparams, cnn_precision=self.cnn_precision, stream=s)
            host_out.copy_(y, non_blocking=True)
            ev = torch.cuda.Event()
            ev.record(s)
        self.inflight.append((batch, si, ev, (host_in, host_out, x, y), fp))
        self.inflight_bytes += fp
        self.stats.launches += 1
        self.stats.max_batch = max(self.stats.max_batch, len(batch))
        self.stats.max_inflight_bytes = max(self.stats.max_inflight_bytes, self.inflight_bytes)
        self.stats.max_inflight = max(self.stats.max_inflight, sum(len(b[0]) for b in self.inflight))

    def _poll(self, t0: float, keep_results: bool):
        still = []
        for item in self.inflight:
            batch, si, ev, bufs, fp = item
            if ev.query():
                done = time.perf_counter() - t0
                for k, req in enumerate(batch):
                    req.done = done
                    if keep_results:
                        req.result = bufs[1][k].numpy().copy()
                    self.stats.latencies_ms.append(1e3 * (req.done - req.arrival))
                    C, H, W = req.image.shape
                    self.stats.pixels += H * W
                    self.stats.channel_pixels += C * H * W
                self.inflight_bytes -= fp
                self.free_streams.append(si)
            else:
                still.append(item)
        self.inflight = still

    def run(self, requests, realtime=True, keep_results=False):
        """Serve `requests` (sorted by arrival).  realtime=True replays the
        arrival times; False submits everything at t = 0.  Returns stats."""
        queue = collections.deque()
        pending = collections.deque(sorted(requests, key=lambda r: r.arrival))
        for r in pending:
            C, H, W = r.image.shape
            r.footprint = self.footprint(C, H, W)
        t0 = time.perf_counter()
        while pending or queue or self.inflight:
            now = time.perf_counter() - t0
            while pending and (not realtime or pending[0].arrival <= now):
                r = pending.popleft()
                if not realtime:
                    r.arrival = 0.0
                if r.footprint > self.budget:
                    r.rejected = True
                    self.stats.rejected += 1
                    continue
                queue.append(r)
            self._poll(t0, keep_results)
            while queue and self.free_streams:
                batch, fp = self._take_batch(queue)
                if batch is None:
                    break
                self._launch(batch, fp, t0)
            if not (queue and self.free_streams) and self.inflight:
                time.sleep(0.0002)
            elif not self.inflight and not queue and pending and realtime:
                time.sleep(max(0.0, min(0.002, pending[0].arrival - (time.perf_counter() - t0))))
        torch.cuda.synchronize(self.dev)
        self.stats.makespan_s = time.perf_counter() - t0
        return self.stats


def load_weights(device="cuda"):
    p = os.path.join(HERE, "weights", "resnet10x32_bm3d.npy")
    return torch.from_numpy(np.load(p).astype(np.float32)).to(device).contiguous()


def replay(rate=200.0, n=2000, seed=0, budget_gb=60.0, slots=8, bm3d_precision=api.DN_FP32,
           cnn_precision=api.DN_BF16, side=(128, 2048), warm=True, max_batch=8):
    """Builds the trace (host images first, outside the timed replay) and serves it."""
    specs = make_trace(n, rate, seed, side=side)
    pool = ScenePool(seed, side=max(side[1], 256))
    reqs = [pool.build(s) for s in specs]
    srv = Server(load_weights(), budget_bytes=int(budget_gb * (1 << 30)), slots=slots,
                 bm3d_precision=bm3d_precision, cnn_precision=cnn_precision, max_batch=max_batch)
    if warm:
        Server(srv.weights, srv.budget, 2, bm3d_precision, cnn_precision).run(
            [build_request(dict(rid=-1, arrival=0.0, H=160, W=144, C=c, sigma=25.0, seed=7 + c)) for c in (1, 3)],
            realtime=False)
    stats = srv.run(reqs, realtime=True)
    out = stats.summary()
    out["offered_mpix_s"] = float(sum(s["H"] * s["W"] for s in specs) / 1e6 / (specs[-1]["arrival"] + 1e-9))
    out["rate"] = rate
    out["trace"] = "%d Poisson requests at %.0f/s, sides U[%d,%d], grey/RGB p=0.5, sigma in {15,25,50}" % (
        n, rate, side[0], side[1])
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--rate", type=float, default=200.0)
    ap.add_argument("--requests", type=int, default=2000)
    ap.add_argument("--budget-gb", type=float, default=60.0)
    ap.add_argument("--slots", type=int, default=8)
    ap.add_argument("--max-batch", type=int, default=8)
    ap.add_argument("--plain", action="store_true", help="FP32 plain path (BM3D FP32 + CNN FP32)")
    args = ap.parse_args()
    res = replay(args.rate, args.requests, budget_gb=args.budget_gb, slots=args.slots,
                 cnn_precision=api.DN_FP32 if args.plain else api.DN_BF16, max_batch=args.max_batch)
    print(json.dumps(res))


if __name__ == "__main__":
    main()
