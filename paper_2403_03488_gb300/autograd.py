"""The residual CNN of Sec. II (Fig. 1, Eq. 2-3) on the library's kernels.

Conv3x3Fn is a torch.autograd.Function whose forward and backward are the
hand-written conv kernels (dn_conv3x3_fwd / _bwd_data / _bwd_weight, ReLU
backward by dn_relu_bwd).  ResidualNet keeps its FP32 master parameters in
one flat device buffer laid out exactly as the C ABI's dn_cnn weights
(per layer W [Cout][3][3][Cin] then b [Cout]), so the same buffer feeds
denoise_hybrid, and trains with an explicit step: forward through the
kernels, the L1 loss gradient of Eq. 2, backward through the kernels, Adam.
"""
from __future__ import annotations

import numpy as np
import torch

from . import api
from .synth import he_normal_weights


class Conv3x3Fn(torch.autograd.Function):
    """y = conv3x3(x, w) + b, optionally followed by ReLU (NCHW, w [Cout,3,3,Cin])."""

    @staticmethod
    def forward(ctx, x, w, b, relu=False):
        x = x.contiguous()
        w = w.contiguous()
        b = b.contiguous()
        y = api.conv3x3_fwd(x, w, b, relu=relu)
        ctx.relu = bool(relu)
        ctx.save_for_backward(x, w, y)
        return y

    @staticmethod
    def backward(ctx, gy):
        x, w, y = ctx.saved_tensors
        g = gy.contiguous()
        if ctx.relu:
            g = api.relu_bwd(g, y)
        gx = api.conv3x3_bwd_data(g, w) if ctx.needs_input_grad[0] else None
        gw, gb = api.conv3x3_bwd_weight(x, g)
        return gx, gw, gb, None


class ResidualOutFn(torch.autograd.Function):
    """out = pre + 255 r (Eq. 2) by the library's dn_cnn_residual_out; the
    gradient reaching r, 255 g, is the same kernel applied to (0, g)."""

    @staticmethod
    def forward(ctx, pre, r):
        return api.cnn_residual_out(pre, r)

    @staticmethod
    def backward(ctx, g):
        g = g.contiguous()
        gr = api.cnn_residual_out(torch.zeros_like(g), g) if ctx.needs_input_grad[1] else None
        return g, gr


class ResidualNet(torch.nn.Module):
    """K 3x3 conv layers, `width` channels, 2 inputs (pre/255, noisy/255), 1 output."""

    def __init__(self, layers: int = 10, width: int = 32, seed: int = 0, flat: torch.Tensor = None):
        super().__init__()
        self.layers, self.width = layers, width
        n = api.cnn_param_count(layers, width)
        if flat is None:
            flat = torch.from_numpy(np.concatenate(
                [np.concatenate([w.ravel(), b.ravel()]) for w, b in he_normal_weights(seed, layers, width)]))
        assert flat.numel() == n
        self.flat = torch.nn.Parameter(flat.float().contiguous())
        self.register_buffer("m", torch.zeros(n))
        self.register_buffer("v", torch.zeros(n))
        self.register_buffer("grad_flat", torch.zeros(n))
        self.t = 0
        self._before = None
        self.shapes = []
        off, kin = 0, 2
        for l in range(layers):
            kout = 1 if l == layers - 1 else width
            nw = kout * 9 * kin
            self.shapes.append((off, (kout, 3, 3, kin), off + nw, kout))
            off += nw + kout
            kin = kout

    def params(self, buf=None):
        buf = self.flat if buf is None else buf
        return [(buf[o:o + int(np.prod(s))].view(s), buf[ob:ob + k]) for o, s, ob, k in self.shapes]

    def flat_weights(self) -> torch.Tensor:
        return self.flat.detach()

    def numpy_params(self):
        return [(w.detach().cpu().numpy(), b.detach().cpu().numpy()) for w, b in self.params()]

    def numpy_params_before_step(self):
        return self._before

    def last_grads(self):
        return self.params(self.grad_flat)

    def _grad_ws(self, like):
        """Workspace of dn_cnn_grad for this batch shape, kept between steps."""
        import ctypes
        from . import _lib as L
        N, H, W = like.shape
        cnn = api.make_cnn(self.flat.data, self.layers, self.width, api.DN_BF16, 1)
        nbytes = int(L.lib().dn_cnn_grad_workspace_bytes(N, H, W, ctypes.byref(cnn)))
        ws = getattr(self, "_gws", None)
        if ws is None or ws.numel() < nbytes or ws.device != like.device:
            self._gws = torch.empty(nbytes, dtype=torch.uint8, device=like.device)
        return self._gws

    def forward(self, noisy: torch.Tensor, pre: torch.Tensor) -> torch.Tensor:
        """Autograd path: noisy, pre [N, H, W] -> pre + 255 F(z) (Eq. 2-3)."""
        z = api.cnn_pack_input(pre.contiguous(), noisy.contiguous())
        h = z
        for l, (w, b) in enumerate(self.params()):
            h = Conv3x3Fn.apply(h, w, b, l < self.layers - 1)
        return ResidualOutFn.apply(pre.contiguous(), h[:, 0].contiguous())

    @torch.no_grad()
    def train_step(self, noisy, pre, clean, lr=1e-3, sync=True, precision=api.DN_FP32):
        """One explicit L1 + Adam step entirely on the library's kernels:
        precision DN_FP32 runs the FP32 CUDA-core layers one by one,
        DN_BF16 (grey, width 32) the tensor-core forward and backward of
        dn_cnn_grad with the FP32 master weights.  Returns the mean L1 loss
        (a host float when sync, else a device tensor)."""
        self._before = self.numpy_params() if sync else None
        noisy, pre, clean = noisy.contiguous(), pre.contiguous(), clean.contiguous()
        if precision == api.DN_BF16:
            _, loss = api.cnn_grad(noisy, pre, clean, self.flat.data, self.layers, self.width, grad=self.grad_flat,
                                   workspace=self._grad_ws(noisy))
            self.t += 1
            api.adam_step(self.flat.data, self.grad_flat, self.m, self.v, self.t, lr=lr)
            count = noisy.numel()
            return float(loss.item()) / count if sync else loss / count
        z = api.cnn_pack_input(pre, noisy)
        acts = [z]
        prm = self.params()
        for l, (w, b) in enumerate(prm):
            acts.append(api.conv3x3_fwd(acts[-1], w, b, relu=l < self.layers - 1))
        r = acts[-1]
        loss = torch.zeros(1, dtype=torch.float64, device=noisy.device)
        g = api.l1_residual_grad(r[:, 0].contiguous(), pre, clean, loss).unsqueeze(1)
        gparams = self.params(self.grad_flat)
        for l in range(self.layers - 1, -1, -1):
            api.conv3x3_bwd_weight(acts[l], g, dw=gparams[l][0], db=gparams[l][1])
            if l > 0:
                g = api.conv3x3_bwd_data(g, prm[l][0], mask=acts[l])
        self.t += 1
        api.adam_step(self.flat.data, self.grad_flat, self.m, self.v, self.t, lr=lr)
        if sync:
            return float(loss.item()) / r[:, 0].numel()
        return loss / r[:, 0].numel()
