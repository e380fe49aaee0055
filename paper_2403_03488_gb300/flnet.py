"""The flexible lightweight network of Sec. III ("Ours-FL") on the library's kernels.

Structure (Sec. III and its Fig. 3 caption): a U-Net with 4 encoders and 4
decoders built from 3x3 depthwise-separable convolutions, a stride-2
depthwise-separable convolution for every downsampling, a 2x2 transposed
convolution (stride 2) for every upsampling and skip connections; like
FFDNet it takes the noise level as an input plane, so one network serves
every sigma.  The paper leaves out the widths and the block internals (its
Fig. 3 is not part of the text); the readings taken here:

  input   z = [pre / 255, noisy / 255, sigma / 255]      (3 planes; pre = the
          nonlocal prefilter's output, as in Eq. 3)
  DS(cin -> cout, s)  depthwise 3x3 (stride s, bias) -> pointwise cin -> cout
          (bias) -> ReLU
  e0 = DS(DS(z; 3 -> c0); c0 -> c0)                       full resolution
  e_k = DS(DS(e_{k-1}; c_{k-1} -> c_k, stride 2); c_k -> c_k), k = 1..4
  d_4 = e_4;  d_{k-1} = DS(up(d_k; c_k -> c_{k-1}) + e_{k-1}; c_{k-1} -> c_{k-1}), k = 4..1
  r = pointwise(d_0; c0 -> 1) (bias, no ReLU);  out = pre + 255 r   (Eq. 2)

with widths c = (48, 64, 96, 128, 192): 17,348 multiply-adds per pixel, 4.55
GMAC for a 512 x 512 image against the paper's 4.52 (Table III).  Image sides
must be multiples of 16 (four halvings).

Parameters live in one flat FP32 buffer, layer by layer in the order above:
DS: dw_w [cin, 3, 3], dw_b [cin], pw_w [cout, cin], pw_b [cout]; up: w [cin,
cout, 2, 2], b [cout]; output: w [1, c0], b [1]; every slice starts at a
multiple of 4 floats.  The forward and backward passes are the library's
FP32 kernels (dn_dw3x3_*, dn_pw_*, dn_deconv2x2_*, dn_relu_bwd), sequenced
by torch.autograd; the L1 loss gradient (Eq. 2) and Adam are library kernels
too.
"""
from __future__ import annotations

import numpy as np
import torch

from . import api

WIDTHS = (48, 64, 96, 128, 192)


def layer_specs(widths=WIDTHS):
    """[(kind, cin, cout, stride)] in network order; kind in {"ds", "up", "out"}."""
    c = tuple(widths)
    L = [("ds", 3, c[0], 1), ("ds", c[0], c[0], 1)]
    for k in range(1, 5):
        L += [("ds", c[k - 1], c[k], 2), ("ds", c[k], c[k], 1)]
    for k in range(4, 0, -1):
        L += [("up", c[k], c[k - 1], 2), ("ds", c[k - 1], c[k - 1], 1)]
    L.append(("out", c[0], 1, 1))
    return L


def param_shapes(widths=WIDTHS):
    """Shapes of the parameter tensors in buffer order."""
    out = []
    for kind, cin, cout, _ in layer_specs(widths):
        if kind == "ds":
            out += [(cin, 3, 3), (cin,), (cout, cin), (cout,)]
        elif kind == "up":
            out += [(cin, cout, 2, 2), (cout,)]
        else:
            out += [(1, cin), (1,)]
    return out


def macs_per_pixel(widths=WIDTHS):
    """Multiply-adds per full-resolution pixel of one forward pass."""
    c = tuple(widths)
    t = 9 * 3 + 3 * c[0] + 9 * c[0] + c[0] * c[0]
    for k in range(1, 5):
        t += (9 * c[k - 1] + c[k - 1] * c[k] + 9 * c[k] + c[k] * c[k]) / 4 ** k
    for k in range(4, 0, -1):
        t += (c[k] * c[k - 1] + 9 * c[k - 1] + c[k - 1] ** 2) / 4 ** (k - 1)
    return t + c[0]


def work_per_pixel(widths=WIDTHS):
    """Algorithmic work of one forward pass per full-resolution pixel, by layer
    kind: multiply-adds of the depthwise, pointwise (output layer included) and
    transposed layers, and the FP32 bytes the depthwise layers must move (input
    plane read once, output plane written once)."""
    w = {"dw_macs": 0.0, "pw_macs": 0.0, "up_macs": 0.0, "dw_bytes": 0.0, "pw_bytes": 0.0, "up_bytes": 0.0}
    level = 0
    for kind, cin, cout, s in layer_specs(widths):
        if kind == "ds":
            lo = level + (1 if s == 2 else 0)
            w["dw_macs"] += 9 * cin / 4 ** lo
            w["pw_macs"] += cin * cout / 4 ** lo
            w["dw_bytes"] += 4 * cin / 4 ** level + 4 * cin / 4 ** lo
            w["pw_bytes"] += 4 * (cin + cout) / 4 ** lo
            level = lo
        elif kind == "up":
            # input plane of the coarser level read, output and skip planes of the finer level
            w["up_bytes"] += 4 * cin / 4 ** level + 2 * 4 * cout / 4 ** (level - 1)
            level -= 1
            w["up_macs"] += cin * cout / 4 ** level
        else:
            w["pw_macs"] += cin * cout / 4 ** level
            w["pw_bytes"] += 4 * (cin + cout) / 4 ** level
    return w


def init_params(widths=WIDTHS, seed=0):
    """He-normal weights (fan-in 9 for depthwise, cin for pointwise, cin for the
    transposed 2x2, whose outputs each see one tap), zero biases."""
    rng = np.random.default_rng(seed)
    out = []
    for shp in param_shapes(widths):
        if len(shp) == 1:
            out.append(np.zeros(shp, np.float32))
            continue
        fan = 9 if len(shp) == 3 else shp[0] if len(shp) == 4 else shp[1]
        out.append((rng.standard_normal(shp) * np.sqrt(2.0 / fan)).astype(np.float32))
    return out


class DwFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x, w, b, stride):
        x = x.contiguous()
        ctx.stride = stride
        ctx.save_for_backward(x, w)
        return api.dw3x3_fwd(x, w, b, stride=stride)

    @staticmethod
    def backward(ctx, g):
        x, w = ctx.saved_tensors
        dx, dw, db = api.dw3x3_bwd(x, g.contiguous(), w, stride=ctx.stride, need_dx=ctx.needs_input_grad[0])
        return dx, dw, db, None


class PwFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x, w, b, relu, precision=api.DN_FP32):
        x = x.contiguous()
        y = api.pw_fwd(x, w, b, relu=relu, precision=precision)
        ctx.relu = bool(relu)
        ctx.precision = precision
        ctx.save_for_backward(x, w, y)
        return y

    @staticmethod
    def backward(ctx, g):
        x, w, y = ctx.saved_tensors
        g = g.contiguous()
        if ctx.relu:
            g = api.relu_bwd(g, y)
        dx = api.pw_fwd(g, w, None, transposed=True, precision=ctx.precision) if ctx.needs_input_grad[0] else None
        dw, db = api.pw_bwd_weight(x, g)
        return dx, dw, db, None, None


class UpFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x, w, b, skip, precision=api.DN_FP32):
        x = x.contiguous()
        ctx.save_for_backward(x, w)
        return api.deconv2x2_fwd(x, w, b, skip.contiguous(), precision=precision)

    @staticmethod
    def backward(ctx, g):
        x, w = ctx.saved_tensors
        g = g.contiguous()
        dx, dw, db = api.deconv2x2_bwd(x, g, w, need_dx=ctx.needs_input_grad[0])
        return dx, dw, db, g, None


class FLNet(torch.nn.Module):
    """precision DN_FP32: every layer on the FP32 CUDA-core kernels; DN_BF16:
    the pointwise layers (forward and data gradient) and the transposed 2x2
    convolutions on the tensor cores (BF16 operands, FP32 accumulation, FP32
    activations), the depthwise layers and the weight gradients in FP32."""

    def __init__(self, widths=WIDTHS, seed=0, flat: torch.Tensor = None, precision=api.DN_FP32):
        super().__init__()
        self.precision = precision
        self.widths = tuple(widths)
        self.shapes = param_shapes(self.widths)
        self.offsets = []
        off = 0
        for shp in self.shapes:
            self.offsets.append(off)
            off += (int(np.prod(shp)) + 3) // 4 * 4
        if flat is None:
            flat = torch.zeros(off)
            for o, a in zip(self.offsets, init_params(self.widths, seed)):
                flat[o:o + a.size] = torch.from_numpy(a.ravel())
        assert flat.numel() == off
        self.flat = torch.nn.Parameter(flat.float().contiguous())
        self.register_buffer("m", torch.zeros(off))
        self.register_buffer("v", torch.zeros(off))
        self.t = 0

    def params(self):
        return [self.flat[o:o + int(np.prod(s))].view(s) for o, s in zip(self.offsets, self.shapes)]

    def numpy_params(self):
        return [p.detach().cpu().numpy() for p in self.params()]

    def residual(self, noisy, pre, sigma):
        """r [N, H, W] (the network output before out = pre + 255 r)."""
        N, H, W = noisy.shape
        if H % 16 or W % 16:
            raise ValueError("image sides must be multiples of 16")
        P = self.params()
        i = 0

        def ds(h, s):
            nonlocal i
            dw_w, dw_b, pw_w, pw_b = P[i:i + 4]
            i += 4
            return PwFn.apply(DwFn.apply(h, dw_w, dw_b, s), pw_w, pw_b, True, self.precision)

        h = ds(ds(api.fl_pack_input(pre.contiguous(), noisy.contiguous(), sigma), 1), 1)
        e = [h]
        for _ in range(4):  # encoders 1..4: stride-2 block, then a block
            h = ds(ds(h, 2), 1)
            e.append(h)
        for k in range(4, 0, -1):  # decoders: up to level k-1, add its encoder output, a block
            h = UpFn.apply(h, P[i], P[i + 1], e[k - 1], self.precision)
            i += 2
            h = ds(h, 1)
        r = PwFn.apply(h, P[i], P[i + 1], False, self.precision)
        return r[:, 0]

    def forward(self, noisy, pre, sigma, out=None):
        """out = pre + 255 r for planes [N, H, W] (written into `out` when given)."""
        r = self.residual(noisy, pre, sigma)
        return api.cnn_residual_out(pre.contiguous(), r.contiguous(), out=out)

    def train_step(self, noisy, pre, clean, sigma, lr=1e-3, sync=True):
        """One L1 (Eq. 2) + Adam step; every kernel is the library's."""
        self.flat.grad = None
        r = self.residual(noisy, pre, sigma).contiguous()
        loss = torch.zeros(1, dtype=torch.float64, device=noisy.device)
        dr = api.l1_residual_grad(r, pre.contiguous(), clean.contiguous(), loss)
        r.backward(dr)
        self.t += 1
        api.adam_step(self.flat.data, self.flat.grad.contiguous(), self.m, self.v, self.t, lr=lr)
        if sync:
            return float(loss.item()) / r.numel()
        return loss / r.numel()
