"""CPU reference of the proposal network (numpy, float64).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py): the CUDA network kernels
are checked against it; nothing in the product imports it.

The network is not in the paper.  It is the learned proposal that predicts a
per-pixel displacement centre, so that EDP can then run on a small label box
around that centre.  Six 3x3 convolutions with zero padding.  Channels go
5 -> 32 -> 32 -> 32 -> 32 -> 32 -> 2, with a ReLU after every layer but the
last.  The loss is smooth-L1 (beta = 1) between the output and the target
centre, averaged over pixels and channels.

Precision contract, shared with the GPU kernels:
  - Weights and activations are stored as bfloat16.  Rounding is
    round-to-nearest-even of the float32 value.
  - Every product is accumulated in float64 here (float32 on the GPU).
  - The bias and the last layer's output stay in float32.
  - In the backward pass, the gradient entering each layer's input is rounded
    to bfloat16 before it is used, as the GPU stores it.
"""
from __future__ import annotations

import numpy as np

CHANNELS = [5, 32, 32, 32, 32, 32, 2]


def bf16(a: np.ndarray) -> np.ndarray:
    """Round to the nearest bfloat16 (ties to even), returned as float64."""
    f = np.ascontiguousarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16) << 16
    nan = np.isnan(f)
    out = (r & 0xFFFFFFFF).astype(np.uint32).view(np.float32).astype(np.float64)
    out[nan] = np.nan
    return out


def conv3x3(x: np.ndarray, w: np.ndarray, b: np.ndarray | None) -> np.ndarray:
    """x [N][Ci][H][W], w [Co][Ci][3][3] -> [N][Co][H][W]; zero padding 1.

    Cross-correlation written as a sum of nine shifted matmuls."""
    N, Ci, H, W = x.shape
    Co = w.shape[0]
    xp = np.zeros((N, Ci, H + 2, W + 2))
    xp[:, :, 1:H + 1, 1:W + 1] = x
    out = np.zeros((N, Co, H, W))
    for dy in range(3):
        for dx in range(3):
            patch = xp[:, :, dy:dy + H, dx:dx + W]               # [N][Ci][H][W]
            out += np.einsum("oc,nchw->nohw", w[:, :, dy, dx], patch)
    if b is not None:
        out += b[None, :, None, None]
    return out


def conv3x3_dgrad(g: np.ndarray, w: np.ndarray) -> np.ndarray:
    """Gradient w.r.t. the input of conv3x3: g [N][Co][H][W] -> [N][Ci][H][W]."""
    N, Co, H, W = g.shape
    Ci = w.shape[1]
    gp = np.zeros((N, Co, H + 2, W + 2))
    gp[:, :, 1:H + 1, 1:W + 1] = g
    out = np.zeros((N, Ci, H, W))
    for dy in range(3):
        for dx in range(3):
            # out[y][x] += sum_o w[o][c][dy][dx] * g[o][y - dy + 1][x - dx + 1]
            patch = gp[:, :, 2 - dy:2 - dy + H, 2 - dx:2 - dx + W]
            out += np.einsum("oc,nohw->nchw", w[:, :, dy, dx], patch)
    return out


def conv3x3_wgrad(g: np.ndarray, x: np.ndarray) -> np.ndarray:
    """Gradient w.r.t. the weights: -> [Co][Ci][3][3]."""
    N, Ci, H, W = x.shape
    xp = np.zeros((N, Ci, H + 2, W + 2))
    xp[:, :, 1:H + 1, 1:W + 1] = x
    Co = g.shape[1]
    out = np.zeros((Co, Ci, 3, 3))
    for dy in range(3):
        for dx in range(3):
            out[:, :, dy, dx] = np.einsum("nohw,nchw->oc", g, xp[:, :, dy:dy + H, dx:dx + W])
    return out


def init_params(seed: int = 0) -> list[tuple[np.ndarray, np.ndarray]]:
    """He-uniform weights (then bf16-rounded) and zero biases."""
    rng = np.random.default_rng(seed)
    ps = []
    for ci, co in zip(CHANNELS[:-1], CHANNELS[1:]):
        lim = np.sqrt(6.0 / (ci * 9))
        w = bf16(rng.uniform(-lim, lim, size=(co, ci, 3, 3)))
        ps.append((w, np.zeros(co)))
    return ps


def _exact(a):
    return np.asarray(a, dtype=np.float64)


def forward(x: np.ndarray, params, keep: bool = False, rounding=bf16):
    """x [N][5][H][W] (bf16-representable).  Returns the output [N][2][H][W]
    and, if keep, the stored activations (inputs of every layer).
    rounding=None computes in plain float64 (for derivative checks)."""
    rnd = rounding or _exact
    f32 = (lambda a: a.astype(np.float32).astype(np.float64)) if rounding else _exact
    acts = [rnd(x)]
    h = acts[0]
    nl = len(params)
    for i, (w, b) in enumerate(params):
        z = conv3x3(h, rnd(w), f32(np.asarray(b, dtype=np.float64)))
        if i < nl - 1:
            h = rnd(np.maximum(z, 0.0))
            acts.append(h)
        else:
            h = f32(z)
    return (h, acts) if keep else h


def smooth_l1(out: np.ndarray, target: np.ndarray) -> tuple[float, np.ndarray]:
    """Mean smooth-L1 (beta = 1) and its gradient w.r.t. out."""
    d = out - target
    a = np.abs(d)
    loss = np.where(a < 1.0, 0.5 * d * d, a - 0.5)
    grad = np.where(a < 1.0, d, np.sign(d)) / d.size
    return float(loss.mean()), grad


def backward(x: np.ndarray, params, target: np.ndarray, rounding=bf16):
    """Loss and gradients [(dW, db)] with the precision contract above."""
    rnd = rounding or _exact
    out, acts = forward(x, params, keep=True, rounding=rounding)
    loss, g = smooth_l1(out, target)
    grads = [None] * len(params)
    for i in range(len(params) - 1, -1, -1):
        w, _ = params[i]
        gz = rnd(g)  # gradient at this layer's output, stored as bf16
        grads[i] = (conv3x3_wgrad(gz, acts[i]), gz.sum(axis=(0, 2, 3)))
        if i > 0:
            gx = conv3x3_dgrad(gz, rnd(w))
            g = gx * (acts[i] > 0)  # ReLU of the previous layer
    return loss, grads


def features(I0: np.ndarray, I1: np.ndarray, wta_flow: np.ndarray, wta_cost: np.ndarray,
             flow_scale: float, cost_scale: float) -> np.ndarray:
    """Network input [5][H][W]: both frames (/255), the winner-take-all
    displacement (/flow_scale, 2 channels) and its cost (/cost_scale)."""
    return np.stack([I0 / 255.0, I1 / 255.0, wta_flow[..., 0] / flow_scale, wta_flow[..., 1] / flow_scale,
                     wta_cost / cost_scale]).astype(np.float64)
