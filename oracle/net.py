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


def backward(x: np.ndarray, params, target: np.ndarray, rounding=bf16, acts=None, out=None):
    """Loss and gradients [(dW, db)] with the precision contract above.

    acts / out: the stored layer inputs and the output of a forward pass to
    differentiate (default: this reference's own forward pass of x)."""
    rnd = rounding or _exact
    if acts is None:
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


def gradient_magnitudes(x: np.ndarray, params, target: np.ndarray, rounding=bf16, acts=None, out=None):
    """Per parameter, the sum of the absolute values of the terms whose sum
    is its gradient: sum |dL/dz| |input| for a weight, sum |dL/dz| for a
    bias (same layout as the gradients of backward; acts / out as there).
    Where bf16 rounding of an intermediate gradient can go either way, a
    gradient moves by about one bf16 step of some of its terms, so these sums
    scale the absolute error a gradient can carry from that rounding."""
    rnd = rounding or _exact
    if acts is None:
        out, acts = forward(x, params, keep=True, rounding=rounding)
    _, g = smooth_l1(out, target)
    mags = [None] * len(params)
    for i in range(len(params) - 1, -1, -1):
        w, _ = params[i]
        gz = rnd(g)
        mags[i] = (conv3x3_wgrad(np.abs(gz), np.abs(acts[i])), np.abs(gz).sum(axis=(0, 2, 3)))
        if i > 0:
            g = conv3x3_dgrad(gz, rnd(w)) * (acts[i] > 0)
    return mags


def features(I0: np.ndarray, I1: np.ndarray, wta_flow: np.ndarray, wta_cost: np.ndarray,
             flow_scale: float, cost_scale: float) -> np.ndarray:
    """Network input [5][H][W]: both frames (/255), the winner-take-all
    displacement (/flow_scale, 2 channels) and its cost (/cost_scale)."""
    return np.stack([I0 / 255.0, I1 / 255.0, wta_flow[..., 0] / flow_scale, wta_flow[..., 1] / flow_scale,
                     wta_cost / cost_scale]).astype(np.float64)


# ---------------------------------------------------------------------------
# Coarse-level proposal inputs (not in the paper either): the image pyramid
# step, the coarse-to-fine label map, the network input built from a
# labeling, and the residual centre / target conventions.
# ---------------------------------------------------------------------------

def pyr_down2(I: np.ndarray) -> np.ndarray:
    """2x2 box average, rounded half up; odd sizes repeat the last row/column.
    Output shape ((H+1)//2, (W+1)//2), uint8."""
    H, W = I.shape
    Hc, Wc = (H + 1) // 2, (W + 1) // 2
    out = np.zeros((Hc, Wc), dtype=np.uint8)
    for yc in range(Hc):
        for xc in range(Wc):
            ys = (min(2 * yc, H - 1), min(2 * yc + 1, H - 1))
            xs = (min(2 * xc, W - 1), min(2 * xc + 1, W - 1))
            total = sum(int(I[y, x]) for y in ys for x in xs)
            out[yc, xc] = (total + 2) // 4
    return out


def halved_space(vmin: tuple[int, int], Q: tuple[int, int]) -> tuple[tuple[int, int], tuple[int, int]]:
    """Offsets o in [vmin, vmin + Q - 1] per axis -> the coarse axis holding
    the integers in [ceil(vmin / 2), floor((vmin + Q - 1) / 2)]: (vmin_c, Q_c)."""
    vc, qc = [], []
    for v, q in zip(vmin, Q):
        lo = -((-v) // 2)          # ceil(v / 2)
        hi = (v + q - 1) // 2      # floor
        vc.append(lo)
        qc.append(max(1, hi - lo + 1))
    return tuple(vc), tuple(qc)


def labels_up2(lc: np.ndarray, vmin_c, Qc, vmin, Q, H: int, W: int) -> np.ndarray:
    """Coarse labels (linear index, axis 0 fastest) -> full resolution: pixel
    (x, y) takes coarse pixel (x//2, y//2), offsets doubled, clamped."""
    Hc, Wc = lc.shape
    out = np.zeros((H, W), dtype=np.int64)
    for y in range(H):
        for x in range(W):
            q = int(lc[min(y // 2, Hc - 1), min(x // 2, Wc - 1)])
            o = (2 * (vmin_c[0] + q % Qc[0]), 2 * (vmin_c[1] + q // Qc[0]))
            q0 = min(max(o[0] - vmin[0], 0), Q[0] - 1)
            q1 = min(max(o[1] - vmin[1], 0), Q[1] - 1)
            out[y, x] = q0 + Q[0] * q1
    return out


def features_from_labels(I0, I1, labels, vmin, Q, l2: int, cmax: int, scale: float) -> np.ndarray:
    """Network input [5][H][W] from a labeling: both frames / 255, the label
    coordinates minus (Q_r - 1)/2, / scale, and the label's data cost
    min(|I1(x + o) - I0(x)|^l2, cmax) / cmax (out of the image: cmax)."""
    H, W = I0.shape
    f = np.zeros((5, H, W))
    for y in range(H):
        for x in range(W):
            q = int(labels[y, x])
            q0, q1 = q % Q[0], q // Q[0]
            xs, ys = x + vmin[0] + q0, y + vmin[1] + q1
            c = cmax
            if 0 <= xs < W and 0 <= ys < H:
                d = abs(int(I1[ys, xs]) - int(I0[y, x]))
                c = min(d if l2 == 1 else d * d, cmax)
            f[:, y, x] = (I0[y, x] / 255.0, I1[y, x] / 255.0, (q0 - 0.5 * (Q[0] - 1)) / scale,
                          (q1 - 0.5 * (Q[1] - 1)) / scale, c / cmax)
    return f


def targets(labels: np.ndarray, Q, base: np.ndarray | None = None) -> np.ndarray:
    """[..][2] label coordinates minus the base labeling's (or minus the
    space's middle without one)."""
    q0, q1 = labels % Q[0], labels // Q[0]
    if base is None:
        b0, b1 = 0.5 * (Q[0] - 1), 0.5 * (Q[1] - 1)
    else:
        b0, b1 = base % Q[0], base // Q[0]
    return np.stack([q0 - b0, q1 - b1], axis=-1).astype(np.float64)


def centres_residual(out: np.ndarray, base: np.ndarray, Q, min_shift: int = 0) -> np.ndarray:
    """[..][2] int centres: base coordinates + out rounded half away from
    zero (dropped when its larger component is below min_shift), clamped
    into the space."""
    r = np.where(out >= 0, np.floor(out + 0.5), -np.floor(-out + 0.5)).astype(np.int64)
    small = np.maximum(np.abs(r[..., 0]), np.abs(r[..., 1])) < min_shift
    r = np.where(small[..., None], 0, r)
    c0 = np.clip(base % Q[0] + r[..., 0], 0, Q[0] - 1)
    c1 = np.clip(base // Q[0] + r[..., 1], 0, Q[1] - 1)
    return np.stack([c0, c1], axis=-1)


def window_edge_count(labels: np.ndarray, centre: np.ndarray, win: int, Q) -> int:
    """Pixels whose label lies on an inner edge of its win x win box (centre
    clamped so the box fits): an edge that is not an edge of the label space."""
    h = (win - 1) // 2
    l0, l1 = labels % Q[0], labels // Q[0]
    lo0 = np.clip(centre[..., 0], h, Q[0] - 1 - h) - h
    lo1 = np.clip(centre[..., 1], h, Q[1] - 1 - h) - h
    e0 = ((l0 == lo0) & (lo0 > 0)) | ((l0 == lo0 + win - 1) & (lo0 + win - 1 < Q[0] - 1))
    e1 = ((l1 == lo1) & (lo1 > 0)) | ((l1 == lo1 + win - 1) & (lo1 + win - 1 < Q[1] - 1))
    return int((e0 | e1).sum())
