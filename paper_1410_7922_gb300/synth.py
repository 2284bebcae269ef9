"""Seeded synthetic stereo / motion inputs (numpy only).

This module holds no arithmetic of the method: it only draws images, ground
truth displacement fields and the per-workload label spaces and parameters.
Both the CUDA path and the CPU oracle consume what it produces, so it imports
neither of them.

The paper evaluates on Middlebury *Cones* (stereo, 450x375) and *Back Yard*
(motion, 320x265), Sec. 5; those images are not available here, so every
workload is a seeded stand-in with the same shape and the same kind of
structure: smoothed-noise texture, piecewise planar disparity or piecewise
affine motion, right/next image warped from the first and N(0, 2) noise.
Seeds: 14107922 + 1000 * workload_id + pair_id.
"""
from __future__ import annotations

import numpy as np

SEED_BASE = 14107922


def seed_for(workload: int, pair: int = 0) -> int:
    return SEED_BASE + 1000 * workload + pair


def _gauss_blur(img: np.ndarray, sigma: float) -> np.ndarray:
    r = max(1, int(np.ceil(3 * sigma)))
    t = np.arange(-r, r + 1, dtype=np.float64)
    k = np.exp(-0.5 * (t / sigma) ** 2)
    k /= k.sum()
    p = np.pad(img, r, mode="reflect")
    # separable: rows then columns
    p = np.apply_along_axis(lambda v: np.convolve(v, k, mode="valid"), 1, p)
    p = np.apply_along_axis(lambda v: np.convolve(v, k, mode="valid"), 0, p)
    return p


def texture(rng: np.random.Generator, H: int, W: int, sigma: float = 1.5) -> np.ndarray:
    """Uniform noise, Gaussian-blurred, contrast-stretched to 0..255 (float)."""
    t = _gauss_blur(rng.uniform(0.0, 1.0, size=(H, W)), sigma)
    t -= t.min()
    t *= 255.0 / max(t.max(), 1e-9)
    return t


def _sample_rows(img: np.ndarray, xs: np.ndarray) -> np.ndarray:
    """Linear interpolation of img[y, xs[y, x]] along x (edge-clamped)."""
    H, W = img.shape
    x0 = np.clip(np.floor(xs), 0, W - 1).astype(np.int64)
    x1 = np.clip(x0 + 1, 0, W - 1)
    f = np.clip(xs - np.floor(xs), 0.0, 1.0)
    yy = np.arange(H)[:, None]
    return img[yy, x0] * (1 - f) + img[yy, x1] * f


def _bilinear(img: np.ndarray, xs: np.ndarray, ys: np.ndarray) -> np.ndarray:
    H, W = img.shape
    xs = np.clip(xs, 0, W - 1)
    ys = np.clip(ys, 0, H - 1)
    x0 = np.floor(xs).astype(np.int64)
    y0 = np.floor(ys).astype(np.int64)
    x1 = np.minimum(x0 + 1, W - 1)
    y1 = np.minimum(y0 + 1, H - 1)
    fx = xs - x0
    fy = ys - y0
    return (img[y0, x0] * (1 - fx) * (1 - fy) + img[y0, x1] * fx * (1 - fy)
            + img[y1, x0] * (1 - fx) * fy + img[y1, x1] * fx * fy)


def _to_u8(rng: np.random.Generator, img: np.ndarray, noise_sigma: float = 2.0) -> np.ndarray:
    img = img + rng.normal(0.0, noise_sigma, size=img.shape)
    return np.clip(np.rint(img), 0, 255).astype(np.uint8)


def stereo_bands(seed: int, W: int, H: int, dmax: int):
    """Left/right pair with piecewise-constant disparity (4-6 vertical bands
    and one rectangle), disparity in 0..dmax, sampled in right coordinates:
    IR(x, y) = IL(x + d(x, y), y)."""
    rng = np.random.default_rng(seed)
    IL = texture(rng, H, W)
    n = int(rng.integers(4, 7))
    cuts = np.sort(rng.choice(np.arange(1, W), size=n - 1, replace=False))
    d = np.zeros((H, W), dtype=np.int64)
    edges = [0, *cuts.tolist(), W]
    for i in range(n):
        d[:, edges[i]:edges[i + 1]] = int(rng.integers(0, dmax + 1))
    x0, x1 = sorted(rng.integers(0, W, size=2).tolist())
    y0, y1 = sorted(rng.integers(0, H, size=2).tolist())
    d[y0:y1 + 1, x0:x1 + 1] = int(rng.integers(0, dmax + 1))
    xs = np.arange(W)[None, :] + d
    IR = _sample_rows(IL, xs.astype(np.float64))
    return _to_u8(rng, IL), _to_u8(rng, IR), d.astype(np.int32)


def stereo_planes(seed: int, W: int, H: int, dmax: int):
    """Left/right pair with 8-20 Voronoi segments, each a plane d = a + bx + cy
    rounded and clipped to 0..dmax."""
    rng = np.random.default_rng(seed)
    IL = texture(rng, H, W)
    n = int(rng.integers(8, 21))
    sx = rng.uniform(0, W, n)
    sy = rng.uniform(0, H, n)
    yy, xx = np.mgrid[0:H, 0:W]
    dist = (xx[None] - sx[:, None, None]) ** 2 + (yy[None] - sy[:, None, None]) ** 2
    seg = np.argmin(dist, axis=0)
    a = rng.uniform(0, dmax, n)
    b = rng.uniform(-0.05, 0.05, n)
    c = rng.uniform(-0.05, 0.05, n)
    d = a[seg] + b[seg] * (xx - sx[seg]) + c[seg] * (yy - sy[seg])
    d = np.clip(np.rint(d), 0, dmax).astype(np.int64)
    IR = _sample_rows(IL, (xx + d).astype(np.float64))
    return _to_u8(rng, IL), _to_u8(rng, IR), d.astype(np.int32)


def motion_layers(seed: int, W: int, H: int, vmax: int, nlayers: tuple[int, int] = (2, 4)):
    """Frame pair: a background plus 2-4 elliptical textured layers, each
    moving with an affine flow inside [-vmax, vmax]^2, composited in painter's
    order.  I1(p + v(p)) = I0(p).  Returns (I0, I1, flow [H][W][2])."""
    rng = np.random.default_rng(seed)
    yy, xx = np.mgrid[0:H, 0:W].astype(np.float64)
    n = int(rng.integers(nlayers[0], nlayers[1] + 1))
    tex, masks, flows = [], [], []
    for i in range(n + 1):
        tex.append(texture(rng, H, W))
        u0, v0 = rng.uniform(-0.7 * vmax, 0.7 * vmax, 2)
        A = rng.uniform(-0.02, 0.02, (2, 2))
        cx, cy = W / 2, H / 2
        fu = u0 + A[0, 0] * (xx - cx) + A[0, 1] * (yy - cy)
        fv = v0 + A[1, 0] * (xx - cx) + A[1, 1] * (yy - cy)
        flows.append((np.clip(fu, -vmax, vmax), np.clip(fv, -vmax, vmax)))
        if i == 0:
            masks.append(np.ones((H, W), dtype=bool))
        else:
            ex, ey = rng.uniform(0.15 * W, 0.85 * W), rng.uniform(0.15 * H, 0.85 * H)
            rx, ry = rng.uniform(0.1 * W, 0.3 * W), rng.uniform(0.1 * H, 0.3 * H)
            masks.append(((xx - ex) / rx) ** 2 + ((yy - ey) / ry) ** 2 <= 1.0)
    I0 = np.zeros((H, W))
    flow = np.zeros((H, W, 2))
    I1 = np.zeros((H, W))
    for i in range(n + 1):
        m = masks[i]
        I0[m] = tex[i][m]
        flow[m, 0] = flows[i][0][m]
        flow[m, 1] = flows[i][1][m]
        # next frame: layer i seen at p comes from p - v (backward sampling);
        # the flow is smooth, so v(p - v) ~ v(p)
        fu, fv = flows[i]
        srcx, srcy = xx - fu, yy - fv
        mw = _bilinear(m.astype(np.float64), srcx, srcy) > 0.5
        I1[mw] = _bilinear(tex[i], srcx, srcy)[mw]
    return _to_u8(rng, I0), _to_u8(rng, I1), np.rint(flow).astype(np.int32)


# --------------------------------------------------------------------------
# Workloads.  Label-space and prior parameters per workload; the parameter
# names follow the paper: lam = lambda, g = truncation threshold (K),
# l1 / l2 = prior / cost powers, cmax = cost truncation, iters = j.
# --------------------------------------------------------------------------

def space_stereo(Q: int) -> dict:
    # label q is disparity d = q; I1 (right) is sampled at x - d
    return {"R": 1, "Q": (Q, 1, 1), "vmin": (0, 0, 0), "step": (-1, 1, 1)}


def space_motion(Qx: int, Qy: int | None = None) -> dict:
    Qy = Qx if Qy is None else Qy
    return {"R": 2, "Q": (Qx, Qy, 1), "vmin": (-(Qx // 2), -(Qy // 2), 0), "step": (1, 1, 1)}


def space_motion_stereo(Qx: int, Qy: int, Qd: int) -> dict:
    return {"R": 3, "Q": (Qx, Qy, Qd), "vmin": (-(Qx // 2), -(Qy // 2), 0), "step": (1, 1, -1)}


def workload_scanline_64x48(pair: int = 0) -> dict:
    """64x48 stereo, Q=16, C = min(|IL-IR|, 20), prior 20*min(|d-d'|, 4)."""
    IL, IR, d = stereo_bands(seed_for(1, pair), 64, 48, 15)
    return {"name": "stereo_scanline_64x48_Q16", "I0": IL, "I1": IR, "I2": None, "gt": d,
            "space": space_stereo(16), "prior": {"lam": 20, "g": 4, "l1": 1, "mode": "joint"},
            "l2": 1, "cmax": 20, "cost_mode": "pair", "iters": 1}


def workload_stereo_450x375(pair: int = 0, W: int = 450, H: int = 375) -> dict:
    """450x375 stereo (Cones-sized), Q=64, T=20, lambda=20, K=4, full EDP."""
    IL, IR, d = stereo_planes(seed_for(2, pair), W, H, 63)
    return {"name": f"stereo_edp_{W}x{H}_Q64", "I0": IL, "I1": IR, "I2": None, "gt": d,
            "space": space_stereo(64), "prior": {"lam": 20, "g": 4, "l1": 1, "mode": "joint"},
            "l2": 1, "cmax": 20, "cost_mode": "pair", "iters": 1}


def workload_motion_320x240(pair: int = 0, W: int = 320, H: int = 240, mode: str = "per_axis") -> dict:
    """320x240 motion, 33x33 labels in [-16, 16]^2, lambda=15, K=3 per axis."""
    I0, I1, f = motion_layers(seed_for(3, pair), W, H, 16)
    return {"name": f"motion_edp_{W}x{H}_Q33x33", "I0": I0, "I1": I1, "I2": None, "gt": f,
            "space": space_motion(33), "prior": {"lam": 15, "g": 3, "l1": 1, "mode": mode},
            "l2": 1, "cmax": 20, "cost_mode": "pair", "iters": 1}


BATCH_SIZES = [(160, 120), (240, 180), (320, 240), (480, 360), (640, 480)]
BATCH_1D_Q = [32, 48, 64, 96, 128]
BATCH_2D_Q = [17, 25, 33]


def workload_batch(n_pairs: int = 64, scale: float = 1.0) -> list[dict]:
    """64 heterogeneous problems: sizes uniform over 160x120..640x480, kinds
    round-robin 1D stereo (Q 32..128) / 2D motion (17^2..33^2) / 3D (17x17x9)
    with a third image.  ``scale`` shrinks the images (tests)."""
    out = []
    for i in range(n_pairs):
        rng = np.random.default_rng(seed_for(4, i))
        W, H = BATCH_SIZES[int(rng.integers(0, len(BATCH_SIZES)))]
        W, H = max(4, int(W * scale)), max(3, int(H * scale))
        kind = i % 3
        if kind == 0:
            Q = BATCH_1D_Q[int(rng.integers(0, len(BATCH_1D_Q)))]
            I0, I1, gt = stereo_planes(seed_for(4, i), W, H, Q - 1)
            w = {"I0": I0, "I1": I1, "I2": None, "gt": gt, "space": space_stereo(Q),
                 "prior": {"lam": 20, "g": 4, "l1": 1, "mode": "joint"}, "cost_mode": "pair"}
        elif kind == 1:
            Q = BATCH_2D_Q[int(rng.integers(0, len(BATCH_2D_Q)))]
            I0, I1, gt = motion_layers(seed_for(4, i), W, H, Q // 2)
            w = {"I0": I0, "I1": I1, "I2": None, "gt": gt, "space": space_motion(Q),
                 "prior": {"lam": 15, "g": 3, "l1": 1, "mode": "per_axis"}, "cost_mode": "pair"}
        else:
            I0, I1, gt = motion_layers(seed_for(4, i), W, H, 8)
            # third image: a stereo partner of I0 (disparity 0..8 bands)
            I2 = _stereo_partner(I0, seed_for(4, 500 + i), 8)
            w = {"I0": I0, "I1": I1, "I2": I2, "gt": gt, "space": space_motion_stereo(17, 17, 9),
                 "prior": {"lam": 15, "g": 3, "l1": 1, "mode": "per_axis"},
                 "cost_mode": "pair_stereo3"}
        w.update({"name": f"batch{i}_{W}x{H}", "l2": 1, "cmax": 20, "iters": 1})
        out.append(w)
    return out


def _stereo_partner(I0: np.ndarray, seed: int, dmax: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    H, W = I0.shape
    n = int(rng.integers(3, 6))
    cuts = np.sort(rng.choice(np.arange(1, W), size=n - 1, replace=False))
    d = np.zeros((H, W))
    edges = [0, *cuts.tolist(), W]
    for i in range(n):
        d[:, edges[i]:edges[i + 1]] = int(rng.integers(0, dmax + 1))
    return _to_u8(rng, _sample_rows(I0.astype(np.float64), np.arange(W)[None, :] + d))


def workload_motion_640x480(pair: int = 0, W: int = 640, H: int = 480, vmax: int = 32) -> dict:
    """640x480 motion with the full 65x65 label space ([-32, 32]^2); smaller
    images / label spaces for tests through W, H, vmax."""
    I0, I1, f = motion_layers(seed_for(5, pair), W, H, vmax)
    Q = 2 * vmax + 1
    return {"name": f"motion_{W}x{H}_Q{Q}x{Q}", "I0": I0, "I1": I1, "I2": None, "gt": f,
            "space": space_motion(Q), "prior": {"lam": 15, "g": 3, "l1": 1, "mode": "per_axis"},
            "l2": 1, "cmax": 20, "cost_mode": "pair", "iters": 1}


def random_cost(seed: int, H: int, W: int, Q: int, cmax: int = 20) -> np.ndarray:
    """Uniform random integer cost volume in 0..cmax (parity edge cases)."""
    rng = np.random.default_rng(seed)
    return rng.integers(0, cmax + 1, size=(H, W, Q), dtype=np.int64).astype(np.int32)
