"""Learned proposal + windowed EDP (two-axis motion label spaces).

Pipeline, every arithmetic step in libedp.so:
  1. winner-take-all over the full label space (edp_wta) and the network
     features (edp_net_features);
  2. the proposal network predicts each pixel's label centre
     (edp_net_forward, edp_net_centres);
  3. EDP runs on a win x win label box around that centre
     (edp_cost_window, edp_solve_windowed);
  4. the energy of the result is evaluated on the full label space
     (edp_cost_volume, edp_energy): full-label EDP is the reference the gap is
     measured against.
Training targets are labelings that full-label EDP (edp_solve_images)
produces on synthetic pairs; training is Adam on the smooth-L1 loss with the
project's forward/backward kernels.  torch only holds device memory.
"""
from __future__ import annotations

import time

import numpy as np
import torch

from . import edp, synth

FLOW_SCALE = 16.0
WTA_RADIUS = 3  # winner-take-all feature on costs summed over 7x7 pixels


def pair(pair_id: int, W: int, H: int, vmax: int = 32) -> dict:
    return synth.workload_motion_640x480(pair=pair_id, W=W, H=H, vmax=vmax)


def to_device(w: dict) -> tuple[torch.Tensor, torch.Tensor]:
    return torch.from_numpy(w["I0"]).cuda(), torch.from_numpy(w["I1"]).cuda()


def features(I0, I1, w: dict, radius: int = WTA_RADIUS) -> torch.Tensor:
    lab, cost = edp.wta(I0, I1, w["space"], w["l2"], w["cmax"], radius=radius)
    area = (2 * radius + 1) ** 2
    return edp.net_features(I0, I1, lab, cost, w["space"], FLOW_SCALE, float(w["cmax"] * area))


def targets(labels: torch.Tensor, space: dict) -> torch.Tensor:
    """Label coordinates of a labeling, centred on the space's middle (the
    network's output convention)."""
    Q0, Q1 = space["Q"][0], space["Q"][1]
    q0 = (labels % Q0).float() - 0.5 * (Q0 - 1)
    q1 = torch.div(labels, Q0, rounding_mode="floor").float() - 0.5 * (Q1 - 1)
    return torch.stack([q0, q1], dim=-1).contiguous()


def full_edp(I0, I1, w: dict, iters: int = 1, ws=None):
    """Full-label EDP: (labels, energy4)."""
    return edp.solve_images(I0, I1, None, w["space"], w["prior"], w["l2"], w["cmax"], iters=iters, ws=ws)


def init_params(seed: int = 0) -> torch.Tensor:
    """He-uniform weights, zero biases, flat float32 on the device."""
    g = torch.Generator().manual_seed(seed)
    chans = [5, 32, 32, 32, 32, 32, 2]
    parts = []
    for ci, co in zip(chans[:-1], chans[1:]):
        lim = (6.0 / (ci * 9)) ** 0.5
        parts.append((torch.rand(co * ci * 9, generator=g, dtype=torch.float64) * 2 - 1) * lim)
        parts.append(torch.zeros(co, dtype=torch.float64))
    p = torch.cat(parts).float().cuda()
    assert p.numel() == edp.net_param_count()
    return p


def build_training_set(n_pairs: int, W: int, H: int, first_pair: int = 0, iters: int = 1, vmax: int = 32):
    """Features and full-label EDP targets of n_pairs synthetic pairs."""
    xs, ts = [], []
    ws = None
    for k in range(n_pairs):
        w = pair(first_pair + k, W, H, vmax)
        I0, I1 = to_device(w)
        if ws is None:
            ws = edp.workspace(edp.OP_SOLVE_IMAGES, W, H, w["space"], w["prior"], iters)
        lab, _ = full_edp(I0, I1, w, iters, ws)
        xs.append(features(I0, I1, w))
        ts.append(targets(lab, w["space"]))
    return torch.stack(xs).contiguous(), torch.stack(ts).contiguous()


def train(x: torch.Tensor, t: torch.Tensor, epochs: int = 30, batch: int = 8, lr: float = 2e-3, seed: int = 0,
          log=None) -> tuple[torch.Tensor, list[float]]:
    """Adam on the smooth-L1 loss; x bf16 [P][H][W][5], t float32 [P][H][W][2]."""
    P = init_params(seed)
    m, v = torch.zeros_like(P), torch.zeros_like(P)
    n = x.shape[0]
    H, W = x.shape[1], x.shape[2]
    ws = edp.net_workspace(batch, H, W)
    g = torch.Generator().manual_seed(seed + 1)
    step, losses = 0, []
    grad = torch.empty_like(P)
    loss = torch.empty(1, dtype=torch.float64, device="cuda")
    for ep in range(epochs):
        perm = torch.randperm(n, generator=g)
        ep_loss = 0.0
        nb = 0
        for b0 in range(0, n - batch + 1, batch):
            idx = perm[b0:b0 + batch].cuda()
            xb = x.index_select(0, idx).contiguous()
            tb = t.index_select(0, idx).contiguous()
            out = edp.net_forward(P, xb, ws)
            edp.net_backward(P, out, tb, ws, grad=grad, loss=loss)
            step += 1
            edp.net_adam(P, grad, m, v, lr, step)
            ep_loss += float(loss.item())
            nb += 1
        losses.append(ep_loss / max(nb, 1))
        if log:
            log(f"epoch {ep}: loss {losses[-1]:.4f}")
    return P, losses


def propose(P: torch.Tensor, I0, I1, w: dict) -> torch.Tensor:
    """Box centres int32 [H][W][2] from the trained network."""
    x = features(I0, I1, w)[None].contiguous()
    H, W = I0.shape
    ws = edp.net_workspace(1, H, W)
    out = edp.net_forward(P, x, ws)
    return edp.net_centres(out[0].contiguous(), w["space"])


def wta_centres(I0, I1, w: dict, radius: int = WTA_RADIUS) -> torch.Tensor:
    """Centres straight from (window-aggregated) winner-take-all: the
    proposal without a network."""
    lab, _ = edp.wta(I0, I1, w["space"], w["l2"], w["cmax"], radius=radius)
    Q0 = w["space"]["Q"][0]
    return torch.stack([lab % Q0, torch.div(lab, Q0, rounding_mode="floor")], dim=-1).int().contiguous()


def windowed_edp(I0, I1, w: dict, centre: torch.Tensor, win: int = 9, iters: int = 1, ws=None):
    Cw = edp.cost_window(I0, I1, None, w["space"], w["l2"], w["cmax"], centre, win)
    return edp.solve_windowed(Cw, centre, win, w["space"], w["prior"], iters=iters, ws=ws)


def label_centres(labels: torch.Tensor, space: dict) -> torch.Tensor:
    """Label coordinates of a labeling as box centres int32 [H][W][2]."""
    Q0 = space["Q"][0]
    return torch.stack([labels % Q0, torch.div(labels, Q0, rounding_mode="floor")], dim=-1).int().contiguous()


def refine(I0, I1, w: dict, centre: torch.Tensor, rounds: int, win: int = 9, iters: int = 1, ws=None):
    """Windowed EDP, then `rounds - 1` more windowed solves re-centred on the
    previous result."""
    lab = windowed_edp(I0, I1, w, centre, win, iters, ws)
    for _ in range(rounds - 1):
        lab = windowed_edp(I0, I1, w, label_centres(lab, w["space"]), win, iters, ws)
    return lab


def evaluate(P: torch.Tensor, pairs: list[int], W: int, H: int, win: int = 9, iters: int = 1, reps: int = 3,
             vmax: int = 32):
    """Energy gap and time of (network + windowed EDP) against full-label EDP,
    and of (WTA centres + windowed EDP), on held-out pairs."""
    rows = []
    ev = lambda: torch.cuda.Event(enable_timing=True)

    def timed(fn):
        fn()
        torch.cuda.synchronize()
        best = None
        for _ in range(reps):
            s, e = ev(), ev()
            s.record()
            r = fn()
            e.record()
            torch.cuda.synchronize()
            ms = s.elapsed_time(e)
            best = ms if best is None else min(best, ms)
        return r, best

    ws_full = ws_win = None
    for pid in pairs:
        w = pair(pid, W, H, vmax)
        I0, I1 = to_device(w)
        if ws_full is None:
            ws_full = edp.workspace(edp.OP_SOLVE_IMAGES, W, H, w["space"], w["prior"], iters)
            ws_win = edp.workspace_windowed(W, H, w["space"], w["prior"], win, iters)
        (lab_f, e_f), ms_full = timed(lambda: full_edp(I0, I1, w, iters, ws_full))
        e_full = int(e_f[3].item())
        C = edp.cost_volume(I0, I1, None, w["space"], w["l2"], w["cmax"])

        def net_path():
            c = propose(P, I0, I1, w)
            return windowed_edp(I0, I1, w, c, win, iters, ws_win)

        def wta_path():
            c = wta_centres(I0, I1, w)
            return windowed_edp(I0, I1, w, c, win, iters, ws_win)

        lab_n, ms_net = timed(net_path)
        lab_w, ms_wta = timed(wta_path)
        e_net = int(edp.energy(C, lab_n, w["space"], w["prior"])[3].item())
        e_wta = int(edp.energy(C, lab_w, w["space"], w["prior"])[3].item())
        del C
        rows.append({"pair": pid, "E_full": e_full, "E_net": e_net, "E_wta": e_wta,
                     "gap_net": (e_net - e_full) / e_full, "gap_wta": (e_wta - e_full) / e_full,
                     "ms_full": ms_full, "ms_net": ms_net, "ms_wta": ms_wta,
                     "label_agree_net": float((lab_n == lab_f).float().mean().item())})
    return rows
