"""Learned proposal + windowed EDP (two-axis motion label spaces).

Pipeline, every arithmetic step in libedp.so:
  1. a coarse labeling: full EDP on the 2x2-averaged images over the label
     space with halved offsets, doubled back to full resolution
     (edp_coarse_labels);
  2. the proposal network reads the frames and that labeling
     (edp_net_features_labels) and predicts a correction of it, in label
     units (edp_net_forward); centre = coarse label + rounded correction
     (edp_net_centres_residual);
  3. EDP runs on a win x win label box around each centre
     (edp_cost_window, edp_solve_windowed), optionally re-centred on its own
     result for more rounds;
  4. full-label EDP stays the reference and the fallback: solve() falls back
     to it when too many windowed labels sit on an inner edge of their box
     (edp_window_edge_count: the box probably cut off a better label), and in
     verify mode it solves the full label space as well and keeps whichever
     labeling has the lower energy (edp_cost_volume, edp_energy).
Training targets are, per synthetic pair, the lower-energy labeling of
full-label EDP (edp_solve_images) and of windowed EDP centred on the coarse
labeling, as corrections of the coarse labeling (edp_net_targets); training
is Adam on the smooth-L1 loss with the project's forward/backward kernels.
torch only holds device memory.
"""
from __future__ import annotations

import time

import numpy as np
import torch

from . import edp, synth

FLOW_SCALE = 16.0
MIN_SHIFT = 2  # network corrections below this many labels are not applied


def pair(pair_id: int, W: int, H: int, vmax: int = 32) -> dict:
    return synth.workload_motion_640x480(pair=pair_id, W=W, H=H, vmax=vmax)


def to_device(w: dict) -> tuple[torch.Tensor, torch.Tensor]:
    return torch.from_numpy(w["I0"]).cuda(), torch.from_numpy(w["I1"]).cuda()


def coarse(I0, I1, w: dict, ws=None, iters: int = 1) -> torch.Tensor:
    """Coarse-level labeling in the full label space (int32 [H][W])."""
    return edp.coarse_labels(I0, I1, w["space"], w["prior"], w["l2"], w["cmax"], iters=iters, ws=ws)


def features(I0, I1, w: dict, base: torch.Tensor) -> torch.Tensor:
    """Network input bf16 [H][W][5] from the frames and the coarse labeling."""
    return edp.net_features_labels(I0, I1, base, w["space"], w["l2"], w["cmax"], FLOW_SCALE)


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


def build_training_set(n_pairs: int, W: int, H: int, first_pair: int = 0, iters: int = 1, vmax: int = 32,
                       pool=None, target: str = "best", win: int = 9):
    """Network inputs (bf16 [P][H][W][5]) and targets (float32 [P][H][W][2],
    corrections of the coarse labeling) of n_pairs synthetic pairs.  target
    "best": per pair the lower-energy labeling of full-label EDP and of
    windowed EDP centred on the coarse labeling; "full": full-label EDP.
    `pool`: an optional process pool (spawn) that synthesises the pairs."""
    ids = [first_pair + k for k in range(n_pairs)]
    gen = pool.imap(_pair_images, [(i, W, H, vmax) for i in ids], chunksize=4) if pool else (
        _pair_images((i, W, H, vmax)) for i in ids)
    xs, ts = [], []
    ws = wsc = wsw = C = None
    for pid, (I0n, I1n) in zip(ids, gen):
        w = pair_meta(W, H, vmax)
        I0, I1 = torch.from_numpy(I0n).cuda(), torch.from_numpy(I1n).cuda()
        if ws is None:
            ws = edp.workspace(edp.OP_SOLVE_IMAGES, W, H, w["space"], w["prior"], iters)
            wsc = edp.workspace(edp.OP_COARSE, W, H, w["space"], w["prior"], iters, l2=w["l2"], cmax=w["cmax"])
            wsw = edp.workspace_windowed(W, H, w["space"], w["prior"], win, iters)
            C = torch.empty((H, W, edp.n_labels(w["space"])), dtype=torch.int32, device="cuda")
        lab, e4 = full_edp(I0, I1, w, iters, ws)
        base = coarse(I0, I1, w, wsc, iters)
        if target == "best":
            lab_c = windowed_edp(I0, I1, w, label_centres(base, w["space"]), win, iters, wsw)
            edp.cost_volume(I0, I1, None, w["space"], w["l2"], w["cmax"], out=C)
            if int(edp.energy(C, lab_c, w["space"], w["prior"])[3].item()) < int(e4[3].item()):
                lab = lab_c
        xs.append(features(I0, I1, w, base))
        ts.append(edp.net_targets(lab, w["space"], base=base))
    return torch.stack(xs).contiguous(), torch.stack(ts).contiguous()


def _pair_images(args):
    pid, W, H, vmax = args
    w = pair(pid, W, H, vmax)
    return w["I0"], w["I1"]


def pair_meta(W: int, H: int, vmax: int = 32) -> dict:
    """Label space, prior and cost parameters of the motion pairs (no images)."""
    Q = 2 * vmax + 1
    return {"space": synth.space_motion(Q), "prior": {"lam": 15, "g": 3, "l1": 1, "mode": "per_axis"},
            "l2": 1, "cmax": 20, "cost_mode": "pair", "W": W, "H": H}


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


def propose(P: torch.Tensor, I0, I1, w: dict, base: torch.Tensor | None = None, ws=None,
            min_shift: int = MIN_SHIFT) -> torch.Tensor:
    """Box centres int32 [H][W][2]: coarse labeling + the network's correction."""
    if base is None:
        base = coarse(I0, I1, w, ws)
    x = features(I0, I1, w, base)[None].contiguous()
    H, W = I0.shape
    out = edp.net_forward(P, x, edp.net_workspace(1, H, W))
    return edp.net_centres_residual(out[0].contiguous(), base, w["space"], min_shift)


def windowed_edp(I0, I1, w: dict, centre: torch.Tensor, win: int = 9, iters: int = 1, ws=None):
    Cw = edp.cost_window(I0, I1, None, w["space"], w["l2"], w["cmax"], centre, win)
    return edp.solve_windowed(Cw, centre, win, w["space"], w["prior"], iters=iters, ws=ws)


def label_centres(labels: torch.Tensor, space: dict) -> torch.Tensor:
    """Label coordinates of a labeling as box centres int32 [H][W][2]."""
    zero = torch.zeros(tuple(labels.shape) + (2,), dtype=torch.float32, device=labels.device)
    return edp.net_centres_residual(zero, labels, space)


def refine(I0, I1, w: dict, centre: torch.Tensor, rounds: int, win: int = 9, iters: int = 1, ws=None):
    """Windowed EDP, then `rounds - 1` more windowed solves re-centred on the
    previous result."""
    lab = windowed_edp(I0, I1, w, centre, win, iters, ws)
    for _ in range(rounds - 1):
        lab = windowed_edp(I0, I1, w, label_centres(lab, w["space"]), win, iters, ws)
    return lab


EDGE_FRAC = 0.02  # fallback when more than this fraction of labels sit on an inner box edge


def solve(P: torch.Tensor, I0, I1, w: dict, win: int = 9, iters: int = 1, edge_frac: float = EDGE_FRAC,
          verify: bool = False, min_shift: int = MIN_SHIFT, ws=None):
    """The proposal path with full-label EDP as its fallback: coarse labeling,
    network correction, windowed EDP; then full-label EDP instead when more
    than `edge_frac` of the pixels got a label on an inner edge of their box
    (the box likely cut off a better label).  verify=True also solves the
    full label space and keeps the lower-energy labeling (the gap to
    full-label EDP is then never positive, at the cost of the full solve).
    ws: optional dict of workspaces reused across calls.  Returns (labels,
    info) with info = {"fallback": bool, "edge_frac": float}."""
    H, W = I0.shape
    ws = {} if ws is None else ws
    if "coarse" not in ws:
        ws["coarse"] = edp.workspace(edp.OP_COARSE, W, H, w["space"], w["prior"], iters, l2=w["l2"], cmax=w["cmax"])
        ws["win"] = edp.workspace_windowed(W, H, w["space"], w["prior"], win, iters)
        ws["net"] = edp.net_workspace(1, H, W)
    base = coarse(I0, I1, w, ws["coarse"], iters)
    x = features(I0, I1, w, base)[None].contiguous()
    out = edp.net_forward(P, x, ws["net"])
    centre = edp.net_centres_residual(out[0].contiguous(), base, w["space"], min_shift)
    lab = windowed_edp(I0, I1, w, centre, win, iters, ws["win"])
    frac = int(edp.window_edge_count(lab, centre, win, w["space"]).item()) / (W * H)
    info = {"fallback": False, "edge_frac": frac}
    if verify or frac > edge_frac:
        if "full" not in ws:
            ws["full"] = edp.workspace(edp.OP_SOLVE_IMAGES, W, H, w["space"], w["prior"], iters)
        lab_f, e4 = full_edp(I0, I1, w, iters, ws["full"])
        use_full = not verify
        if verify:
            C = edp.cost_volume(I0, I1, None, w["space"], w["l2"], w["cmax"])
            use_full = int(edp.energy(C, lab, w["space"], w["prior"])[3].item()) > int(e4[3].item())
            del C
        if use_full:
            lab = lab_f
            info["fallback"] = True
    return lab, info


def coverage(centre: torch.Tensor, labels: torch.Tensor, space: dict, win: int) -> float:
    """Fraction of pixels whose label (e.g. full-label EDP's) lies inside the
    win x win box around the centre, boxes clamped into the space as the
    windowed solve does (evaluation metric)."""
    Q0, Q1 = space["Q"][0], space["Q"][1]
    h = (win - 1) // 2
    c0 = centre[..., 0].clamp(h, Q0 - 1 - h)
    c1 = centre[..., 1].clamp(h, Q1 - 1 - h)
    l0, l1 = labels % Q0, torch.div(labels, Q0, rounding_mode="floor")
    inside = ((l0 - c0).abs() <= h) & ((l1 - c1).abs() <= h)
    return float(inside.float().mean().item())


def evaluate(P: torch.Tensor, pairs: list[int], W: int, H: int, win: int = 9, iters: int = 1, reps: int = 3,
             vmax: int = 32, rounds: int = 1, min_shift: int = MIN_SHIFT):
    """Energy gap and time against full-label EDP on held-out pairs of
    (coarse labeling + network + windowed EDP) and of the same path without
    the network (windows centred on the coarse labeling)."""
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

    ws_full = ws_win = ws_c = None
    net_ws = edp.net_workspace(1, H, W)
    for pid in pairs:
        w = pair(pid, W, H, vmax)
        I0, I1 = to_device(w)
        if ws_full is None:
            ws_full = edp.workspace(edp.OP_SOLVE_IMAGES, W, H, w["space"], w["prior"], iters)
            ws_win = edp.workspace_windowed(W, H, w["space"], w["prior"], win, iters)
            ws_c = edp.workspace(edp.OP_COARSE, W, H, w["space"], w["prior"], iters, l2=w["l2"], cmax=w["cmax"])
        (lab_f, e_f), ms_full = timed(lambda: full_edp(I0, I1, w, iters, ws_full))
        e_full = int(e_f[3].item())
        C = edp.cost_volume(I0, I1, None, w["space"], w["l2"], w["cmax"])

        centres = {}

        def net_path():
            base = coarse(I0, I1, w, ws_c, iters)
            x = features(I0, I1, w, base)[None].contiguous()
            out = edp.net_forward(P, x, net_ws)
            c = edp.net_centres_residual(out[0].contiguous(), base, w["space"], min_shift)
            centres["net"] = c
            return refine(I0, I1, w, c, rounds, win, iters, ws_win)

        def coarse_path():
            base = coarse(I0, I1, w, ws_c, iters)
            c = label_centres(base, w["space"])
            centres["coarse"] = c
            return refine(I0, I1, w, c, rounds, win, iters, ws_win)

        lab_n, ms_net = timed(net_path)
        lab_c, ms_coarse = timed(coarse_path)
        solve_ws = {}
        (lab_s, info), ms_solve = timed(lambda: solve(P, I0, I1, w, win, iters, min_shift=min_shift, ws=solve_ws))
        # held-out smooth-L1 of the network's correction against full-label
        # EDP, and of no correction (the coarse labeling as it is)
        base = coarse(I0, I1, w, ws_c, iters)
        out = edp.net_forward(P, features(I0, I1, w, base)[None].contiguous(), net_ws)
        tgt = edp.net_targets(lab_f, w["space"], base=base)[None].contiguous()
        loss_net = float(edp.net_backward(P, out, tgt, net_ws)[1].item())
        loss_zero = float(edp.net_backward(P, torch.zeros_like(out), tgt, net_ws)[1].item())
        e_net = int(edp.energy(C, lab_n, w["space"], w["prior"])[3].item())
        e_coarse = int(edp.energy(C, lab_c, w["space"], w["prior"])[3].item())
        e_solve = int(edp.energy(C, lab_s, w["space"], w["prior"])[3].item())
        del C
        rows.append({"pair": pid, "E_full": e_full, "E_net": e_net, "E_coarse": e_coarse, "E_solve": e_solve,
                     "gap_net": (e_net - e_full) / e_full, "gap_coarse": (e_coarse - e_full) / e_full,
                     "gap_solve": (e_solve - e_full) / e_full, "fallback": info["fallback"],
                     "edge_frac": info["edge_frac"],
                     "ms_full": ms_full, "ms_net": ms_net, "ms_coarse": ms_coarse, "ms_solve": ms_solve,
                     "label_agree_net": float((lab_n == lab_f).float().mean().item()),
                     "label_agree_coarse": float((lab_c == lab_f).float().mean().item()),
                     "loss_net": loss_net, "loss_zero": loss_zero,
                     "cover_net": coverage(centres["net"], lab_f, w["space"], win),
                     "cover_coarse": coverage(centres["coarse"], lab_f, w["space"], win)})
    return rows
