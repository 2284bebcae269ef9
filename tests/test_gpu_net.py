"""GPU proposal network against its CPU reference (oracle/net.py): forward
outputs and parameter gradients within 1e-2 relative (bf16 storage on both
sides, float32 vs float64 accumulation), with the 32 -> 32 convolutions on
the tensor cores (the default) and on the CUDA cores; features, centres, the
winner-take-all kernel, and a short training run that lowers the loss."""
import numpy as np
import pytest
import torch

import oracle
from oracle import net as rnet
from paper_1410_7922_gb300 import synth

pytestmark = pytest.mark.gpu


def flat_params(ps):
    return np.concatenate([np.concatenate([w.ravel(), b.ravel()]) for w, b in ps]).astype(np.float32)


def unflat(v):
    out, o = [], 0
    for ci, co in zip(rnet.CHANNELS[:-1], rnet.CHANNELS[1:]):
        w = v[o:o + co * ci * 9].reshape(co, ci, 3, 3).astype(np.float64)
        o += co * ci * 9
        b = v[o:o + co].astype(np.float64)
        o += co
        out.append((w, b))
    return out


def rel_err(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30))


RTOL = 1e-2


# bf16 carries 8 significant bits: half a step is 2^-8 of the value
HALF_BF16_STEP = 2.0 ** -8


def assert_close(got, want, what, mags=None):
    """Element by element: |got - want| <= 1e-2 |want| + floor.  For an
    output the absolute floor of near-zero entries is 1e-2 of the array's
    RMS.  For a gradient it is half a bf16 step of the sum of the absolute
    values of its terms (oracle.net.gradient_magnitudes): a gradient that is
    a small difference of large terms moves by their bf16 rounding where
    the two sides round an intermediate value differently."""
    got, want = np.asarray(got, np.float64), np.asarray(want, np.float64)
    if mags is None:
        floor = RTOL * float(np.sqrt(np.mean(want * want)))
    else:
        floor = HALF_BF16_STEP * np.asarray(mags, np.float64)
    err = np.abs(got - want)
    bad = err > RTOL * np.abs(want) + floor
    assert not bad.any(), (f"{what}: {int(bad.sum())} of {bad.size} entries off; worst "
                           f"{float(err.max()):.3g} at {np.unravel_index(np.argmax(err), err.shape)}")


# 21 x 35: ragged against every conv tile; 96 x 128: several tiles and thread
# blocks of the conv kernels in both directions; 37 x 61: ragged against the
# tensor-core tile (8 x 16 pixels) in both directions, one image; a single
# pixel, and three tiny images (one partial tile each)
SIZES = [(2, 21, 35), (2, 96, 128), (1, 37, 61), (1, 1, 1), (3, 5, 9)]


@pytest.fixture(params=[True, False], ids=["tensor_cores", "cuda_cores"])
def tc(request, edp_lib):
    edp_lib.set_net_tensor_cores(request.param)
    yield request.param
    edp_lib.set_net_tensor_cores(True)


def make_setup(edp_lib, N, H, W):
    rng = np.random.default_rng(5 + H)
    ps = rnet.init_params(11)
    ps = [(w, rng.normal(0, 0.05, size=b.shape)) for w, b in ps]
    P = flat_params(ps)
    assert P.size == edp_lib.net_param_count()
    x = rnet.bf16(rng.uniform(-1, 1, size=(N, 5, H, W)))
    tgt = rng.normal(0, 3, size=(N, 2, H, W)).astype(np.float32)
    return ps, P, x, tgt


@pytest.mark.parametrize("N,H,W", SIZES)
def test_net_forward_parity(edp_lib, tc, N, H, W):
    ps, P, x, tgt = make_setup(edp_lib, N, H, W)
    want = rnet.forward(x, unflat(P))                       # [N][2][H][W]
    xg = torch.from_numpy(x.transpose(0, 2, 3, 1).astype(np.float32)).to(torch.bfloat16).cuda().contiguous()
    Pg = torch.from_numpy(P).cuda()
    ws = edp_lib.net_workspace(N, H, W)
    out = edp_lib.net_forward(Pg, xg, ws).cpu().numpy().transpose(0, 3, 1, 2)
    assert edp_lib.net_device_status(ws) == 0
    assert_close(out, want, "forward output")
    # every hidden activation, one layer at a time: the reference layer run
    # on the GPU's own input to that layer (as the backward test does), so
    # that a pre-activation rounded to the other side of zero upstream does
    # not show as a ReLU decision here
    acts = [a.float().cpu().numpy().astype(np.float64).transpose(0, 3, 1, 2)
            for a in edp_lib.net_activations(ws, N, H, W)]
    ps_ = unflat(P)
    for layer in range(1, 6):
        w, b = ps_[layer - 1]
        z = rnet.conv3x3(acts[layer - 1], rnet.bf16(w), np.asarray(b, np.float32).astype(np.float64))
        assert_close(acts[layer], rnet.bf16(np.maximum(z, 0.0)), f"activation {layer}")


@pytest.mark.parametrize("N,H,W", SIZES)
def test_net_backward_parity(edp_lib, tc, N, H, W):
    """The backward kernels element by element against the reference
    backward run on the activations and output of the GPU's own forward pass
    (read back from the workspace; the forward pass is checked element by
    element above).  Differentiating one forward pass isolates the backward
    arithmetic: two forward passes that accumulate in different precisions
    can round a pre-activation near zero to opposite signs, and the ReLU then
    drops or keeps a whole gradient term.  The end-to-end gradients (GPU
    forward + backward against the reference's own forward + backward) agree
    within 1e-2 in norm."""
    ps, P, x, tgt = make_setup(edp_lib, N, H, W)
    xg = torch.from_numpy(x.transpose(0, 2, 3, 1).astype(np.float32)).to(torch.bfloat16).cuda().contiguous()
    Pg = torch.from_numpy(P).cuda()
    tg = torch.from_numpy(np.ascontiguousarray(tgt.transpose(0, 2, 3, 1))).cuda()
    ws = edp_lib.net_workspace(N, H, W)
    out = edp_lib.net_forward(Pg, xg, ws)
    acts = [a.float().cpu().numpy().astype(np.float64).transpose(0, 3, 1, 2)
            for a in edp_lib.net_activations(ws, N, H, W)]
    assert np.array_equal(acts[0], x)
    out_np = out.cpu().numpy().astype(np.float64).transpose(0, 3, 1, 2)
    g, loss = edp_lib.net_backward(Pg, out, tg, ws)
    assert edp_lib.net_device_status(ws) == 0
    loss_want, grads = rnet.backward(x, unflat(P), tgt.astype(np.float64), acts=acts, out=out_np)
    assert abs(float(loss.item()) - loss_want) <= RTOL * abs(loss_want)
    gp = unflat(g.cpu().numpy())
    mags = rnet.gradient_magnitudes(x, unflat(P), tgt.astype(np.float64), acts=acts, out=out_np)
    for layer, ((gw, gb), (ww, wb), (mw, mb)) in enumerate(zip(gp, grads, mags)):
        assert_close(gw, ww, f"layer {layer} weight gradient", mw)
        assert_close(gb, wb, f"layer {layer} bias gradient", mb)
    _, grads_ref = rnet.backward(x, unflat(P), tgt.astype(np.float64))
    for layer, ((gw, gb), (ww, wb)) in enumerate(zip(gp, grads_ref)):
        assert rel_err(gw, ww) < RTOL and rel_err(gb, wb) < RTOL, layer


def test_wta_and_features(edp_lib):
    w = synth.workload_motion_640x480(W=48, H=40)
    space = w["space"]
    C = oracle.cost_volume(w["I0"], w["I1"], None, space, w["l2"], w["cmax"])
    I0, I1 = torch.from_numpy(w["I0"]).cuda(), torch.from_numpy(w["I1"]).cuda()
    lab, cost = edp_lib.wta(I0, I1, space, w["l2"], w["cmax"])
    assert np.array_equal(lab.cpu().numpy(), np.argmin(C, axis=2))
    assert np.array_equal(cost.cpu().numpy(), np.min(C, axis=2))
    # window-aggregated: costs summed over a 5x5 pixel window, edge pixels repeated
    r = 2
    Cp = np.pad(C.astype(np.int64), ((r, r), (r, r), (0, 0)), mode="edge")
    Hh, Ww = C.shape[:2]
    agg = sum(Cp[dy:dy + Hh, dx:dx + Ww] for dy in range(2 * r + 1) for dx in range(2 * r + 1))
    lab2, cost2 = edp_lib.wta(I0, I1, space, w["l2"], w["cmax"], radius=r)
    assert np.array_equal(lab2.cpu().numpy(), np.argmin(agg, axis=2))
    assert np.array_equal(cost2.cpu().numpy(), np.min(agg, axis=2))
    x = edp_lib.net_features(I0, I1, lab, cost, space, 16.0, float(w["cmax"])).float().cpu().numpy()
    q = np.argmin(C, axis=2)
    Q0, Q1 = space["Q"][0], space["Q"][1]
    feats = rnet.features(w["I0"].astype(np.float64), w["I1"].astype(np.float64),
                          np.stack([q % Q0 - (Q0 - 1) / 2, q // Q0 - (Q1 - 1) / 2], -1), np.min(C, axis=2), 16.0,
                          float(w["cmax"]))
    # same float32 inputs on both sides; allow one bf16 step where a float32/float64 quotient straddles a tie
    assert np.allclose(x.transpose(2, 0, 1), rnet.bf16(feats), rtol=8e-3, atol=1e-7)
    out = torch.tensor([[[0.4, -0.6], [31.7, -40.0]]], dtype=torch.float32, device="cuda")
    c = edp_lib.net_centres(out, space).cpu().numpy()
    assert c.tolist() == [[[32, 31], [64, 0]]]


@pytest.mark.parametrize("W,H,vmax", [(24, 20, 4), (23, 17, 3)])
def test_coarse_labels(edp_lib, W, H, vmax):
    """edp_coarse_labels = 2x2 pyramid, EDP on the halved label space,
    labels doubled back to full resolution (odd sizes included)."""
    w = synth.workload_motion_640x480(pair=3, W=W, H=H, vmax=vmax)
    space, prior = w["space"], w["prior"]
    h0, h1 = rnet.pyr_down2(w["I0"]), rnet.pyr_down2(w["I1"])
    vc, qc = rnet.halved_space(space["vmin"][:2], space["Q"][:2])
    sc = {"R": 2, "Q": (qc[0], qc[1], 1), "vmin": (vc[0], vc[1], 0), "step": (1, 1, 1)}
    lc = oracle.edp(oracle.cost_volume(h0, h1, None, sc, w["l2"], w["cmax"]), sc, prior, iters=1, tier=1)
    want = rnet.labels_up2(lc, vc, qc, space["vmin"][:2], space["Q"][:2], H, W)
    I0, I1 = torch.from_numpy(w["I0"]).cuda(), torch.from_numpy(w["I1"]).cuda()
    got = edp_lib.coarse_labels(I0, I1, space, prior, w["l2"], w["cmax"]).cpu().numpy()
    assert np.array_equal(got, want)


def test_features_labels_targets_residual_centres(edp_lib):
    w = synth.workload_motion_640x480(pair=4, W=37, H=29, vmax=6)
    space = w["space"]
    Q = space["Q"][:2]
    rng = np.random.default_rng(5)
    lab = rng.integers(0, Q[0] * Q[1], size=(29, 37)).astype(np.int32)
    base = rng.integers(0, Q[0] * Q[1], size=(29, 37)).astype(np.int32)
    I0, I1 = torch.from_numpy(w["I0"]).cuda(), torch.from_numpy(w["I1"]).cuda()
    x = edp_lib.net_features_labels(I0, I1, torch.from_numpy(lab).cuda(), space, w["l2"], w["cmax"], 16.0)
    want = rnet.features_from_labels(w["I0"], w["I1"], lab, space["vmin"][:2], Q, w["l2"], w["cmax"], 16.0)
    assert np.allclose(x.float().cpu().numpy().transpose(2, 0, 1), rnet.bf16(want), rtol=8e-3, atol=1e-7)
    t = edp_lib.net_targets(torch.from_numpy(lab).cuda(), space, base=torch.from_numpy(base).cuda())
    assert np.array_equal(t.cpu().numpy(), rnet.targets(lab, Q, base))
    t0 = edp_lib.net_targets(torch.from_numpy(lab).cuda(), space)
    assert np.array_equal(t0.cpu().numpy(), rnet.targets(lab, Q))
    out = (rng.standard_normal((29, 37, 2)) * 3).astype(np.float32)
    out[0, :4, 0] = [0.5, -0.5, 1.5, -2.5]  # ties round away from zero
    for gate in (0, 2, 3):
        c = edp_lib.net_centres_residual(torch.from_numpy(out).cuda(), torch.from_numpy(base).cuda(), space, gate)
        assert np.array_equal(c.cpu().numpy(), rnet.centres_residual(out.astype(np.float64), base, Q, gate))


def test_net_training_lowers_loss(edp_lib):
    rng = np.random.default_rng(9)
    N, H, W = 4, 32, 32
    x = torch.from_numpy(rng.uniform(-1, 1, size=(N, H, W, 5)).astype(np.float32)).to(torch.bfloat16).cuda()
    # target: a smooth function of the inputs the network can fit
    xf = x.float()
    tgt = torch.stack([3 * xf[..., 2] + xf[..., 0], -2 * xf[..., 3]], dim=-1).contiguous()
    P = torch.from_numpy(flat_params(rnet.init_params(2))).cuda()
    m, v = torch.zeros_like(P), torch.zeros_like(P)
    ws = edp_lib.net_workspace(N, H, W)
    losses = []
    for step in range(1, 61):
        out = edp_lib.net_forward(P, x, ws)
        g, loss = edp_lib.net_backward(P, out, tgt, ws)
        edp_lib.net_adam(P, g, m, v, 3e-3, step)
        losses.append(float(loss.item()))
    assert losses[-1] < 0.5 * losses[0]


def test_window_edge_count(edp_lib):
    rng = np.random.default_rng(12)
    Q = (17, 13)
    space = {"R": 2, "Q": (17, 13, 1), "vmin": (-8, -6, 0), "step": (1, 1, 1)}
    for win in (3, 5, 9):
        centre = np.stack([rng.integers(-3, 20, size=(37, 29)), rng.integers(-3, 16, size=(37, 29))], -1)
        h = (win - 1) // 2
        lo0 = np.clip(centre[..., 0], h, Q[0] - 1 - h) - h
        lo1 = np.clip(centre[..., 1], h, Q[1] - 1 - h) - h
        # labels inside each box, many on its edges
        l0 = lo0 + rng.integers(0, win, size=lo0.shape)
        l1 = lo1 + rng.integers(0, win, size=lo1.shape)
        lab = (l0 + Q[0] * l1).astype(np.int32)
        want = rnet.window_edge_count(lab, centre, win, Q)
        got = edp_lib.window_edge_count(torch.from_numpy(lab).cuda(),
                                        torch.from_numpy(centre.astype(np.int32)).cuda(), win, space)
        assert int(got.item()) == want
