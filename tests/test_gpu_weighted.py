"""GPU parity of the locally adaptive prior (per-edge multipliers of the
prior, the text below Eq. Smooth_value_t): edge weights, weighted EDP and
weighted energy against the oracle, bit for bit."""
import numpy as np
import pytest
import torch

import oracle
from paper_1410_7922_gb300 import synth

pytestmark = pytest.mark.gpu


def sp(Q):
    R = len(Q)
    return {"R": R, "Q": tuple(Q), "vmin": (0,) * R, "step": (1,) * R}


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def host(t):
    return t.cpu().numpy()


@pytest.fixture(autouse=True)
def reset(edp_lib):
    edp_lib.set_tuning(0, 0, 0)
    edp_lib.set_pass_pairs(edp_lib.PAIRS_AUTO)
    yield
    edp_lib.set_tuning(0, 0, 0)
    edp_lib.set_pass_pairs(edp_lib.PAIRS_AUTO)


@pytest.mark.parametrize("H,W", [(1, 1), (1, 17), (13, 1), (37, 45)])
@pytest.mark.parametrize("thresh,factor", [(10, 2), (0, 3), (256, 4)])
def test_edge_weights(edp_lib, H, W, thresh, factor):
    I = np.random.default_rng(H * 100 + W).integers(0, 256, size=(H, W)).astype(np.uint8)
    I[:, ::3] = I[:, :1]  # some equal neighbours
    wh, wv = edp_lib.edge_weights(dev(I), thresh, factor)
    owh, owv = oracle.edge_weights(I, thresh, factor)
    assert np.array_equal(host(wh), owh) and np.array_equal(host(wv), owv)


@pytest.mark.parametrize("Q", [7, 33, 64, 130, 256])
@pytest.mark.parametrize("iters", [1, 2])
@pytest.mark.parametrize("pairs", [False, True])
def test_weighted_edp_random(edp_lib, Q, iters, pairs):
    rng = np.random.default_rng(Q * 10 + iters + 100 * pairs)
    H, W = 19, 23
    C = rng.integers(0, 21, size=(H, W, Q)).astype(np.int32)
    wh = rng.integers(0, 4, size=(H, W)).astype(np.uint8)
    wv = rng.integers(0, 4, size=(H, W)).astype(np.uint8)
    prior = {"lam": int(rng.integers(1, 12)), "g": int(rng.integers(1, 6)), "l1": 1, "mode": "joint"}
    want = oracle.edp_weighted(C, sp((Q,)), prior, wh, wv, iters=iters)
    edp_lib.set_pass_pairs(pairs)
    edp_lib.set_tuning(3, 0, 0)
    got = host(edp_lib.solve_weighted(dev(C), sp((Q,)), prior, dev(wh), dev(wv), 3, iters=iters))
    assert np.array_equal(got, want)


@pytest.mark.parametrize("Q,mode", [((9, 9), "per_axis"), ((17, 9), "joint"), ((33, 33), "per_axis"),
                                    ((65, 65), "joint"), ((17, 17, 9), "per_axis")])
@pytest.mark.parametrize("pairs", [False, True])
def test_weighted_edp_whole_line_form(edp_lib, Q, mode, pairs):
    """Multi-axis spaces on the whole-line form of the multi-axis kernel."""
    rng = np.random.default_rng(sum(Q) * 7 + pairs)
    n = int(np.prod(Q))
    H, W = (9, 13) if n > 1000 else (15, 19)
    C = rng.integers(0, 21, size=(H, W, n)).astype(np.int32)
    wh = rng.integers(0, 4, size=(H, W)).astype(np.uint8)
    wv = rng.integers(0, 4, size=(H, W)).astype(np.uint8)
    prior = {"lam": int(rng.integers(1, 9)), "g": int(rng.integers(1, 5)), "l1": 1, "mode": mode}
    want = oracle.edp_weighted(C, sp(Q), prior, wh, wv, iters=2)
    edp_lib.set_pass_pairs(pairs)
    edp_lib.set_tuning(2, 0, 0)
    got = host(edp_lib.solve_weighted(dev(C), sp(Q), prior, dev(wh), dev(wv), 3, iters=2))
    assert np.array_equal(got, want)


@pytest.mark.parametrize("Q,g", [(16, 3), (64, 5)])
def test_weighted_edp_quadratic_prior(edp_lib, Q, g):
    rng = np.random.default_rng(Q + g)
    C = rng.integers(0, 40, size=(15, 21, Q)).astype(np.int32)
    wh = rng.integers(0, 3, size=(15, 21)).astype(np.uint8)
    wv = rng.integers(0, 3, size=(15, 21)).astype(np.uint8)
    prior = {"lam": 2, "g": g, "l1": 2, "mode": "joint"}
    want = oracle.edp_weighted(C, sp((Q,)), prior, wh, wv, iters=2)
    got = host(edp_lib.solve_weighted(dev(C), sp((Q,)), prior, dev(wh), dev(wv), 2, iters=2))
    assert np.array_equal(got, want)


def test_adaptive_prior_on_the_stereo_workload(edp_lib):
    """The paper's rule (2 lambda below an intensity step of 10) on the
    64x48 stereo stand-in: weights, labels and energy as the oracle."""
    w = synth.workload_scanline_64x48()
    I0, I1 = dev(w["I0"]), dev(w["I1"])
    C = edp_lib.cost_volume(I0, I1, None, w["space"], w["l2"], w["cmax"])
    wh, wv = edp_lib.edge_weights(I0, 10, 2)
    Cc = oracle.cost_volume(w["I0"], w["I1"], None, w["space"], w["l2"], w["cmax"])
    owh, owv = oracle.edge_weights(w["I0"], 10, 2)
    prior = dict(w["prior"], l1=1)
    want = oracle.edp_weighted(Cc, w["space"], prior, owh, owv, iters=2)
    got = edp_lib.solve_weighted(C, w["space"], prior, wh, wv, 2, iters=2)
    assert np.array_equal(host(got), want)
    e = host(edp_lib.energy_weighted(C, got, w["space"], prior, wh, wv))
    assert tuple(int(v) for v in e) == oracle.energy_weighted(Cc, want, w["space"], prior, owh, owv)


@pytest.mark.parametrize("Q,mode", [((9,), "joint"), ((5, 4), "per_axis"), ((3, 3, 2), "joint")])
def test_weighted_energy(edp_lib, Q, mode):
    rng = np.random.default_rng(int(np.prod(Q)))
    H, W = 17, 29
    n = int(np.prod(Q))
    C = rng.integers(0, 50, size=(H, W, n)).astype(np.int32)
    lab = rng.integers(0, n, size=(H, W)).astype(np.int32)
    wh = rng.integers(0, 5, size=(H, W)).astype(np.uint8)
    wv = rng.integers(0, 5, size=(H, W)).astype(np.uint8)
    prior = {"lam": 3, "g": 2, "l1": 1, "mode": mode}
    got = host(edp_lib.energy_weighted(dev(C), dev(lab), sp(Q), prior, dev(wh), dev(wv)))
    assert tuple(int(v) for v in got) == oracle.energy_weighted(C, lab, sp(Q), prior, wh, wv)


def test_weighted_unsupported_and_invalid(edp_lib):
    """The lane-group form of the multi-axis kernel (a 5x4 space) takes no weights."""
    C = torch.zeros((4, 5, 20), dtype=torch.int32, device="cuda")
    w = torch.ones((4, 5), dtype=torch.uint8, device="cuda")
    prior = {"lam": 2, "g": 2, "l1": 1, "mode": "per_axis"}
    with pytest.raises(RuntimeError, match="UNSUPPORTED"):
        edp_lib.solve_weighted(C, sp((5, 4)), prior, w, w, 1)
    with pytest.raises(RuntimeError, match="INVALID_ARG"):
        edp_lib.solve_weighted(C, sp((20,)), prior, w, w, 300)
