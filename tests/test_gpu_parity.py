"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle.

All arithmetic is integer, so labels, costs, row energies and energies must
match bit for bit.  Inputs are the seeded synthetic workloads and random cost
volumes (including tie-heavy ones), at sizes the oracle finishes in seconds
that still span several blocks, bands and a ragged tail; the full-size
450x375 stereo and 320x240 motion workloads run once each.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1410_7922_gb300 import synth

pytestmark = pytest.mark.gpu


def sp(Q, vmin=None, step=None):
    R = len(Q)
    return {"R": R, "Q": tuple(Q), "vmin": tuple(vmin or [0] * R), "step": tuple(step or [1] * R)}


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def host(t):
    return t.cpu().numpy()


@pytest.fixture(autouse=True)
def reset_tuning(edp_lib):
    edp_lib.set_tuning(0, 0, False)
    edp_lib.set_pass_pairs(edp_lib.PAIRS_AUTO)
    yield
    edp_lib.set_tuning(0, 0, False)
    edp_lib.set_pass_pairs(edp_lib.PAIRS_AUTO)


# --------------------------------------------------------------------------
# cost volume
# --------------------------------------------------------------------------

@pytest.mark.parametrize("case", [
    ("stereo", sp((16,), (0,), (-1,)), "pair", 1, 20),
    ("stereo_l2", sp((24,), (0,), (-1,)), "pair", 2, 900),
    ("motion", sp((9, 7), (-4, -3), (1, 1)), "pair", 1, 20),
    ("stereo3", sp((5, 5, 4), (-2, -2, 0), (1, 1, -1)), "pair_stereo3", 1, 30),
    ("composite", sp((12,), (0,), (1,)), "composite", 2, 400),
    ("composite2d", sp((5, 5), (-2, -2), (1, 1)), "composite", 1, 25),
])
def test_cost_volume_parity(edp_lib, case):
    name, space, mode, l2, cmax = case
    rng = np.random.default_rng(len(name))
    H, W = 37, 53
    I0, I1, I2 = (rng.integers(0, 256, size=(H, W)).astype(np.uint8) for _ in range(3))
    use2 = mode != "pair"
    want = oracle.cost_volume(I0, I1, I2 if use2 else None, space, l2, cmax, mode)
    got = edp_lib.cost_volume(dev(I0), dev(I1), dev(I2) if use2 else None, space, l2, cmax, mode)
    assert np.array_equal(host(got), want)


def test_cost_volume_pitched_rows(edp_lib):
    rng = np.random.default_rng(1)
    H, W, P = 20, 30, 48
    big0 = rng.integers(0, 256, size=(H, P)).astype(np.uint8)
    big1 = rng.integers(0, 256, size=(H, P)).astype(np.uint8)
    space = sp((8,), (0,), (-1,))
    want = oracle.cost_volume(big0[:, :W].copy(), big1[:, :W].copy(), None, space, 1, 20)
    t0, t1 = dev(big0), dev(big1)
    # the binding takes contiguous tensors; pass the pitched buffers through the C ABI directly
    import ctypes
    lib = edp_lib.load()
    out = torch.empty((H, W, 8), dtype=torch.int32, device="cuda")
    ls, pr = edp_lib.label_space(space), edp_lib.params({"lam": 0, "g": 1}, l2=1, cmax=20)
    rc = lib.edp_cost_volume(ctypes.c_void_p(t0.data_ptr()), ctypes.c_void_p(t1.data_ptr()), None, W, H, P,
                             ctypes.byref(ls), ctypes.byref(pr), ctypes.c_void_p(out.data_ptr()),
                             ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == 0
    assert np.array_equal(host(out), want)


@pytest.mark.parametrize("case", [
    ("motion_65x65", sp((65, 65), (-32, -32)), "pair", 1, 20),
    ("motion_9x7_steps", {"R": 2, "Q": (9, 7), "vmin": (4, -3), "step": (-1, 1)}, "pair", 1, 20),
    ("stereo_63", sp((63,), (-62,)), "pair", 1, 300),
    ("stereo_63_sq", sp((63,), (-62,)), "pair", 2, 3000),
    ("axis3", sp((5, 3, 3), (-2, -1, 0)), "pair_stereo3", 1, 40),
    ("composite", sp((7, 5), (-3, -2)), "composite", 1, 30),
])
@pytest.mark.parametrize("shift", [0, 1, 2, 3])
def test_cost_volume_vector_and_scalar_forms(edp_lib, case, shift):
    """The cost volume in each of its forms: one warp per pixel (the pair
    cost with 32 or more labels on axis 0, any output alignment: the 65 x 65
    and Q = 63 cases), four entries per thread (output 16-byte aligned,
    shift 0; odd Q puts pixel boundaries inside the 16-byte words) and one
    entry per thread (output shifted by 1..3 entries), on a frame whose
    borders cut the label windows; I1 also from a base that is not 4-byte
    aligned."""
    import ctypes
    name, space, mode, l2, cmax = case
    rng = np.random.default_rng(len(name) * 7 + shift)
    H, W, P = 19, 41, 45
    I0, I1, I2 = (rng.integers(0, 256, size=(H, P)).astype(np.uint8) for _ in range(3))
    use2 = mode != "pair"
    want = oracle.cost_volume(I0[:, :W].copy(), I1[:, :W].copy(), I2[:, :W].copy() if use2 else None, space,
                              l2, cmax, mode)
    Q = want.shape[2]
    lib = edp_lib.load()
    ls = edp_lib.label_space(space)
    pr = edp_lib.params({"lam": 0, "g": 1}, l2=l2, cmax=cmax, cost_mode=mode)
    t0, t2 = dev(I0), dev(I2)
    for i1_off in (0, 1):
        # I1 from a buffer one byte longer, the image at byte i1_off
        big1 = np.zeros(H * P + 1, np.uint8)
        big1[i1_off:i1_off + H * P] = I1.reshape(-1)
        t1 = dev(big1)
        buf = torch.full((H * W * Q + 4,), -7, dtype=torch.int32, device="cuda")
        rc = lib.edp_cost_volume(ctypes.c_void_p(t0.data_ptr()), ctypes.c_void_p(t1.data_ptr() + i1_off),
                                 ctypes.c_void_p(t2.data_ptr()) if use2 else None, W, H, P, ctypes.byref(ls),
                                 ctypes.byref(pr), ctypes.c_void_p(buf.data_ptr() + 4 * shift),
                                 ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
        assert rc == 0
        b = host(buf)
        assert np.array_equal(b[shift:shift + H * W * Q].reshape(H, W, Q), want), (name, shift, i1_off)
        assert (b[:shift] == -7).all() and (b[shift + H * W * Q:] == -7).all()


# --------------------------------------------------------------------------
# scanline DP
# --------------------------------------------------------------------------

def test_scanline_stereo_64x48(edp_lib):
    w = synth.workload_scanline_64x48()
    C = oracle.cost_volume(w["I0"], w["I1"], None, w["space"], w["l2"], w["cmax"])
    lab, row_e = oracle.scanline_dp(C, w["space"], w["prior"], tier=1)
    glab, grow = edp_lib.scanline_dp(dev(C), w["space"], w["prior"])
    assert np.array_equal(host(glab), lab)
    assert np.array_equal(host(grow), row_e)


@pytest.mark.parametrize("Q,mode", [((5,), "joint"), ((16,), "joint"), ((33,), "joint"), ((100,), "joint"),
                                    ((256,), "joint"), ((300,), "joint"), ((5, 4), "joint"),
                                    ((5, 4), "per_axis"), ((17, 17), "per_axis"), ((17, 17), "joint"),
                                    ((3, 3, 2), "per_axis"), ((4, 3, 5), "joint"), ((1,), "joint")])
def test_scanline_random(edp_lib, Q, mode):
    rng = np.random.default_rng(sum(Q) * 7 + len(mode))
    n = int(np.prod(Q))
    H, W = 13, 29
    for trial in range(2):
        hi = 4 if trial else 21  # trial 1: many ties
        C = rng.integers(0, hi, size=(H, W, n)).astype(np.int32)
        prior = {"lam": int(rng.integers(0, 9)), "g": int(rng.integers(1, 5)), "l1": 1, "mode": mode}
        lab, row_e = oracle.scanline_dp(C, sp(Q), prior, tier=1)
        glab, grow = edp_lib.scanline_dp(dev(C), sp(Q), prior)
        assert np.array_equal(host(grow), row_e), prior
        assert np.array_equal(host(glab), lab), prior


@pytest.mark.parametrize("Q", [(7,), (20,), (64,), (100,), (300,)])
@pytest.mark.parametrize("g", [1, 2, 3, 5])
def test_scanline_quadratic_prior(edp_lib, Q, g):
    """Truncated quadratic prior (l1 = 2, the taps of Eq. M_decmp) in the
    scanline DP on one label axis: labels and row energies against the
    oracle's definition tier, and the min-marginal mode, on random and
    tie-heavy costs (the lane-group shapes of 7 .. 300 labels)."""
    rng = np.random.default_rng(sum(Q) * 5 + g)
    n = int(np.prod(Q))
    H, W = 11, 23
    for hi in (30, 4):
        C = rng.integers(0, hi, size=(H, W, n)).astype(np.int32)
        prior = {"lam": int(rng.integers(1, 7)), "g": g, "l1": 2, "mode": "joint"}
        lab, row_e = oracle.scanline_dp(C, sp(Q), prior, tier=0)
        glab, grow = edp_lib.scanline_dp(dev(C), sp(Q), prior)
        assert np.array_equal(host(grow), row_e), prior
        assert np.array_equal(host(glab), lab), prior
        S = oracle.min_marginals(C, sp(Q), prior, tier=0)
        mlab, marg = edp_lib.scanline_marginals(dev(C), sp(Q), prior, marginals=True)
        assert np.array_equal(host(marg).astype(np.int64), S), prior
        assert np.array_equal(host(mlab), np.argmin(S, axis=2)), prior


@pytest.mark.parametrize("Q,mode", [((16,), "joint"), ((64,), "joint"), ((130,), "joint"), ((5, 4), "per_axis"),
                                    ((9, 9), "joint"), ((3, 4, 3), "per_axis")])
def test_scanline_min_marginals(edp_lib, Q, mode):
    """Min-marginal mode (Eq. DP_1D_3): S_Omega = M(F(x-1)) + C + M(B(x+1)) and
    its lowest-index argmin against the oracle, on random and tie-heavy costs."""
    rng = np.random.default_rng(sum(Q) * 3 + len(mode))
    n = int(np.prod(Q))
    H, W = 13, 29
    for hi in (21, 3):
        C = rng.integers(0, hi, size=(H, W, n)).astype(np.int32)
        prior = {"lam": int(rng.integers(0, 9)), "g": int(rng.integers(1, 5)), "l1": 1, "mode": mode}
        S = oracle.min_marginals(C, sp(Q), prior, tier=1)
        lab, marg = edp_lib.scanline_marginals(dev(C), sp(Q), prior, marginals=True)
        assert np.array_equal(host(marg).astype(np.int64), S), prior
        assert np.array_equal(host(lab), np.argmin(S, axis=2)), prior


@pytest.mark.parametrize("rb,e", [(1, 1), (3, 2), (7, 3), (2, 8), (5, 16)])
def test_scanline_launch_shapes(edp_lib, rb, e):
    rng = np.random.default_rng(rb * 10 + e)
    C = rng.integers(0, 15, size=(11, 23, 40)).astype(np.int32)
    prior = {"lam": 4, "g": 3, "l1": 1, "mode": "joint"}
    lab, row_e = oracle.scanline_dp(C, sp((40,)), prior, tier=1)
    edp_lib.set_tuning(rb, e, False)
    glab, grow = edp_lib.scanline_dp(dev(C), sp((40,)), prior)
    assert np.array_equal(host(glab), lab) and np.array_equal(host(grow), row_e)


# --------------------------------------------------------------------------
# EDP
# --------------------------------------------------------------------------

LINE_SHAPES = {(17, 17), (25, 25), (33, 33), (65, 65), (27, 15)}


def run_edp(edp_lib, C, space, prior, iters):
    """The oracle's labels and the GPU's.  Two-axis spaces the line kernels
    are built for also run on every other two-axis kernel (multi-axis, line
    with split lines, line with one lane per line; the same labels are
    asserted here)."""
    want = oracle.edp(C, space, prior, iters=iters, tier=1)
    got = host(edp_lib.solve(dev(C), space, prior, iters=iters))
    if tuple(space["Q"][:space["R"]]) in LINE_SHAPES and prior.get("l1", 1) == 1:
        ran = {edp_lib.last_pass_kernel()}
        try:
            for general in (3, 4, 5):
                edp_lib.set_tuning(0, 0, general)
                other = host(edp_lib.solve(dev(C), space, prior, iters=iters))
                ran.add(edp_lib.last_pass_kernel())
                assert np.array_equal(other, want), edp_lib.last_pass_kernel()
        finally:
            edp_lib.set_tuning(0, 0, 0)
        assert len(ran) >= 2, ran
    return want, got


@pytest.mark.parametrize("Q,mode", [((7,), "joint"), ((64,), "joint"), ((33,), "joint"), ((130,), "joint"),
                                    ((5, 4), "per_axis"), ((5, 4), "joint"), ((9, 9), "per_axis"),
                                    ((33, 33), "per_axis"), ((33, 33), "joint"), ((17, 9), "per_axis"),
                                    ((17, 17, 9), "joint"), ((9, 9, 9), "per_axis"), ((65, 65), "per_axis"),
                                    ((65, 65), "joint"), ((3, 4, 3), "joint"),
                                    ((5, 5, 3), "per_axis"), ((1,), "joint")])
@pytest.mark.parametrize("iters", [1, 2])
def test_edp_random(edp_lib, Q, mode, iters):
    rng = np.random.default_rng(sum(Q) * 13 + iters)
    n = int(np.prod(Q))
    H, W = (9, 14) if n > 500 else (17, 23)
    for hi in (21, 3):
        C = rng.integers(0, hi, size=(H, W, n)).astype(np.int32)
        prior = {"lam": int(rng.integers(1, 12)), "g": int(rng.integers(1, 5)), "l1": 1, "mode": mode}
        want, got = run_edp(edp_lib, C, sp(Q), prior, iters)
        assert np.array_equal(got, want), (prior, hi)


@pytest.mark.parametrize("W,H", [(1, 1), (1, 9), (9, 1), (2, 2), (3, 50), (50, 3), (7, 33)])
@pytest.mark.parametrize("general", [False, True])
def test_edp_degenerate_shapes(edp_lib, W, H, general):
    rng = np.random.default_rng(W * 100 + H)
    C = rng.integers(0, 20, size=(H, W, 6)).astype(np.int32)
    prior = {"lam": 5, "g": 2, "l1": 1, "mode": "joint"}
    edp_lib.set_tuning(0, 0, general)
    for iters in (1, 3):
        want, got = run_edp(edp_lib, C, sp((6,)), prior, iters)
        assert np.array_equal(got, want)


@pytest.mark.parametrize("Q,mode", [((7,), "joint"), ((5, 4), "per_axis"), ((9, 9), "joint")])
def test_edp_sixteen_iterations(edp_lib, Q, mode):
    """Long runs of Algorithm 1 (j = 16): later iterations read all four
    message arrays and the sums keep growing."""
    rng = np.random.default_rng(sum(Q) + 16)
    C = rng.integers(0, 21, size=(11, 13, int(np.prod(Q)))).astype(np.int32)
    prior = {"lam": 7, "g": 3, "l1": 1, "mode": mode}
    want, got = run_edp(edp_lib, C, sp(Q), prior, 16)
    assert np.array_equal(got, want)


@pytest.mark.parametrize("Q,mode", [((7,), "joint"), ((64,), "joint"), ((100,), "joint"), ((9, 9), "joint"),
                                    ((9, 9), "per_axis"), ((17, 9), "per_axis"), ((33, 33), "joint"),
                                    ((17, 17, 9), "per_axis"), ((65, 65), "per_axis"), ((27, 15), "per_axis"),
                                    ((27, 15), "joint"), ((25, 25), "per_axis")])
@pytest.mark.parametrize("g", [1, 2, 3, 5])
def test_edp_quadratic_prior(edp_lib, Q, mode, g):
    """Truncated quadratic prior (l1 = 2, the generalized RMS of Eq. M_decmp)
    against the oracle's GRMS tier."""
    rng = np.random.default_rng(sum(Q) * 7 + g)
    n = int(np.prod(Q))
    H, W = (6, 9) if n > 500 else (13, 17)
    C = rng.integers(0, 30, size=(H, W, n)).astype(np.int32)
    prior = {"lam": int(rng.integers(1, 6)), "g": g, "l1": 2, "mode": mode}
    for iters in (1, 2):
        want, got = run_edp(edp_lib, C, sp(Q), prior, iters)
        assert np.array_equal(got, want), (prior, iters)


def test_quadratic_prior_unsupported_shapes(edp_lib):
    """Lines the quadratic taps are not built for say so."""
    C = torch.zeros((4, 5, 20), dtype=torch.int32, device="cuda")
    prior = {"lam": 2, "g": 3, "l1": 2, "mode": "joint"}
    with pytest.raises(edp_lib.EdpError) as e:
        edp_lib.solve(C, sp((5, 4)), prior)
    assert e.value.code == edp_lib.ERR_UNSUPPORTED
    with pytest.raises(edp_lib.EdpError) as e:
        edp_lib.scanline_dp(C, sp((5, 4)), prior)
    assert e.value.code == edp_lib.ERR_UNSUPPORTED


@pytest.mark.parametrize("W,H", [(1, 1), (1, 9), (9, 1), (2, 2), (3, 50), (50, 3)])
@pytest.mark.parametrize("form", [0, 2])
def test_edp_degenerate_shapes_two_axes(edp_lib, W, H, form):
    """Image shapes at the edges of the wavefront, both forms of the
    multi-axis kernel."""
    rng = np.random.default_rng(W * 1000 + H)
    C = rng.integers(0, 20, size=(H, W, 12)).astype(np.int32)
    for mode in ("joint", "per_axis"):
        prior = {"lam": 4, "g": 2, "l1": 1, "mode": mode}
        edp_lib.set_tuning(0, 0, form)
        for iters in (1, 3):
            want, got = run_edp(edp_lib, C, sp((4, 3)), prior, iters)
            assert np.array_equal(got, want), (mode, iters)


@pytest.mark.parametrize("Q", [1, 5, 16, 31, 32, 33, 64, 100, 129, 256])
@pytest.mark.parametrize("g", [1, 2, 4, 9, 300])
def test_edp_one_axis_kernel(edp_lib, Q, g):
    """The warp-per-row kernel: label counts around the lane boundaries and
    truncations from 1 (no carries) to untruncated."""
    rng = np.random.default_rng(Q * 1000 + g)
    C = rng.integers(0, 21, size=(19, 27, Q)).astype(np.int32)
    prior = {"lam": int(rng.integers(1, 25)), "g": g, "l1": 1, "mode": "joint"}
    want, got = run_edp(edp_lib, C, sp((Q,)), prior, 2)
    assert np.array_equal(got, want)


@pytest.mark.parametrize("rows", [2, 3, 5, 8, 16])
def test_edp_one_axis_rows_per_block(edp_lib, rows):
    rng = np.random.default_rng(rows)
    C = rng.integers(0, 21, size=(37, 41, 64)).astype(np.int32)
    prior = {"lam": 20, "g": 4, "l1": 1, "mode": "joint"}
    want = oracle.edp(C, sp((64,)), prior, iters=2, tier=1)
    edp_lib.set_tuning(rows, 0, False)
    got = host(edp_lib.solve(dev(C), sp((64,)), prior, iters=2))
    assert np.array_equal(got, want)


@pytest.mark.parametrize("pairs", [False, True])
@pytest.mark.parametrize("Q,W,H,rows", [(64, 41, 37, 2), (64, 41, 37, 8), (7, 5, 23, 3), (33, 1, 9, 2),
                                        (100, 9, 1, 2), (130, 30, 17, 5)])
@pytest.mark.parametrize("iters", [1, 3])
def test_edp_pass_schedule(edp_lib, pairs, Q, W, H, rows, iters):
    """Paired sweeps (P1 + P2, P3 + P4 in one launch each) and one launch per
    pass give the oracle's labels: the schedule never changes a value."""
    rng = np.random.default_rng(Q * 7 + W + H + iters)
    C = rng.integers(0, 21, size=(H, W, Q)).astype(np.int32)
    prior = {"lam": int(rng.integers(1, 25)), "g": 4, "l1": 1, "mode": "joint"}
    want = oracle.edp(C, sp((Q,)), prior, iters=iters, tier=1)
    edp_lib.set_pass_pairs(pairs)
    edp_lib.set_tuning(rows, 0, False)
    got = host(edp_lib.solve(dev(C), sp((Q,)), prior, iters=iters))
    assert edp_lib.last_pass_launches() == (2 if pairs else 4) * iters
    assert np.array_equal(got, want)


@pytest.mark.parametrize("pairs", [False, True])
@pytest.mark.parametrize("Q,mode,form", [((9, 9), "per_axis", 0), ((33, 33), "joint", 0), ((17, 9), "per_axis", 0),
                                         ((5, 4), "per_axis", 2), ((17, 17, 9), "joint", 0),
                                         ((5, 5, 3), "per_axis", 2), ((16,), "joint", 1)])
@pytest.mark.parametrize("iters", [1, 3])
def test_edp_pass_schedule_multi_axis(edp_lib, pairs, Q, mode, form, iters):
    """The multi-axis kernel (whole-line form 0, lane-group form 2, one-axis
    spaces on it with form 1) under both schedules, with bands spanning
    several blocks and teams (2 rows per block)."""
    rng = np.random.default_rng(sum(Q) * 11 + form + iters)
    n = int(np.prod(Q))
    H, W = (11, 13) if n > 500 else (19, 25)
    C = rng.integers(0, 21, size=(H, W, n)).astype(np.int32)
    prior = {"lam": int(rng.integers(1, 12)), "g": int(rng.integers(1, 5)), "l1": 1, "mode": mode}
    want = oracle.edp(C, sp(Q), prior, iters=iters, tier=1)
    edp_lib.set_pass_pairs(pairs)
    edp_lib.set_tuning(2, 0, form)
    got = host(edp_lib.solve(dev(C), sp(Q), prior, iters=iters))
    assert np.array_equal(got, want)


@pytest.mark.parametrize("mode", [0, 1, 2])
@pytest.mark.parametrize("Q,mode_prior", [((16,), "joint"), ((5, 4), "per_axis"), ((9, 9), "per_axis")])
def test_edp_pass_schedule_many_bands(edp_lib, mode, Q, mode_prior):
    """More row bands than blocks can be resident at once (12000 rows, 2 per
    block, more than 152 SMs x 32 blocks): the automatic schedule falls back to
    one launch per pass, a forced pairing holds each block for a paired band;
    every schedule gives the oracle's labels."""
    rng = np.random.default_rng(sum(Q) + mode)
    H, W = 12000, 3
    n = int(np.prod(Q))
    C = rng.integers(0, 21, size=(H, W, n)).astype(np.int32)
    prior = {"lam": int(rng.integers(1, 12)), "g": 3, "l1": 1, "mode": mode_prior}
    want = oracle.edp(C, sp(Q), prior, iters=2, tier=1)
    edp_lib.set_pass_pairs(mode)
    edp_lib.set_tuning(2, 0, 0)
    got = host(edp_lib.solve(dev(C), sp(Q), prior, iters=2))
    launches = edp_lib.last_pass_launches()
    assert np.array_equal(got, want)
    assert launches == (4 if mode == 1 else 8)


@pytest.mark.parametrize("pairs", [False, True])
@pytest.mark.parametrize("Q,win,l1", [((13, 13), 5, 1), ((11,), 7, 1), ((13, 13), 5, 2)])
def test_windowed_pass_schedule(edp_lib, pairs, Q, win, l1):
    rng = np.random.default_rng(sum(Q) + win + l1)
    H, W = 13, 19
    R = len(Q)
    space = sp(Q, [-(q // 2) for q in Q], [1] * R)
    I0 = rng.integers(0, 256, size=(H, W)).astype(np.uint8)
    I1 = rng.integers(0, 256, size=(H, W)).astype(np.uint8)
    centre = np.stack([rng.integers(-2, q + 2, size=(H, W)) for q in Q], axis=-1).astype(np.int32)
    prior = {"lam": int(rng.integers(2, 9)), "g": 3, "l1": l1, "mode": "per_axis"}
    Cw = oracle.cost_window(I0, I1, None, space, 1, 30, centre, win)
    want = oracle.edp_windowed(Cw, centre, space, prior, win, iters=2)
    edp_lib.set_pass_pairs(pairs)
    edp_lib.set_tuning(3, 0, 0)
    got = edp_lib.solve_windowed(dev(Cw), dev(centre), win, space, prior, iters=2)
    assert np.array_equal(host(got), want)


@pytest.mark.parametrize("form", [1, 2])
@pytest.mark.parametrize("rb,t", [(1, 1), (2, 2), (3, 4), (6, 3), (4, 8), (1, 12), (15, 1)])
def test_edp_launch_shapes(edp_lib, rb, t, form):
    """Results never depend on the launch shape of the multi-axis kernel
    (rows per block, warps per row) nor on its form (whole lines per lane /
    lane groups)."""
    rng = np.random.default_rng(rb * 31 + t)
    for Q, mode in (((24,), "joint"), ((7, 6), "per_axis"), ((7, 6), "joint"), ((33, 33), "joint"),
                    ((5, 4, 3), "per_axis")):
        n = int(np.prod(Q))
        H, W = (7, 11) if n > 500 else (21, 19)
        C = rng.integers(0, 21, size=(H, W, n)).astype(np.int32)
        prior = {"lam": 6, "g": 3, "l1": 1, "mode": mode}
        want = oracle.edp(C, sp(Q), prior, iters=2, tier=1)
        edp_lib.set_tuning(rb, 0, form, warps_per_row=t)
        got = host(edp_lib.solve(dev(C), sp(Q), prior, iters=2))
        assert np.array_equal(got, want), (Q, mode, rb, t, form)


def test_edp_stereo_450x375_full_size(edp_lib):
    """The full Cones-sized stereo workload (Q = 64), j = 1 and j = 6."""
    w = synth.workload_stereo_450x375()
    C = oracle.cost_volume(w["I0"], w["I1"], None, w["space"], w["l2"], w["cmax"])
    gC = edp_lib.cost_volume(dev(w["I0"]), dev(w["I1"]), None, w["space"], w["l2"], w["cmax"])
    assert np.array_equal(host(gC), C)
    for iters in (1, 6):
        want = oracle.edp(C, w["space"], w["prior"], iters=iters, tier=1)
        got = edp_lib.solve(gC, w["space"], w["prior"], iters=iters)
        assert np.array_equal(host(got), want), iters
        e_want = oracle.energy(C, want, w["space"], w["prior"])
        e_got = tuple(int(v) for v in host(edp_lib.energy(gC, got, w["space"], w["prior"])))
        assert e_got == e_want


def test_edp_motion_320x240_full_size(edp_lib):
    """The full 320x240 motion workload, 33x33 labels, per-axis prior."""
    w = synth.workload_motion_320x240()
    C = oracle.cost_volume(w["I0"], w["I1"], None, w["space"], w["l2"], w["cmax"])
    gC = edp_lib.cost_volume(dev(w["I0"]), dev(w["I1"]), None, w["space"], w["l2"], w["cmax"])
    assert np.array_equal(host(gC), C)
    want = oracle.edp(C, w["space"], w["prior"], iters=1, tier=1)
    got = edp_lib.solve(gC, w["space"], w["prior"], iters=1)
    assert np.array_equal(host(got), want)


def test_edp_motion_joint_crop(edp_lib):
    w = synth.workload_motion_320x240(W=96, H=64, mode="joint")
    C = oracle.cost_volume(w["I0"], w["I1"], None, w["space"], w["l2"], w["cmax"])
    want, got = run_edp(edp_lib, C, w["space"], w["prior"], 2)
    assert np.array_equal(got, want)


# --------------------------------------------------------------------------
# energy and the image-level entry points
# --------------------------------------------------------------------------

@pytest.mark.parametrize("Q,mode,l1", [((16,), "joint", 1), ((6, 5), "per_axis", 1), ((6, 5), "joint", 2),
                                       ((3, 3, 3), "per_axis", 2)])
def test_energy_parity(edp_lib, Q, mode, l1):
    rng = np.random.default_rng(3)
    n = int(np.prod(Q))
    C = rng.integers(0, 50, size=(31, 47, n)).astype(np.int32)
    lab = rng.integers(0, n, size=(31, 47)).astype(np.int32)
    prior = {"lam": 7, "g": 2, "l1": l1, "mode": mode}
    want = oracle.energy(C, lab, sp(Q), prior)
    got = tuple(int(v) for v in host(edp_lib.energy(dev(C), dev(lab), sp(Q), prior)))
    assert got == want


def test_solve_images_device_and_host(edp_lib):
    w = synth.workload_stereo_450x375(W=120, H=90)
    C = oracle.cost_volume(w["I0"], w["I1"], None, w["space"], w["l2"], w["cmax"])
    want = oracle.edp(C, w["space"], w["prior"], iters=2, tier=1)
    e_want = oracle.energy(C, want, w["space"], w["prior"])
    lab, e = edp_lib.solve_images(dev(w["I0"]), dev(w["I1"]), None, w["space"], w["prior"], w["l2"], w["cmax"],
                                  iters=2)
    assert np.array_equal(host(lab), want)
    assert tuple(int(v) for v in host(e)) == e_want
    ws = edp_lib.workspace(edp_lib.OP_SOLVE_IMAGES, 120, 90, w["space"], w["prior"], 2)
    hl, he = edp_lib.solve_images_host(w["I0"], w["I1"], None, w["space"], w["prior"], w["l2"], w["cmax"], ws,
                                       iters=2)
    assert np.array_equal(hl, want) and tuple(int(v) for v in he) == e_want
    assert edp_lib.get_device_status(ws) == 0


@pytest.mark.parametrize("W,H,iters", [(10, 24, 1), (7, 33, 2)])
def test_solve_images_fused_cost_65x65(edp_lib, W, H, iters):
    """edp_solve_images on a 65 x 65 motion space (the split line kernel):
    with the pair cost computed from the images inside the scan passes and
    the energy, and with the cost volume built first (the default); both
    equal the oracle's labels and energy.  Also through the C ABI with
    pitched image rows (pitch > W), and through the host entry point, both
    fused."""
    import ctypes
    w = synth.workload_motion_640x480(W=W, H=H)
    C = oracle.cost_volume(w["I0"], w["I1"], None, w["space"], w["l2"], w["cmax"])
    want = oracle.edp(C, w["space"], w["prior"], iters=iters, tier=1)
    e_want = oracle.energy(C, want, w["space"], w["prior"])
    try:
        for fused in (True, False):
            edp_lib.set_fused_cost(fused)
            lab, e = edp_lib.solve_images(dev(w["I0"]), dev(w["I1"]), None, w["space"], w["prior"], w["l2"],
                                          w["cmax"], iters=iters)
            assert edp_lib.last_pass_kernel() == "edp_pass_line2_kernel"
            assert np.array_equal(host(lab), want), fused
            assert tuple(int(v) for v in host(e)) == e_want, fused
        edp_lib.set_fused_cost(True)
        # pitched rows: the images inside wider buffers
        P = W + 5
        big0 = np.zeros((H, P), np.uint8)
        big1 = np.full((H, P), 255, np.uint8)
        big0[:, :W], big1[:, :W] = w["I0"], w["I1"]
        t0, t1 = dev(big0), dev(big1)
        ws = edp_lib.workspace(edp_lib.OP_SOLVE_IMAGES, W, H, w["space"], w["prior"], iters)
        lab = torch.empty((H, W), dtype=torch.int32, device="cuda")
        e4 = torch.empty(4, dtype=torch.int64, device="cuda")
        ls = edp_lib.label_space(w["space"])
        pr = edp_lib.params(w["prior"], l2=w["l2"], cmax=w["cmax"], iters=iters)
        rc = edp_lib.load().edp_solve_images(ctypes.c_void_p(t0.data_ptr()), ctypes.c_void_p(t1.data_ptr()), None,
                                             W, H, P, ctypes.byref(ls), ctypes.byref(pr),
                                             ctypes.c_void_p(lab.data_ptr()), ctypes.c_void_p(e4.data_ptr()),
                                             ctypes.c_void_p(ws.data_ptr()), ws.numel(),
                                             ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
        assert rc == 0
        assert np.array_equal(host(lab), want)
        assert tuple(int(v) for v in host(e4)) == e_want
        hl, he = edp_lib.solve_images_host(w["I0"], w["I1"], None, w["space"], w["prior"], w["l2"], w["cmax"], ws,
                                           iters=iters)
        assert np.array_equal(hl, want) and tuple(int(v) for v in he) == e_want
        assert edp_lib.get_device_status(ws) == 0
    finally:
        edp_lib.set_fused_cost(False)


def test_solve_images_fused_cost_full_frame(edp_lib):
    """The 640x480 frame with 65 x 65 labels (the bench's launch shape):
    fused and unfused solves give the same labels and energy."""
    w = synth.workload_motion_640x480()
    I0, I1 = dev(w["I0"]), dev(w["I1"])
    try:
        out = {}
        for fused in (True, False):
            edp_lib.set_fused_cost(fused)
            lab, e = edp_lib.solve_images(I0, I1, None, w["space"], w["prior"], w["l2"], w["cmax"], iters=1)
            out[fused] = (host(lab), tuple(int(v) for v in host(e)))
        assert np.array_equal(out[True][0], out[False][0])
        assert out[True][1] == out[False][1]
    finally:
        edp_lib.set_fused_cost(False)


def test_range_and_argument_errors(edp_lib):
    C = torch.zeros((4, 4, 8), dtype=torch.int32, device="cuda")
    with pytest.raises(edp_lib.EdpError) as ei:
        edp_lib.solve(C, sp((8,)), {"lam": 2**21, "g": 1, "l1": 1, "mode": "joint"})
    assert ei.value.code == edp_lib.ERR_RANGE
    with pytest.raises(edp_lib.EdpError) as ei:  # quadratic taps: not built for 5 x 4 lines
        edp_lib.solve(torch.zeros((4, 4, 20), dtype=torch.int32, device="cuda"), sp((5, 4)),
                      {"lam": 1, "g": 2, "l1": 2, "mode": "joint"})
    assert ei.value.code == edp_lib.ERR_UNSUPPORTED
    ws = torch.empty(1024, dtype=torch.uint8, device="cuda")
    with pytest.raises(edp_lib.EdpError) as ei:
        edp_lib.solve(C, sp((8,)), {"lam": 1, "g": 2}, ws=ws)
    assert ei.value.code == edp_lib.ERR_WORKSPACE


# --------------------------------------------------------------------------
# batched persistent solve
# --------------------------------------------------------------------------

def _batch_items(edp_lib, scale=0.12, n=9, iters=1):
    items = []
    for w in synth.workload_batch(n_pairs=n, scale=scale):
        H, W = w["I0"].shape
        it = dict(w)
        it["I0"], it["I1"] = dev(w["I0"]), dev(w["I1"])
        it["I2"] = dev(w["I2"]) if w["I2"] is not None else None
        it["labels"] = torch.empty((H, W), dtype=torch.int32, device="cuda")
        it["energy4"] = torch.empty(4, dtype=torch.int64, device="cuda")
        it["iters"] = iters
        it["_w"] = w
        items.append(it)
    return items


def _oracle_problem(w, iters):
    C = oracle.cost_volume(w["I0"], w["I1"], w["I2"], w["space"], w["l2"], w["cmax"], w["cost_mode"])
    lab = oracle.edp(C, w["space"], w["prior"], iters=iters, tier=1)
    return lab, oracle.energy(C, lab, w["space"], w["prior"])


@pytest.mark.parametrize("pairs", [False, True])
@pytest.mark.parametrize("iters", [1, 2])
def test_batched_matches_oracle(edp_lib, iters, pairs):
    """Every body of the batched kernel, one pass per work item or paired sweeps."""
    edp_lib.set_pass_pairs(pairs)
    items = _batch_items(edp_lib, iters=iters)
    probs = edp_lib.make_problems(items)
    ws = torch.empty(edp_lib.batch_workspace_size(probs), dtype=torch.uint8, device="cuda")
    edp_lib.solve_batched(probs, ws)
    torch.cuda.synchronize()
    assert edp_lib.get_device_status(ws) == 0
    for it in items:
        lab, e = _oracle_problem(it["_w"], iters)
        assert np.array_equal(host(it["labels"]), lab), it["name"]
        assert tuple(int(v) for v in host(it["energy4"])) == e, it["name"]


def test_batched_waves_and_replay(edp_lib):
    """A workspace too small for all problems runs them in waves; a second
    call on the same workspace gives the same result."""
    items = _batch_items(edp_lib, n=6)
    probs = edp_lib.make_problems(items)
    full = edp_lib.batch_workspace_size(probs)
    big = max(edp_lib.batch_workspace_size(edp_lib.make_problems([it])) for it in items)
    ws = torch.empty(max(big, full // 3), dtype=torch.uint8, device="cuda")
    for _ in range(2):
        for it in items:
            it["labels"].fill_(-1)
        edp_lib.solve_batched(probs, ws)
        torch.cuda.synchronize()
        for it in items:
            lab, e = _oracle_problem(it["_w"], 1)
            assert np.array_equal(host(it["labels"]), lab), it["name"]
            assert tuple(int(v) for v in host(it["energy4"])) == e


# --------------------------------------------------------------------------
# windowed EDP (per-pixel label boxes)
# --------------------------------------------------------------------------

@pytest.mark.parametrize("Q,win,mode,l1", [((13, 13), 5, "per_axis", 1), ((13, 13), 5, "joint", 1),
                                           ((11, 9), 9, "per_axis", 1), ((20,), 7, "joint", 1), ((9, 9), 9, "joint", 1),
                                           ((17, 17), 15, "per_axis", 1), ((13, 13), 5, "per_axis", 2),
                                           ((13, 13), 7, "joint", 2), ((20,), 7, "joint", 2), ((17, 17), 9, "per_axis", 2)])
@pytest.mark.parametrize("iters", [1, 2])
def test_windowed_matches_oracle(edp_lib, Q, win, mode, l1, iters):
    rng = np.random.default_rng(sum(Q) * 10 + win + iters)
    H, W = 15, 21
    R = len(Q)
    space = sp(Q, [-(q // 2) for q in Q], [1] * R)
    I0 = rng.integers(0, 256, size=(H, W)).astype(np.uint8)
    I1 = rng.integers(0, 256, size=(H, W)).astype(np.uint8)
    # centres: a smooth field plus jumps, some outside the valid range (clamped)
    centre = np.stack([rng.integers(-2, q + 2, size=(H, W)) for q in Q], axis=-1).astype(np.int32)
    prior = {"lam": int(rng.integers(2, 9)), "g": 3, "l1": l1, "mode": mode}
    Cw = oracle.cost_window(I0, I1, None, space, 1, 30, centre, win)
    gCw = edp_lib.cost_window(dev(I0), dev(I1), None, space, 1, 30, dev(centre), win)
    assert np.array_equal(host(gCw), Cw)
    want = oracle.edp_windowed(Cw, centre, space, prior, win, iters=iters)
    got = edp_lib.solve_windowed(gCw, dev(centre), win, space, prior, iters=iters)
    assert np.array_equal(host(got), want)


def test_windowed_full_box_equals_full_edp(edp_lib):
    rng = np.random.default_rng(77)
    Q = (9, 9)
    space = sp(Q, (-4, -4), (1, 1))
    H, W = 23, 29
    I0 = rng.integers(0, 256, size=(H, W)).astype(np.uint8)
    I1 = rng.integers(0, 256, size=(H, W)).astype(np.uint8)
    prior = {"lam": 6, "g": 3, "l1": 1, "mode": "per_axis"}
    centre = np.full((H, W, 2), 4, np.int32)
    C = edp_lib.cost_volume(dev(I0), dev(I1), None, space, 1, 25)
    full = host(edp_lib.solve(C, space, prior, iters=2))
    Cw = edp_lib.cost_window(dev(I0), dev(I1), None, space, 1, 25, dev(centre), 9)
    assert np.array_equal(host(Cw), host(C))
    win = host(edp_lib.solve_windowed(Cw, dev(centre), 9, space, prior, iters=2))
    assert np.array_equal(win, full)
