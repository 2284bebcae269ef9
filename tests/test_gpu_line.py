"""GPU parity of the two-axis line kernels against the oracle: one label
line per lane, and (65 x 65 labels) each line split over two lanes.
Random and tie-heavy costs, both truncations, several iterations, every
rows-per-block shape and both pass schedules, per-edge prior multipliers,
and the 480-row schedule of the 640x480 workload.  All arithmetic is
integer: labels and energies must match bit for bit."""
import numpy as np
import pytest
import torch

import oracle
from paper_1410_7922_gb300 import synth

pytestmark = pytest.mark.gpu

# the label-space shapes the line kernel is built for (Q0, Q1)
LINE_SHAPES = [(17, 17), (25, 25), (33, 33), (65, 65), (27, 15)]


def sp(Q, vmin=None):
    R = len(Q)
    return {"R": R, "Q": tuple(Q), "vmin": tuple(vmin or [0] * R), "step": (1,) * R}


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


LINE = 4  # general_kernel value: the line kernel wherever it is built
ONE_LANE = 5  # the same, with one lane per label line also at 65 x 65
LINE1, LINE2 = "edp_pass_line_kernel", "edp_pass_line2_kernel"


def kernel_for(Q, general=LINE):
    """The kernel the planner picks for a two-axis shape under `general`."""
    return LINE2 if tuple(Q) == (65, 65) and general == LINE else LINE1


@pytest.fixture(autouse=True)
def reset_tuning(edp_lib):
    edp_lib.set_tuning(0, 0, LINE)
    edp_lib.set_pass_pairs(edp_lib.PAIRS_AUTO)
    yield
    edp_lib.set_tuning(0, 0, 0)
    edp_lib.set_pass_pairs(edp_lib.PAIRS_AUTO)


SHAPE_FORMS = [(Q, LINE) for Q in LINE_SHAPES] + [((65, 65), ONE_LANE)]


@pytest.mark.parametrize("Q,general", SHAPE_FORMS)
@pytest.mark.parametrize("mode", ["per_axis", "joint"])
@pytest.mark.parametrize("iters", [1, 2])
def test_line_kernel_random(edp_lib, Q, general, mode, iters):
    rng = np.random.default_rng(Q[0] * 31 + Q[1] + iters + (mode == "joint"))
    n = Q[0] * Q[1]
    H, W = (11, 9) if n > 2000 else (17, 13)
    edp_lib.set_tuning(0, 0, general)
    for hi in (21, 3):  # 3: tie-heavy
        C = rng.integers(0, hi, size=(H, W, n)).astype(np.int32)
        prior = {"lam": int(rng.integers(1, 12)), "g": int(rng.integers(1, 6)), "l1": 1, "mode": mode}
        want = oracle.edp(C, sp(Q), prior, iters=iters, tier=1)
        got = edp_lib.solve(dev(C), sp(Q), prior, iters=iters).cpu().numpy()
        assert edp_lib.last_pass_kernel() == kernel_for(Q, general)
        assert np.array_equal(got, want), (prior, hi)


@pytest.mark.parametrize("rows", [1, 2, 3, 4])
@pytest.mark.parametrize("pairs", [0, 1])
def test_split_kernel_rows_per_block_and_schedule(edp_lib, rows, pairs):
    """The split form (65 x 65): rows per block 1..4 (hand-offs through the
    shared-memory mailbox and through the published value ring between
    blocks) under both pass schedules, a ragged last band, two iterations,
    large and small lambda."""
    rng = np.random.default_rng(rows * 11 + pairs)
    H, W = 23, 6
    C = rng.integers(0, 21, size=(H, W, 65 * 65)).astype(np.int32)
    for prior in ({"lam": 9, "g": 3, "l1": 1, "mode": "per_axis"}, {"lam": 1, "g": 40, "l1": 1, "mode": "joint"}):
        want = oracle.edp(C, sp((65, 65)), prior, iters=2, tier=1)
        edp_lib.set_tuning(rows, 0, LINE)
        edp_lib.set_pass_pairs(pairs)
        got = edp_lib.solve(dev(C), sp((65, 65)), prior, iters=2).cpu().numpy()
        assert edp_lib.last_pass_kernel() == LINE2
        assert edp_lib.last_pass_launches() == (2 if pairs else 4) * 2
        assert np.array_equal(got, want), prior


@pytest.mark.parametrize("W,H", [(1, 1), (1, 7), (7, 1), (2, 2), (3, 19)])
def test_split_kernel_degenerate_shapes(edp_lib, W, H):
    """The split form on degenerate frames: one pixel, one column, one row
    (a single band, no hand-off), and a ragged narrow strip."""
    rng = np.random.default_rng(W * 100 + H + 7)
    C = rng.integers(0, 20, size=(H, W, 65 * 65)).astype(np.int32)
    for mode in ("joint", "per_axis"):
        prior = {"lam": 4, "g": 3, "l1": 1, "mode": mode}
        for iters in (1, 2):
            want = oracle.edp(C, sp((65, 65)), prior, iters=iters, tier=1)
            got = edp_lib.solve(dev(C), sp((65, 65)), prior, iters=iters).cpu().numpy()
            assert edp_lib.last_pass_kernel() == LINE2
            assert np.array_equal(got, want), (mode, iters)


def test_split_kernel_lambda_bound(edp_lib):
    """Above the split form's lambda bound the planner takes the one-lane
    form; both equal the oracle."""
    rng = np.random.default_rng(3)
    H, W = 5, 4
    C = rng.integers(0, 1000, size=(H, W, 65 * 65)).astype(np.int32)
    for lam, kern in ((2 ** 30 // (34 * 255), LINE2), (2 ** 30 // (34 * 255) + 1, LINE1)):
        prior = {"lam": lam, "g": 1, "l1": 1, "mode": "per_axis"}
        want = oracle.edp(C, sp((65, 65)), prior, iters=1, tier=1)
        got = edp_lib.solve(dev(C), sp((65, 65)), prior, iters=1).cpu().numpy()
        assert edp_lib.last_pass_kernel() == kern
        assert np.array_equal(got, want), lam


@pytest.mark.parametrize("rows", [1, 2, 3, 4])
@pytest.mark.parametrize("pairs", [0, 1])
@pytest.mark.parametrize("Q", [(33, 33), (17, 17), (27, 15)])
def test_line_kernel_rows_per_block_and_schedule(edp_lib, rows, pairs, Q):
    """Rows per block 1..4 (hand-offs through the shared-memory mailbox and
    through the record ring between blocks) under both pass schedules, with
    a ragged last band."""
    rng = np.random.default_rng(rows * 7 + pairs + Q[0])
    H, W = 23, 10
    n = Q[0] * Q[1]
    C = rng.integers(0, 21, size=(H, W, n)).astype(np.int32)
    prior = {"lam": 9, "g": 3, "l1": 1, "mode": "per_axis"}
    want = oracle.edp(C, sp(Q), prior, iters=3, tier=1)
    edp_lib.set_tuning(rows, 0, LINE)
    edp_lib.set_pass_pairs(pairs)
    got = edp_lib.solve(dev(C), sp(Q), prior, iters=3).cpu().numpy()
    assert edp_lib.last_pass_kernel() == LINE1
    assert edp_lib.last_pass_launches() == (2 if pairs else 4) * 3
    assert np.array_equal(got, want)


@pytest.mark.parametrize("W,H", [(1, 1), (1, 7), (7, 1), (2, 2), (3, 19), (19, 3)])
def test_line_kernel_degenerate_shapes(edp_lib, W, H):
    rng = np.random.default_rng(W * 100 + H)
    C = rng.integers(0, 20, size=(H, W, 17 * 17)).astype(np.int32)
    for mode in ("joint", "per_axis"):
        prior = {"lam": 4, "g": 2, "l1": 1, "mode": mode}
        for iters in (1, 3):
            want = oracle.edp(C, sp((17, 17)), prior, iters=iters, tier=1)
            got = edp_lib.solve(dev(C), sp((17, 17)), prior, iters=iters).cpu().numpy()
            assert np.array_equal(got, want), (mode, iters)


@pytest.mark.parametrize("Q", [(33, 33), (27, 15), (65, 65)])
def test_line_kernel_weighted_prior(edp_lib, Q):
    """Per-edge prior multipliers (the locally adaptive prior) in the line
    kernel against oracle_edp_weighted, and the weighted energy."""
    rng = np.random.default_rng(Q[0] + 5)
    H, W = (12, 11) if Q != (65, 65) else (7, 6)
    n = Q[0] * Q[1]
    C = rng.integers(0, 21, size=(H, W, n)).astype(np.int32)
    wh = rng.integers(0, 4, size=(H, W)).astype(np.uint8)
    wv = rng.integers(0, 4, size=(H, W)).astype(np.uint8)
    for mode in ("per_axis", "joint"):
        prior = {"lam": 5, "g": 3, "l1": 1, "mode": mode}
        want = oracle.edp_weighted(C, sp(Q), prior, wh, wv, iters=2, tier=1)
        got = edp_lib.solve_weighted(dev(C), sp(Q), prior, dev(wh), dev(wv), 3, iters=2)
        assert edp_lib.last_pass_kernel() == kernel_for(Q)
        assert np.array_equal(got.cpu().numpy(), want), mode


@pytest.mark.parametrize("kernel", ["line", "line1", "team"])
def test_motion_65x65_480_rows(edp_lib, kernel):
    """The schedule of the 640x480 workload with 65 x 65 labels: 480 rows
    (line kernels, split and one lane per line: two rows per block, every
    band resident, paired sweeps; multi-axis kernel: 185 KB rows, more bands
    than can be resident, one launch per pass), on a narrow 8-pixel-wide
    crop the oracle solves in seconds; labels and energy bit-exact."""
    w = synth.workload_motion_640x480(W=8, H=480)
    C = oracle.cost_volume(w["I0"], w["I1"], None, w["space"], w["l2"], w["cmax"])
    want = oracle.edp(C, w["space"], w["prior"], iters=1, tier=1)
    edp_lib.set_tuning(0, 0, {"line": LINE, "line1": ONE_LANE, "team": 3}[kernel])
    gC = dev(C)
    got = edp_lib.solve(gC, w["space"], w["prior"], iters=1)
    if kernel != "team":
        assert edp_lib.last_pass_kernel() == (LINE2 if kernel == "line" else LINE1)
        assert edp_lib.last_pass_launches() == 2
    else:
        assert edp_lib.last_pass_kernel() == "edp_pass_team_kernel"
        assert edp_lib.last_pass_launches() == 4
    assert np.array_equal(got.cpu().numpy(), want)
    e = tuple(int(v) for v in edp_lib.energy(gC, got, w["space"], w["prior"]).cpu().numpy())
    assert e == oracle.energy(C, want, w["space"], w["prior"])


def test_motion_640x480_full_size(edp_lib):
    """The full 640x480 workload with 65 x 65 labels in the launch shape the
    bench times (split line kernel), j = 1.  The oracle cannot solve the
    frame in test time, so: the cost volume against the oracle's, the labels
    of the split kernel against those of the one-lane line kernel and of the
    independent multi-axis kernel, and the energy of those labels against the
    oracle's energy function."""
    w = synth.workload_motion_640x480()
    space, prior = w["space"], w["prior"]
    I0, I1 = dev(w["I0"]), dev(w["I1"])
    gC = edp_lib.cost_volume(I0, I1, None, space, w["l2"], w["cmax"])
    # rows 0..39 look at most 32 rows down: a 72-row crop has the same costs there
    C = oracle.cost_volume(w["I0"][:72], w["I1"][:72], None, space, w["l2"], w["cmax"])
    assert np.array_equal(gC[:40].cpu().numpy(), C[:40])
    edp_lib.set_tuning(0, 0, 0)  # the default choice for this shape
    lab_line = edp_lib.solve(gC, space, prior, iters=1)
    assert edp_lib.last_pass_kernel() == LINE2
    edp_lib.set_tuning(0, 0, ONE_LANE)
    lab_line1 = edp_lib.solve(gC, space, prior, iters=1)
    assert edp_lib.last_pass_kernel() == LINE1
    edp_lib.set_tuning(0, 0, 3)
    lab_team = edp_lib.solve(gC, space, prior, iters=1)
    assert edp_lib.last_pass_kernel() == "edp_pass_team_kernel"
    assert torch.equal(lab_line, lab_team)
    assert torch.equal(lab_line1, lab_team)
    e_gpu = tuple(int(v) for v in edp_lib.energy(gC, lab_line, space, prior).cpu().numpy())
    del gC
    torch.cuda.empty_cache()
    Cfull = oracle.cost_volume(w["I0"], w["I1"], None, space, w["l2"], w["cmax"])
    assert e_gpu == oracle.energy(Cfull, lab_line.cpu().numpy(), space, prior)


def test_line_kernel_repeatable_320x240(edp_lib):
    """Repeated solves of the full 320x240 motion workload (33 x 33 labels)
    on the line kernel, with one and two rows per block (every row, or every
    second row, gets its messages from the block above through the record
    ring) under both pass schedules: every run equals the oracle.  Hand-off
    timing differs from run to run, so a protocol hazard would show as a
    difference here."""
    w = synth.workload_motion_320x240()
    C = oracle.cost_volume(w["I0"], w["I1"], None, w["space"], w["l2"], w["cmax"])
    want = oracle.edp(C, w["space"], w["prior"], iters=1, tier=1)
    gC = dev(C)
    for rows in (1, 2):
        for pairs in (0, 1):
            edp_lib.set_tuning(rows, 0, LINE)
            edp_lib.set_pass_pairs(pairs)
            for _ in range(3):
                got = edp_lib.solve(gC, w["space"], w["prior"], iters=1).cpu().numpy()
                assert edp_lib.last_pass_kernel() == LINE1
                assert np.array_equal(got, want), (rows, pairs)


def test_split_kernel_repeatable_320x240(edp_lib):
    """Repeated solves of a 320x240 motion pair with 65 x 65 labels on the
    split kernel, one and two rows per block (every row, or every second
    row, reads the published value ring), both pass schedules: every run
    equals the one-lane line kernel's labels (an independent body and
    hand-off protocol).  A protocol hazard would show as a difference."""
    w = synth.workload_motion_640x480(W=320, H=240)
    gC = edp_lib.cost_volume(dev(w["I0"]), dev(w["I1"]), None, w["space"], w["l2"], w["cmax"])
    edp_lib.set_tuning(0, 0, ONE_LANE)
    ref = edp_lib.solve(gC, w["space"], w["prior"], iters=1)
    assert edp_lib.last_pass_kernel() == LINE1
    for rows in (1, 2):
        for pairs in (0, 1):
            edp_lib.set_tuning(rows, 0, LINE)
            edp_lib.set_pass_pairs(pairs)
            for _ in range(3):
                got = edp_lib.solve(gC, w["space"], w["prior"], iters=1)
                assert edp_lib.last_pass_kernel() == LINE2
                assert torch.equal(got, ref), (rows, pairs)
