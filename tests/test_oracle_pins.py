"""Pins for the CPU oracle against things other than itself.

Each test checks the oracle against a value the paper or mathematics fixes:
hand-worked examples (tests/golden/), exhaustive enumeration of labelings on
tiny chains and grids, the paper's exactness claim for the recursive minimum
search (RMS == straightforward search, Sec. 1 and Sec. 3), the modified-DP
min-marginal identity (Eq. DP_1D_3), closed-form special cases and
invariances.  None of these needs a GPU.
"""
import itertools
import json
import os
import zlib

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def sp(Q, vmin=None, step=None):
    R = len(Q)
    return {"R": R, "Q": tuple(Q), "vmin": tuple(vmin or [0] * R), "step": tuple(step or [1] * R)}


def coords(q, Q):
    c = []
    for n in Q:
        c.append(q % n)
        q //= n
    return c


def V_def(a, b, Q, lam, g, l1, mode):
    """Eq. Smooth_value_t on label coordinates, for the enumeration tests."""
    ca, cb = coords(a, Q), coords(b, Q)
    f = [abs(x - y) ** l1 for x, y in zip(ca, cb)]
    if mode == "joint":
        return lam * min(sum(f), g ** l1)
    return sum(lam * min(v, g ** l1) for v in f)


# --------------------------------------------------------------------------
# prior and cost: hand-worked values
# --------------------------------------------------------------------------

def test_prior_handworked():
    gold = json.load(open(os.path.join(GOLDEN, "prior_and_cost_handworked.json")))
    for c in gold["prior_cases"]:
        Q = c["Q"]
        qa = sum(v * int(np.prod(Q[:i])) for i, v in enumerate(c["a"]))
        qb = sum(v * int(np.prod(Q[:i])) for i, v in enumerate(c["b"]))
        pr = {"lam": c["lam"], "g": c["g"], "l1": c["l1"], "mode": c["mode"]}
        assert oracle.prior_value(sp(Q), pr, qa, qb) == c["V"], c
        assert oracle.prior_value(sp(Q), pr, qb, qa) == c["V"], c


def test_cost_handworked():
    gold = json.load(open(os.path.join(GOLDEN, "prior_and_cost_handworked.json")))
    im = {k: np.array(v, dtype=np.uint8) for k, v in gold["cost_image"].items()}
    for c in gold["cost_cases"]:
        s = c["space"]
        space = sp(s["Q"], s["vmin"], s["step"])
        I2 = im["I2"] if c["mode"] == "composite" else None
        C = oracle.cost_volume(im["I0"], im["I1"], I2, space, c["l2"], c["cmax"], c["mode"])
        assert C.tolist() == c["C"], c


def test_cost_3d_sum_and_oob():
    # R = 3: |I1(x+o0, y+o1) - I0|^l2 + |I2(x+o2, y) - I0|^l2, Cmax if either is outside
    I0 = np.array([[10, 20], [30, 40]], np.uint8)
    I1 = np.array([[11, 25], [30, 49]], np.uint8)
    I2 = np.array([[12, 18], [33, 0]], np.uint8)
    space = sp((2, 2, 2), (0, 0, 0), (1, 1, -1))
    C = oracle.cost_volume(I0, I1, I2, space, 1, 100, "pair_stereo3")
    # pixel (x=0, y=0), q = (0,0,0): |11-10| + |12-10| = 3
    assert C[0, 0, 0] == 3
    # pixel (1, 1), q = (0, 0, 1): o2 = -1 -> I2(0, 1) = 33: |49-40| + |33-40| = 16
    assert C[1, 1, 0 + 2 * 2 * 1] == 16
    # pixel (1, 1), q = (1, 0, 0): o0 = 1 -> x = 2 outside -> Cmax
    assert C[1, 1, 1] == 100
    # pixel (0, 0), q = (0, 0, 1): o2 = -1 -> x = -1 outside -> Cmax
    assert C[0, 0, 4] == 100


# --------------------------------------------------------------------------
# min-search operator M
# --------------------------------------------------------------------------

SPACES = [(1,), (7,), (16,), (5, 4), (3, 3, 2), (1, 6), (6, 1)]


@pytest.mark.parametrize("Q", SPACES)
@pytest.mark.parametrize("mode", ["joint", "per_axis"])
@pytest.mark.parametrize("l1", [1, 2])
def test_rms_equals_straightforward(Q, mode, l1):
    """Sec. 1 / Sec. 3: the RMS result equals the straightforward search."""
    rng = np.random.default_rng(zlib.crc32(repr((Q, mode, l1)).encode()))
    space = sp(Q)
    n = int(np.prod(Q))
    for lam in (0, 1, 20):
        for g in sorted({1, 2, 4, max(Q)}):
            pr = {"lam": lam, "g": g, "l1": l1, "mode": mode}
            for _ in range(30):
                h = rng.integers(-2000, 2000, size=n)
                if rng.random() < 0.3:
                    h = rng.integers(-3, 3, size=n)  # many ties
                a = oracle.message(h, space, pr, tier=0)
                b = oracle.message(h, space, pr, tier=1)
                assert np.array_equal(a, b), (pr, h)


@pytest.mark.parametrize("Q", [(9,), (4, 5), (3, 2, 4)])
def test_message_matches_enumerated_definition(Q):
    """M(h)(q) = min_q' h(q') + V(q', q) with V from Eq. Smooth_value_t."""
    rng = np.random.default_rng(7)
    n = int(np.prod(Q))
    for mode in ("joint", "per_axis"):
        for l1 in (1, 2):
            pr = {"lam": 3, "g": 2, "l1": l1, "mode": mode}
            h = rng.integers(-50, 50, size=n)
            want = [min(h[a] + V_def(a, b, Q, 3, 2, l1, mode) for a in range(n)) for b in range(n)]
            assert oracle.message(h, sp(Q), pr, 0).tolist() == want


def test_message_special_cases():
    rng = np.random.default_rng(3)
    for Q in [(12,), (4, 6), (3, 3, 3)]:
        n = int(np.prod(Q))
        h = rng.integers(-100, 100, size=n)
        for tier in (0, 1):
            # lambda = 0: M is the constant min h
            m = oracle.message(h, sp(Q), {"lam": 0, "g": 3, "l1": 1, "mode": "joint"}, tier)
            assert np.all(m == h.min())
            # g = 1, joint: every other label costs exactly lambda
            m = oracle.message(h, sp(Q), {"lam": 5, "g": 1, "l1": 1, "mode": "joint"}, tier)
            assert np.array_equal(m, np.minimum(h, h.min() + 5))
            # shift invariance M(h + c) = M(h) + c
            pr = {"lam": 7, "g": 2, "l1": 1, "mode": "per_axis"}
            assert np.array_equal(oracle.message(h + 11, sp(Q), pr, tier),
                                  oracle.message(h, sp(Q), pr, tier) + 11)


def test_message_untruncated_l1_closed_form():
    # R = 1, g >= Q: M(delta at q0)(q) = lambda |q - q0| (plus the delta value)
    Q = 10
    for q0 in range(Q):
        h = np.full(Q, 10**6, dtype=np.int64)
        h[q0] = -4
        for tier in (0, 1):
            m = oracle.message(h, sp((Q,)), {"lam": 3, "g": Q, "l1": 1, "mode": "joint"}, tier)
            assert m.tolist() == [-4 + 3 * abs(q - q0) for q in range(Q)]


# --------------------------------------------------------------------------
# scanline DP (Sec. 4.1): exhaustive enumeration on tiny chains
# --------------------------------------------------------------------------

def chain_energy(Crow, lab, Q, pr):
    e = sum(int(Crow[x, l]) for x, l in enumerate(lab))
    e += sum(V_def(lab[x], lab[x + 1], Q, pr["lam"], pr["g"], pr["l1"], pr["mode"])
             for x in range(len(lab) - 1))
    return e


@pytest.mark.parametrize("Q,W", [((2,), 6), ((3,), 5), ((4,), 4), ((2, 2), 4), ((3, 1), 3)])
@pytest.mark.parametrize("tier", [0, 1])
def test_scanline_dp_enumeration(Q, W, tier):
    rng = np.random.default_rng(11)
    n = int(np.prod(Q))
    for trial in range(6):
        H = 2
        C = rng.integers(0, 6 if trial % 2 else 30, size=(H, W, n)).astype(np.int32)
        pr = {"lam": int(rng.integers(0, 8)), "g": int(rng.integers(1, 4)), "l1": 1,
              "mode": "joint" if trial % 3 else "per_axis"}
        labels, row_e = oracle.scanline_dp(C, sp(Q), pr, tier)
        for y in range(H):
            best, best_lab = None, None
            for lab in itertools.product(range(n), repeat=W):
                e = chain_energy(C[y], lab, Q, pr)
                # ties: smallest label at the last pixel, then the one before...
                key = (e, lab[::-1])
                if best is None or key < best:
                    best, best_lab = key, lab
            assert row_e[y] == best[0]
            assert tuple(labels[y]) == best_lab
            assert chain_energy(C[y], labels[y], Q, pr) == row_e[y]


@pytest.mark.parametrize("tier", [0, 1])
def test_min_marginals_enumeration(tier):
    """Eq. DP_1D_3: S_Omega(x, q) = minimum energy over labelings with v(x) = q."""
    rng = np.random.default_rng(5)
    for Q, W in [((3,), 5), ((2, 2), 4)]:
        n = int(np.prod(Q))
        C = rng.integers(0, 25, size=(1, W, n)).astype(np.int32)
        pr = {"lam": 4, "g": 2, "l1": 1, "mode": "joint"}
        S = oracle.min_marginals(C, sp(Q), pr, tier)
        want = np.full((W, n), 10**9)
        for lab in itertools.product(range(n), repeat=W):
            e = chain_energy(C[0], lab, Q, pr)
            for x in range(W):
                want[x, lab[x]] = min(want[x, lab[x]], e)
        assert np.array_equal(S[0], want)


def test_scanline_lambda_zero_is_wta():
    rng = np.random.default_rng(1)
    C = rng.integers(0, 5, size=(3, 9, 6)).astype(np.int32)
    labels, _ = oracle.scanline_dp(C, sp((6,)), {"lam": 0, "g": 2, "l1": 1, "mode": "joint"}, 1)
    assert np.array_equal(labels, np.argmin(C, axis=2))


def test_row_energy_is_data_plus_horizontal():
    rng = np.random.default_rng(2)
    C = rng.integers(0, 21, size=(5, 12, 8)).astype(np.int32)
    pr = {"lam": 6, "g": 3, "l1": 1, "mode": "joint"}
    labels, row_e = oracle.scanline_dp(C, sp((8,)), pr, 1)
    d, sh, sv, tot = oracle.energy(C, labels, sp((8,)), pr)
    assert d + sh == int(row_e.sum())
    assert tot == d + sh + sv


# --------------------------------------------------------------------------
# energy (Eq. GE_objective_function)
# --------------------------------------------------------------------------

def test_energy_enumerated_definition():
    rng = np.random.default_rng(4)
    Q = (3, 2)
    C = rng.integers(0, 9, size=(3, 4, 6)).astype(np.int32)
    lab = rng.integers(0, 6, size=(3, 4)).astype(np.int32)
    pr = {"lam": 2, "g": 2, "l1": 1, "mode": "per_axis"}
    d = sum(int(C[y, x, lab[y, x]]) for y in range(3) for x in range(4))
    sh = sum(V_def(lab[y, x], lab[y, x + 1], Q, 2, 2, 1, "per_axis") for y in range(3) for x in range(3))
    sv = sum(V_def(lab[y, x], lab[y + 1, x], Q, 2, 2, 1, "per_axis") for y in range(2) for x in range(4))
    assert oracle.energy(C, lab, sp(Q), pr) == (d, sh, sv, d + sh + sv)


# --------------------------------------------------------------------------
# EDP (Sec. 4.2, Algorithm 1).  The paper calls the recursion a heuristic
# (no closed form); the pins are hand-worked grids, a scalar restatement for
# label-independent costs, special cases, invariances and a lower bound.
# --------------------------------------------------------------------------

@pytest.mark.parametrize("tier", [0, 1])
def test_edp_handworked_chains(tier):
    gold = json.load(open(os.path.join(GOLDEN, "edp_chain_2px_handworked.json")))
    pr = {k: gold["prior"][k] for k in ("lam", "g", "l1", "mode")}
    space = sp(gold["prior"]["Q"])
    for c in gold["cases"]:
        C = np.array(c["C"], dtype=np.int32)
        labels, S, So = oracle.edp(C, space, pr, iters=1, tier=tier, return_sums=True,
                                   return_marginal=True)
        assert labels.tolist() == c["labels"], c["name"]
        for k, name in enumerate(["S_px", "S_mx", "S_py", "S_my"]):
            assert S[k].tolist() == c[name], (c["name"], name)
        assert So.tolist() == c["S_omega"], c["name"]
        assert list(oracle.energy(C, labels, space, pr)) == c["energy"]


def scalar_edp(c, W, H, iters):
    """Algorithm 1 for one label (Q = 1): then M is the identity, so each sum
    is one integer; written independently of the oracle, loops in the order
    of P1..P4 (Sec. 4.2)."""
    S = {k: [[0] * W for _ in range(H)] for k in ("+x", "-x", "+y", "-y")}
    opp = {"+x": "-x", "-x": "+x", "+y": "-y", "-y": "+y"}
    nb = {"+x": (-1, 0), "-x": (1, 0), "+y": (0, -1), "-y": (0, 1)}

    def msg(k, x, y):
        dx, dy = nb[k]
        xn, yn = x + dx, y + dy
        if 0 <= xn < W and 0 <= yn < H:
            return S[k][yn][xn] // 2  # python // is floor division
        return 0

    passes = [(("+x", "+y"), True, True), (("-x", "+y"), False, True),
              (("+x", "-y"), True, False), (("-x", "-y"), False, False)]
    for _ in range(iters):
        for upd, incx, incy in passes:
            for y in (range(H) if incy else range(H - 1, -1, -1)):
                for x in (range(W) if incx else range(W - 1, -1, -1)):
                    m = {k: msg(k, x, y) for k in S}
                    new = {}
                    for kp in upd:
                        new[kp] = c[y][x] + sum(m[k] for k in S if k != opp[kp]) - m[opp[kp]]
                    for kp in upd:
                        S[kp][y][x] = new[kp]
    return S


@pytest.mark.parametrize("W,H,iters", [(5, 4, 1), (3, 6, 2), (7, 2, 3), (1, 5, 1)])
def test_edp_label_independent_cost_matches_scalar_recursion(W, H, iters):
    rng = np.random.default_rng(W * 100 + H)
    c = rng.integers(0, 40, size=(H, W))
    want = scalar_edp(c.tolist(), W, H, iters)
    # Q = 1, and Q = 5 with the same cost on every label: all sums are flat in q
    for Q in (1, 5):
        C = np.repeat(c[:, :, None], Q, axis=2).astype(np.int32)
        for tier in (0, 1):
            labels, S = oracle.edp(C, sp((Q,)), {"lam": 9, "g": 2, "l1": 1, "mode": "joint"},
                                   iters=iters, tier=tier, return_sums=True)
            for k, name in enumerate(["+x", "-x", "+y", "-y"]):
                assert np.array_equal(S[k], np.repeat(np.array(want[name])[:, :, None], Q, 2))
            assert np.all(labels == 0)


@pytest.mark.parametrize("Q", [(6,), (3, 4)])
def test_edp_lambda_zero_is_wta(Q):
    rng = np.random.default_rng(8)
    n = int(np.prod(Q))
    C = rng.integers(0, 20, size=(5, 6, n)).astype(np.int32)
    labels = oracle.edp(C, sp(Q), {"lam": 0, "g": 2, "l1": 1, "mode": "joint"}, iters=2, tier=1)
    assert np.array_equal(labels, np.argmin(C, axis=2))


def test_edp_translation_equivariance():
    """Prepending one label with a prohibitive cost shifts every label by one."""
    rng = np.random.default_rng(9)
    C = rng.integers(0, 20, size=(4, 5, 6)).astype(np.int32)
    big = np.full((4, 5, 1), 100000, dtype=np.int32)
    Cs = np.concatenate([big, C], axis=2)
    for mode in ("joint", "per_axis"):
        pr = {"lam": 5, "g": 2, "l1": 1, "mode": mode}
        a = oracle.edp(C, sp((6,)), pr, iters=2, tier=1)
        b = oracle.edp(Cs, sp((7,)), pr, iters=2, tier=1)
        assert np.array_equal(a + 1, b)
    # 2D: shift along axis 1 (rows of the label grid)
    C2 = rng.integers(0, 20, size=(3, 4, 12)).astype(np.int32)  # Q = 4 x 3
    C2s = np.concatenate([np.full((3, 4, 4), 100000, np.int32), C2], axis=2)  # Q = 4 x 4
    pr = {"lam": 5, "g": 2, "l1": 1, "mode": "per_axis"}
    a = oracle.edp(C2, sp((4, 3)), pr, iters=1, tier=1)
    b = oracle.edp(C2s, sp((4, 4)), pr, iters=1, tier=1)
    assert np.array_equal(a + 4, b)


def test_edp_energy_not_below_global_minimum():
    """EDP is an approximation: its energy is >= the exhaustive optimum on a
    3x3 grid with 3 labels (3^9 labelings)."""
    rng = np.random.default_rng(10)
    Q = 3
    labs = np.array(list(itertools.product(range(Q), repeat=9))).reshape(-1, 3, 3)
    for trial in range(4):
        C = rng.integers(0, 20, size=(3, 3, Q)).astype(np.int32)
        pr = {"lam": int(rng.integers(1, 10)), "g": 2, "l1": 1, "mode": "joint"}
        lab = oracle.edp(C, sp((Q,)), pr, iters=3, tier=0)
        e = oracle.energy(C, lab, sp((Q,)), pr)[3]
        V = np.array([[V_def(a, b, (Q,), pr["lam"], 2, 1, "joint") for b in range(Q)]
                      for a in range(Q)])
        yy, xx = np.mgrid[0:3, 0:3]
        data = C[yy[None], xx[None], labs].sum(axis=(1, 2))
        sh = V[labs[:, :, :-1], labs[:, :, 1:]].sum(axis=(1, 2))
        sv = V[labs[:, :-1, :], labs[:, 1:, :]].sum(axis=(1, 2))
        assert e >= int((data + sh + sv).min())


@pytest.mark.parametrize("Q", [(5,), (3, 4), (2, 2, 3)])
def test_edp_tiers_agree(Q):
    rng = np.random.default_rng(12)
    n = int(np.prod(Q))
    C = rng.integers(0, 21, size=(6, 7, n)).astype(np.int32)
    for mode in ("joint", "per_axis"):
        pr = {"lam": 6, "g": 2, "l1": 1, "mode": mode}
        a, Sa = oracle.edp(C, sp(Q), pr, iters=2, tier=0, return_sums=True)
        b, Sb = oracle.edp(C, sp(Q), pr, iters=2, tier=1, return_sums=True)
        assert np.array_equal(a, b) and np.array_equal(Sa, Sb)


def test_edp_range_error():
    C = np.full((2, 2, 2), 2**31 - 1, dtype=np.int32)
    with pytest.raises(oracle.OracleError):
        oracle.edp(C, sp((2,)), {"lam": 1, "g": 1, "l1": 1, "mode": "joint"}, iters=1)


# --------------------------------------------------------------------------
# windowed EDP
# --------------------------------------------------------------------------

def test_windowed_full_window_equals_full_edp():
    rng = np.random.default_rng(13)
    for Q, mode in [((7,), "joint"), ((5, 5), "per_axis"), ((5, 5), "joint")]:
        n = int(np.prod(Q))
        C = rng.integers(0, 20, size=(4, 5, n)).astype(np.int32)
        pr = {"lam": 4, "g": 2, "l1": 1, "mode": mode}
        centre = np.zeros((4, 5, len(Q)), np.int32) + np.array([q // 2 for q in Q], np.int32)
        a = oracle.edp(C, sp(Q), pr, iters=2, tier=0)
        b = oracle.edp_windowed(C, centre, sp(Q), pr, win=Q[0], iters=2)
        assert np.array_equal(a, b)


def test_windowed_common_box_equals_cropped_space():
    """All pixels sharing one box = full EDP on the cropped label space."""
    rng = np.random.default_rng(14)
    Q = (9, 8)
    I0 = rng.integers(0, 256, size=(5, 6)).astype(np.uint8)
    I1 = rng.integers(0, 256, size=(5, 6)).astype(np.uint8)
    space = sp(Q, (-4, -4), (1, 1))
    pr = {"lam": 3, "g": 2, "l1": 1, "mode": "per_axis"}
    centre = np.zeros((5, 6, 2), np.int32) + np.array([5, 3], np.int32)  # box [3..7] x [1..5]
    Cw = oracle.cost_window(I0, I1, None, space, 1, 30, centre, 5)
    lab_w = oracle.edp_windowed(Cw, centre, space, pr, 5, iters=2)
    crop = sp((5, 5), (-4 + 3, -4 + 1), (1, 1))
    Cc = oracle.cost_volume(I0, I1, None, crop, 1, 30)
    assert np.array_equal(Cw, Cc)
    lab_c = oracle.edp(Cc, crop, pr, iters=2, tier=0)
    q0, q1 = lab_c % 5 + 3, lab_c // 5 + 1
    assert np.array_equal(lab_w, q0 + 9 * q1)


def test_windowed_centre_clamped():
    rng = np.random.default_rng(15)
    I0 = rng.integers(0, 256, size=(3, 4)).astype(np.uint8)
    I1 = rng.integers(0, 256, size=(3, 4)).astype(np.uint8)
    space = sp((7,), (0,), (-1,))
    a = oracle.cost_window(I0, I1, None, space, 1, 30, np.full((3, 4, 1), -5, np.int32), 3)
    b = oracle.cost_window(I0, I1, None, space, 1, 30, np.full((3, 4, 1), 1, np.int32), 3)
    assert np.array_equal(a, b)


@pytest.mark.parametrize("name", ["horizontal 2x1, A left, B right", "vertical 1x2, A top, B bottom"])
def test_windowed_distinct_boxes_handworked(name):
    """Two pixels whose boxes differ: every sum and label worked by hand
    (tests/golden/edp_window_2px_distinct_boxes_handworked.json)."""
    gold = json.load(open(os.path.join(GOLDEN, "edp_window_2px_distinct_boxes_handworked.json")))
    pr = {k: gold["prior"][k] for k in ("lam", "g", "l1", "mode")}
    space = sp(gold["prior"]["Q"])
    (c,) = [c for c in gold["cases"] if c["name"] == name]
    Cw = np.array(c["Cw"], dtype=np.int32)
    centre = np.array(c["centre"], dtype=np.int32)
    labels, S = oracle.edp_windowed(Cw, centre, space, pr, gold["win"], iters=1, return_sums=True)
    assert labels.tolist() == c["labels"]
    for k, key in enumerate(["S_px", "S_mx", "S_py", "S_my"]):
        assert S[k].tolist() == c[key], key


def py_windowed_edp(Cw, centre, Q, pr, win, iters):
    """Windowed Algorithm 1 restated in plain Python, independently of the
    oracle: per-pixel boxes of win^R labels (centre clamped so the box fits),
    messages by direct search over the source box evaluated on the target
    box, passes P1..P4 of Sec. 4.2 in place, then Eq. DP_2D_1 / DP_2D_2 with
    the lowest box index on ties.  Returns (full-space labels, sums)."""
    H, W, R = len(Cw), len(Cw[0]), len(Q)
    n = win ** R
    half = (win - 1) // 2
    lam, g, l1, mode = pr["lam"], pr["g"], pr["l1"], pr["mode"]

    def lo(y, x):
        return [min(max(centre[y][x][r], half), Q[r] - 1 - half) - half for r in range(R)]

    def full(box_lo, w):
        q = box_lo[0] + w % win
        if R == 2:
            q += Q[0] * (box_lo[1] + w // win)
        return q

    S = {k: [[[0] * n for _ in range(W)] for _ in range(H)] for k in ("+x", "-x", "+y", "-y")}
    opp = {"+x": "-x", "-x": "+x", "+y": "-y", "-y": "+y"}
    nb = {"+x": (-1, 0), "-x": (1, 0), "+y": (0, -1), "-y": (0, 1)}

    def msg(k, x, y):
        xn, yn = x + nb[k][0], y + nb[k][1]
        if not (0 <= xn < W and 0 <= yn < H):
            return [0] * n
        ls, ld, src = lo(yn, xn), lo(y, x), S[k][yn][xn]
        return [min(src[u] // 2 + V_def(full(ls, u), full(ld, v), Q, lam, g, l1, mode) for u in range(n))
                for v in range(n)]

    passes = [(("+x", "+y"), True, True), (("-x", "+y"), False, True),
              (("+x", "-y"), True, False), (("-x", "-y"), False, False)]
    for _ in range(iters):
        for upd, incx, incy in passes:
            for y in (range(H) if incy else range(H - 1, -1, -1)):
                for x in (range(W) if incx else range(W - 1, -1, -1)):
                    m = {k: msg(k, x, y) for k in S}
                    new = {kp: [Cw[y][x][v] + sum(m[k][v] for k in S if k != opp[kp]) - m[opp[kp]][v]
                                for v in range(n)] for kp in upd}
                    for kp in upd:
                        S[kp][y][x] = new[kp]
    labels = [[0] * W for _ in range(H)]
    for y in range(H):
        for x in range(W):
            m = {k: msg(k, x, y) for k in S}
            tot = [Cw[y][x][v] + sum(m[k][v] for k in S) for v in range(n)]
            labels[y][x] = full(lo(y, x), tot.index(min(tot)))
    return labels, S


@pytest.mark.parametrize("Q,win,mode,l1,iters", [((7,), 3, "joint", 1, 2), ((6, 5), 3, "per_axis", 1, 1),
                                                  ((5, 6), 3, "joint", 1, 2), ((6, 6), 3, "per_axis", 2, 1),
                                                  ((9,), 5, "joint", 2, 1)])
def test_windowed_random_boxes_match_python_restatement(Q, win, mode, l1, iters):
    """3x3 grids whose pixels all have different (random, partly clamped)
    boxes: the oracle equals the independent Python restatement in every sum
    and label."""
    rng = np.random.default_rng(sum(Q) * 10 + win + l1)
    R = len(Q)
    n = win ** R
    for trial in range(2):
        Cw = rng.integers(0, 25, size=(3, 3, n)).astype(np.int32)
        centre = np.stack([rng.integers(-1, Q[r] + 1, size=(3, 3)) for r in range(R)], axis=2).astype(np.int32)
        pr = {"lam": int(rng.integers(1, 6)), "g": int(rng.integers(1, 4)), "l1": l1, "mode": mode}
        want_lab, want_S = py_windowed_edp(Cw.tolist(), centre.tolist(), Q, pr, win, iters)
        lab, S = oracle.edp_windowed(Cw, centre, sp(Q), pr, win, iters=iters, return_sums=True)
        assert lab.tolist() == want_lab
        for k, key in enumerate(["+x", "-x", "+y", "-y"]):
            assert S[k].tolist() == want_S[key], key
