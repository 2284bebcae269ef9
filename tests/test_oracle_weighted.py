"""Oracle pins for the locally adaptive prior (the text below Eq.
Smooth_value_t: lambda(x) = 2 lambda where the local image gradient is below
10, lambda elsewhere), read as per-edge multipliers of the prior: the edge
(x, y)-(x+1, y) carries wh[y][x] * lambda, the edge (x, y)-(x, y+1) wv[y][x] *
lambda.  The pins tie the weighted oracle to the unweighted one (whose pins
are in test_oracle_pins.py) through identities that a misplaced or transposed
weight breaks, and to brute force on tiny grids."""
import itertools

import numpy as np
import pytest

import oracle

SP1 = {"R": 1, "Q": (5, 1, 1), "vmin": (0, 0, 0), "step": (1, 1, 1)}
SP2 = {"R": 2, "Q": (3, 4, 1), "vmin": (0, 0, 0), "step": (1, 1, 1)}


def _prior(lam=3, g=2, l1=1, mode="joint"):
    return {"lam": lam, "g": g, "l1": l1, "mode": mode}


def test_edge_weights_handworked():
    # I = [[10, 15, 40], [12, 30, 31]], threshold 10, factor 2:
    # horizontal steps |15-10| = 5 -> 2, |40-15| = 25 -> 1, |30-12| = 18 -> 1,
    # |31-30| = 1 -> 2; vertical steps |12-10| = 2 -> 2, |30-15| = 15 -> 1,
    # |31-40| = 9 -> 2; entries without an edge are 1.
    I = np.array([[10, 15, 40], [12, 30, 31]], dtype=np.uint8)
    wh, wv = oracle.edge_weights(I, 10, 2)
    assert wh.tolist() == [[2, 1, 1], [1, 2, 1]]
    assert wv.tolist() == [[2, 1, 2], [1, 1, 1]]
    # the step equal to the threshold is not below it
    wh, wv = oracle.edge_weights(np.array([[0, 10]], dtype=np.uint8), 10, 3)
    assert wh.tolist() == [[1, 1]] and wv.tolist() == [[1, 1]]


@pytest.mark.parametrize("space", [SP1, SP2])
@pytest.mark.parametrize("tier", [0, 1])
@pytest.mark.parametrize("mode", ["joint", "per_axis"])
def test_unit_weights_are_the_plain_prior(space, tier, mode):
    rng = np.random.default_rng(3 + tier)
    Q = int(np.prod(space["Q"][:space["R"]]))
    C = rng.integers(0, 20, size=(6, 7, Q)).astype(np.int32)
    ones = np.ones((6, 7), dtype=np.uint8)
    p = _prior(mode=mode)
    want = oracle.edp(C, space, p, iters=2, tier=tier)
    got = oracle.edp_weighted(C, space, p, ones, ones, iters=2, tier=tier)
    assert np.array_equal(got, want)
    assert oracle.energy_weighted(C, want, space, p, ones, ones) == oracle.energy(C, want, space, p)


@pytest.mark.parametrize("k", [0, 2, 3])
def test_uniform_weight_scales_lambda(k):
    """Every edge at k: the prior is (k lambda) f, labels and energy as with k lambda."""
    rng = np.random.default_rng(10 + k)
    C = rng.integers(0, 25, size=(5, 6, 5)).astype(np.int32)
    w = np.full((5, 6), k, dtype=np.uint8)
    got = oracle.edp_weighted(C, SP1, _prior(lam=3), w, w, iters=2)
    want = oracle.edp(C, SP1, _prior(lam=3 * k), iters=2)
    assert np.array_equal(got, want)
    assert oracle.energy_weighted(C, want, SP1, _prior(lam=3), w, w) == oracle.energy(C, want, SP1,
                                                                                    _prior(lam=3 * k))


def test_one_row_reads_only_horizontal_weights():
    """A single row has no vertical edges: wv is never read, wh alone scales."""
    rng = np.random.default_rng(21)
    C = rng.integers(0, 25, size=(1, 9, 5)).astype(np.int32)
    wh = np.full((1, 9), 3, dtype=np.uint8)
    wv = rng.integers(0, 9, size=(1, 9)).astype(np.uint8)
    got = oracle.edp_weighted(C, SP1, _prior(lam=2), wh, wv, iters=2)
    assert np.array_equal(got, oracle.edp(C, SP1, _prior(lam=6), iters=2))


def test_one_column_reads_only_vertical_weights():
    rng = np.random.default_rng(22)
    C = rng.integers(0, 25, size=(9, 1, 5)).astype(np.int32)
    wv = np.full((9, 1), 3, dtype=np.uint8)
    wh = rng.integers(0, 9, size=(9, 1)).astype(np.uint8)
    got = oracle.edp_weighted(C, SP1, _prior(lam=2), wh, wv, iters=2)
    assert np.array_equal(got, oracle.edp(C, SP1, _prior(lam=6), iters=2))


def test_weighted_energy_brute_force():
    """energy_weighted against a literal sum over the grid edges."""
    rng = np.random.default_rng(5)
    H, W = 3, 4
    C = rng.integers(0, 30, size=(H, W, 5)).astype(np.int32)
    lab = rng.integers(0, 5, size=(H, W)).astype(np.int32)
    wh = rng.integers(0, 4, size=(H, W)).astype(np.uint8)
    wv = rng.integers(0, 4, size=(H, W)).astype(np.uint8)
    p = _prior(lam=4, g=2)

    def V(a, b):
        return 4 * min(abs(int(a) - int(b)), 2)

    data = sum(int(C[y, x, lab[y, x]]) for y in range(H) for x in range(W))
    sh = sum(int(wh[y, x]) * V(lab[y, x], lab[y, x + 1]) for y in range(H) for x in range(W - 1))
    sv = sum(int(wv[y, x]) * V(lab[y, x], lab[y + 1, x]) for y in range(H - 1) for x in range(W))
    assert oracle.energy_weighted(C, lab, SP1, p, wh, wv) == (data, sh, sv, data + sh + sv)


@pytest.mark.parametrize("seed", range(4))
def test_weighted_edp_not_below_the_optimum(seed):
    """EDP is a heuristic: its weighted energy is never below the exhaustive
    optimum of the same weighted energy (2x3 grid, 3 labels)."""
    rng = np.random.default_rng(40 + seed)
    H, W, Q = 2, 3, 3
    sp = {"R": 1, "Q": (Q, 1, 1), "vmin": (0, 0, 0), "step": (1, 1, 1)}
    C = rng.integers(0, 12, size=(H, W, Q)).astype(np.int32)
    wh = rng.integers(0, 4, size=(H, W)).astype(np.uint8)
    wv = rng.integers(0, 4, size=(H, W)).astype(np.uint8)
    p = _prior(lam=3, g=2)
    best = min(oracle.energy_weighted(C, np.array(l, dtype=np.int32).reshape(H, W), sp, p, wh, wv)[3]
               for l in itertools.product(range(Q), repeat=H * W))
    lab = oracle.edp_weighted(C, sp, p, wh, wv, iters=3)
    assert oracle.energy_weighted(C, lab, sp, p, wh, wv)[3] >= best


def test_weighted_tiers_agree():
    """The RMS tier equals the definition tier under random edge weights."""
    rng = np.random.default_rng(77)
    C = rng.integers(0, 20, size=(5, 6, 12)).astype(np.int32)
    wh = rng.integers(0, 4, size=(5, 6)).astype(np.uint8)
    wv = rng.integers(0, 4, size=(5, 6)).astype(np.uint8)
    sp = {"R": 2, "Q": (4, 3, 1), "vmin": (0, 0, 0), "step": (1, 1, 1)}
    for mode in ("joint", "per_axis"):
        p = _prior(lam=2, g=2, mode=mode)
        assert np.array_equal(oracle.edp_weighted(C, sp, p, wh, wv, iters=2, tier=0),
                              oracle.edp_weighted(C, sp, p, wh, wv, iters=2, tier=1))


@pytest.mark.parametrize("k", [1, 3])
def test_weighted_quadratic_prior(k):
    """The same identities for the truncated quadratic prior (l1 = 2): a
    uniform multiplier k is the prior k lambda min(d^2, g^2), in both tiers."""
    rng = np.random.default_rng(90 + k)
    C = rng.integers(0, 40, size=(5, 6, 7)).astype(np.int32)
    sp = {"R": 1, "Q": (7, 1, 1), "vmin": (0, 0, 0), "step": (1, 1, 1)}
    w = np.full((5, 6), k, dtype=np.uint8)
    for tier in (0, 1):
        got = oracle.edp_weighted(C, sp, _prior(lam=2, g=3, l1=2), w, w, iters=2, tier=tier)
        want = oracle.edp(C, sp, _prior(lam=2 * k, g=3, l1=2), iters=2, tier=tier)
        assert np.array_equal(got, want)

