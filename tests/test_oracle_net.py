"""Pins for the CPU reference of the proposal network (oracle/net.py):
bfloat16 rounding against torch's conversion, the convolution and its two
gradients against torch's conv2d and autograd in float64, and the whole
backward pass against central finite differences."""
import numpy as np
import pytest
import torch

from oracle import net


def test_bf16_rounding_matches_torch():
    rng = np.random.default_rng(0)
    x = np.concatenate([rng.normal(0, 10, 5000), [1.0, 1 + 2**-8, 1 + 3 * 2**-9, -1 - 2**-8, 0.0, 3e38]])
    want = torch.from_numpy(x.astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(net.bf16(x), want)
    assert net.bf16(np.array([1 + 2**-8]))[0] == 1.0          # tie to even
    assert net.bf16(np.array([1 + 3 * 2**-9]))[0] == 1 + 2**-7


def test_conv_and_gradients_match_torch():
    rng = np.random.default_rng(1)
    x = rng.normal(size=(2, 3, 7, 9))
    w = rng.normal(size=(4, 3, 3, 3))
    b = rng.normal(size=4)
    g = rng.normal(size=(2, 4, 7, 9))
    xt = torch.from_numpy(x).requires_grad_(True)
    wt = torch.from_numpy(w).requires_grad_(True)
    out = torch.nn.functional.conv2d(xt, wt, torch.from_numpy(b), padding=1)
    assert np.allclose(net.conv3x3(x, w, b), out.detach().numpy(), rtol=1e-12, atol=1e-12)
    out.backward(torch.from_numpy(g))
    assert np.allclose(net.conv3x3_dgrad(g, w), xt.grad.numpy(), rtol=1e-12, atol=1e-12)
    assert np.allclose(net.conv3x3_wgrad(g, x), wt.grad.numpy(), rtol=1e-12, atol=1e-12)


def test_backward_finite_differences():
    rng = np.random.default_rng(2)
    params = net.init_params(3)
    params = [(w, rng.normal(0, 0.1, size=b.shape)) for w, b in params]
    x = rng.uniform(0, 1, size=(1, 5, 6, 5))
    tgt = rng.normal(0, 2, size=(1, 2, 6, 5))
    loss, grads = net.backward(x, params, tgt, rounding=None)
    eps = 1e-6
    for li in (0, 3, 5):
        w, b = params[li]
        for idx in [(0, 0, 1, 1), (1, 2, 0, 2)]:
            if idx[1] >= w.shape[1] or idx[0] >= w.shape[0]:
                continue
            wp, wm = w.copy(), w.copy()
            wp[idx] += eps
            wm[idx] -= eps
            pp = list(params); pp[li] = (wp, b)
            pm = list(params); pm[li] = (wm, b)
            lp = net.smooth_l1(net.forward(x, pp, rounding=None), tgt)[0]
            lm = net.smooth_l1(net.forward(x, pm, rounding=None), tgt)[0]
            assert abs((lp - lm) / (2 * eps) - grads[li][0][idx]) < 1e-6 * max(1.0, abs(grads[li][0][idx]))
        bp, bm = b.copy(), b.copy()
        bp[0] += eps
        bm[0] -= eps
        pp = list(params); pp[li] = (w, bp)
        pm = list(params); pm[li] = (w, bm)
        lp = net.smooth_l1(net.forward(x, pp, rounding=None), tgt)[0]
        lm = net.smooth_l1(net.forward(x, pm, rounding=None), tgt)[0]
        assert abs((lp - lm) / (2 * eps) - grads[li][1][0]) < 1e-6 * max(1.0, abs(grads[li][1][0]))


def test_smooth_l1_closed_form():
    out = np.array([0.0, 0.5, 3.0, -2.0])
    tgt = np.zeros(4)
    loss, g = net.smooth_l1(out, tgt)
    assert loss == pytest.approx((0 + 0.125 + 2.5 + 1.5) / 4)
    assert np.allclose(g, np.array([0.0, 0.5, 1.0, -1.0]) / 4)


# --------------------------------------------------------------------------
# coarse-level proposal inputs: hand-worked cases
# --------------------------------------------------------------------------

def test_pyr_down2_hand_worked():
    I = np.arange(9, dtype=np.uint8).reshape(3, 3)
    # (0+1+3+4+2)//4 = 2; odd edge repeats: (2+2+5+5+2)//4 = 4, (6+7+6+7+2)//4 = 7, (4*8+2)//4 = 8
    assert net.pyr_down2(I).tolist() == [[2, 4], [7, 8]]
    # rounding half up: 1+1+1+2 = 5 -> (5+2)//4 = 1; 1+2+2+2 = 7 -> 2
    assert net.pyr_down2(np.array([[1, 1], [1, 2]], dtype=np.uint8)).tolist() == [[1]]
    assert net.pyr_down2(np.array([[1, 2], [2, 2]], dtype=np.uint8)).tolist() == [[2]]


def test_halved_space():
    assert net.halved_space((-32, -32), (65, 65)) == ((-16, -16), (33, 33))
    # offsets -3..2 -> -1..1; offsets 0..4 -> 0..2
    assert net.halved_space((-3, 0), (6, 5)) == ((-1, 0), (3, 3))


def test_labels_up2_hand_worked():
    # coarse space offsets -1..1 per axis; label 2 = offset (1, -1)
    lc = np.array([[2]])
    up = net.labels_up2(lc, (-1, -1), (3, 3), (-2, -2), (5, 5), 2, 3)
    # doubled offset (2, -2) -> label (4, 0) = 4 everywhere
    assert up.tolist() == [[4, 4, 4], [4, 4, 4]]
    # clamped into a smaller space: offsets -1..1 -> label (2, 0)
    assert net.labels_up2(lc, (-1, -1), (3, 3), (-1, -1), (3, 3), 1, 1).tolist() == [[2]]


def test_features_from_labels_hand_worked():
    I0 = np.array([[10, 20]], dtype=np.uint8)
    I1 = np.array([[30, 40]], dtype=np.uint8)
    lab = np.array([[5, 5]])  # (q0, q1) = (2, 1): offset (+1, 0) in vmin (-1, -1)
    f = net.features_from_labels(I0, I1, lab, (-1, -1), (3, 3), 1, 50, 2.0)
    assert f[:, 0, 0].tolist() == pytest.approx([10 / 255, 30 / 255, 0.5, 0.0, 30 / 50])
    assert f[4, 0, 1] == 1.0  # x + 1 leaves the image: cmax


def test_targets_and_residual_centres():
    Q = (5, 4)
    lab = np.array([7])            # (2, 1)
    base = np.array([5])           # (0, 1)
    assert net.targets(lab, Q, base).tolist() == [[2.0, 0.0]]
    assert net.targets(lab, Q).tolist() == [[0.0, -0.5]]
    out = np.array([[0.5, -0.5], [1.49, -2.6], [9.0, 9.0]])
    b = np.array([6, 6, 6])        # (1, 1)
    assert net.centres_residual(out, b, Q).tolist() == [[2, 0], [2, 0], [4, 3]]
    # corrections below 2 labels dropped: (1, -1) -> base; (1, -3) and (9, 9) kept
    assert net.centres_residual(out, b, Q, min_shift=2).tolist() == [[1, 1], [2, 0], [4, 3]]


def test_gradient_magnitudes_bound_the_gradients():
    """The absolute-value sums bound every gradient (triangle inequality) and
    equal its magnitude where every term has one sign: the last layer's bias
    gradient with all outputs above their targets."""
    rng = np.random.default_rng(4)
    params = net.init_params(6)
    params = [(w, rng.normal(0, 0.1, size=b.shape)) for w, b in params]
    x = net.bf16(rng.uniform(0, 1, size=(1, 5, 6, 7)))
    tgt = rng.normal(0, 2, size=(1, 2, 6, 7))
    _, grads = net.backward(x, params, tgt)
    mags = net.gradient_magnitudes(x, params, tgt)
    for (gw, gb), (mw, mb) in zip(grads, mags):
        assert np.all(mw >= np.abs(gw) - 1e-15) and np.all(mb >= np.abs(gb) - 1e-15)
    out = net.forward(x, params)
    _, grads = net.backward(x, params, out - 5.0)
    mags = net.gradient_magnitudes(x, params, out - 5.0)
    assert np.allclose(mags[-1][1], np.abs(grads[-1][1]), rtol=1e-12)


def test_window_edge_count_hand_worked():
    """Q = 5 x 7 labels, 3 x 3 boxes: a label on a box edge counts unless
    that edge is also an edge of the label space (centres clamped first)."""
    Q = (5, 7)
    cases = [((2, 3), (1, 3), 1),   # box [1..3] x [2..4], left edge, inside the space
             ((2, 3), (2, 3), 0),   # interior
             ((0, 0), (0, 0), 0),   # box clamped to [0..2] x [0..2]: both edges are space edges
             ((0, 0), (2, 1), 1),   # right edge of [0..2], inside the space
             ((4, 6), (4, 6), 0),   # box [2..4] x [4..6]: corner on the space's edges
             ((4, 6), (2, 6), 1)]   # left edge of [2..4]
    centre = np.array([c for c, _, _ in cases], np.int64)
    labels = np.array([l0 + Q[0] * l1 for _, (l0, l1), _ in cases], np.int64)
    for k, (_, _, want) in enumerate(cases):
        assert net.window_edge_count(labels[k:k + 1], centre[k:k + 1], 3, Q) == want, k
    assert net.window_edge_count(labels, centre, 3, Q) == 3
