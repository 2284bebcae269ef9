"""The timeout path of the bounded waits between row bands, made to run out
without any fault: the test hook edp_test_hold_band makes the first row of
one band wait for hand-off data no producer publishes.  The wait
gives up after the spin limit, the launch writes EDP_ERR_TIMEOUT to the
device status word, every kernel of the solve returns, and the next normal
solve on the same workspace is bit-exact against the oracle."""
import numpy as np
import pytest
import torch

import oracle
from paper_1410_7922_gb300 import synth

pytestmark = pytest.mark.gpu


def _case(kind):
    """Workload and the general_kernel tuning value that selects the kernel."""
    if kind == "one_axis":  # warp-per-row kernel, 8 rows per band
        return synth.workload_scanline_64x48(), 0
    if kind == "multi_axis_33":  # multi-axis kernel, 33 x 33 labels
        return synth.workload_motion_320x240(W=24, H=40), 3
    if kind == "line_33":  # two-axis line kernel, 33 x 33 labels
        return synth.workload_motion_320x240(W=24, H=40), 4
    if kind == "line_65":  # two-axis line kernel, lines split over lane pairs, 65 x 65 labels
        return synth.workload_motion_640x480(W=12, H=36), 4
    return synth.workload_motion_640x480(W=20, H=36, vmax=4), 0  # multi-axis, 9 x 9 labels


@pytest.mark.parametrize("kind", ["one_axis", "multi_axis_33", "line_33", "line_65", "multi_axis_9"])
@pytest.mark.parametrize("pairs", [0, 1])
def test_timeout_sets_status_and_next_solve_is_exact(edp_lib, kind, pairs):
    edp = edp_lib
    w, general = _case(kind)
    edp.set_tuning(0, 0, general)
    I0, I1 = torch.from_numpy(w["I0"]).cuda(), torch.from_numpy(w["I1"]).cuda()
    C = edp.cost_volume(I0, I1, None, w["space"], w["l2"], w["cmax"])
    H, W, _ = C.shape
    want = oracle.edp(C.cpu().numpy(), w["space"], w["prior"], iters=1, tier=1)
    ws = edp.workspace(edp.OP_SOLVE, W, H, w["space"], w["prior"], 1)
    lab = torch.full((H, W), -1, dtype=torch.int32, device="cuda")
    edp.set_pass_pairs(pairs)
    try:
        edp.set_spin_limit(20000)
        edp.test_hold_band(2)
        edp.solve(C, w["space"], w["prior"], iters=1, ws=ws, labels=lab)
        torch.cuda.synchronize()
        assert edp.get_device_status(ws) == edp.ERR_TIMEOUT
    finally:
        edp.test_hold_band(0)
        edp.set_spin_limit(0)
        edp.set_pass_pairs(edp.PAIRS_AUTO)
    # the context is usable and the workspace is reset by the next solve
    try:
        edp.solve(C, w["space"], w["prior"], iters=1, ws=ws, labels=lab)
        assert edp.get_device_status(ws) == 0
        assert np.array_equal(lab.cpu().numpy(), want)
    finally:
        edp.set_tuning(0, 0, 0)
