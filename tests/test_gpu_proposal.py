"""Learned proposal + windowed EDP, end to end on the GPU at a small size.
The network is trained by the project's kernels on full-label EDP
labelings.  On held-out pairs the whole proposal path (coarse labeling +
network + windowed EDP) is compared with full-label EDP (energies on the
full label space), and the network's own contribution with the path without
it (no correction of the coarse labeling)."""
import numpy as np
import pytest
import torch

from paper_1410_7922_gb300 import edp, proposal

pytestmark = pytest.mark.gpu


def test_proposal_path(edp_lib):
    W, H, vmax = 128, 96, 12
    x, t = proposal.build_training_set(32, W, H, first_pair=100, vmax=vmax)
    P, losses = proposal.train(x, t, epochs=20, batch=8, lr=2e-3)
    assert losses[-1] < losses[0]
    rows = proposal.evaluate(P, [900, 901, 902], W, H, win=9, reps=1, vmax=vmax, min_shift=0)
    assert all(r["E_full"] > 0 for r in rows)
    # the proposal path (coarse labeling, network, 9x9 windows) stays close to full-label EDP
    assert np.mean([r["gap_net"] for r in rows]) < 0.05, rows
    assert np.mean([r["gap_coarse"] for r in rows]) < 0.05, rows
    # what the trained network gains over the path without it: on held-out
    # pairs its correction predicts the full-label EDP labeling better than
    # the coarse labeling alone does
    assert np.mean([r["loss_net"] for r in rows]) < np.mean([r["loss_zero"] for r in rows]), rows


def test_no_correction_is_the_coarse_labeling(edp_lib):
    """With every correction dropped the centres are the coarse labels."""
    w = proposal.pair(7, 40, 30, 6)
    I0, I1 = proposal.to_device(w)
    base = proposal.coarse(I0, I1, w)
    P = proposal.init_params(3)
    c = proposal.propose(P, I0, I1, w, base=base, min_shift=10 ** 6)
    assert torch.equal(c, proposal.label_centres(base, w["space"]))
