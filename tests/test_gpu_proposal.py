"""Learned proposal + windowed EDP, end to end on the GPU at a small size:
the network is trained by the project's kernels on full-label EDP
labelings, and on held-out pairs its proposals must give windowed EDP a
lower energy than winner-take-all proposals do (what the network gains),
with the energy measured on the full label space."""
import numpy as np
import pytest
import torch

from paper_1410_7922_gb300 import proposal

pytestmark = pytest.mark.gpu


def test_proposal_gains_over_wta(edp_lib):
    W, H, vmax = 64, 48, 8
    x, t = proposal.build_training_set(32, W, H, first_pair=100, vmax=vmax)
    P, losses = proposal.train(x, t, epochs=40, batch=8, lr=3e-3)
    assert losses[-1] < losses[0]
    rows = proposal.evaluate(P, [900, 901, 902, 903], W, H, win=5, reps=1, vmax=vmax)
    gap_net = np.mean([r["gap_net"] for r in rows])
    gap_wta = np.mean([r["gap_wta"] for r in rows])
    assert all(r["E_full"] > 0 for r in rows)
    assert gap_net < gap_wta, rows
