"""The batched solve beyond plain parity: problems split between their own
launches and the persistent launch, capture in a CUDA graph with two
replays, and the launch-shape autotuner (every candidate shape gives the
same labels).  Integer results: equal to the oracle bit for bit."""
import numpy as np
import pytest
import torch

from paper_1410_7922_gb300 import autotune
from test_gpu_parity import _batch_items, _oracle_problem, host

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def reset(edp_lib):
    yield
    edp_lib.set_tuning(0, 0, 0)
    edp_lib.set_batch_split(172800)
    edp_lib.set_pass_pairs(edp_lib.PAIRS_AUTO)


def _check(items, iters=1):
    for it in items:
        lab, e = _oracle_problem(it["_w"], iters)
        assert np.array_equal(host(it["labels"]), lab), it["name"]
        assert tuple(int(v) for v in host(it["energy4"])) == e, it["name"]


@pytest.mark.parametrize("split", [0, 1, 1500])
def test_batched_split(edp_lib, split):
    """split 0: every problem in the persistent launch; 1: every problem on
    its own launches; 1500 pixels: the larger ones on their own."""
    edp_lib.set_batch_split(split)
    items = _batch_items(edp_lib, n=9)
    probs = edp_lib.make_problems(items)
    ws = torch.empty(edp_lib.batch_workspace_size(probs), dtype=torch.uint8, device="cuda")
    edp_lib.solve_batched(probs, ws)
    torch.cuda.synchronize()
    assert edp_lib.get_device_status(ws) == 0
    _check(items)


def test_batched_graph_capture_and_replay(edp_lib):
    """One uncaptured call (sets the kernels' attributes), a capture, then
    two replays with the outputs cleared in between."""
    edp_lib.set_batch_split(1500)
    items = _batch_items(edp_lib, n=9)
    probs = edp_lib.make_problems(items)
    ws = torch.empty(edp_lib.batch_workspace_size(probs), dtype=torch.uint8, device="cuda")
    edp_lib.solve_batched(probs, ws)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    st = torch.cuda.Stream()
    st.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(st):
        with torch.cuda.graph(g, stream=st):
            edp_lib.solve_batched(probs, ws, stream=st)
    torch.cuda.current_stream().wait_stream(st)
    for _ in range(2):
        for it in items:
            it["labels"].fill_(-1)
            it["energy4"].fill_(-1)
        g.replay()
        torch.cuda.synchronize()
        assert edp_lib.get_device_status(ws) == 0
        _check(items)


def test_batched_autotune_candidates_agree(edp_lib):
    """autotune.tune times every (rows per block, warps per row) candidate;
    each candidate's labels are the same, and equal to the oracle's."""
    items = _batch_items(edp_lib, n=6)
    probs = edp_lib.make_problems(items)
    ws = torch.empty(edp_lib.batch_workspace_size(probs), dtype=torch.uint8, device="cuda")
    results = []

    def run():
        for it in items:
            it["labels"].fill_(-1)
        edp_lib.solve_batched(probs, ws)
        torch.cuda.synchronize()
        results.append([it["labels"].clone() for it in items])

    r, w, ms, table = autotune.tune(run, rows=(0, 1, 2), warps=(0, 2, 4), reps=1)
    assert len(table) >= 2 and ms > 0
    for res in results[1:]:
        assert all(torch.equal(a, b) for a, b in zip(results[0], res))
    _check(items)
