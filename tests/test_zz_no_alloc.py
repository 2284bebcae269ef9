"""edp_solve_noalloc: the workspace-free entry point, for callers that cannot
allocate device memory.  Called through the C ABI twice in a row and compared
with edp_solve (the results are integers: equal bit for bit); sizes beyond
the fixed scratch are rejected before any work is enqueued."""
import ctypes

import numpy as np
import pytest
import torch

from paper_1410_7922_gb300 import synth

pytestmark = pytest.mark.gpu


def call_noalloc(edp, C, space, prior, iters, labels):
    lib = edp.load()
    f = lib.edp_solve_noalloc
    f.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.POINTER(edp.LabelSpace),
                  ctypes.POINTER(edp.Params), ctypes.c_void_p, ctypes.c_void_p]
    f.restype = ctypes.c_int
    H, W, _ = C.shape
    ls, pr = edp.label_space(space), edp.params(prior, iters=iters)
    return f(ctypes.c_void_p(C.data_ptr()), W, H, ctypes.byref(ls), ctypes.byref(pr),
             ctypes.c_void_p(labels.data_ptr()), ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))


@pytest.mark.parametrize("which", ["stereo_64x48", "stereo_240x180", "motion_48x36"])
def test_noalloc_matches_solve_twice(edp_lib, which):
    if which == "stereo_64x48":
        w = synth.workload_scanline_64x48()
    elif which == "stereo_240x180":
        w = synth.workload_stereo_450x375(W=240, H=180)
    else:
        w = synth.workload_motion_320x240(W=48, H=36)
    I0, I1 = torch.from_numpy(w["I0"]).cuda(), torch.from_numpy(w["I1"]).cuda()
    C = edp_lib.cost_volume(I0, I1, None, w["space"], w["l2"], w["cmax"])
    H, W, _ = C.shape
    for iters in (1, 2):
        want = edp_lib.solve(C, w["space"], w["prior"], iters=iters).cpu().numpy()
        for _ in range(2):
            lab = torch.full((H, W), -1, dtype=torch.int32, device="cuda")
            assert call_noalloc(edp_lib, C, w["space"], w["prior"], iters, lab) == edp_lib.OK
            torch.cuda.synchronize()
            assert np.array_equal(lab.cpu().numpy(), want)


def test_noalloc_rejects_oversize(edp_lib):
    space = {"R": 2, "Q": (65, 65, 1), "vmin": (-32, -32, 0), "step": (1, 1, 1)}
    C = torch.zeros((2, 2, 1), dtype=torch.int32, device="cuda")  # never read: the size check comes first
    lab = torch.zeros((480, 640), dtype=torch.int32, device="cuda")
    lib = edp_lib.load()
    f = lib.edp_solve_noalloc
    f.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.POINTER(edp_lib.LabelSpace),
                  ctypes.POINTER(edp_lib.Params), ctypes.c_void_p, ctypes.c_void_p]
    f.restype = ctypes.c_int
    ls, pr = edp_lib.label_space(space), edp_lib.params({"lam": 15, "g": 3, "mode": "per_axis"})
    rc = f(ctypes.c_void_p(C.data_ptr()), 640, 480, ctypes.byref(ls), ctypes.byref(pr),
           ctypes.c_void_p(lab.data_ptr()), None)
    assert rc == edp_lib.ERR_WORKSPACE
