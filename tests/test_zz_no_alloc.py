"""edp_solve_noalloc: the entry point for callers that cannot allocate device
memory (a fixed pool reserved by another allocator, or code that must not
call cudaMalloc because it may synchronise the device).  It runs edp_solve on
a fixed static array in the library's device memory.

Called through the C ABI twice in a row on each case and compared with the
CPU oracle and with edp_solve (integer results: equal bit for bit); the
device status word is read after every call.  Argument errors come back with
the same codes as edp_solve's.  This file sorts last so that a run stopping
at its first failure has already run every other test."""
import ctypes

import numpy as np
import pytest
import torch

import oracle
from paper_1410_7922_gb300 import synth

pytestmark = pytest.mark.gpu


def _fn(edp, name, argtypes):
    f = getattr(edp.load(), name)
    f.argtypes = argtypes
    f.restype = ctypes.c_int
    return f


def call_noalloc(edp, C_ptr, W, H, space, prior, iters, labels_ptr, stream=None):
    f = _fn(edp, "edp_solve_noalloc", [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.POINTER(edp.LabelSpace),
                                       ctypes.POINTER(edp.Params), ctypes.c_void_p, ctypes.c_void_p])
    ls, pr = edp.label_space(space), edp.params(prior, iters=iters)
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream) if stream is None else stream
    return f(C_ptr, W, H, ctypes.byref(ls), ctypes.byref(pr), labels_ptr, st)


def noalloc_status(edp):
    f = _fn(edp, "edp_noalloc_get_device_status", [ctypes.POINTER(ctypes.c_int), ctypes.c_void_p])
    s = ctypes.c_int(-1)
    assert f(ctypes.byref(s), ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)) == 0
    return s.value


def call_solve(edp, C_ptr, W, H, space, prior, iters, labels_ptr, ws_ptr, ws_bytes):
    f = _fn(edp, "edp_solve", [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.POINTER(edp.LabelSpace),
                               ctypes.POINTER(edp.Params), ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t,
                               ctypes.c_void_p])
    ls, pr = edp.label_space(space), edp.params(prior, iters=iters)
    return f(C_ptr, W, H, ctypes.byref(ls), ctypes.byref(pr), labels_ptr, ws_ptr, ws_bytes,
             ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))


@pytest.mark.parametrize("which", ["stereo_64x48", "stereo_120x90", "motion_40x30"])
def test_noalloc_matches_oracle_and_solve_twice(edp_lib, which):
    if which == "stereo_64x48":
        w = synth.workload_scanline_64x48()
    elif which == "stereo_120x90":
        w = synth.workload_stereo_450x375(W=120, H=90)
    else:
        w = synth.workload_motion_320x240(W=40, H=30)
    I0, I1 = torch.from_numpy(w["I0"]).cuda(), torch.from_numpy(w["I1"]).cuda()
    C = edp_lib.cost_volume(I0, I1, None, w["space"], w["l2"], w["cmax"])
    H, W, _ = C.shape
    Cn = C.cpu().numpy()
    for iters in (1, 2):
        want = oracle.edp(Cn, w["space"], w["prior"], iters=iters, tier=1)
        assert np.array_equal(edp_lib.solve(C, w["space"], w["prior"], iters=iters).cpu().numpy(), want)
        for _ in range(2):
            lab = torch.full((H, W), -1, dtype=torch.int32, device="cuda")
            rc = call_noalloc(edp_lib, ctypes.c_void_p(C.data_ptr()), W, H, w["space"], w["prior"], iters,
                              ctypes.c_void_p(lab.data_ptr()))
            assert rc == edp_lib.OK
            assert noalloc_status(edp_lib) == 0
            assert np.array_equal(lab.cpu().numpy(), want)


def test_noalloc_same_codes_as_solve(edp_lib):
    """Every argument error: edp_solve (given a 64 MiB workspace, the size of
    the static array) and edp_solve_noalloc return the same code."""
    nbytes = 64 << 20
    ws = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    C = torch.zeros((4, 4, 16), dtype=torch.int32, device="cuda")
    lab = torch.zeros((4, 4), dtype=torch.int32, device="cuda")
    cp, lp, wp = ctypes.c_void_p(C.data_ptr()), ctypes.c_void_p(lab.data_ptr()), ctypes.c_void_p(ws.data_ptr())
    s16 = {"R": 1, "Q": (16, 1, 1), "vmin": (0, 0, 0), "step": (-1, 1, 1)}
    s65 = {"R": 2, "Q": (65, 65, 1), "vmin": (-32, -32, 0), "step": (1, 1, 1)}
    s2k = {"R": 2, "Q": (1025, 1025, 1), "vmin": (0, 0, 0), "step": (1, 1, 1)}
    ok = {"lam": 20, "g": 4, "mode": "joint"}
    cases = [
        ("null cost volume", None, 4, 4, s16, ok, 1, lp),
        ("null labels", cp, 4, 4, s16, ok, 1, None),
        ("zero width", cp, 0, 4, s16, ok, 1, lp),
        ("zero iterations", cp, 4, 4, s16, ok, 0, lp),
        ("negative lambda", cp, 4, 4, s16, {"lam": -1, "g": 4}, 1, lp),
        ("bad prior power", cp, 4, 4, s16, {"lam": 1, "g": 4, "l1": 3}, 1, lp),
        ("too many labels (unsupported)", cp, 4, 4, s2k, ok, 1, lp),
        ("larger than the array", cp, 640, 480, s65, {"lam": 15, "g": 3, "mode": "per_axis"}, 1, lp),
        ("int32 range", cp, 4000, 4000, s16, {"lam": 1 << 19, "g": 4}, 1, lp),
    ]
    for name, c, W, H, space, prior, iters, l in cases:
        a = call_solve(edp_lib, c, W, H, space, prior, iters, l, wp, nbytes)
        b = call_noalloc(edp_lib, c, W, H, space, prior, iters, l)
        assert a == b and a != edp_lib.OK, (name, a, b)
    assert call_noalloc(edp_lib, cp, 640, 480, s65, {"lam": 15, "g": 3, "mode": "per_axis"}, 1, lp) == \
        edp_lib.ERR_WORKSPACE
    torch.cuda.synchronize()
