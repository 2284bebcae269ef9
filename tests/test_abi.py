"""C-ABI checks that need no GPU: the library builds, loads, and exports every
function include/edp.h declares; host-side argument validation."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_functions():
    txt = open(os.path.join(ROOT, "include", "edp.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(edp_[a-z_0-9]+)\s*\(", txt)))


@pytest.fixture(scope="module")
def lib():
    from paper_1410_7922_gb300 import build
    build.build()
    from paper_1410_7922_gb300 import edp
    return edp.load()


def test_header_declares_core_calls():
    names = header_functions()
    for n in ("edp_cost_volume", "edp_scanline_dp", "edp_solve", "edp_energy"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    for name in header_functions():
        assert hasattr(lib, name), name


def test_binding_covers_header():
    from paper_1410_7922_gb300 import edp
    assert sorted(edp.exported_symbols()) == header_functions()


def test_host_validation_without_gpu(lib):
    from paper_1410_7922_gb300 import edp
    space = {"R": 1, "Q": (16, 1, 1), "vmin": (0, 0, 0), "step": (-1, 1, 1)}
    prior = {"lam": 20, "g": 4}
    ls, pr = edp.label_space(space), edp.params(prior)
    # null pointers are rejected before any CUDA call
    assert lib.edp_solve(None, 8, 8, ctypes.byref(ls), ctypes.byref(pr), None, None, 0, None) == edp.ERR_INVALID_ARG
    assert lib.edp_energy(None, None, 8, 8, ctypes.byref(ls), ctypes.byref(pr), None, None) == edp.ERR_INVALID_ARG
    # bad label space
    bad = edp.label_space({"R": 4, "Q": (2, 2, 2)})
    assert lib.edp_workspace_size(edp.OP_SOLVE, 8, 8, ctypes.byref(bad), ctypes.byref(pr)) == 0
    bad2 = edp.label_space({"R": 1, "Q": (16, 1, 1)})
    bad2.Q[1] = 2  # an unused axis with more than one label
    assert lib.edp_workspace_size(edp.OP_SOLVE, 8, 8, ctypes.byref(bad2), ctypes.byref(pr)) == 0
    # workspace sizes grow with the image and iterations
    a = edp.workspace_size(edp.OP_SOLVE, 64, 48, space, prior, 1)
    b = edp.workspace_size(edp.OP_SOLVE, 64, 48, space, prior, 6)
    assert a >= 4 * 64 * 48 * 16 * 4 and b > a
    assert edp.status_string(edp.ERR_TIMEOUT) == "EDP_ERR_TIMEOUT"
    assert lib.edp_set_tuning(-1, 0, 0, 0) == edp.ERR_INVALID_ARG
    assert lib.edp_set_tuning(0, 0, 0, 6) == edp.ERR_INVALID_ARG
    assert lib.edp_set_tuning(0, 0, 13, 0) == edp.ERR_INVALID_ARG
    # the cost-volume and network switches take 0 or 1 (and are left at their defaults)
    assert lib.edp_set_fused_cost(2) == edp.ERR_INVALID_ARG
    assert lib.edp_set_fused_cost(-1) == edp.ERR_INVALID_ARG
    assert lib.edp_set_net_tensor_cores(2) == edp.ERR_INVALID_ARG
    edp.set_fused_cost(False)
    edp.set_net_tensor_cores(True)
    # the network status reader checks its arguments before touching the device
    assert lib.edp_net_get_device_status(None, 0, None, None) == edp.ERR_INVALID_ARG
    # pass schedule: off, on, or paired when every band is resident (default)
    assert lib.edp_set_pass_pairs(3) == edp.ERR_INVALID_ARG
    assert lib.edp_set_pass_pairs(-1) == edp.ERR_INVALID_ARG
    for mode in (edp.PAIRS_OFF, edp.PAIRS_ON, True, False, edp.PAIRS_AUTO):
        edp.set_pass_pairs(mode)
    assert edp.last_pass_launches() >= 0
