"""Thin Python binding of libedp.so (the C ABI in include/edp.h).

Argument marshalling only: every step of the computation runs in the CUDA
library.  Device buffers are torch tensors (torch provides device memory and
streams); the functions take the same names as the C entry points without the
``edp_`` prefix.  There is no fallback: if the library cannot be loaded, every
call raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libedp.so")

OK, ERR_INVALID_ARG, ERR_UNSUPPORTED, ERR_WORKSPACE, ERR_RANGE, ERR_TIMEOUT, ERR_CUDA = range(7)
PRIOR = {"joint": 0, "per_axis": 1}
COST = {"pair": 0, "pair_stereo3": 1, "composite": 2}
OP_SCANLINE_DP, OP_SOLVE, OP_SOLVE_IMAGES, OP_COARSE, OP_SCANLINE_MARGINALS = 1, 2, 3, 4, 5


class EdpError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__(f"{what}: {status_string(code)} ({code})")
        self.code = code


class LabelSpace(ctypes.Structure):
    _fields_ = [("R", ctypes.c_int32), ("Q", ctypes.c_int32 * 3), ("vmin", ctypes.c_int32 * 3),
                ("step", ctypes.c_int32 * 3)]


class Params(ctypes.Structure):
    _fields_ = [("lam", ctypes.c_int32), ("g", ctypes.c_int32), ("l1", ctypes.c_int32),
                ("prior_mode", ctypes.c_int32), ("l2", ctypes.c_int32), ("cmax", ctypes.c_int32),
                ("cost_mode", ctypes.c_int32), ("iters", ctypes.c_int32)]


class Problem(ctypes.Structure):
    _fields_ = [("I0", ctypes.c_void_p), ("I1", ctypes.c_void_p), ("I2", ctypes.c_void_p),
                ("W", ctypes.c_int32), ("H", ctypes.c_int32), ("pitch", ctypes.c_int32),
                ("space", LabelSpace), ("params", Params), ("labels", ctypes.c_void_p),
                ("energy4", ctypes.c_void_p)]


_lib = None


def load() -> ctypes.CDLL:
    """Load libedp.so (built by paper_1410_7922_gb300.build)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: run paper_1410_7922_gb300/build.py "
                           "(or __graft_entry__.build()); there is no CPU fallback")
    lib = ctypes.CDLL(LIB_PATH)
    P, I, SZ = ctypes.c_void_p, ctypes.c_int, ctypes.c_size_t
    LS, PR = ctypes.POINTER(LabelSpace), ctypes.POINTER(Params)
    sig = {
        "edp_version": ([], I),
        "edp_status_string": ([I], ctypes.c_char_p),
        "edp_workspace_size": ([I, I, I, LS, PR], SZ),
        "edp_set_tuning": ([I, I, I, I], I),
        "edp_set_profile_events": ([P, I], I),
        "edp_set_pass_pairs": ([I], I),
        "edp_set_fused_cost": ([I], I),
        "edp_last_pass_launches": ([], I),
        "edp_last_pass_kernel": ([], ctypes.c_char_p),
        "edp_set_spin_limit": ([ctypes.c_longlong], I),
        "edp_set_batch_split": ([ctypes.c_longlong], I),
        "edp_test_hold_band": ([I], I),
        "edp_set_trace": ([P, SZ], I),
        "edp_cost_volume": ([P, P, P, I, I, I, LS, PR, P, P], I),
        "edp_scanline_dp": ([P, I, I, LS, PR, P, P, P, SZ, P], I),
        "edp_solve": ([P, I, I, LS, PR, P, P, SZ, P], I),
        "edp_scanline_marginals": ([P, I, I, LS, PR, P, P, P, SZ, P], I),
        "edp_energy": ([P, P, I, I, LS, PR, P, P], I),
        "edp_edge_weights": ([P, I, I, I, I, I, P, P, P], I),
        "edp_solve_weighted": ([P, I, I, LS, PR, P, P, I, P, P, SZ, P], I),
        "edp_energy_weighted": ([P, P, I, I, LS, PR, P, P, P, P], I),
        "edp_solve_images": ([P, P, P, I, I, I, LS, PR, P, P, P, SZ, P], I),
        "edp_solve_images_host": ([P, P, P, I, I, LS, PR, P, P, P, SZ, P], I),
        "edp_get_device_status": ([P, SZ, ctypes.POINTER(I), P], I),
        "edp_batch_workspace_size": ([ctypes.POINTER(Problem), I], SZ),
        "edp_workspace_size_windowed": ([I, I, LS, PR, I], SZ),
        "edp_cost_window": ([P, P, P, I, I, I, LS, PR, P, I, P, P], I),
        "edp_solve_windowed": ([P, P, I, I, I, LS, PR, P, P, SZ, P], I),
        "edp_wta": ([P, P, I, I, I, LS, PR, I, P, P, P], I),
        "edp_coarse_labels": ([P, P, I, I, I, LS, PR, P, P, SZ, P], I),
        "edp_net_features_labels": ([P, P, P, I, I, I, LS, PR, ctypes.c_float, P, P], I),
        "edp_net_centres_residual": ([P, P, I, LS, I, P, P], I),
        "edp_net_targets": ([P, P, I, LS, P, P], I),
        "edp_window_edge_count": ([P, P, I, I, LS, P, P], I),
        "edp_net_param_count": ([], ctypes.c_longlong),
        "edp_net_workspace_size": ([I, I, I], SZ),
        "edp_net_activation_offset": ([I, I, I, I], SZ),
        "edp_net_forward": ([P, P, I, I, I, P, P, SZ, P], I),
        "edp_net_backward": ([P, P, P, I, I, I, P, P, P, SZ, P], I),
        "edp_net_adam": ([P, P, P, P, ctypes.c_float, ctypes.c_float, ctypes.c_float, ctypes.c_float, I, P], I),
        "edp_net_features": ([P, P, P, P, I, I, LS, ctypes.c_float, ctypes.c_float, P, P], I),
        "edp_net_centres": ([P, I, LS, P, P], I),
        "edp_solve_noalloc": ([P, I, I, LS, PR, P, P], I),
        "edp_noalloc_get_device_status": ([ctypes.POINTER(I), P], I),
        "edp_set_net_tensor_cores": ([I], I),
        "edp_net_get_device_status": ([P, SZ, ctypes.POINTER(I), P], I),
        "edp_solve_batched": ([ctypes.POINTER(Problem), I, P, SZ, P], I),
    }
    for name, (args, res) in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    _lib = lib
    return lib


def exported_symbols() -> list[str]:
    return ["edp_version", "edp_status_string", "edp_workspace_size", "edp_set_tuning", "edp_set_profile_events",
            "edp_set_trace",
            "edp_cost_volume", "edp_scanline_dp", "edp_solve", "edp_energy", "edp_solve_images",
            "edp_solve_images_host", "edp_get_device_status", "edp_batch_workspace_size",
            "edp_solve_batched", "edp_workspace_size_windowed", "edp_cost_window", "edp_solve_windowed",
            "edp_wta", "edp_net_param_count", "edp_net_workspace_size", "edp_net_activation_offset", "edp_net_forward", "edp_net_backward",
            "edp_net_adam", "edp_net_features", "edp_net_centres", "edp_solve_noalloc",
            "edp_noalloc_get_device_status", "edp_coarse_labels",
            "edp_net_features_labels", "edp_net_centres_residual", "edp_net_targets", "edp_window_edge_count", "edp_scanline_marginals",
            "edp_set_pass_pairs", "edp_set_fused_cost", "edp_last_pass_launches", "edp_last_pass_kernel", "edp_set_spin_limit",
            "edp_test_hold_band", "edp_set_batch_split", "edp_edge_weights", "edp_solve_weighted",
            "edp_energy_weighted", "edp_set_net_tensor_cores", "edp_net_get_device_status"]


def status_string(code: int) -> str:
    return load().edp_status_string(int(code)).decode()


def _check(rc: int, what: str) -> None:
    if rc != OK:
        raise EdpError(rc, what)


def label_space(space: dict) -> LabelSpace:
    s = LabelSpace()
    s.R = int(space["R"])
    Q = list(space["Q"]) + [1] * 3
    vmin = list(space.get("vmin", (0, 0, 0))) + [0] * 3
    step = list(space.get("step", (1, 1, 1))) + [1] * 3
    for r in range(3):
        s.Q[r] = int(Q[r]) if r < s.R else 1
        s.vmin[r] = int(vmin[r])
        s.step[r] = int(step[r])
    return s


def params(prior: dict, l2: int = 1, cmax: int = 20, cost_mode: str = "pair", iters: int = 1) -> Params:
    p = Params()
    p.lam = int(prior["lam"])
    p.g = int(prior["g"])
    p.l1 = int(prior.get("l1", 1))
    p.prior_mode = PRIOR[prior.get("mode", "joint")]
    p.l2 = int(l2)
    p.cmax = int(cmax)
    p.cost_mode = COST[cost_mode]
    p.iters = int(iters)
    return p


def n_labels(space: dict) -> int:
    q = 1
    for r in range(int(space["R"])):
        q *= int(space["Q"][r])
    return q


def _dev(t: torch.Tensor | None, dtype, name: str):
    if t is None:
        return None
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream) -> ctypes.c_void_p:
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


def version() -> int:
    return load().edp_version()


def set_tuning(rows_per_block: int = 0, labels_per_lane: int = 0, general_kernel: int = 0,
               warps_per_row: int = 0) -> None:
    """Launch shape of the DP kernels (0 = automatic); results never depend on it.
    general_kernel: 1 = one-axis spaces take the multi-axis kernel, 2 = and
    multi-axis spaces its lane-group form, 3 = two-axis spaces take the
    multi-axis kernel instead of the two-axis line kernel, 4 = two-axis spaces
    take the line kernel wherever it is built, 5 = as 4 with one lane per label
    line also where lines are split over lane pairs by default (65 x 65)."""
    _check(load().edp_set_tuning(int(rows_per_block), int(labels_per_lane), int(warps_per_row),
                                 int(general_kernel)), "set_tuning")


_prof_keep = None


PAIRS_OFF, PAIRS_ON, PAIRS_AUTO = 0, 1, 2


def set_pass_pairs(mode) -> None:
    """Pass schedule: PAIRS_OFF (one launch per pass), PAIRS_ON (paired sweeps
    P1 + P2, P3 + P4) or PAIRS_AUTO (paired when every row band is resident;
    the default).  A bool selects PAIRS_ON / PAIRS_OFF."""
    if isinstance(mode, bool):
        mode = PAIRS_ON if mode else PAIRS_OFF
    _check(load().edp_set_pass_pairs(int(mode)), "set_pass_pairs")


def last_pass_launches() -> int:
    """Scan-pass launches of the most recent solve in this process."""
    return int(load().edp_last_pass_launches())


def set_spin_limit(polls: int = 0) -> None:
    """Polls before a wait between row bands gives up (0: the default)."""
    _check(load().edp_set_spin_limit(int(polls)), "set_spin_limit")


def set_batch_split(min_pixels: int) -> None:
    """edp_solve_batched: problems of at least min_pixels pixels get their
    own launches (0: every problem in the persistent launch)."""
    _check(load().edp_set_batch_split(int(min_pixels)), "set_batch_split")


def test_hold_band(band: int = 0) -> None:
    """Timeout test hook: the first row of `band` (> 0) waits for records
    that are never written (0: off)."""
    _check(load().edp_test_hold_band(int(band)), "test_hold_band")


def last_pass_kernel() -> str:
    """Name of the scan-pass kernel the most recent solve launched."""
    return load().edp_last_pass_kernel().decode()


def set_profile_events(events) -> None:
    """Record torch.cuda.Event pairs around each scan-pass launch (None: off)."""
    global _prof_keep
    lib = load()
    if not events:
        _check(lib.edp_set_profile_events(None, 0), "set_profile_events")
        _prof_keep = None
        return
    for e in events:  # torch creates the CUDA event lazily, on first record
        if not e.cuda_event:
            e.record()
    arr = (ctypes.c_void_p * len(events))(*[ctypes.c_void_p(e.cuda_event) for e in events])
    _prof_keep = (arr, events)
    _check(lib.edp_set_profile_events(arr, len(events)), "set_profile_events")


def set_trace(buf) -> None:
    """Per-band trace of the scan passes into a CUDA uint8/int64 tensor (None: off)."""
    if buf is None:
        _check(load().edp_set_trace(None, 0), "set_trace")
        return
    _check(load().edp_set_trace(ctypes.c_void_p(buf.data_ptr()), buf.numel() * buf.element_size()), "set_trace")


def workspace_size(op: int, W: int, H: int, space: dict, prior: dict, iters: int = 1, **kw) -> int:
    ls, pr = label_space(space), params(prior, iters=iters, **kw)
    n = load().edp_workspace_size(int(op), int(W), int(H), ctypes.byref(ls), ctypes.byref(pr))
    if n == 0:
        raise EdpError(ERR_INVALID_ARG, "workspace_size")
    return int(n)


def workspace(op: int, W: int, H: int, space: dict, prior: dict, iters: int = 1, device="cuda", **kw):
    """A device workspace tensor of the right size (256-byte aligned)."""
    n = workspace_size(op, W, H, space, prior, iters, **kw)
    return torch.empty(n, dtype=torch.uint8, device=device)


def cost_volume(I0, I1, I2, space: dict, l2: int, cmax: int, cost_mode: str = "pair", out=None, stream=None):
    """edp_cost_volume: uint8 [H][W] images -> int32 [H][W][Q]."""
    H, W = I0.shape
    if out is None:
        out = torch.empty((H, W, n_labels(space)), dtype=torch.int32, device=I0.device)
    ls = label_space(space)
    pr = params({"lam": 0, "g": 1}, l2=l2, cmax=cmax, cost_mode=cost_mode)
    rc = load().edp_cost_volume(_dev(I0, torch.uint8, "I0"), _dev(I1, torch.uint8, "I1"),
                                _dev(I2, torch.uint8, "I2"), W, H, I0.stride(0), ctypes.byref(ls),
                                ctypes.byref(pr), _dev(out, torch.int32, "C"), _stream(stream))
    _check(rc, "cost_volume")
    return out


def scanline_dp(C, space: dict, prior: dict, ws=None, labels=None, row_energy=None, stream=None):
    """edp_scanline_dp: returns (labels int32 [H][W], row_energy int64 [H])."""
    H, W, _ = C.shape
    if ws is None:
        ws = workspace(OP_SCANLINE_DP, W, H, space, prior, device=C.device)
    if labels is None:
        labels = torch.empty((H, W), dtype=torch.int32, device=C.device)
    if row_energy is None:
        row_energy = torch.empty(H, dtype=torch.int64, device=C.device)
    ls, pr = label_space(space), params(prior)
    rc = load().edp_scanline_dp(_dev(C, torch.int32, "C"), W, H, ctypes.byref(ls), ctypes.byref(pr),
                                _dev(labels, torch.int32, "labels"), _dev(row_energy, torch.int64, "row_energy"),
                                _dev(ws, torch.uint8, "ws"), ws.numel(), _stream(stream))
    _check(rc, "scanline_dp")
    return labels, row_energy


def scanline_marginals(C, space: dict, prior: dict, ws=None, labels=None, marginals=False, stream=None):
    """edp_scanline_marginals: labels int32 [H][W] (argmin of the min-marginals),
    and the marginals int32 [H][W][Q] when marginals=True."""
    H, W, Q = C.shape
    if ws is None:
        ws = workspace(OP_SCANLINE_MARGINALS, W, H, space, prior, device=C.device)
    if labels is None:
        labels = torch.empty((H, W), dtype=torch.int32, device=C.device)
    marg = torch.empty((H, W, Q), dtype=torch.int32, device=C.device) if marginals else None
    ls, pr = label_space(space), params(prior)
    rc = load().edp_scanline_marginals(_dev(C, torch.int32, "C"), W, H, ctypes.byref(ls), ctypes.byref(pr),
                                       _dev(labels, torch.int32, "labels"),
                                       _dev(marg, torch.int32, "marginals") if marginals else None,
                                       _dev(ws, torch.uint8, "ws"), ws.numel(), _stream(stream))
    _check(rc, "scanline_marginals")
    return (labels, marg) if marginals else labels


def solve(C, space: dict, prior: dict, iters: int = 1, ws=None, labels=None, stream=None):
    """edp_solve (Algorithm 1): labels int32 [H][W]."""
    H, W, _ = C.shape
    if ws is None:
        ws = workspace(OP_SOLVE, W, H, space, prior, iters, device=C.device)
    if labels is None:
        labels = torch.empty((H, W), dtype=torch.int32, device=C.device)
    ls, pr = label_space(space), params(prior, iters=iters)
    rc = load().edp_solve(_dev(C, torch.int32, "C"), W, H, ctypes.byref(ls), ctypes.byref(pr),
                          _dev(labels, torch.int32, "labels"), _dev(ws, torch.uint8, "ws"), ws.numel(),
                          _stream(stream))
    _check(rc, "solve")
    return labels


def energy(C, labels, space: dict, prior: dict, out=None, stream=None):
    """edp_energy: int64 [4] = (data, smooth_h, smooth_v, total) on the device."""
    H, W = labels.shape
    if out is None:
        out = torch.empty(4, dtype=torch.int64, device=labels.device)
    ls, pr = label_space(space), params(prior)
    rc = load().edp_energy(_dev(C, torch.int32, "C"), _dev(labels, torch.int32, "labels"), W, H,
                           ctypes.byref(ls), ctypes.byref(pr), _dev(out, torch.int64, "out4"), _stream(stream))
    _check(rc, "energy")
    return out


def edge_weights(I, threshold: int = 10, factor: int = 2, wh=None, wv=None, stream=None):
    """edp_edge_weights: per-edge prior multipliers (wh, wv) uint8 [H][W] of
    the locally adaptive prior from a device image."""
    H, W = I.shape
    if wh is None:
        wh = torch.empty((H, W), dtype=torch.uint8, device=I.device)
    if wv is None:
        wv = torch.empty((H, W), dtype=torch.uint8, device=I.device)
    rc = load().edp_edge_weights(_dev(I, torch.uint8, "I"), W, H, I.stride(0), int(threshold), int(factor),
                                 _dev(wh, torch.uint8, "wh"), _dev(wv, torch.uint8, "wv"), _stream(stream))
    _check(rc, "edge_weights")
    return wh, wv


def solve_weighted(C, space: dict, prior: dict, wh, wv, max_weight: int, iters: int = 1, ws=None, labels=None,
                   stream=None):
    """edp_solve_weighted: EDP with per-edge prior multipliers (one-axis spaces)."""
    H, W, _ = C.shape
    if ws is None:
        ws = workspace(OP_SOLVE, W, H, space, prior, iters, device=C.device)
    if labels is None:
        labels = torch.empty((H, W), dtype=torch.int32, device=C.device)
    ls, pr = label_space(space), params(prior, iters=iters)
    rc = load().edp_solve_weighted(_dev(C, torch.int32, "C"), W, H, ctypes.byref(ls), ctypes.byref(pr),
                                   _dev(wh, torch.uint8, "wh"), _dev(wv, torch.uint8, "wv"), int(max_weight),
                                   _dev(labels, torch.int32, "labels"), _dev(ws, torch.uint8, "ws"), ws.numel(),
                                   _stream(stream))
    _check(rc, "solve_weighted")
    return labels


def energy_weighted(C, labels, space: dict, prior: dict, wh, wv, out=None, stream=None):
    """edp_energy_weighted: int64 [4] with per-edge prior multipliers."""
    H, W = labels.shape
    if out is None:
        out = torch.empty(4, dtype=torch.int64, device=labels.device)
    ls, pr = label_space(space), params(prior)
    rc = load().edp_energy_weighted(_dev(C, torch.int32, "C"), _dev(labels, torch.int32, "labels"), W, H,
                                    ctypes.byref(ls), ctypes.byref(pr), _dev(wh, torch.uint8, "wh"),
                                    _dev(wv, torch.uint8, "wv"), _dev(out, torch.int64, "out4"), _stream(stream))
    _check(rc, "energy_weighted")
    return out


def solve_images(I0, I1, I2, space: dict, prior: dict, l2: int, cmax: int, cost_mode: str = "pair",
                 iters: int = 1, ws=None, labels=None, energy4=None, stream=None):
    """edp_solve_images: device images -> (labels, energy4)."""
    H, W = I0.shape
    if ws is None:
        ws = workspace(OP_SOLVE_IMAGES, W, H, space, prior, iters, device=I0.device)
    if labels is None:
        labels = torch.empty((H, W), dtype=torch.int32, device=I0.device)
    if energy4 is None:
        energy4 = torch.empty(4, dtype=torch.int64, device=I0.device)
    ls = label_space(space)
    pr = params(prior, l2=l2, cmax=cmax, cost_mode=cost_mode, iters=iters)
    rc = load().edp_solve_images(_dev(I0, torch.uint8, "I0"), _dev(I1, torch.uint8, "I1"),
                                 _dev(I2, torch.uint8, "I2"), W, H, I0.stride(0), ctypes.byref(ls),
                                 ctypes.byref(pr), _dev(labels, torch.int32, "labels"),
                                 _dev(energy4, torch.int64, "energy4"), _dev(ws, torch.uint8, "ws"),
                                 ws.numel(), _stream(stream))
    _check(rc, "solve_images")
    return labels, energy4


def solve_images_host(I0, I1, I2, space: dict, prior: dict, l2: int, cmax: int, ws, cost_mode: str = "pair",
                      iters: int = 1, labels_out: np.ndarray | None = None, energy_out: np.ndarray | None = None,
                      stream=None):
    """edp_solve_images_host: host uint8 images (numpy or pinned CPU tensors)
    -> host labels and energy; synchronises the stream."""
    def hptr(a):
        if a is None:
            return None
        if isinstance(a, torch.Tensor):
            assert a.device.type == "cpu" and a.is_contiguous()
            return ctypes.c_void_p(a.data_ptr())
        assert a.flags["C_CONTIGUOUS"]
        return a.ctypes.data_as(ctypes.c_void_p)

    H, W = I0.shape
    if labels_out is None:
        labels_out = np.empty((H, W), dtype=np.int32)
    if energy_out is None:
        energy_out = np.empty(4, dtype=np.int64)
    ls = label_space(space)
    pr = params(prior, l2=l2, cmax=cmax, cost_mode=cost_mode, iters=iters)
    rc = load().edp_solve_images_host(hptr(I0), hptr(I1), hptr(I2), W, H, ctypes.byref(ls), ctypes.byref(pr),
                                      hptr(labels_out), hptr(energy_out), _dev(ws, torch.uint8, "ws"),
                                      ws.numel(), _stream(stream))
    _check(rc, "solve_images_host")
    return labels_out, energy_out


def get_device_status(ws, stream=None) -> int:
    st = ctypes.c_int(0)
    rc = load().edp_get_device_status(_dev(ws, torch.uint8, "ws"), ws.numel(), ctypes.byref(st), _stream(stream))
    _check(rc, "get_device_status")
    return int(st.value)


def make_problems(items) -> ctypes.Array:
    """Problem descriptors from dicts with device tensors I0, I1, I2 (or
    None), labels, energy4 (or None) and space / prior / l2 / cmax /
    cost_mode / iters.  Keep the returned array alive while it is in use."""
    arr = (Problem * len(items))()
    for k, it in enumerate(items):
        H, W = it["I0"].shape
        pr = arr[k]
        pr.I0 = _dev(it["I0"], torch.uint8, "I0")
        pr.I1 = _dev(it["I1"], torch.uint8, "I1")
        pr.I2 = _dev(it.get("I2"), torch.uint8, "I2")
        pr.W, pr.H, pr.pitch = W, H, it["I0"].stride(0)
        pr.space = label_space(it["space"])
        pr.params = params(it["prior"], l2=it.get("l2", 1), cmax=it.get("cmax", 20),
                           cost_mode=it.get("cost_mode", "pair"), iters=it.get("iters", 1))
        pr.labels = _dev(it["labels"], torch.int32, "labels")
        pr.energy4 = _dev(it.get("energy4"), torch.int64, "energy4")
    return arr


def batch_workspace_size(problems: ctypes.Array) -> int:
    n = load().edp_batch_workspace_size(problems, len(problems))
    if n == 0:
        raise EdpError(ERR_INVALID_ARG, "batch_workspace_size")
    return int(n)


def solve_batched(problems: ctypes.Array, ws, stream=None) -> None:
    """edp_solve_batched over descriptors from make_problems."""
    rc = load().edp_solve_batched(problems, len(problems), _dev(ws, torch.uint8, "ws"), ws.numel(), _stream(stream))
    _check(rc, "solve_batched")


def cost_window(I0, I1, I2, space: dict, l2: int, cmax: int, centre, win: int, cost_mode: str = "pair",
                out=None, stream=None):
    """edp_cost_window: box costs int32 [H][W][win^R] around int32 centres [H][W][R]."""
    H, W = I0.shape
    R = int(space["R"])
    if out is None:
        out = torch.empty((H, W, win ** R), dtype=torch.int32, device=I0.device)
    ls = label_space(space)
    pr = params({"lam": 0, "g": 1}, l2=l2, cmax=cmax, cost_mode=cost_mode)
    rc = load().edp_cost_window(_dev(I0, torch.uint8, "I0"), _dev(I1, torch.uint8, "I1"),
                                _dev(I2, torch.uint8, "I2"), W, H, I0.stride(0), ctypes.byref(ls),
                                ctypes.byref(pr), _dev(centre, torch.int32, "centre"), int(win),
                                _dev(out, torch.int32, "Cw"), _stream(stream))
    _check(rc, "cost_window")
    return out


def workspace_windowed(W: int, H: int, space: dict, prior: dict, win: int, iters: int = 1, device="cuda"):
    ls, pr = label_space(space), params(prior, iters=iters)
    n = load().edp_workspace_size_windowed(int(W), int(H), ctypes.byref(ls), ctypes.byref(pr), int(win))
    if n == 0:
        raise EdpError(ERR_INVALID_ARG, "workspace_size_windowed")
    return torch.empty(int(n), dtype=torch.uint8, device=device)


def solve_windowed(Cw, centre, win: int, space: dict, prior: dict, iters: int = 1, ws=None, labels=None,
                   stream=None):
    """edp_solve_windowed: full-space labels int32 [H][W]."""
    H, W, _ = Cw.shape
    if ws is None:
        ws = workspace_windowed(W, H, space, prior, win, iters, device=Cw.device)
    if labels is None:
        labels = torch.empty((H, W), dtype=torch.int32, device=Cw.device)
    ls, pr = label_space(space), params(prior, iters=iters)
    rc = load().edp_solve_windowed(_dev(Cw, torch.int32, "Cw"), _dev(centre, torch.int32, "centre"), int(win), W, H,
                                   ctypes.byref(ls), ctypes.byref(pr), _dev(labels, torch.int32, "labels"),
                                   _dev(ws, torch.uint8, "ws"), ws.numel(), _stream(stream))
    _check(rc, "solve_windowed")
    return labels


def wta(I0, I1, space: dict, l2: int, cmax: int, radius: int = 0, stream=None):
    """edp_wta: (labels int32 [H][W], cost int32 [H][W]) over the full label
    space, costs summed over a (2 radius + 1)^2 pixel window."""
    H, W = I0.shape
    lab = torch.empty((H, W), dtype=torch.int32, device=I0.device)
    cost = torch.empty((H, W), dtype=torch.int32, device=I0.device)
    ls = label_space(space)
    pr = params({"lam": 0, "g": 1}, l2=l2, cmax=cmax)
    rc = load().edp_wta(_dev(I0, torch.uint8, "I0"), _dev(I1, torch.uint8, "I1"), W, H, I0.stride(0),
                        ctypes.byref(ls), ctypes.byref(pr), int(radius), _dev(lab, torch.int32, "labels"),
                        _dev(cost, torch.int32, "cost"), _stream(stream))
    _check(rc, "wta")
    return lab, cost


def net_param_count() -> int:
    return int(load().edp_net_param_count())


def net_workspace(N: int, H: int, W: int, device="cuda"):
    n = load().edp_net_workspace_size(int(N), int(H), int(W))
    if n == 0:
        raise EdpError(ERR_INVALID_ARG, "net_workspace_size")
    return torch.empty(int(n), dtype=torch.uint8, device=device)


NET_CHANNELS = (5, 32, 32, 32, 32, 32, 2)


def set_fused_cost(on: bool) -> None:
    """edp_set_fused_cost: edp_solve_images computes the pair cost from the
    images inside the split line kernel (True) or always builds the cost
    volume first (False, the default)."""
    _check(load().edp_set_fused_cost(1 if on else 0), "set_fused_cost")


def set_net_tensor_cores(on: bool) -> None:
    """edp_set_net_tensor_cores: the 32 -> 32 convolutions on the tensor cores
    (True, the default) or on the CUDA cores (False)."""
    _check(load().edp_set_net_tensor_cores(1 if on else 0), "set_net_tensor_cores")


def net_device_status(ws, stream=None) -> int:
    """edp_net_get_device_status: the network workspace's status word."""
    s = ctypes.c_int(-1)
    _check(load().edp_net_get_device_status(_dev(ws, torch.uint8, "ws"), ws.numel(), ctypes.byref(s), _stream(stream)),
           "net_get_device_status")
    return s.value


def net_activations(ws, N: int, H: int, W: int) -> list:
    """The inputs of the six layers that the last net_forward left in ws
    (bf16 [N][H][W][C] views)."""
    out = []
    for layer in range(6):
        off = int(load().edp_net_activation_offset(int(N), int(H), int(W), layer))
        n = N * H * W * NET_CHANNELS[layer]
        out.append(ws[off:off + 2 * n].view(torch.bfloat16).view(N, H, W, NET_CHANNELS[layer]))
    return out


def net_forward(params_f32, x_bf16, ws, out=None, stream=None):
    """edp_net_forward: x bf16 [N][H][W][5] -> float32 [N][H][W][2]."""
    N, H, W, _ = x_bf16.shape
    if out is None:
        out = torch.empty((N, H, W, 2), dtype=torch.float32, device=x_bf16.device)
    rc = load().edp_net_forward(_dev(params_f32, torch.float32, "params"), _dev(x_bf16, torch.bfloat16, "x"), N, H, W,
                                _dev(out, torch.float32, "out"), _dev(ws, torch.uint8, "ws"), ws.numel(),
                                _stream(stream))
    _check(rc, "net_forward")
    return out


def net_backward(params_f32, out, target, ws, grad=None, loss=None, stream=None):
    """edp_net_backward after net_forward: (grad float32 like params, loss float64 [1])."""
    N, H, W, _ = out.shape
    if grad is None:
        grad = torch.empty_like(params_f32)
    if loss is None:
        loss = torch.empty(1, dtype=torch.float64, device=out.device)
    rc = load().edp_net_backward(_dev(params_f32, torch.float32, "params"), _dev(out, torch.float32, "out"),
                                 _dev(target, torch.float32, "target"), N, H, W, _dev(grad, torch.float32, "grad"),
                                 _dev(loss, torch.float64, "loss"), _dev(ws, torch.uint8, "ws"), ws.numel(),
                                 _stream(stream))
    _check(rc, "net_backward")
    return grad, loss


def net_adam(params_f32, grad, m, v, lr: float, step: int, b1: float = 0.9, b2: float = 0.999, eps: float = 1e-8,
             stream=None) -> None:
    rc = load().edp_net_adam(_dev(params_f32, torch.float32, "params"), _dev(grad, torch.float32, "grad"),
                             _dev(m, torch.float32, "m"), _dev(v, torch.float32, "v"), float(lr), float(b1), float(b2),
                             float(eps), int(step), _stream(stream))
    _check(rc, "net_adam")


def net_features(I0, I1, wta_labels, wta_cost, space: dict, scale: float, cmax: float, out=None, stream=None):
    """edp_net_features: bf16 [H][W][5]."""
    H, W = I0.shape
    if out is None:
        out = torch.empty((H, W, 5), dtype=torch.bfloat16, device=I0.device)
    ls = label_space(space)
    rc = load().edp_net_features(_dev(I0, torch.uint8, "I0"), _dev(I1, torch.uint8, "I1"),
                                 _dev(wta_labels, torch.int32, "wta_labels"), _dev(wta_cost, torch.int32, "wta_cost"),
                                 W, H, ctypes.byref(ls), float(scale), float(cmax), _dev(out, torch.bfloat16, "x"),
                                 _stream(stream))
    _check(rc, "net_features")
    return out


def coarse_labels(I0, I1, space: dict, prior: dict, l2: int, cmax: int, cost_mode: str = "pair", iters: int = 1,
                  ws=None, labels=None, stream=None):
    """edp_coarse_labels: full-resolution labels (int32 [H][W]) from EDP on the
    halved images and label space."""
    H, W = I0.shape
    pr = params(prior, iters=iters, l2=l2, cmax=cmax, cost_mode=cost_mode)
    ls = label_space(space)
    if ws is None:
        ws = workspace(OP_COARSE, W, H, space, prior, iters, device=I0.device, l2=l2, cmax=cmax, cost_mode=cost_mode)
    if labels is None:
        labels = torch.empty((H, W), dtype=torch.int32, device=I0.device)
    rc = load().edp_coarse_labels(_dev(I0, torch.uint8, "I0"), _dev(I1, torch.uint8, "I1"), W, H, I0.stride(0),
                                  ctypes.byref(ls), ctypes.byref(pr), _dev(labels, torch.int32, "labels"),
                                  _dev(ws, torch.uint8, "ws"), ws.numel(), _stream(stream))
    _check(rc, "coarse_labels")
    return labels


def net_features_labels(I0, I1, labels, space: dict, l2: int, cmax: int, scale: float, out=None, stream=None):
    """edp_net_features_labels: bf16 [H][W][5] from a labeling."""
    H, W = I0.shape
    if out is None:
        out = torch.empty((H, W, 5), dtype=torch.bfloat16, device=I0.device)
    ls = label_space(space)
    pr = params({"lam": 0, "g": 1}, l2=l2, cmax=cmax)
    rc = load().edp_net_features_labels(_dev(I0, torch.uint8, "I0"), _dev(I1, torch.uint8, "I1"),
                                        _dev(labels, torch.int32, "labels"), W, H, I0.stride(0), ctypes.byref(ls),
                                        ctypes.byref(pr), float(scale), _dev(out, torch.bfloat16, "x"),
                                        _stream(stream))
    _check(rc, "net_features_labels")
    return out


def net_centres_residual(out, base, space: dict, min_shift: int = 0, centre=None, stream=None):
    """edp_net_centres_residual: int32 [..][2] centres = base label + network
    output (corrections below min_shift labels dropped)."""
    n = out.numel() // 2
    if centre is None:
        centre = torch.empty(out.shape[:-1] + (2,), dtype=torch.int32, device=out.device)
    ls = label_space(space)
    rc = load().edp_net_centres_residual(_dev(out, torch.float32, "out"), _dev(base, torch.int32, "base"), n,
                                         ctypes.byref(ls), int(min_shift), _dev(centre, torch.int32, "centre"),
                                         _stream(stream))
    _check(rc, "net_centres_residual")
    return centre


def window_edge_count(labels, centre, win: int, space: dict, out=None, stream=None):
    """edp_window_edge_count: pixels whose label lies on an inner edge of its
    box (device int64 [1])."""
    n = labels.numel()
    if out is None:
        out = torch.empty(1, dtype=torch.int64, device=labels.device)
    ls = label_space(space)
    rc = load().edp_window_edge_count(_dev(labels, torch.int32, "labels"), _dev(centre, torch.int32, "centre"), n,
                                      int(win), ctypes.byref(ls), _dev(out, torch.int64, "count"), _stream(stream))
    _check(rc, "window_edge_count")
    return out


def net_targets(labels, space: dict, base=None, out=None, stream=None):
    """edp_net_targets: float [..][2] label coordinates minus the base's (or
    minus the space's middle without a base)."""
    n = labels.numel()
    if out is None:
        out = torch.empty(tuple(labels.shape) + (2,), dtype=torch.float32, device=labels.device)
    ls = label_space(space)
    bp = _dev(base, torch.int32, "base") if base is not None else None
    rc = load().edp_net_targets(_dev(labels, torch.int32, "labels"), bp, n, ctypes.byref(ls),
                                _dev(out, torch.float32, "target"), _stream(stream))
    _check(rc, "net_targets")
    return out


def net_centres(out, space: dict, centre=None, stream=None):
    """edp_net_centres: int32 [..][2] box centres from network outputs [..][2]."""
    n = out.numel() // 2
    if centre is None:
        centre = torch.empty(out.shape[:-1] + (2,), dtype=torch.int32, device=out.device)
    ls = label_space(space)
    rc = load().edp_net_centres(_dev(out, torch.float32, "out"), n, ctypes.byref(ls),
                                _dev(centre, torch.int32, "centre"), _stream(stream))
    _check(rc, "net_centres")
    return centre
