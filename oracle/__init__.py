"""CPU oracle for the EDP / RMS hot path (arXiv 1410.7922).

TEST INFRASTRUCTURE ONLY.  The test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` are the only callers.  The product library in
``paper_1410_7922_gb300`` never imports this package and shares no code with
it: the oracle is plain C (``edp_oracle.c``, exact int64 arithmetic) plus this
ctypes wrapper, and a numpy reference of the proposal network (``net.py``).

Label spaces and parameters are passed as plain dicts:
  space  = {"R": R, "Q": (Q0, Q1, Q2), "vmin": (...), "step": (...)}
  prior  = {"lam": lambda, "g": g, "l1": 1 | 2, "mode": "joint" | "per_axis"}
Tier 0 is the brute-force min search (the definition, Eq. M_strf); tier 1 is
the recursive minimum search of Sec. 3, trusted only through the tests that
compare it with tier 0.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "edp_oracle.c")
_SO = os.path.join(_HERE, "liboracle.so")
_lib = None

OK, ERR_ARG, ERR_RANGE, ERR_NOMEM = 0, 1, 2, 3
MODES = {"joint": 0, "per_axis": 1}
COST_MODES = {"pair": 0, "pair_stereo3": 1, "composite": 2}


class OracleError(RuntimeError):
    pass


class _Prior(ctypes.Structure):
    _fields_ = [
        ("R", ctypes.c_int32),
        ("Q", ctypes.c_int32 * 3),
        ("lam", ctypes.c_int32),
        ("g", ctypes.c_int32),
        ("l1", ctypes.c_int32),
        ("mode", ctypes.c_int32),
    ]


def build(force: bool = False) -> str:
    """Compile the oracle with gcc into ``oracle/liboracle.so``."""
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-o", tmp, _SRC])
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_SO)
        P = ctypes.c_void_p
        i32 = ctypes.c_int
        lib.oracle_prior.restype = ctypes.c_int64
        lib.oracle_prior.argtypes = [ctypes.POINTER(_Prior), ctypes.c_int64, ctypes.c_int64]
        lib.oracle_cost_volume.argtypes = [P, P, P, i32, i32, i32, P, P, P, i32, i32, i32, P]
        lib.oracle_cost_window.argtypes = [P, P, P, i32, i32, i32, P, P, P, i32, i32, i32, P, i32, P]
        lib.oracle_message.argtypes = [ctypes.POINTER(_Prior), i32, P, P]
        lib.oracle_scanline_dp.argtypes = [P, i32, i32, ctypes.POINTER(_Prior), i32, P, P]
        lib.oracle_min_marginals.argtypes = [P, i32, i32, ctypes.POINTER(_Prior), i32, P]
        lib.oracle_edp.argtypes = [P, i32, i32, ctypes.POINTER(_Prior), i32, i32, P, P, P]
        lib.oracle_edp_windowed.argtypes = [P, P, i32, i32, ctypes.POINTER(_Prior), i32, i32, P, P]
        lib.oracle_energy.argtypes = [P, P, i32, i32, ctypes.POINTER(_Prior), P]
        lib.oracle_edp_weighted.argtypes = [P, i32, i32, ctypes.POINTER(_Prior), i32, i32, P, P, P]
        lib.oracle_energy_weighted.argtypes = [P, P, i32, i32, ctypes.POINTER(_Prior), P, P, P]
        lib.oracle_edge_weights.argtypes = [P, i32, i32, i32, i32, i32, P, P]
        for f in ("oracle_cost_volume", "oracle_cost_window", "oracle_message",
                  "oracle_scanline_dp", "oracle_min_marginals", "oracle_edp",
                  "oracle_edp_windowed", "oracle_energy", "oracle_edp_weighted",
                  "oracle_energy_weighted", "oracle_edge_weights"):
            getattr(lib, f).restype = ctypes.c_int
        _lib = lib
    return _lib


def _check(rc: int, what: str) -> None:
    if rc != OK:
        name = {ERR_ARG: "invalid argument", ERR_RANGE: "int32 range exceeded",
                ERR_NOMEM: "out of memory"}.get(rc, str(rc))
        raise OracleError(f"{what}: {name}")


def _ptr(a: np.ndarray | None):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _i32x3(t) -> np.ndarray:
    v = list(t) + [1] * (3 - len(t))
    return np.ascontiguousarray(v[:3], dtype=np.int32)


def n_labels(space: dict) -> int:
    q = 1
    for r in range(space["R"]):
        q *= int(space["Q"][r])
    return q


def make_prior(space: dict, prior: dict) -> _Prior:
    p = _Prior()
    p.R = int(space["R"])
    Q = list(space["Q"]) + [1] * (3 - len(space["Q"]))
    for r in range(3):
        p.Q[r] = int(Q[r]) if r < p.R else 1
    p.lam = int(prior["lam"])
    p.g = int(prior["g"])
    p.l1 = int(prior.get("l1", 1))
    p.mode = MODES[prior.get("mode", "joint")]
    return p


def prior_value(space: dict, prior: dict, q: int, qp: int) -> int:
    p = make_prior(space, prior)
    return int(_load().oracle_prior(ctypes.byref(p), int(q), int(qp)))


def cost_volume(I0, I1, I2, space: dict, l2: int, cmax: int, cost_mode: str = "pair") -> np.ndarray:
    """Eq. Cost_value (and Eq. Cost_cmp for ``composite``): int32 [H][W][Q]."""
    I0 = np.ascontiguousarray(I0, dtype=np.uint8)
    I1 = np.ascontiguousarray(I1, dtype=np.uint8)
    I2 = None if I2 is None else np.ascontiguousarray(I2, dtype=np.uint8)
    H, W = I0.shape
    C = np.empty((H, W, n_labels(space)), dtype=np.int32)
    rc = _load().oracle_cost_volume(
        _ptr(I0), _ptr(I1), _ptr(I2), W, H, int(space["R"]), _ptr(_i32x3(space["Q"])),
        _ptr(_i32x3(space["vmin"])), _ptr(_i32x3(space["step"])), int(l2), int(cmax),
        COST_MODES[cost_mode], _ptr(C))
    _check(rc, "cost_volume")
    return C


def cost_window(I0, I1, I2, space: dict, l2: int, cmax: int, centre, win: int,
                cost_mode: str = "pair") -> np.ndarray:
    """Cost restricted to each pixel's box of win^R labels: int32 [H][W][win^R]."""
    I0 = np.ascontiguousarray(I0, dtype=np.uint8)
    I1 = np.ascontiguousarray(I1, dtype=np.uint8)
    I2 = None if I2 is None else np.ascontiguousarray(I2, dtype=np.uint8)
    H, W = I0.shape
    R = int(space["R"])
    centre = np.ascontiguousarray(centre, dtype=np.int32).reshape(H, W, R)
    Cw = np.empty((H, W, win ** R), dtype=np.int32)
    rc = _load().oracle_cost_window(
        _ptr(I0), _ptr(I1), _ptr(I2), W, H, R, _ptr(_i32x3(space["Q"])),
        _ptr(_i32x3(space["vmin"])), _ptr(_i32x3(space["step"])), int(l2), int(cmax),
        COST_MODES[cost_mode], _ptr(centre), int(win), _ptr(Cw))
    _check(rc, "cost_window")
    return Cw


def message(h, space: dict, prior: dict, tier: int = 0) -> np.ndarray:
    """M(h)(q) = min_q' h(q') + V(q', q) (Eq. M_strf), int64."""
    h = np.ascontiguousarray(h, dtype=np.int64)
    out = np.empty_like(h)
    p = make_prior(space, prior)
    _check(_load().oracle_message(ctypes.byref(p), int(tier), _ptr(h), _ptr(out)), "message")
    return out


def scanline_dp(C, space: dict, prior: dict, tier: int = 0):
    """Per-row DP (Eq. base, Eq. DP_1D_2) + backward path recovery.

    Returns (labels int32 [H][W], row_energy int64 [H])."""
    C = np.ascontiguousarray(C, dtype=np.int32)
    H, W, _ = C.shape
    labels = np.empty((H, W), dtype=np.int32)
    row_e = np.empty(H, dtype=np.int64)
    p = make_prior(space, prior)
    _check(_load().oracle_scanline_dp(_ptr(C), W, H, ctypes.byref(p), int(tier), _ptr(labels),
                                      _ptr(row_e)), "scanline_dp")
    return labels, row_e


def min_marginals(C, space: dict, prior: dict, tier: int = 0) -> np.ndarray:
    """Modified DP marginal S_Omega of Eq. DP_1D_3 per row, int64 [H][W][Q]."""
    C = np.ascontiguousarray(C, dtype=np.int32)
    H, W, Q = C.shape
    S = np.empty((H, W, Q), dtype=np.int64)
    p = make_prior(space, prior)
    _check(_load().oracle_min_marginals(_ptr(C), W, H, ctypes.byref(p), int(tier), _ptr(S)),
           "min_marginals")
    return S


def edp(C, space: dict, prior: dict, iters: int = 1, tier: int = 1, return_sums: bool = False,
        return_marginal: bool = False):
    """Algorithm 1 (EDP): labels int32 [H][W] (lowest-index argmin).

    Optionally also the final sums S_k [4][H][W][Q] (k = +x, -x, +y, -y) and the
    marginal estimate S_Omega [H][W][Q]."""
    C = np.ascontiguousarray(C, dtype=np.int32)
    H, W, Q = C.shape
    labels = np.empty((H, W), dtype=np.int32)
    S = np.empty((4, H, W, Q), dtype=np.int32) if return_sums else None
    So = np.empty((H, W, Q), dtype=np.int64) if return_marginal else None
    p = make_prior(space, prior)
    _check(_load().oracle_edp(_ptr(C), W, H, ctypes.byref(p), int(iters), int(tier),
                              _ptr(labels), _ptr(S), _ptr(So)), "edp")
    out = [labels]
    if return_sums:
        out.append(S)
    if return_marginal:
        out.append(So)
    return out[0] if len(out) == 1 else tuple(out)


def edp_windowed(Cw, centre, space: dict, prior: dict, win: int, iters: int = 1, return_sums: bool = False):
    """EDP on per-pixel label boxes; labels are full-space linear indexes.

    Optionally also the final sums S_k [4][H][W][win^R] in box coordinates
    (k = +x, -x, +y, -y)."""
    Cw = np.ascontiguousarray(Cw, dtype=np.int32)
    H, W, QW = Cw.shape
    R = int(space["R"])
    centre = np.ascontiguousarray(centre, dtype=np.int32).reshape(H, W, R)
    labels = np.empty((H, W), dtype=np.int32)
    S = np.empty((4, H, W, QW), dtype=np.int32) if return_sums else None
    p = make_prior(space, prior)
    _check(_load().oracle_edp_windowed(_ptr(Cw), _ptr(centre), W, H, ctypes.byref(p), int(win),
                                       int(iters), _ptr(labels), _ptr(S)), "edp_windowed")
    return (labels, S) if return_sums else labels


def energy(C, labels, space: dict, prior: dict) -> tuple[int, int, int, int]:
    """Eq. GE_objective_function: (data, smooth_h, smooth_v, total), int."""
    labels = np.ascontiguousarray(labels, dtype=np.int32)
    H, W = labels.shape
    Cc = None if C is None else np.ascontiguousarray(C, dtype=np.int32)
    out = np.zeros(4, dtype=np.int64)
    p = make_prior(space, prior)
    _check(_load().oracle_energy(_ptr(Cc), _ptr(labels), W, H, ctypes.byref(p), _ptr(out)),
           "energy")
    return tuple(int(v) for v in out)


def edge_weights(I, thresh: int = 10, factor: int = 2):
    """Per-edge prior multipliers of the locally adaptive lambda (text below
    Eq. Smooth_value_t): (wh, wv) uint8 [H][W]; an edge whose intensity step
    is below `thresh` gets `factor`, every other edge 1."""
    I = np.ascontiguousarray(I, dtype=np.uint8)
    H, W = I.shape
    wh = np.empty((H, W), dtype=np.uint8)
    wv = np.empty((H, W), dtype=np.uint8)
    _check(_load().oracle_edge_weights(_ptr(I), W, H, W, int(thresh), int(factor), _ptr(wh), _ptr(wv)),
           "edge_weights")
    return wh, wv


def edp_weighted(C, space: dict, prior: dict, wh, wv, iters: int = 1, tier: int = 1):
    """EDP with per-edge prior multipliers: the prior of edge (x, y)-(x+1, y)
    is wh[y][x] * lambda * f, of (x, y)-(x, y+1) wv[y][x] * lambda * f."""
    C = np.ascontiguousarray(C, dtype=np.int32)
    H, W, Q = C.shape
    wh = np.ascontiguousarray(wh, dtype=np.uint8)
    wv = np.ascontiguousarray(wv, dtype=np.uint8)
    assert wh.shape == (H, W) and wv.shape == (H, W)
    labels = np.empty((H, W), dtype=np.int32)
    p = make_prior(space, prior)
    _check(_load().oracle_edp_weighted(_ptr(C), W, H, ctypes.byref(p), int(iters), int(tier), _ptr(wh),
                                       _ptr(wv), _ptr(labels)), "edp_weighted")
    return labels


def energy_weighted(C, labels, space: dict, prior: dict, wh, wv) -> tuple[int, int, int, int]:
    """Eq. GE_objective_function with per-edge prior multipliers."""
    labels = np.ascontiguousarray(labels, dtype=np.int32)
    H, W = labels.shape
    Cc = None if C is None else np.ascontiguousarray(C, dtype=np.int32)
    wh = np.ascontiguousarray(wh, dtype=np.uint8)
    wv = np.ascontiguousarray(wv, dtype=np.uint8)
    out = np.zeros(4, dtype=np.int64)
    p = make_prior(space, prior)
    _check(_load().oracle_energy_weighted(_ptr(Cc), _ptr(labels), W, H, ctypes.byref(p), _ptr(wh), _ptr(wv),
                                          _ptr(out)), "energy_weighted")
    return tuple(int(v) for v in out)
