"""Launch-shape autotuner for the scan-pass kernels.

The scan-pass kernels take two shape knobs (edp_set_tuning): rows of the
image per block (one warp per row in the one-axis kernel, one team of warps
per row in the multi-axis kernel) and warps per row of the multi-axis
kernel.  Results never depend on them; only the time does.  The tuner times
each candidate with CUDA events on the caller's workload and leaves the
fastest one set.
"""
from __future__ import annotations

import itertools
import json
import os

import torch

from . import edp

DEFAULT_ROWS = (0, 1, 2, 4, 8)
DEFAULT_WARPS = (0, 1, 2, 4, 8)


def _time(fn, reps: int) -> float:
    fn()
    torch.cuda.synchronize()
    best = None
    for _ in range(reps):
        s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s.record()
        fn()
        e.record()
        torch.cuda.synchronize()
        ms = s.elapsed_time(e)
        best = ms if best is None else min(best, ms)
    return best


def tune(fn, rows=DEFAULT_ROWS, warps=DEFAULT_WARPS, reps: int = 3, log=None):
    """Time fn() under every (rows per block, warps per row) pair; set and
    return the fastest as (rows, warps_per_row, ms, table).  Shapes the
    kernels cannot run are skipped."""
    table = []
    for r, w in itertools.product(rows, warps):
        edp.set_tuning(r, 0, False, warps_per_row=w)
        try:
            ms = _time(fn, reps)
        except edp.EdpError:
            continue
        table.append((r, w, ms))
        if log:
            log(f"rows={r} warps_per_row={w}: {ms:.3f} ms")
    r, w, ms = min(table, key=lambda t: t[2])
    edp.set_tuning(r, 0, False, warps_per_row=w)
    return r, w, ms, table


def save(path: str, key: str, result) -> None:
    d = json.load(open(path)) if os.path.exists(path) else {}
    d[key] = {"rows": result[0], "warps_per_row": result[1], "ms": result[2]}
    with open(path, "w") as f:
        json.dump(d, f, indent=1)
