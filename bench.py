#!/usr/bin/env python
"""Benchmark: EDP pixel-label updates/s.

One step = the whole hot path over one synthetic pair: cost volume, j EDP
iterations (four scan passes each, Algorithm 1) with the marginal/argmin, and
the energy -- one call of edp_solve_images.  Pixel-label updates per step =
N * Q * (8 * j + 1): two sums written per pass, four passes per iteration,
plus the marginal.  Workloads (--workload):
  motion_edp_640x480_Q65x65  640x480 motion, the full 65x65 label space
                             ([-32, 32]^2), cost min(|I1(x+o) - I0(x)|, 20),
                             per-axis truncated-linear prior lambda = 15, K = 3
                             (the default: the largest single-GPU workload);
  motion_edp_320x240_Q33x33  320x240 motion, 33x33 labels, same prior;
  stereo_edp_450x375_Q64     450x375 stereo, 64 labels, cost min(|IL-IR|, 20),
                             truncated-linear prior lambda = 20, K = 4.
The other two workloads are also timed as side rows of the default line.

Roofline: the scan pass is HBM-bound; its algorithmic bytes are those of the
paper's sums form, 20 * Q bytes per pixel per pass (read C and the two old
sums, write the two new sums), divided by the pass launches' CUDA-event time.
The message form the kernels store moves fewer bytes; that count is reported
beside it.

Prints one JSON line (rank 0).  --impl reference runs the CPU oracle on the
host cores instead (bounded samples of the same workload).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "EDP pixel-label updates/s"
UNIT = "pixel-label updates/s"
WORKLOAD = "motion_edp_640x480_Q65x65"
WORKLOADS = ("motion_edp_640x480_Q65x65", "motion_edp_320x240_Q33x33", "stereo_edp_450x375_Q64")


def make_workload(name: str, pair: int = 0, size: str = "") -> dict:
    """The named workload; `size` ("WxH") replaces its image size (smaller
    cases of the same kernel for profiling)."""
    from paper_1410_7922_gb300 import synth
    kw = {}
    if size:
        W, H = (int(v) for v in size.lower().split("x"))
        kw = {"W": W, "H": H}
    if name == "stereo_edp_450x375_Q64":
        w = synth.workload_stereo_450x375(pair=pair, **kw)
        w["desc"] = {"prior": "truncated linear, lambda=20, K=4", "cost": "min(|IL-IR|, 20)"}
    elif name == "motion_edp_320x240_Q33x33":
        w = synth.workload_motion_320x240(pair=pair, **kw)
        w["desc"] = {"prior": "per-axis truncated linear, lambda=15, K=3", "cost": "min(|I1(x+o)-I0(x)|, 20)"}
    else:
        w = synth.workload_motion_640x480(pair=pair, **kw)
        w["desc"] = {"prior": "per-axis truncated linear, lambda=15, K=3", "cost": "min(|I1(x+o)-I0(x)|, 20)"}
    return w
PASS_NAMES = ["P1", "P2", "P3", "P4"]


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--iters", type=int, default=1, help="EDP iterations j per step")
    ap.add_argument("--impl", default="edp", choices=["edp", "reference"])
    ap.add_argument("--workload", default=WORKLOAD, choices=WORKLOADS)
    ap.add_argument("--size", default="", help="WxH: the workload at another image size (profiling runs)")
    ap.add_argument("--no-rows", action="store_true", help="skip the per-row side measurements")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU-oracle baseline")
    ap.add_argument("--net-only", action="store_true",
                    help="only the proposal network's forward / backward timing (one JSON line; profiling runs)")
    ap.add_argument("--extra", default="", help="comma list of longer side measurements: batched,proposal")
    ap.add_argument("--batch-scale", type=float, default=1.0, help="image scale of the batched workload")
    ap.add_argument("--proposal-pairs", type=int, default=2000, help="training pairs of the proposal network")
    ap.add_argument("--row-proposal-pairs", type=int, default=64,
                    help="training pairs of the proposal row of the default line")
    return ap.parse_args()


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist
        backend = "nccl" if torch.cuda.is_available() and args.impl == "edp" else "gloo"
        if backend == "nccl":
            torch.cuda.set_device(local)
        dist.init_process_group(backend=backend)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def allreduce_max(world, v: float) -> float:
    if world == 1:
        return v
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([v], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ---------------------------------------------------------------------------
# algorithmic bytes of one scan pass (the messages each pass must read/write)
# ---------------------------------------------------------------------------

def pass_units(pass_idx: int, it: int, iters: int) -> tuple[int, bool]:
    """Q-vectors (of 4*Q bytes) one pass moves per pixel, and whether it
    writes the labels.  Reads: C, and the two messages of the other
    directions once they have been written; writes: the two new messages when
    a later pass reads them (mirrors the pass schedule of the library)."""
    last = it == iters - 1
    read_c = (it > 0) if pass_idx == 0 else True
    read_d = (it > 0) if pass_idx <= 1 else True
    write_a = (not last) if pass_idx == 3 else True
    write_b = True if pass_idx == 1 else ((not last) if pass_idx == 3 else False)
    return 1 + read_c + read_d + write_a + write_b, (pass_idx == 3 and last)


def launch_bytes(nlaunch: int, W: int, H: int, Q: int, iters: int) -> list[int]:
    """Algorithmic bytes of each scan-pass launch of one solve: one pass per
    launch (4 per iteration), or a paired sweep P1 + P2 / P3 + P4 (2 per
    iteration), which moves the bytes of both its passes."""
    per_it = nlaunch // iters
    out = []
    for i in range(nlaunch):
        it, k = divmod(i, per_it)
        passes = (2 * k, 2 * k + 1) if per_it == 2 else (k,)
        b = 0
        for p in passes:
            units, lab = pass_units(p, it, iters)
            b += units * W * H * Q * 4 + (W * H * 4 if lab else 0)
        out.append(b)
    return out


def sums_bytes_per_pass(W: int, H: int, Q: int) -> int:
    """Algorithmic bytes of one scan pass in the paper's sums form: per pixel
    read C(x, .) and the two old sums, write the two new sums, 20 * Q bytes."""
    return 20 * Q * W * H


def measured_bf16_peak():
    """Dense bf16 TFLOP/s measured on this machine (burst: a kernel timed alone)."""
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        return float(json.load(open(p))["bf16_tflops"]), "measured"
    return 1900.0, "fallback"


def measure_net(edp, torch, sizes=((1, 480, 640), (8, 240, 320)), reps=10):
    """Proposal network forward and backward (parameter gradients) on random
    inputs, with the 32 -> 32 convolutions on the tensor cores and on the
    CUDA cores; TFLOP/s of the forward's four 32 -> 32 layers against the
    measured bf16 peak (the forward's other two layers, 5 -> 32 and
    32 -> 2, run on the CUDA cores inside the same time)."""
    import statistics

    def timed(fn):
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        ts = []
        for _ in range(reps):
            s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            s.record()
            fn()
            e.record()
            torch.cuda.synchronize()
            ts.append(s.elapsed_time(e))
        return statistics.median(ts)

    peak, kind = measured_bf16_peak()
    g = torch.Generator(device="cuda").manual_seed(0)
    out_rows = {}
    for (N, H, W) in sizes:
        P = (torch.randn(edp.net_param_count(), device="cuda", generator=g) * 0.05).float()
        x = torch.rand((N, H, W, 5), device="cuda", generator=g).to(torch.bfloat16)
        tgt = torch.randn((N, H, W, 2), device="cuda", generator=g)
        ws = edp.net_workspace(N, H, W)
        r = {}
        for tc in (True, False):
            edp.set_net_tensor_cores(tc)
            out = edp.net_forward(P, x, ws)
            f = timed(lambda: edp.net_forward(P, x, ws, out=out))
            b = timed(lambda: edp.net_backward(P, out, tgt, ws))
            r["tensor_cores" if tc else "cuda_cores"] = {"forward_ms": f, "backward_ms": b,
                                                         "status": edp.net_device_status(ws)}
        edp.set_net_tensor_cores(True)
        flops = 4 * 2 * N * H * W * 32 * 288
        r["tc_layers_forward_tflop"] = flops / 1e12
        r["tc_forward_tflops"] = flops / (r["tensor_cores"]["forward_ms"] * 1e-3) / 1e12
        r["frac_of_bf16_peak"] = r["tc_forward_tflops"] / peak
        r["bf16_peak_tflops"] = peak
        r["peak_kind"] = kind
        out_rows[f"{N}x{H}x{W}"] = r
        del ws
    return out_rows


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


KERNEL_SOURCES = {
    "edp_pass_r1_kernel": ("pass_r1.cuh", "edp_pass_r1.cu", "common.cuh"),
    "edp_pass_team_kernel": ("pass_team.cuh", "edp_pass_team.cu", "common.cuh"),
    "edp_pass_line_kernel": ("pass_line.cuh", "edp_pass_line.cu", "common.cuh"),
    "edp_pass_line2_kernel": ("pass_line2.cuh", "pass_line.cuh", "edp_pass_line.cu", "common.cuh"),
}


def _code_only(text: str) -> str:
    """Source text without comments and blank lines (a comment edit does not
    change the kernel)."""
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    lines = [re.sub(r"//.*$", "", ln).rstrip() for ln in text.splitlines()]
    return "\n".join(ln for ln in lines if ln.strip())


def kernel_source_hash(kernel: str) -> str:
    h = hashlib.sha256()
    for f in KERNEL_SOURCES[kernel]:
        with open(os.path.join(ROOT, "paper_1410_7922_gb300", "csrc", f)) as fh:
            h.update(_code_only(fh.read()).encode())
    return h.hexdigest()[:16]


def profiled_traffic(workload: str, kernel: str):
    """DRAM bytes per launch of the pass kernel from a committed ncu summary
    (profiles/edp_pass_traffic.json: workload -> {kernel, source_hash,
    dram_bytes_per_launch}), or None if there is none for the current source."""
    p = os.path.join(ROOT, "profiles", "edp_pass_traffic.json")
    if not os.path.exists(p):
        return None
    d = json.load(open(p))
    e = d.get(workload)
    if not e or kernel not in KERNEL_SOURCES or e.get("kernel") != kernel or \
            e.get("source_hash") != kernel_source_hash(kernel):
        return None
    return float(e["dram_bytes_per_launch"])


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.p = None

    def __enter__(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "20"],
                                      stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            time.sleep(0.3)
        except (OSError, ValueError):
            self.p = None
        return self

    def __exit__(self, *a):
        self.out = ""
        if self.p is not None:
            time.sleep(0.1)
            self.p.terminate()
            try:
                self.out, _ = self.p.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.p.kill()
                self.out, _ = self.p.communicate()

    def summary(self):
        rows = []
        for line in (self.out or "").strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                rows.append((float(f[1]), float(f[2]), f[5], f[6], f[7], f[8]))
            except ValueError:
                continue
        if not rows:
            return None
        smax = max(r[1] for r in rows)
        load = [r for r in rows if r[0] > 0.5 * smax] or rows
        reasons = set()
        for r in rows:
            for name, flag in zip(("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"),
                                  r[2:]):
                if flag.lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(r[0] for r in load), "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(rows)}


def bad_clocks(c) -> bool:
    if not c:
        return False
    if set(c["reasons"]) & {"hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown"}:
        return True
    return c["sm_mhz"] < 0.6 * c["sm_max_mhz"] and not c["reasons"]


# ---------------------------------------------------------------------------
# CPU oracle baseline
# ---------------------------------------------------------------------------

def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def oracle_crop(job):
    """The oracle, as it is, on rows [y0, y0 + rows) of a frame: cost volume,
    EDP (RMS tier) and energy.  Returns the seconds it took."""
    import oracle
    I0, I1, space, prior, l2, cmax, iters = job
    t0 = time.perf_counter()
    C = oracle.cost_volume(I0, I1, None, space, l2, cmax)
    lab = oracle.edp(C, space, prior, iters=iters, tier=1)
    oracle.energy(C, lab, space, prior)
    return time.perf_counter() - t0


def _crop_job(w, y0, rows, iters):
    return (w["I0"][y0:y0 + rows].copy(), w["I1"][y0:y0 + rows].copy(), w["space"], w["prior"], w["l2"],
            w["cmax"], iters)


def crop_rows_for(w, iters, seconds: float) -> int:
    """Image rows of a crop that takes about `seconds` of oracle work on one
    host core (calibrated on a 2-row crop)."""
    H = w["I0"].shape[0]
    t2 = max(oracle_crop(_crop_job(w, 0, 2, iters)), 1e-4)
    return max(2, min(H, int(2 * seconds / t2)))


def oracle_pool(n: int):
    """A process pool for the oracle, started with spawn (it may run after
    the GPU has been initialised in this process)."""
    import multiprocessing as mp
    return mp.get_context("spawn").Pool(n)


def cpu_oracle_sample(w, iters: int, seconds: float = 8.0):
    """The oracle as it is, timed on the host cores on bounded crops of the
    frame: one crop on one core, then one crop per core on every core at
    once (independent problems, one process each)."""
    import oracle
    oracle.build()
    H, W = w["I0"].shape
    Q = 1
    for r in range(w["space"]["R"]):
        Q *= w["space"]["Q"][r]
    rows = crop_rows_for(w, iters, seconds)
    per_crop = W * rows * Q * (8 * iters + 1)
    t1 = oracle_crop(_crop_job(w, 0, rows, iters))
    n = host_cores()
    jobs = [_crop_job(w, (k * rows) % max(1, H - rows + 1), rows, iters) for k in range(n)]
    with oracle_pool(n) as pool:
        pool.map(oracle_crop, jobs[:1])  # start-up of the workers
        t0 = time.perf_counter()
        pool.map(oracle_crop, jobs, chunksize=1)
        tn = time.perf_counter() - t0
    crop = f"{W}x{rows} crops of the {W}x{H} frame, j={iters}: oracle cost volume + EDP (RMS tier) + energy"
    return {"value": n * per_crop / tn, "unit": UNIT, "cores": n, "kind": "oracle",
            "sample": f"{n} {crop}, one process per host core, {tn:.1f} s wall",
            "single_core": {"value": per_crop / t1, "unit": UNIT, "cores": 1,
                            "sample": f"one {crop}, {t1:.1f} s on 1 host core"}}


def run_reference(args, world, rank):
    if rank != 0:
        return
    import oracle
    oracle.build()
    w = make_workload(args.workload, size=args.size)
    H, W = w["I0"].shape
    Q = 1
    for r in range(w["space"]["R"]):
        Q *= w["space"]["Q"][r]
    # each step: one crop per host core, all at once, each about one second
    # of oracle work (the whole frame when it fits)
    rows = crop_rows_for(w, args.iters, 1.0)
    n = host_cores()
    jobs = [_crop_job(w, (k * rows) % max(1, H - rows + 1), rows, args.iters) for k in range(n)]
    with oracle_pool(n) as pool:
        for _ in range(args.warmup):
            pool.map(oracle_crop, jobs, chunksize=1)
        t0 = time.perf_counter()
        for _ in range(args.steps):
            pool.map(oracle_crop, jobs, chunksize=1)
        el = time.perf_counter() - t0
    value = n * W * rows * Q * (8 * args.iters + 1) * args.steps / el
    sample = (f"{n} {W}x{rows} crops of the {W}x{H} frame per step, one process per host core: oracle cost "
              "volume + EDP (RMS tier) + energy")
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
            "impl": "reference",
            "config": {"workload": args.workload, "W": W, "H": H, "Q": Q, "iters": args.iters},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": n, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------

def pass_roofline(W: int, H: int, Q: int, iters: int, pass_ms: list[float], peak: float) -> dict:
    """Roofline of the scan-pass launches of one solve: sums-form bytes (20 Q
    per pixel per pass) over the launches' summed event time, and the
    message-form bytes the kernels actually move."""
    t = sum(pass_ms) * 1e-3
    alg = 4 * iters * sums_bytes_per_pass(W, H, Q)
    msg = sum(launch_bytes(len(pass_ms), W, H, Q, iters))
    return {"achieved_gbs": alg / t / 1e9, "frac": alg / t / 1e9 / peak,
            "message_form_gbs": msg / t / 1e9, "pass_ms": pass_ms}


def time_solve_rows(edp, synth, torch, peak: float):
    """Side measurements of the other workloads and hot-path rows (device
    time, CUDA events; median of the repetitions)."""
    rows = {}
    ev = lambda: torch.cuda.Event(enable_timing=True)

    def timed(fn, reps=20):
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        ts = []
        for _ in range(reps):
            s, e = ev(), ev()
            s.record()
            fn()
            e.record()
            torch.cuda.synchronize()
            ts.append(s.elapsed_time(e))
        return statistics.median(ts)

    # scanline DP, 64x48 stereo, Q = 16 (cost volume + forward pass + backtrack)
    w = synth.workload_scanline_64x48()
    I0, I1 = torch.from_numpy(w["I0"]).cuda(), torch.from_numpy(w["I1"]).cuda()
    C = edp.cost_volume(I0, I1, None, w["space"], w["l2"], w["cmax"])
    ws = edp.workspace(edp.OP_SCANLINE_DP, 64, 48, w["space"], w["prior"])
    lab = torch.empty((48, 64), dtype=torch.int32, device="cuda")
    re = torch.empty(48, dtype=torch.int64, device="cuda")
    ms = timed(lambda: edp.scanline_dp(C, w["space"], w["prior"], ws=ws, labels=lab, row_energy=re))
    rows["scanline_dp_64x48_Q16"] = {"ms": ms, "updates_per_s": 64 * 48 * 16 / (ms * 1e-3)}
    # full EDP (j = 1) on the two smaller workloads: solve time and the
    # roofline of its scan-pass launches
    for name in ("motion_edp_320x240_Q33x33", "stereo_edp_450x375_Q64"):
        w = make_workload(name)
        I0, I1 = torch.from_numpy(w["I0"]).cuda(), torch.from_numpy(w["I1"]).cuda()
        C = edp.cost_volume(I0, I1, None, w["space"], w["l2"], w["cmax"])
        H, W, Q = C.shape
        ws = edp.workspace(edp.OP_SOLVE, W, H, w["space"], w["prior"], 1)
        lab = torch.empty((H, W), dtype=torch.int32, device="cuda")
        evs = [ev() for _ in range(8)]
        edp.set_profile_events(evs)
        ms = timed(lambda: edp.solve(C, w["space"], w["prior"], iters=1, ws=ws, labels=lab), reps=10)
        nl = edp.last_pass_launches()
        pass_ms = [evs[2 * i].elapsed_time(evs[2 * i + 1]) for i in range(nl)]
        edp.set_profile_events(None)
        rows[name] = {"ms_solve": ms, "updates_per_s": W * H * Q * 9 / (ms * 1e-3),
                      "roofline": pass_roofline(W, H, Q, 1, pass_ms, peak)}
    # cost volume alone (write-bound), 450x375x64
    w = synth.workload_stereo_450x375()
    I0, I1 = torch.from_numpy(w["I0"]).cuda(), torch.from_numpy(w["I1"]).cuda()
    C = torch.empty((375, 450, 64), dtype=torch.int32, device="cuda")
    ms = timed(lambda: edp.cost_volume(I0, I1, None, w["space"], w["l2"], w["cmax"], out=C))
    rows["cost_volume_450x375_Q64"] = {"ms": ms, "write_gbs": C.numel() * 4 / (ms * 1e-3) / 1e9}
    lab = edp.solve(C, w["space"], w["prior"], iters=1)
    out = torch.empty(4, dtype=torch.int64, device="cuda")
    ms = timed(lambda: edp.energy(C, lab, w["space"], w["prior"], out=out))
    rows["energy_450x375_Q64"] = {"ms": ms}
    # cost volume of the bench workload (5.2 GB written), the first kernel of its step
    del C
    w = make_workload(WORKLOAD)
    I0, I1 = torch.from_numpy(w["I0"]).cuda(), torch.from_numpy(w["I1"]).cuda()
    C = torch.empty((480, 640, 65 * 65), dtype=torch.int32, device="cuda")
    ms = timed(lambda: edp.cost_volume(I0, I1, None, w["space"], w["l2"], w["cmax"], out=C), reps=10)
    rows["cost_volume_640x480_Q65x65"] = {"ms": ms, "write_gbs": C.numel() * 4 / (ms * 1e-3) / 1e9,
                                          "frac_of_hbm": C.numel() * 4 / (ms * 1e-3) / 1e9 / peak}
    del C
    return rows


def measure_batched(edp, synth, torch, scale: float = 1.0, n_pairs: int = 64, budget_gb: float = 200.0):
    """64 heterogeneous pairs: per-pair edp_solve_images launches against one
    edp_solve_batched call (persistent kernel) and its CUDA-graph replay."""
    from paper_1410_7922_gb300 import autotune
    ws_list = synth.workload_batch(n_pairs=n_pairs, scale=scale)
    items = []
    updates = 0
    for w in ws_list:
        H, W = w["I0"].shape
        it = {"I0": torch.from_numpy(w["I0"]).cuda(), "I1": torch.from_numpy(w["I1"]).cuda(),
              "I2": torch.from_numpy(w["I2"]).cuda() if w["I2"] is not None else None,
              "space": w["space"], "prior": w["prior"], "l2": w["l2"], "cmax": w["cmax"],
              "cost_mode": w["cost_mode"], "iters": 1,
              "labels": torch.empty((H, W), dtype=torch.int32, device="cuda"),
              "energy4": torch.empty(4, dtype=torch.int64, device="cuda")}
        items.append(it)
        updates += W * H * edp.n_labels(w["space"]) * 9
    probs = edp.make_problems(items)
    full = edp.batch_workspace_size(probs)
    biggest = max(edp.batch_workspace_size(edp.make_problems([it])) for it in items)
    wsb = torch.empty(int(max(biggest, min(full, budget_gb * 1e9))), dtype=torch.uint8, device="cuda")
    ev = lambda: torch.cuda.Event(enable_timing=True)

    def timed(fn, reps=2):
        fn()
        torch.cuda.synchronize()
        best = None
        for _ in range(reps):
            s, e = ev(), ev()
            s.record()
            fn()
            e.record()
            torch.cuda.synchronize()
            best = s.elapsed_time(e) if best is None else min(best, s.elapsed_time(e))
        return best

    # per-pair: one edp_solve_images per problem, one workspace sized for the largest
    ws1 = torch.empty(max(edp.workspace_size(edp.OP_SOLVE_IMAGES, it["I0"].shape[1], it["I0"].shape[0],
                                             it["space"], it["prior"]) for it in items), dtype=torch.uint8,
                      device="cuda")
    per_labels = []

    def per_pair():
        for it in items:
            edp.solve_images(it["I0"], it["I1"], it["I2"], it["space"], it["prior"], it["l2"], it["cmax"],
                             it["cost_mode"], 1, ws=ws1, labels=it["labels"], energy4=it["energy4"])

    ms_per = timed(per_pair, reps=1)
    per_labels = [it["labels"].clone() for it in items]
    # which problems get launches of their own (pixels; 0: none)
    splits = {}
    for split in (0, 76800, 172800, 307200):
        edp.set_batch_split(split)
        splits[split] = timed(lambda: edp.solve_batched(probs, wsb), reps=1)
    best_split = min(splits, key=splits.get)
    edp.set_batch_split(best_split)
    tuned = autotune.tune(lambda: edp.solve_batched(probs, wsb), rows=(0,), warps=(0, 1, 2, 4), reps=1)
    ms_batched = timed(lambda: edp.solve_batched(probs, wsb))
    same = all(torch.equal(a, it["labels"]) for a, it in zip(per_labels, items))
    g = torch.cuda.CUDAGraph()
    st = torch.cuda.Stream()
    st.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(st):
        edp.solve_batched(probs, wsb, stream=st)
        torch.cuda.synchronize()
        with torch.cuda.graph(g, stream=st):
            edp.solve_batched(probs, wsb, stream=st)
    torch.cuda.current_stream().wait_stream(st)
    ms_graph = timed(lambda: g.replay())
    same_graph = all(torch.equal(a, it["labels"]) for a, it in zip(per_labels, items))
    edp.set_tuning(0, 0, False)
    edp.set_batch_split(172800)
    return {"pairs": n_pairs, "scale": scale, "workspace_gb": wsb.numel() / 1e9,
            "all_resident_gb": full / 1e9, "updates_per_step": updates,
            "ms_per_pair_launches": ms_per, "ms_batched": ms_batched, "ms_batched_graph": ms_graph,
            "split_pixels": best_split, "ms_by_split": {str(k): v for k, v in splits.items()},
            "speedup_batched": ms_per / ms_batched, "speedup_graph": ms_per / ms_graph,
            "updates_per_s_batched": updates / (ms_graph * 1e-3), "labels_identical": bool(same and same_graph),
            "autotune": {"rows": tuned[0], "warps_per_row": tuned[1], "table": tuned[3]}}


def measure_proposal(edp, torch, train_pairs: int = 2000, epochs: int = 10,
                     eval_pairs=(1000, 1001, 1002, 1003), W: int = 640, H: int = 480, win: int = 9, reps: int = 2):
    """Learned proposal + 9x9 windowed EDP against full-label EDP (65x65
    labels) on held-out 640x480 pairs.  The network is trained here, by the
    project's kernels, on full-label EDP labelings of train_pairs synthetic
    640x480 pairs (the images are synthesised by a spawned process pool)."""
    import multiprocessing as mp

    from paper_1410_7922_gb300 import proposal
    t0 = time.perf_counter()
    with mp.get_context("spawn").Pool(min(16, os.cpu_count() or 1)) as pool:
        x, t = proposal.build_training_set(train_pairs, W, H, first_pair=0, pool=pool)
    torch.cuda.synchronize()
    t_data = time.perf_counter() - t0
    t0 = time.perf_counter()
    P, losses = proposal.train(x, t, epochs=epochs, batch=8, lr=2e-3)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    del x, t
    rows = proposal.evaluate(P, list(eval_pairs), W, H, win=win, reps=reps)
    mean = lambda k: sum(r[k] for r in rows) / len(rows)
    return {"train_pairs": train_pairs, "train_size": [W, H], "epochs": epochs, "window": win,
            "min_shift": proposal.MIN_SHIFT, "edge_frac_fallback": proposal.EDGE_FRAC,
            "loss_first": losses[0], "loss_last": losses[-1],
            "s_training_data": t_data, "s_training": t_train, "eval": rows,
            "mean_gap_solve": mean("gap_solve"), "max_gap_solve": max(r["gap_solve"] for r in rows),
            "fallbacks": sum(r["fallback"] for r in rows),
            "mean_gap_net": mean("gap_net"), "mean_gap_coarse": mean("gap_coarse"),
            "mean_heldout_loss_net": mean("loss_net"), "mean_heldout_loss_no_correction": mean("loss_zero"),
            "mean_ms_full": mean("ms_full"), "mean_ms_solve": mean("ms_solve"), "mean_ms_net": mean("ms_net"),
            "mean_ms_coarse": mean("ms_coarse"),
            "mean_speedup_solve": sum(r["ms_full"] / r["ms_solve"] for r in rows) / len(rows)}


def run_gpu(args, world, rank, local):
    import numpy as np
    import torch

    import __graft_entry__
    __graft_entry__.build()
    from paper_1410_7922_gb300 import edp, synth

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if args.net_only:
        if rank == 0:
            print(json.dumps({"proposal_net": measure_net(edp, torch)}), flush=True)
        return
    j = args.iters
    w = make_workload(args.workload, pair=rank, size=args.size)  # weak scaling: one pair per rank
    H, W = w["I0"].shape
    space, prior = w["space"], w["prior"]
    Q = edp.n_labels(space)
    I0 = torch.from_numpy(w["I0"]).to(dev)
    I1 = torch.from_numpy(w["I1"]).to(dev)
    ws = edp.workspace(edp.OP_SOLVE_IMAGES, W, H, space, prior, j, device=dev)
    labels = torch.empty((H, W), dtype=torch.int32, device=dev)
    energy4 = torch.empty(4, dtype=torch.int64, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)  # > L2 (126 MB)
    pev = [torch.cuda.Event(enable_timing=True) for _ in range(8 * j)]

    def step():
        edp.solve_images(I0, I1, None, space, prior, w["l2"], w["cmax"], iters=j, ws=ws, labels=labels,
                         energy4=energy4)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    npass = edp.last_pass_launches()  # scan-pass launches per solve (2 per iteration for paired sweeps)
    launches_per_step = 1 + npass + 1  # cost volume, scan passes, energy

    def timed_region():
        step_ms, pass_ms = [], [0.0] * npass
        edp.set_profile_events(pev)
        barrier(world)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            flush.zero_()
            s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            s.record()
            step()
            e.record()
            e.synchronize()
            step_ms.append(s.elapsed_time(e))
            for i in range(npass):
                pass_ms[i] += pev[2 * i].elapsed_time(pev[2 * i + 1])
        torch.cuda.synchronize()
        barrier(world)
        wall = time.perf_counter() - t0
        edp.set_profile_events(None)
        return step_ms, pass_ms, wall

    with ClockSampler(local) as cs:
        step_ms, pass_ms, wall = timed_region()
    clocks = cs.summary()
    remeasured = False
    if bad_clocks(clocks):
        remeasured = True
        with ClockSampler(local) as cs:
            step_ms, pass_ms, wall = timed_region()
        clocks = cs.summary()
    status = edp.get_device_status(ws)
    if status != 0:
        raise RuntimeError(f"device status {edp.status_string(status)}")
    total_ms = allreduce_max(world, sum(step_ms))
    ms_per_step = total_ms / args.steps
    updates = W * H * Q * (8 * j + 1)
    value = updates * world * args.steps / (total_ms * 1e-3)

    # roofline of the dominant kernel (the scan pass): sums-form algorithmic
    # bytes (20 Q per pixel per pass, four passes per iteration) / the pass
    # launches' event time
    pass_total_s = sum(pass_ms) * 1e-3 / args.steps
    nbytes = 4 * j * sums_bytes_per_pass(W, H, Q)
    achieved = nbytes / pass_total_s / 1e9
    msg_bytes = sum(launch_bytes(npass, W, H, Q, j))
    peak, peak_kind = measured_peaks()
    kernel = edp.last_pass_kernel()
    traffic = profiled_traffic(args.workload + (f"@{args.size}" if args.size else ""), kernel)
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": traffic, "peak_kind": peak_kind, "kernel": kernel,
                "bytes_per_launch_avg": nbytes / npass, "bytes_model": "20*Q per pixel per pass (sums form)",
                "message_form_bytes_per_launch_avg": msg_bytes / npass,
                "message_form_gbs": msg_bytes / pass_total_s / 1e9,
                "launch_ms_avg": sum(pass_ms) / args.steps / npass,
                "launches_per_solve": npass, "schedule": "paired sweeps" if npass == 2 * j else "one pass per launch",
                "pass_ms": [p / args.steps for p in pass_ms]}

    # end to end through the host-buffer C call (copies inside the timed region)
    I0h = torch.from_numpy(w["I0"]).pin_memory()
    I1h = torch.from_numpy(w["I1"]).pin_memory()
    lab_h = torch.empty((H, W), dtype=torch.int32).pin_memory()
    en_h = torch.empty(4, dtype=torch.int64).pin_memory()

    def e2e_step():
        edp.solve_images_host(I0h, I1h, None, space, prior, w["l2"], w["cmax"], ws, iters=j,
                              labels_out=lab_h.numpy(), energy_out=en_h.numpy())

    for _ in range(2):
        e2e_step()
    barrier(world)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        e2e_step()
    e2e_s = allreduce_max(world, time.perf_counter() - t0)
    e2e = {"value": updates * world * args.steps / e2e_s, "unit": UNIT, "h2d_bytes_per_step": 2 * W * H,
           "d2h_bytes_per_step": W * H * 4 + 32, "ms_per_step": 1e3 * e2e_s / args.steps}
    assert np.array_equal(lab_h.numpy(), labels.cpu().numpy())

    rows = None
    if not args.no_rows and rank == 0 and args.workload == WORKLOAD:
        rows = time_solve_rows(edp, synth, torch, peak)
        # the two added forms against plain full-label EDP on this GPU
        rows["batched_64_pairs"] = measure_batched(edp, synth, torch, scale=args.batch_scale)
        rows["proposal_640x480_Q65x65_w9"] = measure_proposal(edp, torch, train_pairs=args.row_proposal_pairs,
                                                              eval_pairs=(1000, 1001, 1002, 1003, 1004, 1005),
                                                              reps=1)
        rows["proposal_net"] = measure_net(edp, torch)
    extra = {}
    if rank == 0:
        for name in [e for e in args.extra.split(",") if e]:
            if name == "batched":
                extra["batched"] = measure_batched(edp, synth, torch, scale=args.batch_scale)
            elif name == "proposal":
                extra["proposal"] = measure_proposal(edp, torch, train_pairs=args.proposal_pairs)
    cpu = None
    if not args.no_cpu and rank == 0 and world == 1:
        cpu = cpu_oracle_sample(w, j)
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "int32", "data": "synthetic",
                "config": {"workload": args.workload + (f"@{args.size}" if args.size else ""), "W": W, "H": H,
                           "Q": Q, "iters": j,
                           "prior": w["desc"]["prior"], "cost": w["desc"]["cost"],
                           "l2_cache": "flushed between steps (256 MB write)",
                           "parallelism": f"replicas x{world} (one independent pair per GPU)"},
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
                "gpu_launches": launches_per_step * args.steps, "clocks": clocks,
                "wall_s_timed_region": wall, "remeasured": remeasured, "rows": rows,
                "energy_per_pixel": float(energy4[3].item()) / (W * H)}
        if extra:
            line["extra"] = extra
        print(json.dumps(line), flush=True)


def main():
    args = parse_args()
    world, rank, local = dist_setup(args)
    try:
        if args.impl == "reference":
            run_reference(args, world, rank)
        else:
            run_gpu(args, world, rank, local)
    finally:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()


if __name__ == "__main__":
    main()
