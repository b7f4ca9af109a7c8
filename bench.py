#!/usr/bin/env python3
"""Benchmark of the GB300 Gauss-Jordan inversion library.

Default workload: one 8192 x 8192 FP64 matrix, N(0,1) entries + 0.1 n on the diagonal,
partial pivoting, blocked path (cluster panel + rank-b update).  A step is one whole
inversion through the C ABI (copy-in, every panel and update, un-permutation,
determinant) with the input already resident in device memory.  The metric is inverse
GFLOP/s counted as 2 n^3 per inverse.

Other workloads (``--workload``): ``inv128`` (one 128 x 128 N(0,1) matrix, full pivoting)
``batch200k`` (200,000 matrices, orders uniform in 4..64, diagonally dominant,
partial pivoting, one persistent launch replayed as a CUDA graph; metric matrices/s),
``mixed16384`` (one 16384 x 16384 FP32 matrix, kappa 1e6: reduced-precision GJ plus
Newton-Schulz refinement to a 1e-12 normalised residual) and ``mixedbatch4096`` (4,096
FP32 matrices, orders uniform in 128..1024, kappa log-uniform in 1e2..1e8, each refined to
a 1e-12 normalised residual by a pool of host workers with one stream each).

``--impl reference`` times the CPU oracle (plain FP64 C, the test reference) on the host
cores on a bounded sample of the same workload and prints the same JSON line.

Multi-GPU (torchrun): each rank inverts its own matrices (independent problems, no
data-path collective); value = work of all ranks / max time over ranks.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_1401_7962_gb300 import workloads as wl  # noqa: E402

PEAKS_PATH = os.path.join(ROOT, "MEASURED_PEAKS.json")
# Nominal GB300 FP64 rate: 152 SMs x 2 FP64 FMA lanes per clock x 2 FLOP x ~2.06 GHz; used only
# when the run's own probe (gj_measure_peaks) is not available.
FP64_NOMINAL_GFLOPS = 1250.0
PROBED = {}  # this run's gj_measure_peaks result

# DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) per launch of the dominant
# kernel from one ncu capture (profiles/), with the order it was taken at; scaled to the
# benchmark's order by the n^2 elements one update launch touches.  Set an entry to None
# when its kernel changes, until it is captured again.
NCU_TRAFFIC = {
    "update_dfma": None,  # column-window change since profiles/update_dfma_inv6144.md
    # the wide (outer) update of the blocked path, launch 203 of the kernel at n = 6144 (104 CTAs),
    # profiles/ozaki_update_kernel_inv6144.md
    "update_ozaki_wide": {"n": 6144, "bytes": 318.893568e6 + 232.922368e6},
    "update_ozaki_tc": None,
    # the plan replays one kernel per order bin; traffic summed over those kernels
    "batched_plan": None,
}

WORKLOADS = {
    "inv8192": dict(n=8192, shift=0.1, pivot=1, seed=wl.SEED_BASE + 2,
                    name="gj-inverse-8192-fp64-partial-blocked"),
    "inv128": dict(n=128, shift=0.0, pivot=2, seed=wl.SEED_BASE + 1, name="gj-inverse-128-fp64-full-cluster"),
    "batch200k": dict(count=200_000, seed=wl.SEED_BASE + 3, pivot=1,
                      name="gj-batched-200k-n4to64-fp64-partial"),
    "mixed16384": dict(n=16384, kappa=1e6, pivot=1, seed=wl.SEED_BASE + 4,
                       name="gj-inverse-16384-fp32in-mixed-refined"),
    "mixedbatch4096": dict(count=4096, seed=wl.SEED_BASE + 5, pivot=1,
                           name="gj-batched-mixed-4096-n128to1024-fp32in-refined"),
}

_MIXED_BATCH_HOST = {}
_MIXED_BATCH_DEV = {}


def mixed_batch_on_device(count: int, seed: int, dev):
    """The batched mixed recipe generated on the GPU (cached: the QRs take a while)."""
    key = (count, seed, str(dev))
    if key not in _MIXED_BATCH_DEV:
        sizes, kappas, offsets = wl.mixed_batch_params(count, seed)
        _MIXED_BATCH_DEV[key] = (sizes, offsets, wl.mixed_batch_device(sizes, kappas, offsets, seed, device=dev))
    return _MIXED_BATCH_DEV[key]


def mixed_batch_sample(count: int, seed: int):
    """The first ``count`` matrices of the batched mixed recipe (host generator), cached."""
    key = (count, seed)
    if key not in _MIXED_BATCH_HOST:
        sizes, kappas, offsets = wl.mixed_batch_params(count, seed)
        packed32 = wl.mixed_batch_host(sizes, kappas, offsets, seed)
        _MIXED_BATCH_HOST[key] = (sizes, offsets, packed32.astype(np.float64))
    return _MIXED_BATCH_HOST[key]


# ----------------------------------------------------------------- distributed helpers

def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def max_over_ranks(value: float, world: int) -> float:
    if world <= 1:
        return value
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([value], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(world: int) -> None:
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def shard_lpt(sizes: np.ndarray, world: int) -> list[np.ndarray]:
    """Split matrix indices over ranks by n^3, largest first, each to the least-loaded rank."""
    order = np.argsort(-(sizes.astype(np.float64) ** 3), kind="stable")
    load = np.zeros(world)
    parts = [[] for _ in range(world)]
    for m in order:
        r = int(np.argmin(load))
        parts[r].append(int(m))
        load[r] += float(sizes[m]) ** 3
    return [np.array(sorted(p), dtype=np.int64) for p in parts]


# ----------------------------------------------------------------- clocks

class ClockSampler:
    """nvidia-smi samples (200 ms) during the timed region."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines: list[str] = []
        self.t = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, FileNotFoundError):
            self.proc = None
            return
        self.t = threading.Thread(target=self._read, daemon=True)
        self.t.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.t:
            self.t.join(timeout=2)
        sm, smax, power, reasons = [], [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
                power.append(float(f[3]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "power_w_max": max(power) if power else None, "samples": len(sm), "reasons": sorted(reasons)}


# ----------------------------------------------------------------- peaks

def measured_peaks() -> dict:
    try:
        with open(PEAKS_PATH) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def roofline_tensor(tensor_tflops: float, fp64_equiv_tflops, pairs, traffic) -> dict:
    """Roofline entry of a tensor-core update kernel.  With a single slice count, `achieved`
    is the method's own work (2 M N K FP64 FLOP per launch) per second; the BF16 digit-slice
    products the tensor cores actually run (pairs per FP64 term) are reported beside it."""
    peaks = measured_peaks()
    peak = float(peaks.get("bf16_tflops_sustained", 1720.6))
    src = "of measured" if "bf16_tflops_sustained" in peaks else "of fallback"
    ach = fp64_equiv_tflops if fp64_equiv_tflops is not None else tensor_tflops
    return {"bound": "tensor", "achieved": round(ach, 3), "peak": peak, "unit": "TFLOP/s",
            "frac": round(ach / peak, 5), "traffic": traffic,
            "peak_source": f"BF16 dense sustained {src} (kernel timed inside a long step)",
            "work": (f"method FLOP (2 M N K per launch, FP64 accurate); the tensor cores run {pairs} BF16 "
                     "digit-slice products per FP64 term" if pairs else
                     "BF16 digit-slice FLOP (S (S + 1) / 2 products per FP64 term; the mixed path runs several S)"),
            "tensor_slice_tflops": round(tensor_tflops, 2), "tensor_slice_frac": round(tensor_tflops / peak, 4)}


def roofline_fp64(achieved_gflops: float, traffic) -> dict:
    # FP64 FMA is plain ALU work on GB300 (DMMA measures no faster than DFMA), so the
    # peak is the FP64 unit rate, not a tensor rate: this run's DFMA probe when it ran
    if PROBED.get("fp64_fma_gflops"):
        peak = PROBED["fp64_fma_gflops"]
        src = "of measured: FP64 FMA probe (gj_measure_peaks) in this run, independent chains on every SM"
    else:
        peak = FP64_NOMINAL_GFLOPS
        src = "nominal FP64 unit rate (152 SMs x 4 FLOP/clk x 2.06 GHz)"
    return {"bound": "alu", "achieved": round(achieved_gflops / 1000.0, 4), "peak": round(peak / 1000.0, 4),
            "unit": "TFLOP/s", "frac": round(achieved_gflops / peak, 4), "traffic": traffic, "peak_source": src}


# ----------------------------------------------------------------- CPU oracle legs

def cpu_oracle_sample(workload: str, repeat: int = 1) -> dict:
    """The oracle as it stands on a bounded sample of the workload; returns value/unit/cores/sample."""
    import oracle
    W = WORKLOADS[workload]
    if workload == "batch200k":
        sizes, packed, offsets = wl.diag_dominant_batch(W["count"], W["seed"])
        take = 40_000
        sizes, offsets = sizes[:take], offsets[:take]
        cores = os.cpu_count() or 1
        t0 = time.perf_counter()
        for _ in range(repeat):
            oracle.invert_many(sizes, packed, offsets, W["pivot"], threads=cores)
        dt = (time.perf_counter() - t0) / repeat
        return {"value": take / dt, "unit": "matrices/s", "cores": cores, "kind": "oracle",
                "sample": f"first {take} of the 200000 matrices, oracle over {cores} threads",
                "gflops": float((2.0 * sizes.astype(np.float64) ** 3).sum() / dt / 1e9)}
    if workload == "mixedbatch4096":
        # the same recipe's first 192 matrices (orders 128..1024, kappa 1e2..1e8, the FP32
        # values converted exactly), plain FP64 Gauss-Jordan over all host cores
        take = 192
        sizes, offsets, packed = mixed_batch_sample(take, W["seed"])
        cores = os.cpu_count() or 1
        t0 = time.perf_counter()
        for _ in range(repeat):
            oracle.invert_many(sizes, packed, offsets, W["pivot"], threads=cores)
        dt = (time.perf_counter() - t0) / repeat
        return {"value": float((2.0 * sizes.astype(np.float64) ** 3).sum() / dt / 1e9), "unit": "GFLOP/s",
                "cores": cores, "kind": "oracle",
                "sample": f"first {take} of the 4096 matrices (host generator), FP64 oracle over {cores} threads",
                "matrices_per_s": take / dt}
    if workload == "mixed16384":
        n = 1536
        A = wl.svd_conditioned(n, W["kappa"], W["seed"], dtype=np.float32).astype(np.float64)
        t0 = time.perf_counter()
        oracle.invert(A, W["pivot"])
        dt = time.perf_counter() - t0
        return {"value": 2.0 * n ** 3 / dt / 1e9, "unit": "GFLOP/s", "cores": 1, "kind": "oracle",
                "sample": f"FP64 oracle on one {n}x{n} matrix of the same recipe (kappa 1e6), 1 thread"}
    n = 2048 if workload == "inv8192" else W["n"]
    A = wl.gaussian(n, W["seed"], shift=W["shift"] * n)
    reps = repeat if workload == "inv8192" else max(repeat, 50)
    t0 = time.perf_counter()
    for _ in range(reps):
        oracle.invert(A, W["pivot"])
    dt = (time.perf_counter() - t0) / reps
    samp = (f"one {n}x{n} matrix of the same recipe (N(0,1)+0.1nI), partial pivoting, 1 thread"
            if workload == "inv8192" else f"the {n}x{n} matrix, full pivoting, 1 thread, mean of {reps}")
    return {"value": 2.0 * n ** 3 / dt / 1e9, "unit": "GFLOP/s", "cores": 1, "kind": "oracle", "sample": samp}


def run_reference(args) -> None:
    world, rank, _ = dist_env()
    if rank != 0:
        return
    W = WORKLOADS[args.workload]
    for _ in range(args.warmup):
        cpu_oracle_sample(args.workload)
    vals = []
    t0 = time.perf_counter()
    for _ in range(args.steps):
        vals.append(cpu_oracle_sample(args.workload))
    wall = time.perf_counter() - t0
    v = statistics.median([x["value"] for x in vals])
    cb = dict(vals[0])
    cb["value"] = v
    line = {"impl": "reference", "metric": metric_name(args.workload), "value": v, "unit": cb["unit"],
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * wall / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": W["name"], "sample": cb["sample"]},
            "cpu_baseline": {k: cb[k] for k in ("value", "unit", "cores", "kind", "sample")},
            "e2e": {"value": v, "unit": cb["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def metric_name(workload: str) -> str:
    return "inverse GFLOP/s (2n^3)" if workload != "batch200k" else "batched matrices/s"


# ----------------------------------------------------------------- GPU arm

# The other workloads measured beside the 8192 inversion in the default run (one GPU):
# (workload, timed steps, first-inverse slices of the mixed paths).
SUB_WORKLOADS = (("inv128", 50, None), ("batch200k", 10, None), ("mixed16384", 2, 3), ("mixedbatch4096", 2, 7))


def run_gpu(args) -> None:
    import copy
    import torch
    world, rank, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local if world > 1 else 0)
    torch.cuda.set_device(dev)
    from paper_1401_7962_gb300 import _build
    _build.build()
    import paper_1401_7962_gb300 as gj
    L = gj.lib()
    try:
        PROBED.update(gj.measure_peaks())
    except Exception as exc:  # pragma: no cover - reported in the line
        PROBED["error"] = str(exc)
    line = measure(args, gj, L, dev, world, rank)
    if rank == 0 and world == 1 and args.workload == "inv8192" and not args.n and not args.headline_only:
        subs = {}
        for wk, steps, x0 in SUB_WORKLOADS:
            a2 = copy.copy(args)
            a2.workload, a2.steps, a2.slices, a2.update, a2.count = wk, steps, 0, "auto", 0
            if x0 is not None:
                a2.x0_slices = x0
            sub = measure(a2, gj, L, dev, world, rank)
            subs[sub["config"]["workload"]] = sub_entry(sub)
            torch.cuda.synchronize(dev)
            torch.cuda.empty_cache()
            L.gj_trim_memory()
        line["config"]["configs"] = subs
        line["config"]["panel_sweep"] = panel_sweep(args, gj, L, dev)
    if rank == 0 and line:
        line["config"]["peaks_probed"] = {k: (round(v, 1) if isinstance(v, float) else v) for k, v in PROBED.items()}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


GOLDEN_DIR = os.path.join(ROOT, "tests", "golden")


def golden_8192_meta():
    try:
        with open(os.path.join(GOLDEN_DIR, "inv8192_partial_oracle.json")) as f:
            return json.load(f)
    except (OSError, ValueError):
        return None


def oracle_parity_8192(dX, rec) -> dict:
    """The benchmark's last 8192 inverse against the oracle's stored result for the same input
    (tests/golden/inv8192_partial_oracle.*): pivot sequence, det, and the largest difference
    over the 16 stored columns, 16 rows and 4096 entries, relative to max |x| of the oracle's
    inverse."""
    meta = golden_8192_meta()
    if not meta:
        return {"available": False}
    ref = np.load(os.path.join(GOLDEN_DIR, "inv8192_partial_oracle.npz"))
    X = dX.cpu().numpy()
    cols, rows, pairs = ref["cols"], ref["rows"], ref["pairs"]
    d = max(np.max(np.abs(X[:, cols] - ref["X_cols"])), np.max(np.abs(X[rows, :] - ref["X_rows"])),
            np.max(np.abs(X[pairs[:, 0], pairs[:, 1]] - ref["X_pairs"])))
    out = {"available": True, "max_abs_diff_over_max_x": float(d / ref["X_absmax"][0]),
           "compared": "16 columns, 16 rows, 4096 entries"}
    if rec is not None:
        out["pivots_identical"] = bool(np.array_equal(rec["piv_rows"], ref["piv_rows"]))
        out["det_sign_equal"] = rec["det_sign"] == meta["det_sign"]
        out["det_log2_rel_diff"] = abs(rec["det_log2"] - meta["det_log2"]) / abs(meta["det_log2"])
    return out


def panel_sweep(args, gj, L, dev) -> dict:
    """The 8192 inversion with each cluster panel width the blocked path takes at this order
    (the tensor-core update's outer panel is 128 columns; a 64-column cluster panel does not
    fit the shared memory of 16 CTAs at n = 8192): ms per inversion, 3 timed after 2 more."""
    import ctypes
    import torch
    W = WORKLOADS["inv8192"]
    n = W["n"]
    dA = torch.from_numpy(wl.gaussian(n, W["seed"], shift=W["shift"] * n)).to(dev)
    dX = torch.empty_like(dA)
    stream = torch.cuda.Stream(device=dev)
    sgn, lg2 = ctypes.c_int(0), ctypes.c_double(0.0)
    out = {}
    for b in (16, 32):
        opts = gj._Opts()
        opts.stream = stream.cuda_stream
        opts.panel = b
        run = lambda: L.gj_invert_ex(ctypes.byref(opts), n, dA.data_ptr(), n, dX.data_ptr(), W["pivot"],
                                     ctypes.byref(sgn), ctypes.byref(lg2))
        for _ in range(2):
            run()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(3):
            run()
        e1.record(stream)
        e1.synchronize()
        ms = e0.elapsed_time(e1) / 3
        out[f"cluster_panel_{b}"] = {"ms_per_inverse": round(ms, 2), "gflops": round(2.0 * n ** 3 / ms / 1e6, 1)}
    out["outer_panel"] = 128
    return out


def sub_entry(sub: dict) -> dict:
    """The measurement of one more workload, as an entry of the headline line's config."""
    keep = ("metric", "value", "unit", "ms_per_step", "steps", "warmup", "roofline", "cpu_baseline", "e2e", "clocks",
            "gpu_launches")
    e = {k: sub.get(k) for k in keep}
    cfg = dict(sub["config"])
    cfg.pop("profile", None)
    e["config"] = cfg
    return e


def measure(args, gj, L, dev, world: int, rank: int) -> dict:
    """Time one workload (warm-up, then args.steps steps) and return its JSON line (a dict)."""
    import ctypes
    import torch
    W = dict(WORKLOADS[args.workload])
    if args.count and "count" in W:
        W["count"] = args.count
        W["name"] = W["name"].replace("200k", f"{args.count // 1000}k")
    if args.n and "n" in W:
        W["n"] = args.n
        W["name"] = W["name"].replace(str(WORKLOADS[args.workload]["n"]), str(args.n))
    stream = torch.cuda.Stream(device=dev)
    Entry = _profile_struct()[0]
    prof_entries = (Entry * 16)()
    per_launch_flops = 0.0

    extra = {}
    if args.workload == "batch200k":
        sizes, packed, offsets = wl.diag_dominant_batch(W["count"], W["seed"] + rank)
        count = len(sizes)
        dA = torch.from_numpy(packed).to(dev)
        dX = torch.empty_like(dA)
        ap = torch.from_numpy(dA.data_ptr() + 8 * offsets).to(dev)
        xp = torch.from_numpy(dX.data_ptr() + 8 * offsets).to(dev)
        st = torch.zeros(count, dtype=torch.int32, device=dev)
        sg = torch.zeros(count, dtype=torch.int8, device=dev)
        lg = torch.zeros(count, dtype=torch.float64, device=dev)
        # autotuned kernel variant per order bin (choices read from / written to --tune-cache)
        plan = gj.BatchedPlan(sizes, W["pivot"], tune_cache=args.tune_cache)
        extra["bins"] = [{k: b[k] for k in ("lo", "hi", "count", "variant")} for b in plan.bins()]
        flops_step = float((2.0 * sizes.astype(np.float64) ** 3).sum())
        bytes_step = float(16.0 * (sizes.astype(np.float64) ** 2).sum())
        units_step = count

        def step():
            plan.execute(ap, xp, st, sg, lg, stream=stream, use_graph=True)

        dominant = "batched_plan"
        per_launch_flops = flops_step
        h2d = packed.nbytes + 8 * count * 2 + 4 * count
        d2h = packed.nbytes + count * (4 + 1 + 8)
    elif args.workload == "mixed16384":
        n = W["n"]
        dA32 = wl.svd_conditioned_device(n, W["kappa"], W["seed"] + rank, device=dev)
        dX = torch.empty((n, n), dtype=torch.float64, device=dev).t().contiguous().t()
        flops_step = 2.0 * n ** 3
        units_step = 1
        mixed_state = {}

        def step():
            r = gj.invert_mixed(dA32, out=dX, x0_slices=args.x0_slices, corr_slices=4, tol=1e-12, max_iter=10,
                                stream=stream)
            if r["status"] != 0:
                raise RuntimeError(f"gj_invert_mixed: {gj.status_string(r['status'])}")
            mixed_state.update(r)

        dominant = "update_ozaki_tc"
        h2d = 4 * n * n
        d2h = 8 * n * n
    elif args.workload == "mixedbatch4096":
        t_gen = time.perf_counter()
        sizes, offsets, flatA = mixed_batch_on_device(W["count"], W["seed"] + rank, dev)
        torch.cuda.synchronize(dev)
        extra["input_generation_s"] = round(time.perf_counter() - t_gen, 1)
        flatX = torch.empty(flatA.numel(), dtype=torch.float64, device=dev)
        As = [wl.matrix_view(flatA, int(n), int(o)) for n, o in zip(sizes, offsets)]
        Xs = [wl.matrix_view(flatX, int(n), int(o)) for n, o in zip(sizes, offsets)]
        flops_step = float((2.0 * sizes.astype(np.float64) ** 3).sum())
        units_step = len(sizes)
        mixed_state = {}

        def step():
            r = gj.invert_mixed_batched(As, Xs, x0_slices=args.x0_slices, corr_slices=4, tol=1e-12, max_iter=10,
                                        workers=args.workers, stream=stream)
            if r["status"] != 0:
                raise RuntimeError(f"gj_invert_mixed_batched: {gj.status_string(r['status'])}")
            mixed_state.update(r)

        dominant = "update_ozaki_tc"
        h2d = 4 * flatA.numel()
        d2h = 8 * flatX.numel()
    else:
        n = W["n"]
        A = wl.gaussian(n, W["seed"] + rank, shift=W["shift"] * n)
        dA = torch.from_numpy(A).to(dev)
        dX = torch.empty_like(dA)
        flops_step = 2.0 * n ** 3
        units_step = 1
        sgn, lg2 = ctypes.c_int(0), ctypes.c_double(0.0)
        opts = gj._Opts()
        opts.stream = stream.cuda_stream
        opts.update = {"auto": 0, "dfma": 1, "ozaki": 2}[args.update]

        def step():
            stc = L.gj_invert_ex(ctypes.byref(opts), n, dA.data_ptr(), n, dX.data_ptr(), W["pivot"],
                                 ctypes.byref(sgn), ctypes.byref(lg2))
            if stc != 0:
                raise RuntimeError(f"gj_invert_ex failed: {gj.status_string(stc)} {gj.last_error()}")

        opts.slices = args.slices
        opts.panel = args.panel
        opts.update_sms = args.update_sms
        dominant = "update_dfma" if args.workload == "inv8192" else "cluster_single"
        h2d = d2h = n * n * 8

    # ---- warm-up
    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            step()
    stream.synchronize()

    # ---- timed region
    clocks = ClockSampler(dev.index if dev.index is not None else 0)
    barrier(world)
    torch.cuda.synchronize(dev)
    clocks.start()
    # The batched mixed workload makes ~400 launches per matrix from several host threads;
    # an event pair per launch would slow it, so its kernel profile comes from one more
    # step after the timed ones.
    prof_after = args.workload == "mixedbatch4096"
    if not prof_after:
        L.gj_profile_begin()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(stream):
        e0.record(stream)
        for _ in range(args.steps):
            step()
        e1.record(stream)
    e1.synchronize()
    torch.cuda.synchronize(dev)
    barrier(world)
    clk = clocks.stop()
    ms = e0.elapsed_time(e1)
    prof_ms = ms
    launches = ctypes.c_int64(0)
    if prof_after:
        # launch count: one more whole step with the counters on
        L.gj_profile_begin()
        with torch.cuda.stream(stream):
            step()
        torch.cuda.synchronize(dev)
        L.gj_profile_end(prof_entries, 16, ctypes.byref(launches))
        launches.value *= args.steps
        # per-kernel device times: the first 256 matrices on one worker, so that no launch
        # waits for SMs held by another stream's kernels
        L.gj_profile_begin()
        p0 = time.perf_counter()
        gj.invert_mixed_batched(As[:256], Xs[:256], x0_slices=args.x0_slices, corr_slices=4, tol=1e-12,
                                max_iter=10, workers=1, stream=stream)
        torch.cuda.synchronize(dev)
        prof_ms = 1000.0 * (time.perf_counter() - p0)
        extra["profile_sample"] = "first 256 matrices, 1 worker, outside the timed steps"
        extra["profile_sample_ms"] = round(prof_ms, 1)
        dummy = ctypes.c_int64(0)
        cnt = L.gj_profile_end(prof_entries, 16, ctypes.byref(dummy))
    else:
        cnt = L.gj_profile_end(prof_entries, 16, ctypes.byref(launches))
    ms_max = max_over_ranks(ms, world)
    prof = {}
    for i in range(cnt):
        e = prof_entries[i]
        prof[e.kernel.decode()] = {"launches": e.launches, "total_ms": e.total_ms, "flops": e.flops, "bytes": e.bytes}

    total_units = units_step * args.steps * world
    total_flops = flops_step * args.steps * world
    if args.workload == "batch200k":
        value = total_units / (ms_max / 1000.0)
        unit = "matrices/s"
        extra["gflops"] = total_flops / (ms_max / 1000.0) / 1e9
    elif args.workload == "mixedbatch4096":
        value = total_flops / (ms_max / 1000.0) / 1e9
        unit = "GFLOP/s"
        extra["matrices_per_s"] = total_units / (ms_max / 1000.0)
    else:
        value = total_flops / (ms_max / 1000.0) / 1e9
        unit = "GFLOP/s"

    roof = None
    if args.workload == "mixedbatch4096" and prof:
        # many kernels of many matrices: the dominant one is the one with the most device time
        dominant = max(prof, key=lambda k: prof[k]["total_ms"])
    else:
        for name in ("update_ozaki_wide", "update_ozaki_tc"):
            if name in prof and prof[name]["launches"]:
                dominant = name
                break
    if dominant in ("update_ozaki_wide", "update_ozaki_tc"):
        d = prof[dominant]
        avg_ms = d["total_ms"] / d["launches"]
        # the profile counts tensor FLOP (S (S + 1) / 2 slice products per FP64 term); the
        # mixed paths run the update with several slice counts, so no single FP64 equivalent
        S = None if args.workload in ("mixed16384", "mixedbatch4096") else (args.slices or 7)
        pairs = S * (S + 1) // 2 if S else None
        tc_fl = d["flops"] / d["launches"]
        t = NCU_TRAFFIC.get(dominant)
        traffic = args.traffic
        if traffic is None and t and "n" in W:
            traffic = t["bytes"] * (W["n"] / t["n"]) ** 2
        tensor_tflops = tc_fl / (avg_ms / 1000.0) / 1e12
        roof = roofline_tensor(tensor_tflops, tensor_tflops / pairs if pairs else None, pairs, traffic)
        roof["kernel"] = dominant
        roof["avg_launch_ms"] = round(avg_ms, 6)
        roof["share_of_step"] = round(d["total_ms"] / prof_ms, 4)
        if args.workload == "mixedbatch4096":
            roof["note"] = "from the 1-worker profile sample (no contention between streams)"
        if dominant == "update_ozaki_wide" and W.get("n", 0) >= 2048:
            cs = min(16, -(-W["n"] // 256))
            sms = torch.cuda.get_device_properties(dev).multi_processor_count
            roof["grid_sms"] = min(args.update_sms, sms) if args.update_sms > 0 else sms - min(3 * cs, sms // 2)
            roof["note"] = (f"look-ahead: runs on {roof['grid_sms']} of {sms} SMs while the panel stream reduces "
                            "the next panel; share_of_step counts overlapped time")
    elif dominant in prof and prof[dominant]["launches"]:
        d = prof[dominant]
        avg_ms = d["total_ms"] / d["launches"]
        fl = d["flops"] / d["launches"] if d["flops"] else per_launch_flops
        achieved_gflops = fl / (avg_ms / 1000.0) / 1e9
        traffic = args.traffic
        t = NCU_TRAFFIC.get(dominant)
        if traffic is None and t and "n" in W and "n" in t:
            traffic = t["bytes"] * (W["n"] / t["n"]) ** 2
        if traffic is None and t and "count" in W and "count" in t:
            traffic = t["bytes"] * W["count"] / t["count"]
        roof = roofline_fp64(achieved_gflops, traffic)
        roof["kernel"] = dominant
        roof["avg_launch_ms"] = round(avg_ms, 6)
        roof["share_of_step"] = round(d["total_ms"] / prof_ms, 4)
        if args.workload == "mixedbatch4096":
            roof["note"] = ("from the 1-worker profile sample (no contention between streams); a panel launch "
                            "runs on its cluster's 1-4 CTAs, so its fraction of the whole-GPU FP64 rate is "
                            "small by construction")

    if args.workload == "mixedbatch4096":
        rung = np.asarray(mixed_state["rung"])
        its = np.asarray(mixed_state["iters"])
        extra["resid_max"] = float(np.max(mixed_state["resid"]))
        ladder = np.array([min(args.x0_slices, 7), min(max(args.x0_slices, 5), 7), 7])
        used = ladder[rung]
        extra["x0_slices_used_counts"] = {f"{sl}_slices": int((used == sl).sum()) for sl in sorted(set(ladder.tolist()))}
        extra["refinement_steps_mean"] = round(float(its.mean()), 3)
    if args.workload == "mixedbatch4096":
        extra.update(batched_fp64_arm(gj, As, Xs, sizes, flops_step, mixed_state, args.workers, dev))
    if args.workload == "mixed16384":
        n = W["n"]
        extra["resid"] = mixed_state.get("resid")
        extra["refinement_steps"] = mixed_state.get("iters")
        extra["x0_rung_slices"] = [min(args.x0_slices, 7), min(max(args.x0_slices, 5), 7), 7][mixed_state.get("rung", 0)]
        # the plain FP64-level Gauss-Jordan on the same matrix (converted exactly to FP64)
        dA64 = dA32.double().t().contiguous().t()
        for eng, label in ((gj.UPDATE_TC_OZAKI, "fp64_gj_tensor_update"), (gj.UPDATE_DFMA, "fp64_gj_fma_update")):
            if eng == gj.UPDATE_DFMA and not args.compare_fma:
                continue
            c0 = torch.cuda.Event(enable_timing=True)
            c1 = torch.cuda.Event(enable_timing=True)
            c0.record(stream)
            rr = gj.invert(dA64, gj.PIVOT_PARTIAL, out=dX, update=eng, stream=stream)
            c1.record(stream)
            c1.synchronize()
            extra[label + "_ms"] = c0.elapsed_time(c1)
            extra[label + "_gflops"] = 2.0 * n ** 3 / (c0.elapsed_time(c1) / 1000.0) / 1e9
        del dA64

    # ---- end to end through the C ABI with host buffers (copies inside the timed region)
    e2e = None
    if (rank == 0 or world > 1) and not args.no_e2e:
        e2e = run_e2e(args, gj, L, W, stream, dev, h2d, d2h, units_step, flops_step, rank)
        if world > 1:
            e2e["value"] = e2e["value"]  # per-rank; aggregate below
            tmax = max_over_ranks(e2e.pop("_seconds"), world)
            e2e["value"] = (total_units if args.workload == "batch200k" else total_flops / 1e9) / tmax
        else:
            e2e.pop("_seconds", None)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu and not args.n and not args.count:
        cpu = cpu_oracle_sample(args.workload)
        cpu.pop("gflops", None)
        if args.workload == "inv8192":
            meta = golden_8192_meta()
            if meta:
                cpu["full_size_single_core"] = {
                    "seconds": meta["oracle_seconds"], "gflops": round(2.0 * 8192 ** 3 / meta["oracle_seconds"] / 1e9, 3),
                    "where": "the x86 development host, one core, when tests/golden/inv8192_partial_oracle.* was "
                             "written (not this machine; the full-size oracle takes about 11 minutes)"}
    if rank == 0 and args.workload == "inv8192" and not args.n and args.update != "dfma":
        # one more inversion (untimed) with the pivot record, in the timed launch configuration
        rec = gj.invert(dA, W["pivot"], out=dX, record=True, stream=stream, panel=args.panel,
                        update_sms=args.update_sms)
        torch.cuda.synchronize(dev)
        extra["oracle_parity"] = oracle_parity_8192(dX, rec)

    if rank == 0:
        cfg = {"workload": W["name"], "pivot": ["none", "partial", "full"][W["pivot"]],
               "l2": "inputs larger than L2 (no flush)" if args.workload != "inv128" else
               "128 KiB matrix is L2-resident; latency-bound 16-CTA cluster (no flush)",
               "profile": prof}
        if args.workload == "inv8192":
            eng = "fp64 fma" if (args.update == "dfma") else \
                f"tensor cores: bf16 balanced 8-bit digit slices (S={args.slices or 7}), exact fp32 group sums, " \
                "int64 recombination"
            cfg.update({"n": W["n"], "update": args.update, "update_engine": eng,
                        "input": "N(0,1) + 0.1 n I, seed 1403"})
        elif args.workload == "mixed16384":
            cfg.update({"n": W["n"], "kappa": W["kappa"], "tol": 1e-12,
                        "input": "U diag(sigma) V^T, Haar U,V, sigma log-spaced 1..1e6, FP32, seed 1405 (GPU QR)",
                        "method": "reduced-precision blocked GJ (tensor update, x0 slices) + Newton-Schulz, "
                                  "FP64-level residual"})
        elif args.workload == "mixedbatch4096":
            cfg.update({"count": W["count"], "orders": "U{128..1024}", "kappa": "logU[1e2, 1e8]", "tol": 1e-12,
                        "input": "U diag(sigma) V^T, Haar U,V (GPU QR), sigma log-spaced 1..kappa, FP32, seed 1406",
                        "method": f"per matrix: blocked GJ with the tensor update at {args.x0_slices} digit slices "
                                  "(7 = FP64 level) + Newton-Schulz with an FP64-level residual to 1e-12; ladder "
                                  f"{args.x0_slices} -> {max(args.x0_slices, 5)} -> 7 slices for a matrix that does "
                                  "not contract",
                        "launch": f"host worker pool, {args.workers or 16} streams, largest first, update grid "
                                  "capped at 2 x 152 / workers SMs",
                        "x0_slices": args.x0_slices})
        elif args.workload == "inv128":
            cfg.update({"n": W["n"], "input": "N(0,1), seed 1402",
                        "kernel": "one 16-CTA cluster, rows spread over its CTAs (FP64 of 16 SMs)"})
        else:
            cfg.update({"count": W["count"], "orders": "U{4..64}", "input": "U[-1,1], diag 1+sum|row|, seed 1404",
                        "launch": "plan + CUDA graph"})
        cfg.update(extra)
        line = {"metric": metric_name(args.workload), "value": value, "unit": unit, "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max / args.steps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                "data": "synthetic", "config": cfg, "roofline": roof, "cpu_baseline": cpu, "e2e": e2e,
                "clocks": clk, "gpu_launches": int(launches.value)}
        return line
    return {}


def batched_fp64_arm(gj, As, Xs, sizes, flops, mixed_state, workers: int, dev) -> dict:
    """Plain FP64 Gauss-Jordan of the same FP32 matrices (converted exactly to FP64) through the
    public single-matrix call, one host worker thread and stream per worker as in the mixed
    path, timed on the wall clock; then, outside the timing, the per-matrix error of both
    arms against the oracle on the smallest matrices and their residuals on a sample."""
    import threading
    import torch
    import oracle
    order = np.argsort(-sizes, kind="stable")
    workers = max(1, workers or 16)
    Ys = [torch.empty_like(x) for x in Xs]
    streams = [torch.cuda.Stream(device=dev) for _ in range(workers)]
    nxt = [0]
    lock = threading.Lock()
    errs = []

    def work(w):
        st = streams[w]
        while True:
            with lock:
                q = nxt[0]
                nxt[0] += 1
            if q >= len(order):
                return
            m = int(order[q])
            with torch.cuda.stream(st):
                A64 = As[m].to(torch.float64)
                r = gj.invert(A64, gj.PIVOT_PARTIAL, out=Ys[m], stream=st)
            if r["status"] != 0:
                errs.append((m, r["status"]))

    def run_all():
        nxt[0] = 0
        ts = [threading.Thread(target=work, args=(w,)) for w in range(workers)]
        for t in ts:
            t.start()
        for t in ts:
            t.join()
        torch.cuda.synchronize(dev)

    run_all()  # warm-up
    t0 = time.perf_counter()
    run_all()
    dt = time.perf_counter() - t0
    out = {"fp64_gj_batched": {"gflops": flops / dt / 1e9, "matrices_per_s": len(As) / dt, "s_per_batch": dt,
                               "method": "FP64-level blocked GJ (tensor-core update, 7 slices) of every matrix "
                                         f"through gj_invert_ex, {workers} host workers with one stream each",
                               "failures": len(errs)}}
    # per-matrix error against the oracle (smallest matrices) and residuals (sample)
    sample = [int(m) for m in np.argsort(sizes, kind="stable")[:4]]
    e_mixed, e_plain, r_plain = [], [], []
    for m in sample:
        A = As[m].double().cpu().numpy()
        o = oracle.invert(A, oracle.PIVOT_PARTIAL)
        nx = np.linalg.norm(o["X"])
        e_mixed.append(float(np.linalg.norm(Xs[m].cpu().numpy() - o["X"]) / nx))
        Y = Ys[m].cpu().numpy()
        e_plain.append(float(np.linalg.norm(Y - o["X"]) / nx))
        r_plain.append(float(np.linalg.norm(A @ Y - np.eye(A.shape[0])) / (np.linalg.norm(A) * np.linalg.norm(Y))))
    out["oracle_sample"] = {"matrices": sample, "orders": [int(sizes[m]) for m in sample],
                            "mixed_rel_err_F": e_mixed, "fp64_gj_rel_err_F": e_plain,
                            "fp64_gj_resid": r_plain}
    return out


def _profile_struct():
    import ctypes

    class Entry(ctypes.Structure):
        _fields_ = [("kernel", ctypes.c_char_p), ("launches", ctypes.c_int64), ("total_ms", ctypes.c_double),
                    ("flops", ctypes.c_double), ("bytes", ctypes.c_double)]
    return (Entry,)


def run_e2e(args, gj, L, W, stream, dev, h2d, d2h, units_step, flops_step, rank) -> dict:
    """The same metric through the public API with pinned host buffers: every step copies
    the inputs host -> device and the results device -> host inside the timed region."""
    import ctypes
    import torch
    steps = max(1, min(args.steps, 3)) if args.workload in ("inv8192", "mixed16384") else args.steps
    if args.workload == "mixedbatch4096":
        steps = 1
    if args.workload == "mixed16384":
        n = W["n"]
        hA = wl.svd_conditioned_device(n, W["kappa"], W["seed"] + rank, device=dev).cpu().pin_memory()
        hA = hA.t().contiguous().t() if hA.stride(0) != 1 else hA
        hX = torch.empty((n, n), dtype=torch.float64).t().contiguous().t().pin_memory()
        dA = torch.empty((n, n), dtype=torch.float32, device=dev).t().contiguous().t()
        dX = torch.empty((n, n), dtype=torch.float64, device=dev).t().contiguous().t()

        def one():
            with torch.cuda.stream(stream):
                dA.copy_(hA, non_blocking=True)
                gj.invert_mixed(dA, out=dX, x0_slices=args.x0_slices, corr_slices=4, tol=1e-12, stream=stream)
                hX.copy_(dX, non_blocking=True)
            stream.synchronize()
    elif args.workload == "batch200k":
        sizes, packed, offsets = wl.diag_dominant_batch(W["count"], W["seed"] + rank)
        count = len(sizes)
        hA = torch.from_numpy(packed).pin_memory()
        hX = torch.empty_like(hA).pin_memory()
        h_off = torch.from_numpy(offsets).pin_memory()
        h_st = torch.empty(count, dtype=torch.int32).pin_memory()
        h_sg = torch.empty(count, dtype=torch.int8).pin_memory()
        h_lg = torch.empty(count, dtype=torch.float64).pin_memory()
        dA = torch.empty(hA.shape, dtype=torch.float64, device=dev)
        dX = torch.empty_like(dA)
        d_off = torch.empty(count, dtype=torch.int64, device=dev)
        st = torch.empty(count, dtype=torch.int32, device=dev)
        sg = torch.empty(count, dtype=torch.int8, device=dev)
        lg = torch.empty(count, dtype=torch.float64, device=dev)
        n_dev = torch.from_numpy(sizes).to(dev)

        def one():
            with torch.cuda.stream(stream):
                dA.copy_(hA, non_blocking=True)
                d_off.copy_(h_off, non_blocking=True)
                ap = d_off * 8 + dA.data_ptr()
                xp = d_off * 8 + dX.data_ptr()
                gj.invert_batched(n_dev, ap, xp, st, sg, lg, pivot_mode=W["pivot"], nmax=64, stream=stream)
                hX.copy_(dX, non_blocking=True)
                h_st.copy_(st, non_blocking=True)
                h_sg.copy_(sg, non_blocking=True)
                h_lg.copy_(lg, non_blocking=True)
            stream.synchronize()
    elif args.workload == "mixedbatch4096":
        sizes, offsets, flatA = mixed_batch_on_device(W["count"], W["seed"] + rank, dev)
        hA = flatA.cpu().pin_memory()
        hX = torch.empty(hA.numel(), dtype=torch.float64).pin_memory()
        dA = torch.empty(hA.numel(), dtype=torch.float32, device=dev)
        dX = torch.empty(hA.numel(), dtype=torch.float64, device=dev)
        As = [wl.matrix_view(dA, int(n), int(o)) for n, o in zip(sizes, offsets)]
        Xs = [wl.matrix_view(dX, int(n), int(o)) for n, o in zip(sizes, offsets)]

        def one():
            with torch.cuda.stream(stream):
                dA.copy_(hA, non_blocking=True)
                r = gj.invert_mixed_batched(As, Xs, x0_slices=args.x0_slices, corr_slices=4, tol=1e-12,
                                            max_iter=10, workers=args.workers, stream=stream)
                if r["status"] != 0:
                    raise RuntimeError(gj.status_string(r["status"]))
                hX.copy_(dX, non_blocking=True)
            stream.synchronize()
    else:
        n = W["n"]
        A = wl.gaussian(n, W["seed"] + rank, shift=W["shift"] * n)
        hA = torch.from_numpy(A).pin_memory()
        hX = torch.empty_like(hA).pin_memory()
        sgn, lg2 = ctypes.c_int(0), ctypes.c_double(0.0)
        opts = gj._Opts()
        opts.stream = stream.cuda_stream

        def one():
            stc = L.gj_invert_ex(ctypes.byref(opts), n, hA.data_ptr(), n, hX.data_ptr(), W["pivot"],
                                 ctypes.byref(sgn), ctypes.byref(lg2))
            if stc != 0:
                raise RuntimeError(gj.status_string(stc))

    one()
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    for _ in range(steps):
        one()
    torch.cuda.synchronize(dev)
    dt = time.perf_counter() - t0
    if args.workload == "batch200k":
        val = units_step * steps / dt
        unit = "matrices/s"
    else:
        val = flops_step * steps / dt / 1e9
        unit = "GFLOP/s"
    return {"value": val, "unit": unit, "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
            "steps": steps, "_seconds": dt / steps}


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["gj", "reference"], default="gj")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="inv8192")
    ap.add_argument("--update", choices=["auto", "dfma", "ozaki"], default="auto")
    ap.add_argument("--slices", type=int, default=0, help="digit slices of the tensor-core update (0 = 7)")
    ap.add_argument("--panel", type=int, default=0, help="cluster panel width of the blocked path (0 = library choice)")
    ap.add_argument("--update-sms", type=int, default=0,
                    help="SMs of the wide update under look-ahead (0 = library choice)")
    ap.add_argument("--x0-slices", type=int, default=None,
                    help="digit slices of the mixed path's first inverse (default: 3 for mixed16384, the "
                         "reduced-precision start (7 measured faster there at kappa 1e6: 0.73 s against 1.34 s); "
                         "7 for mixedbatch4096, the fastest measured there)")
    ap.add_argument("--workers", type=int, default=16, help="mixedbatch4096: host workers (= streams)")
    ap.add_argument("--compare-fma", action="store_true", help="mixed workload: also time the FP64-FMA update GJ")
    ap.add_argument("--traffic", type=float, default=None,
                    help="DRAM bytes per launch of the dominant kernel from an ncu capture")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--no-e2e", action="store_true", help="skip the end-to-end (host buffer) leg")
    ap.add_argument("--tune-cache", default=None,
                    help="text file for the batched plan's autotuner choices (reused when present)")
    ap.add_argument("--count", type=int, default=0,
                    help="matrices in the batched workload (default: the workload's own); for profiling runs")
    ap.add_argument("--n", type=int, default=0,
                    help="order of the single-matrix workload (default: the workload's own); for profiling runs")
    ap.add_argument("--headline-only", action="store_true",
                    help="measure only the selected workload (the default 8192 run also measures the other "
                         "workloads and reports them under config.configs)")
    args = ap.parse_args()
    if args.x0_slices is None:
        args.x0_slices = 7 if args.workload == "mixedbatch4096" else 3
    if args.warmup < 3 and args.impl == "gj":
        print("warning: fewer than 3 warm-up steps", file=sys.stderr)
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
