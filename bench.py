#!/usr/bin/env python
"""Benchmark of the dynamic-SENSE ADMM reconstruction on GB300.

Workload (one step): a full reconstruction of the cardiac-sized problem,
256 x 256 pixels, 32 frames, 12 coils, variable-density ky-t mask at R=8,
temporal-TV analysis prior (Algorithm 2), lambda=0.005, mu=0.1, rho=0.5,
100 ADMM iterations with the objective J(k) evaluated every iteration:
H'y prologue + 100 iterations + image output, inputs resident in HBM.
Metric: ADMM iterations per second (whole job over all ranks).

Extra keys on the JSON line:
  roofline      the column-inverse kernel (x = A r with the ||y-Hx||^2
                epilogue; it streams every packed inverse once per iteration)
                against the measured HBM copy bandwidth
  e2e           same metric through recon_solve_host with pinned host
                buffers: k-space H2D and image D2H inside the timed region
  cpu_baseline  the FP64 oracle on a bounded sample (a subset of columns,
                single-threaded), scaled to the full workload
  variants      the synthesis prior (Algorithm 1: temporal DFT, and the
                undecimated temporal Haar frame with 2 levels), lambda=0.02,
                and Algorithm 2 with spatio-temporal differences (w = 1) and a
                5-step CG m-update
  batched       64 uneven slices in one batched solve (graph replay)
  precision     384x384x48 frames x16 coils, R=6: FP32 / FP16 / BF16 storage
                (inverses and hybrid coil data; 16-bit k-space for the 16-bit
                runs), iters/s and the inverse kernel's HBM fraction each
  library_comparison  the same TV iteration written with stock PyTorch ops
                (cuFFT for the objective, cuBLAS batched matmul with dense
                per-column inverses from torch.linalg.inv), timed only
  grad          differentiable unrolled Algorithm 2: forward and backward
                (dL/dy, dL/dlambda, dL/dmu) of 4 slices 192x192x24x8,
                20 iterations, checkpoints every 5

Run:  python bench.py [--gpus N --steps K --warmup W] [--impl reference]
For N>1 (torchrun) each rank solves its own slice (weak scaling, no
collective on the data path).
"""

from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = dict(name="cardiac", Nx=256, Ny=256, Nt=32, Nc=12, R=8, lam=0.005, mu=0.1, rho=0.5, iters=100)
METRIC = "ADMM iters/s at 256x256x32 frames x12 coils"
UNIT = "iters/s"
FALLBACK_HBM_GBS = 6800.0
KERNEL_SRC = os.path.join(ROOT, "paper_1203_4587_gb300", "csrc", "iter_kernels.cu")
KERNEL_FILES = ("iter_kernels.cu", "persist_kernels.cu", "colinv.cuh", "common.cuh", "kernels.h", "fft.cuh")
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "col_inverse_traffic.json")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--prior", default="tv", choices=["tv", "dft", "stv"],
                    help="stv: spatio-temporal differences (w = 1), 5 CG steps per iteration")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-variants", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--storage", default="fp32", choices=["fp32", "fp16", "bf16"])
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--batched-slices", type=int, default=64)
    ap.add_argument("--no-grad", action="store_true")
    ap.add_argument("--no-precision", action="store_true")
    ap.add_argument("--no-comparison", action="store_true")
    ap.add_argument("--shard", default="slices", choices=["slices", "columns"],
                    help="slices: each rank solves its own slice (weak scaling); columns: the ranks split one "
                         "problem's image columns, each a slab plan over the whole k-space (strong scaling)")
    ap.add_argument("--persistent", action="store_true",
                    help="temporal-TV solves as one persistent launch (opts.persistent)")
    ap.add_argument("--detail", default=None,
                    help="also write the full record (notes, tunings, every timing) as JSON to this path")
    ap.add_argument("--grad-only", action="store_true",
                    help="only the differentiable-form measurement (one JSON line with its numbers)")
    ap.add_argument("--precision-only", action="store_true",
                    help="only the precision-form measurement (one JSON line with its numbers); --steps sets its "
                         "timed solves")
    ap.add_argument("--precision-frames", type=int, default=None, help="frames of the precision workload (48)")
    ap.add_argument("--precision-iters", type=int, default=None, help="iterations of the precision workload (100)")
    ap.add_argument("--precision-storage", default="fp32,fp16,bf16", help="comma-separated storages to measure")
    ap.add_argument("--batched-only", action="store_true",
                    help="only the batched-form measurement (one JSON line with its numbers); --steps "
                         "sets its timed batches")
    return ap.parse_args()


def finite_json(v):
    """The line with every non-finite float replaced by null (strict JSON has no NaN)."""
    if isinstance(v, float):
        return v if math.isfinite(v) else None
    if isinstance(v, dict):
        return {k: finite_json(x) for k, x in v.items()}
    if isinstance(v, (list, tuple)):
        return [finite_json(x) for x in v]
    return v


def sig(v, n=4):
    """v rounded to n significant digits (ints and non-numbers unchanged)."""
    if isinstance(v, float) and math.isfinite(v) and v != 0.0:
        return round(v, max(0, n - 1 - int(math.floor(math.log10(abs(v))))))
    return v


def compact_forms(line):
    """The forms' headline numbers in a few hundred characters.  The printed
    JSON line ends with this object, so a reader that keeps only the tail of
    the output still sees every form's measurement."""
    out = {}
    if "variants" in line:
        out["variants_iters_s"] = {k: sig(v) for k, v in line["variants"].items()}
    if "stv_step" in line:
        st = line["stv_step"]
        out["stv_step"] = {"ms": sig(st["ms_per_iter"]), "frac": sig(st["frac_hbm"], 3)}
    b = line.get("batched")
    if b:
        out["batched"] = ({"error": b["error"][:120]} if "error" in b else
                          {"recons_s": sig(b["value"]), "ms": sig(b["ms_per_batch"]),
                           "frac": sig(b["hbm_gbs_inverse_stream"] * 1e9 / b["peak_bps"], 3),
                           "recons_s_with_plan": sig(b["recons_per_s_with_plan"], 3),
                           "plan_s": sig(b["plan_s_total"], 3), "slices": b["slices"],
                           "iters": b["iters_per_slice"]})
    pr = line.get("precision")
    if pr:
        if "error" in pr:
            out["precision"] = {"error": pr["error"][:120]}
        else:
            out["precision"] = {k: {"iters_s": sig(v["iters_per_s"]), "inv_frac": sig(v["inverse_frac"], 3),
                                    "inv_share": sig(v["inverse_share"], 3)}
                                for k, v in pr.items() if isinstance(v, dict)}
    g = line.get("grad")
    if g:
        out["grad"] = ({"error": g["error"][:120]} if "error" in g else
                       {"fwd_ms": sig(g["forward_ms"]), "bwd_ms": sig(g["backward_ms"]),
                        "bwd_over_fwd": sig(g["backward_over_forward"], 3), "fwd_frac": sig(g["forward_frac"], 3),
                        "bwd_frac": sig(g["backward_frac"], 3)})
    lc = line.get("library_comparison")
    if lc:
        out["library_iters_s"] = sig(lc["iters_per_s"]) if "iters_per_s" in lc else lc.get("error", "")[:120]
    ca = line.get("cpu_baseline_all_cores")
    if ca and "value" in ca:
        out["cpu_all_cores"] = {"value": sig(ca["value"]), "cores": ca["cores"]}
    return out


def compact_line(line):
    """The JSON line bench.py prints: the contract's keys, then the forms."""
    keys = ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
            "vs_baseline", "dtype", "data", "gpu_launches", "config", "roofline", "cpu_baseline", "clocks", "e2e",
            "plan_s", "set_mu_s", "check")
    out = {k: line[k] for k in keys if k in line}
    for k in ("value", "ms_per_step", "plan_s", "set_mu_s"):
        if k in out:
            out[k] = sig(out[k], 6)
    if "e2e" in out:
        out["e2e"] = dict(out["e2e"], value=sig(out["e2e"]["value"], 6))
    if "check" in out:
        out["check"] = {k: sig(v, 6) for k, v in out["check"].items()}
    rf = out.get("roofline")
    if rf:
        out["roofline"] = {k: (sig(v) if k != "traffic" else v) for k, v in rf.items()}
    forms = compact_forms(line)
    if forms:
        out["forms"] = forms
    return out


def reduce_max(x, dist, device):
    """The largest of every rank's x (the whole job is as slow as its slowest rank)."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def weak_value(world, steps, iters_per_step, ms):
    """Whole-job iterations/s: every rank runs `steps` solves of its own slice."""
    return world * steps * iters_per_step / (ms / 1e3)


def column_shard(Nx, world, rank):
    """The image columns i0 .. i0 + W - 1 that rank `rank` of `world` solves
    when one problem is split along the horizontal axis: contiguous, sizes
    differing by at most one.  Every step of the iteration separates along
    that axis (Section IV-C, Section V), so the ranks need no exchange on the
    data path; each holds the whole k-space (its rows are broadcast once)."""
    base, extra = divmod(Nx, world)
    i0 = rank * base + min(rank, extra)
    return i0, base + (1 if rank < extra else 0)


def strong_value(steps, iters_per_step, ms):
    """Whole-job iterations/s when all ranks together solve one problem per step."""
    return steps * iters_per_step / (ms / 1e3)


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def kernel_hash():
    """Hash of the inverse kernel's sources (its file and the headers it uses):
    DRAM traffic taken from a profile of other sources is not reported."""
    h = hashlib.sha256()
    d = os.path.dirname(KERNEL_SRC)
    for f in KERNEL_FILES:
        with open(os.path.join(d, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def hbm_peak():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle samples during the timed region."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.file = None

    def start(self):
        try:
            self.file = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.file, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.file.flush()
        self.file.seek(0)
        rows = [r.split(",") for r in self.file.read().strip().splitlines() if r.strip()]
        os.unlink(self.file.name)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[0]))
                mx.append(float(r[1]))
                for n, v in zip(names, r[4:8]):
                    if v.strip().lower() in ("active", "1"):
                        reasons.add(n)
            except (ValueError, IndexError):
                continue
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------------------
# CPU side: the FP64 oracle timed on a bounded sample (subprocess, 1 thread)
# ---------------------------------------------------------------------------
ORACLE_SNIPPET = r"""
import json, sys, time
import numpy as np
sys.path.insert(0, {root!r})
import oracle, synthdata
w = json.loads({w!r})
case = synthdata.make_case(w["name"], seed=w.get("seed"))
ncols, budget, prior, col0 = {ncols}, {budget}, {prior!r}, {col0}
t0 = time.perf_counter()
b = oracle.adjoint_op(case.kspace, case.sens, case.mask)
yhat = oracle.hybrid_data(case.kspace, case.mask)
t_pro = time.perf_counter() - t0
cols = (col0 + np.arange(ncols)) % w["Nx"]
P = oracle.Problem(case.kspace, case.sens, case.mask, case.mu, cols)
# size the sample from a 2-iteration probe so that one solve takes about `budget` seconds
t0 = time.perf_counter()
P.solve(prior, case.lam, case.mu, case.rho, 2)
probe = (time.perf_counter() - t0) / 2
n = int(max(2, min(w["iters"], budget / max(probe, 1e-9))))
t0 = time.perf_counter()
_, info = P.solve(prior, case.lam, case.mu, case.rho, n)
el = time.perf_counter() - t0
per_iter_full = el / n * (w["Nx"] / ncols)
solve_s = t_pro + w["iters"] * per_iter_full
print(json.dumps(dict(iters_per_s=w["iters"] / solve_s, prologue_s=t_pro, per_iter_full_s=per_iter_full,
                      sample_iters=n, ncols=ncols, sample_s=el)))
"""


def oracle_sample(prior, ncols=2, budget=10.0, seed=None):
    w = dict(WORKLOAD)
    if seed is not None:
        w["seed"] = seed
    code = ORACLE_SNIPPET.format(root=ROOT, w=json.dumps(w), ncols=ncols, budget=budget, prior=prior, col0=0)
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1",
               CUDA_VISIBLE_DEVICES="")
    t0 = time.perf_counter()
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env)
    if r.returncode != 0:
        raise RuntimeError("oracle sample failed: " + r.stderr[-2000:])
    out = json.loads(r.stdout.strip().splitlines()[-1])
    out["wall_s"] = time.perf_counter() - t0
    return out


def oracle_sample_all_cores(prior, ncols=2, budget=10.0):
    """One single-threaded oracle process per host core, each on its own columns,
    run together: columns are independent, so the all-core rate is the per-column
    rate (measured under full contention) times the core count."""
    procs = max(1, os.cpu_count() or 1)
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1",
               CUDA_VISIBLE_DEVICES="")
    t0 = time.perf_counter()
    ps = []
    for k in range(procs):
        code = ORACLE_SNIPPET.format(root=ROOT, w=json.dumps(WORKLOAD), ncols=ncols, budget=budget, prior=prior,
                                     col0=k * ncols)
        ps.append(subprocess.Popen([sys.executable, "-c", code], stdout=subprocess.PIPE, stderr=subprocess.PIPE,
                                   text=True, env=env))
    outs = []
    for p in ps:
        o, e = p.communicate()
        if p.returncode != 0:
            raise RuntimeError("oracle sample failed: " + e[-2000:])
        outs.append(json.loads(o.strip().splitlines()[-1]))
    per_iter = statistics.mean(o["per_iter_full_s"] for o in outs) / procs
    pro = statistics.mean(o["prologue_s"] for o in outs)
    value = WORKLOAD["iters"] / (pro + WORKLOAD["iters"] * per_iter)
    return {"value": value, "unit": UNIT, "cores": procs, "kind": "oracle",
            "sample": (f"FP64 NumPy oracle, {prior} prior, {procs} single-threaded processes at once, each on "
                       f"{ncols} own columns; per-iteration time = mean per-process time scaled by Nx/{ncols}, "
                       f"divided by {procs}; plus the H'y prologue ({pro:.2f} s, one process)"),
            "wall_s": time.perf_counter() - t0}


def cpu_baseline_obj(res, prior):
    return {"value": res["iters_per_s"], "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": (f"FP64 oracle, 1 thread: {res['sample_iters']} iters on {res['ncols']}/{WORKLOAD['Nx']} "
                       f"columns x Nx/{res['ncols']}, + full H'y ({res['prologue_s']:.2f} s); plan excluded")}


def config_obj(prior, storage):
    w = WORKLOAD
    return {"workload": (f"cardiac {w['Nx']}x{w['Ny']}x{w['Nt']}fr x{w['Nc']}coils R={w['R']} {prior.upper()} "
                         f"lambda={w['lam']} mu={w['mu']} rho={w['rho']}, {w['iters']} iters/solve, J every iter"),
            "prior": prior, "iters_per_step": w["iters"], "storage": storage, "parallelism": "replicas",
            "l2": "inputs > L2: 2.16 GB of inverses per iteration"}


def make_batched_inputs(nslices, seed=64):
    """The batched workload's slices (uneven sizes), generated on host threads."""
    import concurrent.futures as cf

    import numpy as np

    import synthdata
    shapes = synthdata.batched_shapes(nslices, seed)

    def one(sh):
        c = synthdata.make_case("batched", **sh)
        return c.kspace.astype(np.complex64), c.sens.astype(np.complex64), c.mask.astype(np.uint8)

    with cf.ThreadPoolExecutor(max_workers=min(16, os.cpu_count() or 4)) as ex:
        return shapes, list(ex.map(one, shapes))


def measure_batched(nslices, storage, steps=3, persistent=False):
    """64 uneven slices, 80 iterations each, one launch per step, graph replay."""
    import torch

    from paper_1203_4587_gb300 import Batch, Plan
    t0 = time.perf_counter()
    shapes, data = make_batched_inputs(nslices)
    gen_s = time.perf_counter() - t0
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    plans, ks = [], []
    for sh, (k, s_, m) in zip(shapes, data):
        plans.append(Plan(m, torch.from_numpy(s_).cuda(), sh["lam"], sh["mu"], prior=sh["prior"], rho=sh["rho"],
                          max_iters=sh["iters"], storage=storage, persistent=1 if persistent else 0))
        ks.append(torch.from_numpy(k).cuda())
    torch.cuda.synchronize()
    plan_s = time.perf_counter() - t0
    batch = Batch(plans)
    t0 = time.perf_counter()
    tuning = batch.autotune().as_dict()
    tuning["tune_s"] = time.perf_counter() - t0
    outs = [p._img() for p in plans]
    stream = torch.cuda.current_stream()
    batch.solve(ks, outs)            # direct run + graph capture
    batch.solve(ks, outs)            # graph replay (warm)
    torch.cuda.synchronize()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(steps):
        batch.solve(ks, outs)
    b.record(stream)
    torch.cuda.synchronize()
    ms = a.elapsed_time(b) / steps
    infos = batch.info()
    iters = sum(i.iters for i in infos)
    esize = 8 if storage == "fp32" else 4
    # algorithmic bytes: the Hermitian triangle Ny(Ny+1)/2 of every column (i, t)
    A_bytes = sum(esize * sh["Nx"] * sh["Nt"] * sh["Ny"] * (sh["Ny"] + 1) // 2 for sh in shapes)
    A_stored = sum(p.inverse_bytes for p in plans)
    batch.close()
    for p in plans:
        p.close()
    return {"value": nslices / (ms / 1e3), "unit": "recons/s", "slices": nslices,
            "iters_per_slice": shapes[0]["iters"], "ms_per_batch": ms,
            "recons_per_s_with_plan": nslices / (ms / 1e3 + plan_s), "plan_s_total": plan_s,
            "input_gen_s": gen_s, "iters_done": iters, "inverse_bytes_total": A_bytes,
            "inverse_bytes_stored": A_stored, "tuning": tuning,
            "hbm_gbs_inverse_stream": A_bytes * shapes[0]["iters"] / (ms / 1e3) / 1e9,
            "peak_bps": hbm_peak()[0] * 1e9,
            "note": ("Nx, Ny in {128,160,192,256}, Nt in {16,24,32,40}, Nc in {8,12,16}, R in {4,6,8}, TV, "
                     "lambda=0.005, mu=0.1; all slices in one launch per step, the batched solve replayed "
                     "from a captured CUDA graph; plan (double-float inversion) reported separately")}


def measure_precision(steps=3, frames=None, iters=None, storages=("fp32", "fp16", "bf16")):
    """The precision workload with FP32, FP16 and BF16 storage, J(k) every iteration
    (frames / iters: a smaller case of the same shape, e.g. for a profile)."""
    import numpy as np
    import torch

    import synthdata
    from paper_1203_4587_gb300 import Plan
    from paper_1203_4587_gb300.binding import quantize_kspace
    over = {k: v for k, v in (("Nt", frames), ("iters", iters)) if v is not None}
    c = synthdata.make_case("precision", **over)
    sens = torch.from_numpy(c.sens.astype(np.complex64)).cuda()
    k = torch.from_numpy(c.kspace.astype(np.complex64)).cuda()
    mask = c.mask.astype(np.uint8)
    Nt, Ny, Nx = c.x_true.shape
    peak, peak_kind = hbm_peak()
    out = {"workload": f"384x384x{Nt} frames x16 coils, R=6, TV, lambda=0.005, mu=0.1, {c.iters} iterations, "
                       "J(k) every iteration (fused for FP32; explicit for 16-bit, on the tensor cores)",
           "peak_source": f"{peak_kind} hbm_gbs (copy)"}
    stream = torch.cuda.current_stream()
    for storage in storages:
        t0 = time.perf_counter()
        p = Plan(mask, sens, c.lam, c.mu, prior="tv", rho=c.rho, max_iters=c.iters, storage=storage, profile=1)
        torch.cuda.synchronize()
        plan_s = time.perf_counter() - t0
        tn = p.autotune()
        q = quantize_kspace(k, storage) if storage != "fp32" else None
        img = torch.empty((Nt, Ny, Nx), dtype=torch.complex64, device="cuda")

        def run():
            if q is None:
                p.solve(k, img, info=False)
            else:
                p.solve_quantized(q, img, info=False)
        for _ in range(2):
            run()
        torch.cuda.synchronize()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(steps):
            run()
        b.record(stream)
        torch.cuda.synchronize()
        ms = a.elapsed_time(b) / steps
        prof = p.profile()
        A_bytes = (8 if storage == "fp32" else 4) * Nx * Nt * Ny * (Ny + 1) // 2   # algorithmic
        col_ms = prof.inverse_ms / max(prof.inverse_passes, 1)   # per pass over every column
        bytes_launch = A_bytes + 3 * 8 * Nx * Ny * Nt
        out[storage] = {"iters_per_s": c.iters / (ms / 1e3), "ms_per_solve": ms, "plan_s": plan_s,
                        "inverse_bytes": A_bytes, "inverse_bytes_stored": p.inverse_bytes, "inverse_avg_ms": col_ms,
                        "inverse_gbs": bytes_launch / (col_ms / 1e3) / 1e9,
                        "inverse_frac": bytes_launch / (col_ms / 1e3) / 1e9 / peak,
                        "inverse_share": prof.inverse_ms / max(prof.solve_ms, 1e-9),
                        "tuning": {"col_stages": tn.col_stages, "temporal_tile_px": tn.temporal_tile_px,
                                   "objective_coils": tn.objective_coils}}
        p.close()
        del q
        torch.cuda.empty_cache()
    return out


def measure_library_comparison(case, iters=10):
    """Algorithm 2 with stock PyTorch CUDA ops on the cardiac workload: the
    objective through cuFFT (torch.fft), the inverse as a cuBLAS batched
    matrix-vector product with dense per-column inverses (torch.linalg.inv of
    mu I + C_t (.) K_i), the m-update as a dense (rho I + D'D)^{-1} product.
    Timed only: the comparison arm, not part of the library."""
    import numpy as np
    import torch
    dev = "cuda"
    w = WORKLOAD
    Nt, Ny, Nx, Nc = w["Nt"], w["Ny"], w["Nx"], w["Nc"]
    lam, mu, rho = w["lam"], w["mu"], w["rho"]
    t0 = time.perf_counter()
    sens = torch.from_numpy(case.sens.astype(np.complex64)).to(dev)           # [Nc, Ny, Nx]
    mask = torch.from_numpy(case.mask).to(dev)                                # [Nt, Ny]
    y = torch.from_numpy(case.kspace.astype(np.complex64)).to(dev) * mask[:, None, :, None]
    # per-column Gram blocks and inverses
    Kc = torch.einsum("cji,cki->ijk", sens.conj(), sens)                      # [Nx, Ny, Ny]
    P = mask.to(torch.complex64)
    Fv = torch.fft.fft(torch.eye(Ny, dtype=torch.complex64, device=dev), norm="ortho", dim=0)
    Ct = torch.einsum("aj,ta,ak->tjk", Fv.conj(), P, Fv)                       # F_v' P_t F_v  [Nt, Ny, Ny]
    A = torch.empty((Nt, Nx, Ny, Ny), dtype=torch.complex64, device=dev)
    eye = torch.eye(Ny, dtype=torch.complex64, device=dev)
    for t in range(Nt):
        A[t] = torch.linalg.inv(mu * eye + Ct[t][None] * Kc)
    D = torch.zeros((Nt - 1, Nt), dtype=torch.float32, device=dev)
    idx = torch.arange(Nt - 1, device=dev)
    D[idx, idx] = -1.0
    D[idx, idx + 1] = 1.0
    Minv = torch.linalg.inv(rho * torch.eye(Nt, device=dev) + D.T @ D).to(torch.complex64)
    torch.cuda.synchronize()
    setup_s = time.perf_counter() - t0

    def Hop(x):   # [Nt, Ny, Nx] -> [Nt, Nc, Ny, Nx]
        return torch.fft.fft2(sens[None] * x[:, None], norm="ortho") * mask[:, None, :, None]

    b = (sens.conj()[None] * torch.fft.ifft2(y, norm="ortho")).sum(1)        # H'y
    tau = lam * rho / (2 * mu)

    def step(st):
        x, m, d1, d2 = st
        a = m[1:] - m[:-1] + d1
        mag = a.abs()
        v = torch.where(mag > tau, a * (1 - tau / mag.clamp_min(1e-30)), torch.zeros_like(a))
        u = v - d1
        rhs = rho * (x + d2)
        rhs[:-1] -= u
        rhs[1:] += u
        mn = torch.tensordot(Minv, rhs, dims=([1], [0]))
        r = b + mu * (mn - d2)
        xn = torch.matmul(A, r.permute(0, 2, 1).unsqueeze(-1)).squeeze(-1).permute(0, 2, 1)
        d1 = d1 - v + (mn[1:] - mn[:-1])
        d2 = d2 - mn + xn
        J = torch.sum(torch.abs(y - Hop(xn)) ** 2) + lam * torch.sum(torch.abs(xn[1:] - xn[:-1]))
        return (xn, mn, d1, d2), J

    st = (b.clone(), b.clone(), torch.zeros((Nt - 1, Ny, Nx), dtype=torch.complex64, device=dev), torch.zeros_like(b))
    for _ in range(2):
        st, J = step(st)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(iters):
        st, J = step(st)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / iters
    out = {"iters_per_s": 1e3 / ms, "ms_per_iter": ms, "setup_s": setup_s,
           "dense_inverse_bytes": int(A.numel() * 8),
           "note": ("cardiac TV iteration in stock PyTorch: dense per-column inverses (cuBLAS batched matvec), "
                    "dense m-update, J through cuFFT every iteration; timed only")}
    del A, Kc, Ct
    torch.cuda.empty_cache()
    return out


def measure_grad(storage, steps=5):
    """Forward and backward of unrolled Algorithm 2 over a batch of 4 slices."""
    import numpy as np
    import torch

    import synthdata
    from paper_1203_4587_gb300 import Grad, Plan
    cases = [synthdata.make_case("diff", seed=q) for q in range(4)]
    iters = cases[0].iters
    plans = [Plan(c.mask.astype(np.uint8), torch.from_numpy(c.sens.astype(np.complex64)).cuda(), c.lam, c.mu,
                  prior="tv", rho=c.rho, max_iters=iters, objective=0, storage=storage) for c in cases]
    ks = [torch.from_numpy(c.kspace.astype(np.complex64)).cuda() for c in cases]
    xt = [torch.from_numpy(c.x_true.astype(np.complex64)).cuda() for c in cases]
    every = 5
    g = Grad(plans, checkpoint_every=every)
    stream = torch.cuda.current_stream()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    fwd, bwd = [], []
    for s in range(2 + steps):
        ev[0].record(stream)
        xs = g.forward(ks)
        ev[1].record(stream)
        gi = [2.0 * (x - t) for x, t in zip(xs, xt)]
        ev[2].record(stream)
        g.backward(gi)      # fills dL/dlambda, dL/dmu: synchronises
        ev[3].record(stream)
        torch.cuda.synchronize()
        if s >= 2:
            fwd.append(ev[0].elapsed_time(ev[1]))
            bwd.append(ev[2].elapsed_time(ev[3]))
    g.close()
    for p in plans:
        p.close()
    f, b = statistics.median(fwd), statistics.median(bwd)
    # algorithmic bytes: the packed inverses (the Hermitian triangle of every
    # column) streamed once per inverse launch: K forward steps; K reverse
    # steps plus K - K/every recomputed steps backward
    Nt, Ny, Nx = cases[0].x_true.shape
    a_bytes = len(cases) * (8 if storage == "fp32" else 4) * Nx * Nt * Ny * (Ny + 1) // 2
    n_fwd, n_bwd = iters, iters + (iters - iters // every)
    peak, _ = hbm_peak()
    fgbs = n_fwd * a_bytes / (f / 1e3) / 1e9
    bgbs = n_bwd * a_bytes / (b / 1e3) / 1e9
    return {"forward_ms": f, "backward_ms": b, "backward_over_forward": b / f, "slices": 4,
            "iters": iters, "checkpoint_every": every, "inverse_streams_forward": n_fwd,
            "inverse_streams_backward": n_bwd, "inverse_bytes_per_stream": a_bytes,
            "forward_gbs": fgbs, "backward_gbs": bgbs, "forward_frac": fgbs / peak, "backward_frac": bgbs / peak,
            "note": ("192x192x24 frames x8 coils, R=8, TV, lambda=0.005, mu=0.1, rho=0.5; forward = H'y + 20 "
                     "steps keeping checkpoints; backward = segment recomputation + reverse steps + dL/dy = H b_bar "
                     "+ the lambda/mu gradients (host read)")}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    if args.prior == "stv":
        print(json.dumps({"impl": "reference", "unavailable": "the oracle of the spatio-temporal prior couples "
                          "columns, so it has no bounded column sample at this size"}), flush=True)
        return 0
    vals = []
    t_start = time.perf_counter()
    last = None
    for s in range(args.warmup + args.steps):
        res = oracle_sample(args.prior, ncols=1, budget=2.0)
        if s >= args.warmup:
            vals.append(res["iters_per_s"])
            last = res
    value = statistics.mean(vals)
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * WORKLOAD["iters"] / value, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config_obj(args.prior, "fp64"), "impl": "reference",
            "cpu_baseline": cpu_baseline_obj(last, args.prior) | {"value": value},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "wall_s": time.perf_counter() - t_start}
    print(json.dumps(finite_json(line)), flush=True)
    return 0


def run_native(args):
    import numpy as np
    import torch

    import synthdata
    from paper_1203_4587_gb300 import Plan, binding

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    w = WORKLOAD
    by_columns = args.shard == "columns" and world > 1 and args.prior != "stv"
    # slices: each rank its own slice; columns: one problem, the ranks' slabs
    case = synthdata.make_case(w["name"], seed=2 if by_columns else 2 + rank)
    kspace = torch.from_numpy(case.kspace.astype(np.complex64)).cuda()
    sens = torch.from_numpy(case.sens.astype(np.complex64)).cuda()
    mask = case.mask.astype(np.uint8)
    slab = column_shard(w["Nx"], world, rank) if by_columns else None
    t0 = time.perf_counter()
    plan = Plan(mask, sens, w["lam"], w["mu"], prior=args.prior, rho=w["rho"], max_iters=w["iters"],
                profile=1, storage=args.storage, spatial_weight=1.0, cg_steps=5, slab=slab,
                persistent=1 if args.persistent else 0)
    plan_s = time.perf_counter() - t0
    t0 = time.perf_counter()
    plan.set_mu(w["mu"])                     # mu-reuse path: the inverses again, no allocation or upload
    set_mu_s = time.perf_counter() - t0
    t0 = time.perf_counter()
    tuning = plan.autotune().as_dict()       # launch shapes, picked by timing them
    tuning["tune_s"] = time.perf_counter() - t0
    out = torch.empty((w["Nt"], w["Ny"], w["Nx"]), dtype=torch.complex64, device="cuda")
    stream = torch.cuda.current_stream()
    # the timed solves run without per-kernel events (they would serialise the
    # launches); one profiled solve afterwards gives the roofline
    plan.set_profile(False)
    for _ in range(max(args.warmup, 3)):
        plan.solve(kspace, out, info=False)
    barrier()
    sampler = ClockSampler(local) if rank == 0 else None
    if sampler:
        sampler.start()
        time.sleep(0.3)
    launches0 = binding.kernel_launches()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    barrier()
    e0.record(stream)
    for _ in range(args.steps):
        plan.solve(kspace, out, info=False)
    e1.record(stream)
    barrier()
    clocks = sampler.stop() if sampler else None
    launches = binding.kernel_launches() - launches0
    ms = reduce_max(e0.elapsed_time(e1), dist, "cuda")
    value = (strong_value(args.steps, w["iters"], ms) if by_columns else
             weak_value(world, args.steps, w["iters"], ms))
    plan.set_profile(True)
    plan.solve(kspace, out, info=False)
    prof = plan.profile()
    plan.set_profile(False)
    _, info = plan.solve(kspace, out, info=True)

    # roofline of the column-inverse kernel: algorithmic bytes per launch (a
    # slab plan streams its own columns only)
    Ny, Nt, Nc = w["Ny"], w["Nt"], w["Nc"]
    Nx = slab[1] if slab else w["Nx"]
    esize = 8 if args.storage == "fp32" else 4
    total_rows = int(case.mask.sum())
    bytes_A = esize * Nx * Nt * Ny * (Ny + 1) // 2
    # packed inverses + read two input fields (H'y and the state) + write x
    # per pass over every column; the persistent kernel makes K passes per launch
    bytes_pass = bytes_A + 3 * 8 * Nx * Ny * Nt
    passes = max(prof.inverse_passes, 1) // max(prof.inverse_launches, 1)
    bytes_launch = bytes_pass * passes
    avg_s = prof.inverse_ms / max(prof.inverse_launches, 1) / 1e3
    achieved = bytes_launch / avg_s / 1e9
    peak, peak_kind = hbm_peak()
    kname = "k_persist_tv" if prof.persistent else "k_col_inverse"
    traffic = None
    try:
        with open(TRAFFIC_FILE) as f:
            tr = json.load(f)
        if (tr.get("kernel_hash") == kernel_hash() and tr.get("storage", "fp32") == args.storage
                and tr.get("kernel", "").startswith(kname)):
            traffic = tr.get("traffic_bytes_per_launch")
    except Exception:
        pass
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": traffic, "peak_source": f"{peak_kind} copy",
                "kernel": kname, "bytes_per_launch": bytes_launch, "avg_launch_ms": avg_s * 1e3,
                "passes_per_launch": passes, "ms_per_pass": avg_s * 1e3 / passes,
                "share_of_step": prof.inverse_ms / max(prof.solve_ms, 1e-9),
                "temporal_avg_ms": prof.temporal_ms / max(prof.temporal_launches, 1)}

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "strong" if by_columns else "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": dict(config_obj(args.prior, args.storage),
                           parallelism="columns (one slab plan per rank)" if by_columns else "replicas"),
            "roofline": roofline, "clocks": clocks,
            "gpu_launches": launches, "plan_s": plan_s, "set_mu_s": set_mu_s, "tuning": tuning,
            "check": {"iters": info.iters, "J0": info.J0, "J": info.J, "primal_res": info.primal_res,
                      "dual_res": info.dual_res}}

    # end to end through the public API with host buffers
    if not args.no_e2e:
        kh = torch.from_numpy(case.kspace.astype(np.complex64)).pin_memory()
        ih = torch.empty((Nt, Ny, w["Nx"]), dtype=torch.complex64).pin_memory()
        plan.solve_host(kh, ih)
        n_e2e = max(3, args.steps // 2)
        barrier()
        t0 = time.perf_counter()
        for _ in range(n_e2e):
            plan.solve_host(kh, ih)
        el = reduce_max(time.perf_counter() - t0, dist, "cuda")
        e2e_value = (strong_value(n_e2e, w["iters"], el * 1e3) if by_columns else
                     weak_value(world, n_e2e, w["iters"], el * 1e3))
        # pinned k-space is read in place by the prologue: only the sampled rows cross to the device
        h2d = int(case.mask.sum()) * w["Nc"] * w["Nx"] * 8
        line["e2e"] = {"value": e2e_value, "unit": UNIT,
                       "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": int(ih.numel() * 8),
                       "step": "recon_solve_host: sampled k-space rows read from pinned host memory, solve, image D2H"}

    if not args.no_variants and rank == 0:
        var = {}
        for name, prior, lam in (("dft", "dft", 0.005), ("tv_l0.02", "tv", 0.02),
                                 ("dft_l0.02", "dft", 0.02), ("haar2", "haar", 0.005),
                                 ("stv_cg5", "stv", 0.005)):
            if prior == args.prior and lam == w["lam"]:
                continue
            p2 = Plan(mask, sens, lam, w["mu"], prior=prior, rho=w["rho"], max_iters=w["iters"],
                      storage=args.storage, frame_levels=2, spatial_weight=1.0, cg_steps=5,
                      profile=1 if prior == "stv" else 0)
            p2.autotune()
            for _ in range(2):
                p2.solve(kspace, out, info=False)
            torch.cuda.synchronize()
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            for _ in range(3):
                p2.solve(kspace, out, info=False)
            b.record(stream)
            torch.cuda.synchronize()
            var[name] = 3 * w["iters"] / (a.elapsed_time(b) / 1e3)
            if prior == "stv":
                # the spatio-temporal step (r, 5 CG steps, finish) against HBM: per iteration it
                # moves 67 fields of N complex64 at minimum (rhs 7, each CG step 10, finish 10)
                pr = p2.profile()
                step_ms = pr.temporal_ms / max(pr.temporal_launches, 1)
                nbytes = 67 * 8 * w["Nx"] * w["Ny"] * w["Nt"]
                gbs = nbytes / (step_ms / 1e3) / 1e9
                peak, _ = hbm_peak()
                line["stv_step"] = {"ms_per_iter": step_ms, "algorithmic_bytes": nbytes, "gbs": gbs,
                                    "frac_hbm": gbs / peak, "inverse_ms_per_iter":
                                    pr.inverse_ms / max(pr.inverse_launches, 1)}
            p2.close()
        line["variants"] = var

    if not args.no_batched and rank == 0:
        plan.close()
        torch.cuda.empty_cache()
        try:
            line["batched"] = measure_batched(args.batched_slices, args.storage, persistent=args.persistent)
        except Exception as e:  # report, never fake
            line["batched"] = {"error": str(e)[:300]}

    if not args.no_comparison and rank == 0:
        torch.cuda.empty_cache()
        try:
            line["library_comparison"] = measure_library_comparison(case)
        except Exception as e:  # report, never fake
            line["library_comparison"] = {"error": str(e)[:300]}

    if not args.no_precision and rank == 0:
        torch.cuda.empty_cache()
        try:
            line["precision"] = measure_precision()
        except Exception as e:  # report, never fake
            line["precision"] = {"error": str(e)[:300]}

    if not args.no_grad and rank == 0:
        torch.cuda.empty_cache()
        try:
            line["grad"] = measure_grad(args.storage)
        except Exception as e:  # report, never fake
            line["grad"] = {"error": str(e)[:300]}

    if rank == 0 and world == 1 and not args.no_cpu_baseline and args.prior == "stv":
        # the spatio-temporal prior couples columns: no column sample of the oracle
        line["cpu_baseline"] = {"error": "no bounded oracle sample for the spatio-temporal prior (couples columns)"}
    elif rank == 0 and world == 1 and not args.no_cpu_baseline:
        try:
            res = oracle_sample(args.prior, ncols=2, budget=10.0)
            line["cpu_baseline"] = cpu_baseline_obj(res, args.prior)
        except Exception as e:  # report, never fake
            line["cpu_baseline"] = {"error": str(e)[:300]}
        try:
            line["cpu_baseline_all_cores"] = oracle_sample_all_cores(args.prior, ncols=2, budget=6.0)
        except Exception as e:  # report, never fake
            line["cpu_baseline_all_cores"] = {"error": str(e)[:300]}
    if rank == 0:
        if args.detail:
            with open(args.detail, "w") as f:
                json.dump(finite_json(line), f, indent=1)
        print(json.dumps(finite_json(compact_line(line)), separators=(",", ":")), flush=True)
    plan.close()
    if dist is not None:
        dist.destroy_process_group()
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.grad_only:
        print(json.dumps({"grad": measure_grad(args.storage, steps=args.steps)}), flush=True)
        return 0
    if args.precision_only:
        pr = measure_precision(steps=args.steps, frames=args.precision_frames, iters=args.precision_iters,
                               storages=tuple(args.precision_storage.split(",")))
        print(json.dumps({"precision": finite_json(pr)}), flush=True)
        return 0
    if args.batched_only:
        b = measure_batched(args.batched_slices, args.storage, steps=args.steps, persistent=args.persistent)
        print(json.dumps({"batched": finite_json(b)}), flush=True)
        return 0
    return run_native(args)


if __name__ == "__main__":
    sys.exit(main())
