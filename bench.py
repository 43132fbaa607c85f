#!/usr/bin/env python
"""Benchmark of the supernodal factorization on one GB300 (per rank).

Workload: 3-D 7-point variable-coefficient diffusion on a 64^3 grid
(n = 262,144), node coefficients exp(g), g ~ N(0,1), 16 right-hand sides
~ U(-1,1), geometric nested-dissection ordering.  One step is the whole hot
path: assembly + numerical factorization + solve of the 16 right-hand sides to
backward error <= 1e-12 (with refinement when the factor is single
precision).  Each precision mode runs its own steps; the headline is the
fastest mode that reaches the target.

value = exact-pattern factorization flops / step time (GFlop/s), summed over
ranks (independent replicas: the factorization of one system does not shard).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "factorization GFlop/s & time-to-solve at 1e-12 backward error, FP64 vs mixed"
TARGET_BERR = 1e-12
GRID = (64, 64, 64)
NRHS = 16
SEED = 2
WORKLOAD = "diffusion3d_64^3_7pt_expN01_16rhs"
FP64_ALU_PEAK_GFLOPS = 152 * 2 * 2 * 2.07e9 / 1e9        # 2 DFMA / clk / SM
FP32_ALU_PEAK_GFLOPS = 152 * 128 * 2 * 2.07e9 / 1e9      # 128 FFMA / clk / SM
L2_FLUSH_BYTES = 256 << 20
# arithmetic of each factorization mode (the solve's residual and correction
# are FP64 in every mode)
DTYPES = {"fp64": "f64",
          "fp32": "3xtf32 updates (f32 accumulate), f64 diagonal blocks and refinement",
          "tf32": "tf32 updates (f32 accumulate), f64 diagonal blocks and refinement",
          "bf16": "bf16 updates (f32 accumulate), f64 diagonal blocks and refinement"}
NOMINAL_TF32_OVER_BF16 = 1.1 / 2.25                       # nominal dense tensor rates


def measured_peaks() -> dict:
    """HBM GB/s and bf16 TFLOP/s measured on this machine (generated file)."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return {"hbm_gbs": float(d["hbm_gbs"]), "bf16_tflops": float(d["bf16_tflops"]),
                "source": "of measured"}
    except (OSError, KeyError, ValueError):
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "source": "of fallback"}


# DRAM traffic per launch from one ncu capture of the committed kernels
# (dram__bytes_read.sum + dram__bytes_write.sum), with the algorithmic bytes of
# the same launch; profiles/ holds the captures and their commands.
NCU_TRAFFIC = {
    "diag": {"traffic": 132.6e3, "algorithmic_bytes": 2 * 64 * 64 * 4,
             "launch": "potrf_ldl_kernel<float,64>, one 64-wide panel, 48^3 diffusion (cold caches)",
             "source": "profiles/potrf_ldl_kernel_diffusion3d_48.md"},
    "update_tc": {"traffic": 22.6e6, "algorithmic_bytes": None,
                  "launch": "update_tc_persistent<0>, one low level (152 CTAs over its tiles), 48^3 diffusion",
                  "source": "profiles/update_tc_kernel_diffusion3d_48.md"},
}


def class_roofline(cls: str, st: dict, mode: str, peaks: dict) -> dict:
    """Roofline of one kernel class from its algorithmic work and device time."""
    ms = st["ms"]
    tr = NCU_TRAFFIC.get(cls) if mode != "fp64" else None
    out = {"kernel_class": cls, "launches": st["launches"], "device_ms": ms,
           "algorithmic_flops": st["flops"], "algorithmic_bytes": st["bytes"],
           "traffic": tr["traffic"] if tr else None}
    if tr:
        out["traffic_detail"] = tr
    if ms <= 0:
        return out
    if cls in ("assemble", "update_tc"):
        ach = st["bytes"] / (ms / 1e3) / 1e9
        out.update({"bound": "hbm", "achieved": ach, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                    "frac": ach / peaks["hbm_gbs"], "peak_source": peaks["source"]})
        if cls == "update_tc":
            tpeak = peaks["bf16_tflops"] * (1.0 if mode == "bf16" else NOMINAL_TF32_OVER_BF16)
            tach = st["flops"] / (ms / 1e3) / 1e12
            out["tensor"] = {"achieved_tflops": tach, "peak_tflops": tpeak, "frac": tach / tpeak,
                             "peak_source": ("measured bf16" if mode == "bf16" else
                                             "measured bf16 x nominal tf32/bf16 ratio (1.1/2.25)")}
        return out
    if cls == "queue" and mode != "fp64":
        # the task-queue launch of the upper levels: its flops are mostly tensor-core updates
        tpeak = peaks["bf16_tflops"] * (1.0 if mode == "bf16" else NOMINAL_TF32_OVER_BF16)
        tach = st["flops"] / (ms / 1e3) / 1e12
        out.update({"bound": "tensor", "achieved": tach, "peak": tpeak, "unit": "TFLOP/s",
                    "frac": tach / tpeak, "peak_source": peaks["source"]})
        return out
    fp64_arith = mode == "fp64" or cls in ("diag", "queue")
    peak = FP64_ALU_PEAK_GFLOPS if fp64_arith else FP32_ALU_PEAK_GFLOPS
    ach = st["flops"] / (ms / 1e3) / 1e9
    out.update({"bound": "alu", "achieved": ach, "peak": peak, "unit": "GFLOP/s",
                "frac": ach / peak,
                "peak_source": ("derived: 152 SMs x 2 DFMA/clk x 2 flop x 2.07 GHz" if fp64_arith
                                else "derived: 152 SMs x 128 FFMA/clk x 2 flop x 2.07 GHz")})
    return out


def solve_roofline(info: dict, nrhs: int, refine_iters: int, peaks: dict) -> dict:
    """Roofline of a refined solve: each forward + backward sweep pair reads
    the stored factor twice; each residual reads A (values, column indices,
    value map: 8 + 4 + 8 bytes per entry) and X, B, R (n x nrhs FP64).  One
    sweep pair and one residual per refinement step, plus the first solve
    and the final check.  HBM-bound: the bytes over the measured solve time."""
    pairs = 1 + refine_iters
    residuals = refine_iters + (1 if refine_iters > 0 else 0)
    byts = (pairs * 2.0 * info["factor_bytes"]
            + residuals * (20.0 * info["nnz_a"] + 3.0 * 8.0 * info["n"] * nrhs))
    ms = info["solve_ms"]
    out = {"kernel": "fwd_queue_kernel + bwd_queue_kernel (+ residual_kernel)", "bound": "hbm",
           "sweep_pairs": pairs, "algorithmic_bytes": byts, "device_ms": ms, "unit": "GB/s",
           "peak": peaks["hbm_gbs"], "peak_source": peaks["source"], "traffic": None}
    if ms > 0:
        out["achieved"] = byts / (ms / 1e3) / 1e9
        out["frac"] = out["achieved"] / peaks["hbm_gbs"]
    return out


def _args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="spx", choices=["spx", "reference"])
    ap.add_argument("--modes", default="fp64,fp32,tf32,bf16")
    ap.add_argument("--grid", default="64,64,64")
    ap.add_argument("--max-width", type=int, default=64,
                    help="split supernodes wider than this (panel width)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true", help="skip the host-buffer end-to-end pass")
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the batched-LU and differentiation workloads")
    return ap.parse_args()




# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,utilization.gpu,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self) -> dict:
        rows = []
        try:
            for line in open(self.path):
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        finally:
            try:
                os.unlink(self.path)
            except OSError:
                pass
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}

        def num(x):
            try:
                return float(x)
            except ValueError:
                return float("nan")
        busy = [r for r in rows if num(r[4]) >= 50] or rows
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(num(r[1]) for r in busy),
                "sm_max_mhz": max(num(r[2]) for r in rows),
                "power_w_max": max(num(r[3]) for r in rows),
                "reasons": reasons, "samples": len(rows), "samples_under_load": len(busy)}


# ---------------------------------------------------------------------------
# the oracle on the host cores (CPU baseline and reference arm)
# ---------------------------------------------------------------------------
def oracle_rate(grid, seconds_budget: float) -> dict:
    """Oracle factorization + 16-RHS solve on a sub-grid of the same workload."""
    import oracle
    from paper_1405_2636_gb300 import inputs

    A = inputs.diffusion_3d(*grid, SEED)
    B = inputs.rhs(A.shape[0], NRHS, SEED)
    perm = oracle.nd_grid(*grid)
    flops = None
    times = []
    t_end = time.perf_counter() + seconds_budget
    while True:
        t0 = time.perf_counter()
        F = oracle.cholesky(A, perm)
        oracle.solve(F, B)
        times.append(time.perf_counter() - t0)
        flops = oracle.flops(F.sym.counts, "llt")
        if time.perf_counter() > t_end:
            break
    t = statistics.median(times)
    return {"value": flops / t / 1e9, "unit": "GFlop/s", "cores": 1, "kind": "oracle",
            "sample": f"oracle left-looking FP64 Cholesky + 16-RHS solve of the same diffusion "
                      f"generator on a {grid[0]}x{grid[1]}x{grid[2]} sub-grid "
                      f"({flops / 1e9:.2f} GFlop), median of {len(times)} runs",
            "seconds": sum(times)}


def run_reference(args):
    from paper_1405_2636_gb300 import replicas
    _, rank, _ = replicas.env_ranks()
    if rank != 0:
        return
    import oracle
    from paper_1405_2636_gb300 import inputs

    oracle.build()
    grid = (24, 24, 24)
    A = inputs.diffusion_3d(*grid, SEED)
    B = inputs.rhs(A.shape[0], NRHS, SEED)
    perm = oracle.nd_grid(*grid)
    F = None
    for _ in range(args.warmup):
        F = oracle.cholesky(A, perm)
        oracle.solve(F, B)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        F = oracle.cholesky(A, perm)
        X = oracle.solve(F, B)
        times.append(time.perf_counter() - t0)
    flops = oracle.flops(F.sym.counts, "llt")
    berr = oracle.backward_error(A, X, B)
    ms = 1e3 * sum(times) / len(times)
    value = flops / (ms / 1e3) / 1e9
    line = {"metric": METRIC, "value": value, "unit": "GFlop/s", "impl": "reference",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "sample_grid": list(grid),
                       "note": "the oracle (plain single-threaded C, FP64) on a bounded "
                               "sub-grid of the same workload; one step = factorization "
                               "+ 16-RHS solve"},
            "backward_error": berr,
            "cpu_baseline": {"value": value, "unit": "GFlop/s", "cores": 1, "kind": "oracle",
                             "sample": f"{grid[0]}^3 sub-grid of the diffusion workload, "
                                       f"{flops / 1e9:.2f} GFlop per step"},
            "e2e": {"value": value, "unit": "GFlop/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# the other workloads: the batched LU and the differentiable solve
# ---------------------------------------------------------------------------
BATCH_TOL = 1e-10


def run_batched(torch, spx, inputs, steps: int, group, rank: int) -> dict:
    """4096 independent 2-D convection-diffusion systems (sides 12..80),
    static-pivot LU in FP32 with FP64 refinement to 1e-10, one persistent
    launch; the autotuner picks the launch configuration first.  With
    several ranks each takes a flop-balanced bin of the systems and the
    statistics are combined once at the end (max time, summed work)."""
    from paper_1405_2636_gb300 import replicas
    W = inputs.BATCHED_CD_4096
    mine = None
    if group.world > 1:
        work = [replicas.lu_work_estimate(k) for k in inputs.batched_sides(W["count"], W["seed"])]
        mine = replicas.shard_by_work(work, group.world)[rank]
    mats, sides, rhs = inputs.batched_convection_diffusion(W["count"], W["seed"], systems=mine)
    arrs = [inputs.csc_arrays(A) for A in mats]
    b = spx.batch_analyze([(cp, ri) for cp, ri, _ in arrs], grids=[(k, k, 1) for k in sides],
                          ordering=spx.SPX_ORDER_GRID)
    vals_h = np.concatenate([v for _, _, v in arrs])
    vals = torch.from_numpy(vals_h).cuda()
    bd = torch.from_numpy(rhs).cuda()
    ref = spx.default_refine(tol=BATCH_TOL, max_iter=20)
    t0 = time.perf_counter()
    b.tune(vals, bd, precision="fp32", refine=ref)
    tune_s = time.perf_counter() - t0
    out = {}
    i = b.info()
    for prec in ("fp32", "fp64"):
        b.run(vals, bd, precision=prec, refine=ref)
        ms = []
        for _ in range(max(3, steps)):
            _, st = b.run(vals, bd, precision=prec, refine=ref)
            ms.append(b.info()["run_ms"])
        i = b.info()
        si = b.system_info()
        local = {"ms": statistics.median(ms), "flops": i["flops"], "systems": i["nsys"],
                 "n_total": i["n_total"], "nnz_l_total": i["nnz_l_total"],
                 "all_converged": float(np.all(si["converged"] == 1)),
                 "max_backward_error": float(si["berr"].max()) if len(si["berr"]) else 0.0,
                 "max_refine_iters": float(si["iters"].max()) if len(si["iters"]) else 0.0,
                 "pivot_replacements": float(si["npivot_repl"].sum())}
        c = replicas.combine_batch_stats(group, local)
        out[prec] = {"ms": c["ms"], "status": st, "gflops": c["gflops"],
                     "all_converged": bool(c["all_converged"] == 1.0),
                     "max_backward_error": c["max_backward_error"],
                     "max_refine_iters": int(c["max_refine_iters"]),
                     "pivot_replacements": int(c["pivot_replacements"])}
        tot = c
    # end to end through the C ABI with host buffers (copies inside the call)
    Xh = np.empty(b.n_total)
    e2e = []
    for _ in range(3):
        t0 = time.perf_counter()
        b.run(vals_h, rhs, Xh, precision="fp32", refine=ref)
        e2e.append(1e3 * (time.perf_counter() - t0))
    e2e_ms = group.max(statistics.median(e2e))
    peaks = measured_peaks()
    ms32 = out["fp32"]["ms"]
    e = 4.0
    # algorithmic bytes: values and right-hand sides read, the factor written
    # once and read by each of the sweeps (1 + refinement steps, forward and
    # backward), A read by each residual, the solution written
    sweeps = 1 + out["fp32"]["max_refine_iters"]
    byts = group.sum(i["nnz_total"] * 8.0 * (2 + sweeps) + i["factor_elems"] * e * (1 + 2 * sweeps)
                     + i["n_total"] * 8.0 * 3)
    res = {"workload": W["name"], "systems": int(tot["systems"]), "ranks": group.world,
           "sharding": ("flop-balanced bins of whole systems, one per rank; statistics combined "
                        "once after the timed runs" if group.world > 1 else "one rank"),
           "pattern_classes": int(group.max(i["nclasses"])), "n_total": int(tot["n_total"]),
           "n_max": int(group.max(i["n_max"])),
           "nnz_l_total": int(tot["nnz_l_total"]),
           "flops_exact": tot["flops"], "target_backward_error": BATCH_TOL,
           "metric": "time to factorize and solve every system to backward error 1e-10 (one launch)",
           "fp32_refined": out["fp32"], "fp64": out["fp64"],
           "speedup_fp32_over_fp64": out["fp64"]["ms"] / ms32,
           "e2e_host_buffers_ms": e2e_ms,
           "config": {"ctas_per_sm": i["ctas_per_sm"], "leaf_width": i["leaf_width"],
                      "rows_per_thread": i["rows_per_thread"], "tuned_ms": i["tuned_ms"],
                      "tune_seconds": tune_s},
           "roofline": {"bound": "alu", "achieved": out["fp32"]["gflops"],
                        "peak": FP32_ALU_PEAK_GFLOPS, "unit": "GFLOP/s",
                        "frac": out["fp32"]["gflops"] / FP32_ALU_PEAK_GFLOPS,
                        "hbm_achieved_gbs": byts / (ms32 / 1e3) / 1e9,
                        "hbm_frac": byts / (ms32 / 1e3) / 1e9 / peaks["hbm_gbs"],
                        "algorithmic_bytes": byts, "peak_source": peaks["source"],
                        "kernel": "batch_lu_kernel<float> (persistent, one CTA per system)"}}
    b.free()
    return res


def run_differentiation(torch, spx, inputs, steps: int) -> dict:
    """loss = w^T x + log det A on the 48^3 diffusion problem, FP64 factor;
    forward (factorization, solve, log det) and backward (adjoint solve,
    gradient on A's pattern, selected inverse, log det gradient)."""
    from paper_1405_2636_gb300.autograd import SparseSPD

    nx = ny = nz = 48
    seed = 5
    cp, ri, M = inputs.diffusion_3d_coefficient_map(nx, ny, nz)
    n = nx * ny * nz
    g = np.random.default_rng([seed, 9])
    w = torch.from_numpy(g.standard_normal(n)).cuda()
    bvec = torch.from_numpy(g.standard_normal(n)).cuda()
    vals_h = M @ inputs.diffusion_3d_kappa(nx, ny, nz, seed)
    op = SparseSPD(cp, ri, ordering=spx.SPX_ORDER_GRID, grid=(nx, ny, nz), max_width=64)
    fwd, bwd, sel = [], [], []
    for it in range(max(3, steps) + 1):
        v = torch.from_numpy(vals_h).cuda().requires_grad_(True)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        loss = (w * op.solve(v, bvec)).sum() + op.logdet(v)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        torch.autograd.grad(loss, (v,))
        torch.cuda.synchronize()
        t2 = time.perf_counter()
        op.handle.factorize(v.detach(), "fp64")     # a fresh factor: time the selected inverse alone
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        op.handle.selected_inverse()
        e1.record()
        torch.cuda.synchronize()
        if it > 0:
            fwd.append(1e3 * (t1 - t0))
            bwd.append(1e3 * (t2 - t1))
            sel.append(e0.elapsed_time(e1))
    P = op.handle.panels()
    wdt = P["width"].astype(float)
    r = P["height"].astype(float) - wdt
    sel_flops = float(np.sum(2 * r * r * wdt + r * wdt * wdt + wdt ** 3 / 3 + r * wdt * wdt))
    info = op.handle.info()
    op.free()
    sel_ms = statistics.median(sel)
    return {"workload": "diffusion3d_48^3_7pt_expN01: loss = w^T x + log det A",
            "n": n, "nnz_l": info["nnz_l"], "factor_flops_exact": info["flops"],
            "forward_ms": statistics.median(fwd), "backward_ms": statistics.median(bwd),
            "factor_ms": info["factor_ms"],
            "selected_inverse_ms": sel_ms, "selected_inverse_flops": sel_flops,
            "roofline": {"bound": "alu", "achieved": sel_flops / (sel_ms / 1e3) / 1e9,
                         "peak": FP64_ALU_PEAK_GFLOPS, "unit": "GFLOP/s",
                         "frac": sel_flops / (sel_ms / 1e3) / 1e9 / FP64_ALU_PEAK_GFLOPS,
                         "kernel": "selinv_off_kernel + selinv_diag_kernel (FP64)",
                         "peak_source": "derived: 152 SMs x 2 DFMA/clk x 2 flop x 2.07 GHz"},
            "timing": "host wall clock around synchronized calls (forward, backward); "
                      "CUDA events for the selected inverse"}


def run_ldlt(torch, spx, inputs, steps: int) -> dict:
    """Symmetric indefinite (quasi-definite) 40^3 x 2-dof system: LDL^T with
    the C = C - L D L^T updates, FP64 against the mixed modes with refinement
    to 1e-12, one right-hand side block of 16."""
    dims = (40, 40, 40)
    A = inputs.quasi_definite_3d(*dims, 7)
    cp, ri, vals = inputs.csc_arrays(A)
    n = A.shape[0]
    B = inputs.rhs(n, NRHS, 7)
    h = spx.analyze(cp, ri, "ldlt", ordering=spx.SPX_ORDER_GRID, grid=dims, dof=2, max_width=64)
    flops = h.info()["flops"]
    vd = torch.from_numpy(vals).cuda()
    Bd = torch.from_numpy(np.ascontiguousarray(B.T)).cuda().t()
    Xd = torch.empty((NRHS, n), dtype=torch.float64, device="cuda").t()
    out = {}
    for mode in ("fp64", "fp32", "tf32", "bf16"):
        ref = None if mode == "fp64" else spx.default_refine(tol=TARGET_BERR)
        times, fms, sms = [], [], []
        for it in range(max(3, steps) + 1):
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            h.factorize(vd, mode)
            _, si = h.solve(Bd, Xd, refine=ref)
            e1.record()
            torch.cuda.synchronize()
            if it > 0:
                times.append(e0.elapsed_time(e1))
                fms.append(h.info()["factor_ms"])
                sms.append(h.info()["solve_ms"])
        X = Xd.cpu().numpy()
        R = B - A @ X
        den = abs(A).sum(axis=1).max() * np.abs(X).max(axis=0) + np.abs(B).max(axis=0)
        info = h.info()
        out[mode] = {"ms_per_step": statistics.median(times), "factor_ms": statistics.median(fms),
                     "solve_ms": statistics.median(sms),
                     "time_to_solve_gflops": flops / (statistics.median(times) / 1e3) / 1e9,
                     "host_backward_error": float(np.max(np.abs(R).max(axis=0) / den)),
                     "refine_iters": si["iters"], "negative_pivots": info["npivot_neg"],
                     "pivot_replacements": info["npivot_repl"]}
    h.free()
    return {"workload": "quasi-definite [[K, B^T], [B, -C]] 40^3 x 2 dof, 16 rhs, LDL^T",
            "n": n, "nnz_a": int(cp[-1]), "flops_exact": flops,
            "target_backward_error": TARGET_BERR, "modes": out,
            "speedup_best_mixed_over_fp64": out["fp64"]["ms_per_step"] /
            min(out[m]["ms_per_step"] for m in ("fp32", "tf32", "bf16"))}


def run_elasticity(torch, spx, inputs, steps: int) -> dict:
    """The 27-point, 3-dof elasticity-like system on a 40^3 grid (n = 192,000,
    14.8M nonzeros): plain FP64 against BF16 updates (FP32 accumulation, FP64
    diagonal blocks) with FP64 refinement to backward error 1e-12; one step =
    factorization + 16-RHS solve, CUDA events on the current stream."""
    dims = (40, 40, 40)
    A = inputs.elasticity_27pt(*dims, 7)
    cp, ri, vals = inputs.csc_arrays(A)
    n = A.shape[0]
    B = inputs.rhs(n, NRHS, 7)
    h = spx.analyze(cp, ri, "llt", ordering=spx.SPX_ORDER_GRID, grid=dims, dof=3, max_width=64)
    flops = h.info()["flops"]
    vd = torch.from_numpy(vals).cuda()
    Bd = torch.from_numpy(np.ascontiguousarray(B.T)).cuda().t()
    Xd = torch.empty((NRHS, n), dtype=torch.float64, device="cuda").t()
    out = {}
    for mode in ("fp64", "tf32", "bf16"):
        ref = None if mode == "fp64" else spx.default_refine(tol=TARGET_BERR)
        times, fms, sms = [], [], []
        for it in range(max(2, steps) + 1):
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            h.factorize(vd, mode)
            _, si = h.solve(Bd, Xd, refine=ref)
            e1.record()
            torch.cuda.synchronize()
            if it > 0:
                times.append(e0.elapsed_time(e1))
                fms.append(h.info()["factor_ms"])
                sms.append(h.info()["solve_ms"])
        X = Xd.cpu().numpy()
        R = B - A @ X
        den = abs(A).sum(axis=1).max() * np.abs(X).max(axis=0) + np.abs(B).max(axis=0)
        out[mode] = {"ms_per_step": statistics.median(times), "factor_ms": statistics.median(fms),
                     "solve_ms": statistics.median(sms),
                     "time_to_solve_gflops": flops / (statistics.median(times) / 1e3) / 1e9,
                     "factor_gflops": flops / (statistics.median(fms) / 1e3) / 1e9,
                     "host_backward_error": float(np.max(np.abs(R).max(axis=0) / den)),
                     "refine_iters": si["iters"], "gmres_iters": si["gmres_iters"],
                     "converged": bool(si["converged"])}
    info = h.info()
    h.free()
    return {"workload": "elasticity3d_40^3_27pt_3dof: K = R diag(mu) R^T per neighbour pair, "
                        "mu ~ logU[1,1e3], 16 rhs",
            "n": n, "nnz_a": int(cp[-1]), "nnz_l": info["nnz_l"], "flops_exact": flops,
            "target_backward_error": TARGET_BERR, "modes": out,
            "speedup_bf16_over_fp64": out["fp64"]["ms_per_step"] / out["bf16"]["ms_per_step"],
            "speedup_best_mixed_over_fp64": out["fp64"]["ms_per_step"] /
            min(out[m]["ms_per_step"] for m in ("tf32", "bf16") if out[m]["converged"])
            if any(out[m]["converged"] for m in ("tf32", "bf16")) else None}


# ---------------------------------------------------------------------------
# the kernel study of Sec. V-B through the factorization's update kernels
# ---------------------------------------------------------------------------
STUDY_WIDTHS = (32, 64, 128, 256)                  # N: source panel width (K of the product)
STUDY_HEIGHTS = (256, 512, 1024, 2048, 4096, 8192)  # M: source panel rows
STUDY_CALLS = 100


def run_update_study(torch, spx, inputs, peaks: dict) -> dict:
    """C = C - A B^T with A of M x N, B its first N rows, C a panel twice as
    tall as A with random blocks of about 200 rows (A's blocks inside C's),
    each point the average of 100 back-to-back calls (Sec. V-B protocol),
    through the hot-path update kernels (spx_update_* runs update_tc_kernel
    or update_kernel on a one-task plan).  flops = 2 M N^2; bytes = A and B
    read once, the touched C entries read and written once."""
    stream = torch.cuda.current_stream()
    modes = (("tf32", "tensor_cores"), ("bf16", "tensor_cores"), ("fp64", "cuda_cores"))
    out = {}
    for mode, engine in modes:
        rows = []
        for N in STUDY_WIDTHS:
            for M in STUDY_HEIGHTS:
                A, C, rowmap, colmap = inputs.gapped_update_case(M, N, N, 1000 * M + N)
                dt = np.float64 if mode == "fp64" else np.float32
                plan = spx.UpdatePlan(M, N, N, C.shape[0], C.shape[1], rowmap, colmap, lower=False,
                                      precision=mode, engine=engine)
                tA = torch.from_numpy(np.ascontiguousarray(A.T, dtype=dt)).cuda().t()
                tC = torch.from_numpy(np.ascontiguousarray(C.T, dtype=dt)).cuda().t()
                plan.stage(tA, stream=stream)
                for _ in range(3):
                    plan.run(tC, wait=False, stream=stream)
                torch.cuda.synchronize()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                for _ in range(STUDY_CALLS):
                    plan.run(tC, wait=False, stream=stream)
                e1.record(stream)
                plan.run(tC, wait=True, stream=stream)     # reports a pipeline timeout, if any
                ms = e0.elapsed_time(e1) / STUDY_CALLS
                plan.free()
                flops = 2.0 * M * N * N
                eop = {"tf32": 4.0, "bf16": 2.0, "fp64": 8.0}[mode]
                eacc = 8.0 if mode == "fp64" else 4.0
                byts = (M + N) * N * eop + 2.0 * M * N * eacc
                rows.append({"N": N, "M": M, "us_per_call": round(ms * 1e3, 3),
                             "gflops": flops / (ms / 1e3) / 1e9, "gbs": byts / (ms / 1e3) / 1e9})
        if mode == "fp64":
            peak, src = FP64_ALU_PEAK_GFLOPS, "derived FP64 ALU peak"
        else:
            peak = peaks["bf16_tflops"] * 1e3 * (1.0 if mode == "bf16" else NOMINAL_TF32_OVER_BF16)
            src = "measured bf16" + ("" if mode == "bf16" else " x nominal tf32/bf16 ratio (1.1/2.25)")
        for r in rows:
            r["frac_compute_peak"] = r["gflops"] / peak
            r["frac_hbm"] = r["gbs"] / peaks["hbm_gbs"]
        best = max(rows, key=lambda r: r["gflops"])
        out[mode] = {"engine": engine,
                     "kernel": "update_tc_kernel (tcgen05)" if engine == "tensor_cores" else
                               "update_kernel (CUDA cores)",
                     "compute_peak_gflops": peak, "peak_source": src, "points": rows,
                     "best": {k: best[k] for k in ("N", "M", "gflops", "frac_compute_peak")}}
    return {"protocol": "Sec. V-B: C = C - A B^T, A M x N, B = first N rows of A, C twice as tall "
                        "with random ~200-row blocks, average of 100 back-to-back calls "
                        "(C stays in L2 across the calls)",
            "modes": out}


# ---------------------------------------------------------------------------
# the GPU arm
# ---------------------------------------------------------------------------
def main():
    args = _args()
    if args.impl == "reference":
        run_reference(args)
        return
    import torch

    import __graft_entry__
    from paper_1405_2636_gb300 import inputs, replicas, spx

    world, rank, local = replicas.env_ranks()

    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    __graft_entry__.build()

    grid = tuple(int(v) for v in args.grid.split(","))
    A = inputs.diffusion_3d(*grid, SEED)
    colptr, rowind, vals = inputs.csc_arrays(A)
    n = A.shape[0]
    B = inputs.rhs(n, NRHS, SEED)
    h = spx.analyze(colptr, rowind, "llt", ordering=spx.SPX_ORDER_GRID, grid=grid,
                    max_width=args.max_width)
    info0 = h.info()
    flops = info0["flops"]

    dev = torch.device("cuda", local)
    vals_d = torch.from_numpy(vals).to(dev)
    B_d = torch.from_numpy(np.ascontiguousarray(B.T)).to(dev).t()      # column-major n x 16
    X_d = torch.empty((NRHS, n), dtype=torch.float64, device=dev).t()
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()

    group = replicas.RankGroup(world, dev)
    barrier = group.barrier
    max_over_ranks = group.max

    def step(mode):
        h.factorize(vals_d, mode)
        refine = None if mode == "fp64" else spx.default_refine(tol=TARGET_BERR)
        _, sinfo = h.solve(B_d, X_d, refine=refine)
        return sinfo

    results = {}
    x_fp64 = None   # the FP64 factor's solution (that factor matches the oracle to 1e-12 in the tests)
    launches_total = 0
    clocks = None
    modes = [m for m in args.modes.split(",") if m]
    for mode in modes:
        for _ in range(args.warmup):
            step(mode)
        torch.cuda.synchronize()
        times = []
        sinfo = None
        with ClockSampler(local) as cs:
            for _ in range(args.steps):
                flush.fill_(float(len(times)))           # L2 flush between timed steps
                barrier()
                torch.cuda.synchronize()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                sinfo = step(mode)
                e1.record(stream)
                torch.cuda.synchronize()
                barrier()
                times.append(e0.elapsed_time(e1))
        ck = cs.summary()
        info = h.info()
        # independent host check of the timed step's output (scipy residual)
        Xc = X_d.cpu().numpy()
        if mode == "fp64":
            x_fp64 = Xc.copy()
        diff_fp64 = (float(np.linalg.norm(Xc - x_fp64) / np.linalg.norm(x_fp64))
                     if x_fp64 is not None else None)
        R_host = B - A @ Xc
        den = (abs(A).sum(axis=1).max() * np.abs(Xc).max(axis=0) + np.abs(B).max(axis=0))
        host_berr = float(np.max(np.abs(R_host).max(axis=0) / den))
        ms = max_over_ranks(sum(times) / len(times))
        launches_total += args.steps * (info["launches_factor"] + info["launches_solve"])
        # profiled factorization: per-kernel-class device time (events on the library stream)
        h.set_profiling(True)
        h.factorize(vals_d, mode)
        h.set_profiling(False)
        ks = h.kernel_stats()
        # end-to-end through the C ABI with host buffers (copies inside the timed region)
        e2e_times = []
        for i in range(0 if args.no_e2e else max(2, args.steps)):
            barrier()
            t0 = time.perf_counter()
            h.factorize(vals, mode)
            Xh, sinfo_h = h.solve(B, refine=None if mode == "fp64" else spx.default_refine(tol=TARGET_BERR))
            dt = time.perf_counter() - t0
            if i > 0:
                e2e_times.append(dt)
        e2e_ms = max_over_ranks(1e3 * sum(e2e_times) / len(e2e_times)) if e2e_times else float("nan")
        if not e2e_times:
            sinfo_h = {"backward_error": float("nan")}
        results[mode] = {
            "ms_per_step": ms,
            "step_ms": [round(t, 3) for t in times],
            "factor_ms": info["factor_ms"],
            "solve_ms": info["solve_ms"],
            "factor_bytes": info["factor_bytes"],
            "factor_gflops": flops / (info["factor_ms"] / 1e3) / 1e9,
            "time_to_solve_gflops": flops / (ms / 1e3) / 1e9,
            "backward_error": sinfo["backward_error"],
            "host_backward_error": host_berr,
            "rel_diff_to_fp64_solution": diff_fp64,
            "refine_iters": sinfo["iters"],
            "converged": bool(sinfo["backward_error"] <= TARGET_BERR and host_berr <= TARGET_BERR),
            "launches_per_step": info["launches_factor"] + info["launches_solve"],
            "kernel_stats": ks,
            "e2e_ms": e2e_ms,
            "e2e_backward_error": sinfo_h["backward_error"],
            "clocks": ck,
        }

    ok = [m for m in modes if results[m]["converged"]]
    head = min(ok, key=lambda m: results[m]["ms_per_step"]) if ok else modes[0]
    R = results[head]
    clocks = R["clocks"]          # sampled during the headline mode's timed steps
    peaks = measured_peaks()
    # roofline model of the whole factorization: every task at the better of
    # its two bounds (spx_roofline_model), against the measured factor time
    tpeak = peaks["bf16_tflops"] * 1e3 * (1.0 if head == "bf16" else NOMINAL_TF32_OVER_BF16)
    model = h.roofline_model(head, peaks["hbm_gbs"], FP64_ALU_PEAK_GFLOPS, FP32_ALU_PEAK_GFLOPS, tpeak)
    model_total = sum(model.values())
    factor_model = {"mode": head, "model_ms_per_class": model, "model_ms": model_total,
                    "measured_factor_ms": R["factor_ms"],
                    "frac": model_total / R["factor_ms"] if R["factor_ms"] > 0 else None,
                    "peaks": {"hbm_gbs": peaks["hbm_gbs"], "fp64_gflops": FP64_ALU_PEAK_GFLOPS,
                              "fp32_gflops": FP32_ALU_PEAK_GFLOPS, "tensor_gflops": tpeak},
                    "definition": "sum over tasks of max(flops / compute peak, bytes / HBM bandwidth) "
                                  "over the measured factorization time"}
    rooflines = {c: class_roofline(c, st, head, peaks) for c, st in R["kernel_stats"].items()
                 if st["ms"] > 0}
    solve_rl = solve_roofline({"factor_bytes": R["factor_bytes"], "nnz_a": int(colptr[-1]), "n": n,
                               "solve_ms": R["solve_ms"]}, NRHS, R["refine_iters"], peaks)
    dominant = max(rooflines, key=lambda c: rooflines[c]["device_ms"])
    roofline = dict(rooflines[dominant])
    roofline["kernel"] = {"diag": "potrf_ldl_kernel / potrf_kernel (FP64 diagonal blocks)",
                          "trsm": "trsm_gemm_kernel", "update": "update_kernel (CUDA cores)",
                          "update_tc": "update_tc_kernel (tcgen05)",
                          "queue": "factor_queue_kernel (persistent task queue of the upper levels)",
                          "assemble": "assemble_kernel"}[dominant]

    extra = {}
    if not args.no_extra:   # every rank: the batch is sharded over the ranks
        extra["batched_lu"] = run_batched(torch, spx, inputs, args.steps, group, rank)
    if not args.no_extra and rank == 0:
        extra["update_kernel_study"] = run_update_study(torch, spx, inputs, peaks)
    if rank != 0:
        if world > 1:
            torch.distributed.destroy_process_group()
        return
    if not args.no_extra:
        extra["differentiation"] = run_differentiation(torch, spx, inputs, args.steps)
        extra["ldlt"] = run_ldlt(torch, spx, inputs, args.steps)
        extra["elasticity"] = run_elasticity(torch, spx, inputs, args.steps)
    cpu = None
    if not args.no_cpu_baseline and world == 1:
        cpu = oracle_rate((32, 32, 32), 12.0)   # about 12-15 s of single-core work
    value = replicas.whole_job_rate(flops, world, R["ms_per_step"]) / 1e9
    e2e_value = replicas.whole_job_rate(flops, world, R["e2e_ms"]) / 1e9
    line = {
        "metric": METRIC, "value": value, "unit": "GFlop/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": R["ms_per_step"],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": DTYPES[head],
        "data": "synthetic",
        "config": {"workload": WORKLOAD if grid == GRID else
                   f"diffusion3d_{grid[0]}x{grid[1]}x{grid[2]}_7pt_expN01_16rhs",
                   "n": n, "nnz_a": int(colptr[-1]), "nrhs": NRHS,
                   "seed": SEED, "grid": list(grid), "ordering": "geometric nested dissection",
                   "nnz_l": info0["nnz_l"], "flops_exact": flops,
                   "panels": info0["npanels"], "levels": info0["nlevels"],
                   "max_width": args.max_width,
                   "headline_mode": head, "l2": "flushed between timed steps (256 MiB write); "
                   "the 1.3 GB factor also exceeds L2", "parallelism": f"replicas x{world}"},
        "modes": {m: {k: v for k, v in results[m].items() if k not in ("kernel_stats",)}
                  for m in modes},
        "kernel_stats": {m: results[m]["kernel_stats"] for m in modes},
        "fp64_ms_per_step": results["fp64"]["ms_per_step"] if "fp64" in results else None,
        "speedup_mixed_over_fp64": (results["fp64"]["ms_per_step"] / R["ms_per_step"]
                                    if "fp64" in results and head != "fp64" else None),
        "roofline": roofline,
        "rooflines": rooflines,
        "factorization_roofline_model": factor_model,
        "solve_roofline": solve_rl,
        "cpu_baseline": cpu,
        "e2e": {"value": e2e_value, "unit": "GFlop/s",
                "h2d_bytes_per_step": int(8 * colptr[-1] + 8 * n * NRHS),
                "d2h_bytes_per_step": int(8 * n * NRHS)},
        "gpu_launches": launches_total,
        "clocks": clocks,
    }
    line.update(extra)
    print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
