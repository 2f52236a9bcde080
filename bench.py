#!/usr/bin/env python
"""Benchmark of one RK time step of the stage-coupled heat solver on GB300.

Workload (default ``heat2d-1024-radau3``): 2D heat equation u_t = div(kappa grad u) + f
on the unit square, Q1 on 1024 x 1024 quads (1,050,625 nodes), per-cell lognormal
kappa (sigma = 0.5 in log, seed 0), RadauIIA(3), dt = 1/256, FP64 FGMRES (rtol
1e-10) with the block-lower-triangular stage preconditioner, one V(2,2)
weighted-Jacobi (omega = 2/3) V-cycle per block on 6 levels.  Forcing and initial
state are the sine manufactured solution.  A bench "step" is one full time step:
right-hand side, FGMRES solve with V-cycle preconditioning, RK update.

``python bench.py --gpus N --steps K --warmup W`` prints one JSON line.
``--impl reference`` times the FP64 CPU oracle instead (rank 0 only).
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

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402

METRIC = "time-steps/s and DOF·stage/s at fixed L2 error; stencil/V-cycle GB/s vs HBM peak"
# FP64 arithmetic peak: 152 SMs x 2 FP64 FMA/clk/SM x 2 flop x 2.07 GHz (matches the nominal 1.25 TFLOP/s)
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12
FP64_CLASSES = ("stage_apply", "multidot", "axpy")  # always FP64
SPLIT_LABEL = {"ia": "IA: (A^-1 (x) M + dt I (x) K) w = r, k = (A^-1 (x) I) w",
               "ai": "AI: (I (x) M + dt A (x) K) k = r"}


def parse():
    ap = argparse.ArgumentParser(description=__doc__)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--workload", default="heat2d-1024-radau3", choices=sorted(W.WORKLOADS))
    ap.add_argument("--precond", default="lower", choices=["diag", "lower", "upper", "rana_ld", "monolithic"])
    ap.add_argument("--vcycle", default=None, choices=["fp64", "fp32", "bf16"])
    ap.add_argument("--orth", default="cgs", choices=["cgs2", "dgks", "cgs"],
                    help="Arnoldi orthogonalisation; cgs (one pass, true residual checked at convergence) is the "
                         "GMRES default of the PETSc stack the paper used")
    ap.add_argument("--splitting", default="ia", choices=["ia", "ai"],
                    help="form of the stage system: IA (Sec. 3, eq. block_struct_IA, the paper's heat form) or AI")
    ap.add_argument("--tableau", default=None, help="override, e.g. GaussLegendre:4 or Alexander:3")
    ap.add_argument("--restart", type=int, default=50, help="FGMRES restart length (Krylov basis size)")
    ap.add_argument("--no-variants", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--study", default=None, choices=["long-horizon"],
                    help="instead of the benchmark line: time-to-solution at equal final L2 error on the "
                         "2048^2 long-horizon workload (SDIRK vs RadauIIA, FP64 vs FP32 V-cycles)")
    return ap.parse_args()


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# ----------------------------------------------------------------------------
# clock sampling during the timed region
# ----------------------------------------------------------------------------
class Clocks:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_id: str | None):
        self.proc = None
        self.path = tempfile.mktemp(prefix="clocks_", suffix=".csv")
        self.device_id = device_id

    def start(self):
        cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "200"]
        if self.device_id:
            cmd += ["-i", self.device_id]
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(cmd, stdout=self.fh, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self) -> dict | None:
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.fh.close()
        rows = []
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        smax = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": reasons, "samples": len(rows)}


def device_id_for_smi():
    import torch

    try:
        u = str(torch.cuda.get_device_properties(torch.cuda.current_device()).uuid)
        return u if u.startswith("GPU-") else "GPU-" + u
    except Exception:
        return os.environ.get("CUDA_VISIBLE_DEVICES", "").split(",")[0] or None


def source_hash() -> str:
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_2403_08084_gb300", "csrc")
    for f in sorted(os.listdir(d)):
        with open(os.path.join(d, f), "rb") as fh:
            h.update(f.encode() + fh.read())
    return h.hexdigest()[:16]


def ncu_traffic(kernel_class: str, workload: str):
    """The committed ncu record of a kernel class (DRAM bytes per launch, FP64 pipe activity), if it
    was taken on the current kernel sources and this workload; else None."""
    try:
        with open(os.path.join(ROOT, "profiles", "ncu_traffic.json")) as f:
            t = json.load(f)
    except Exception:
        return None
    if t.get("source_sha") != source_hash() or t.get("workload") != workload:
        return None
    return t.get("classes", {}).get(kernel_class)


# ----------------------------------------------------------------------------
# multi-rank aggregation (replicas: no collective on the data path)
# ----------------------------------------------------------------------------
def max_over_ranks(ms: float, device: str) -> float:
    """The slowest rank's time, so that the aggregate throughput counts every rank's work."""
    import torch
    import torch.distributed as td

    t = torch.tensor([ms], dtype=torch.float64, device=device)
    td.all_reduce(t, op=td.ReduceOp.MAX)
    td.barrier()
    return float(t.item())


def aggregate(world: int, steps: int, ms_max: float) -> float:
    """Whole-job time-steps/s: every rank ran ``steps`` steps of its own replica."""
    return world * steps / (ms_max / 1e3)


# ----------------------------------------------------------------------------
# GPU arm
# ----------------------------------------------------------------------------
RESTART = 50


def make_solver(wl, precond, vcycle, orth="cgs2", tableau=None, splitting="ai"):
    from paper_2403_08084_gb300 import Solver
    from paper_2403_08084_gb300 import tableaux as PT

    name, s = tableau or (wl.tableau, wl.s)
    tab = PT.by_name(name, s)
    kap = W.lognormal_kappa(wl.dim, wl.N, 0.5, wl.kappa_seed) if wl.kappa_seed is not None else None
    solver = "dirk_cg" if name.lower() == "alexander" else "fgmres"
    sv = Solver(wl.N, tab, wl.dt, dim=wl.dim, kappa=kap, levels=wl.levels, precond=precond, vcycle=vcycle,
                rtol=wl.rtol, orth=orth, solver=solver, restart=RESTART, splitting=splitting)
    return sv, tab


def run_steps(sv, tab, wl, u, f, n0, count, record=None):
    stats = []
    for n in range(n0, n0 + count):
        t = n * wl.dt
        coef = [W.sine_load_time(wl.dim, t + c * wl.dt) for c in tab.c]
        stats.append(sv.step(u, u, f_space=f, f_coef=coef))
        if record is not None:
            record.append(u.clone())
    return stats


def gpu_arm(args, rank, world):
    import torch

    wl = W.WORKLOADS[args.workload]
    vcycle = args.vcycle or wl.vcycle
    if vcycle == "exact":
        vcycle = "fp64"
    precond = args.precond
    dist = world > 1
    if dist:
        import torch.distributed as td
    tab_override = None
    if args.tableau:
        name, _, s_ = args.tableau.partition(":")
        tab_override = (name, int(s_ or 3))
    if precond == "monolithic":  # monolithic multigrid is built for the AI form
        args.splitting = "ai"
    sv, tab = make_solver(wl, precond, vcycle, args.orth, tab_override, args.splitting)
    nn = (wl.N + 1) ** wl.dim
    u0 = torch.from_numpy(W.sine_initial(wl.dim, wl.N)).cuda()
    f = torch.from_numpy(W.sine_load_space(wl.dim, wl.N)).cuda()
    u = u0.clone()
    stream = torch.cuda.current_stream()

    # warm-up, then one instrumented step to find the kernel class that dominates device time
    run_steps(sv, tab, wl, u, f, 0, args.warmup)
    sv.perf_select([c for c in ("stage_apply", "jacobi", "residual", "restrict", "prolong", "coarse", "multidot",
                                "axpy", "block_rhs", "mg_coarse", "mg_tail")])
    u.copy_(u0)
    run_steps(sv, tab, wl, u, f, 0, 1)
    prof = sv.perf_read()["classes"]
    dominant = max(prof, key=lambda k: prof[k]["timed_ms"] if k != "other" else -1)
    shares = {k: round(v["timed_ms"], 4) for k, v in prof.items() if v["timed_ms"] > 0}
    # every class's algorithmic rate in the instrumented step (events around each launch inflate
    # the shortest kernels' times)
    class_rates = {}
    for k, v in prof.items():
        if v["timed_ms"] > 0 and v["timed_launches"] > 0:
            sec = v["timed_ms"] / 1e3
            fp64 = k in FP64_CLASSES or vcycle == "fp64" or k == "other"
            tfl = v["timed_flops"] / sec / 1e12
            class_rates[k] = {"ms": round(v["timed_ms"], 4), "launches": v["timed_launches"],
                              "gbs": round(v["timed_bytes"] / sec / 1e9, 1),
                              "tflops": round(tfl, 4),
                              "frac": round(tfl / FP64_PEAK_TFLOPS, 4) if fp64 else
                              round(v["timed_bytes"] / sec / 1e9 / peaks()[0], 4),
                              "bound": "alu" if fp64 else "hbm"}

    # timed region: the workload's first K steps from t = 0 (launch counters only, no per-kernel events)
    u.copy_(u0)
    sv.perf_select([])
    clocks = Clocks(device_id_for_smi()) if rank == 0 else None
    if dist:
        td.barrier()
    torch.cuda.synchronize()
    if clocks:
        clocks.start()
        time.sleep(0.3)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    stats = run_steps(sv, tab, wl, u, f, 0, args.steps)
    e1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop() if clocks else None
    ms = e0.elapsed_time(e1)
    if dist:
        ms = max_over_ranks(ms, "cuda")
    launches = sv.perf_read()["launches"]
    u_final = u.clone()
    # the same K steps again with CUDA events around every launch of the dominant kernel class
    # (on the library's stream), for its average launch duration
    u.copy_(u0)
    sv.perf_select([dominant])
    run_steps(sv, tab, wl, u, f, 0, args.steps)
    perf = sv.perf_read()
    # state after the first 5 steps, for the variants' agreement check
    u5 = u0.clone()
    sv.perf_select([])
    run_steps(sv, tab, wl, u5, f, 0, min(5, args.steps))

    steps_per_s = aggregate(world, args.steps, ms)
    s = wl.s
    dof = (wl.N + 1) ** wl.dim
    its = [st["fgmres_its"] for st in stats]
    cls = perf["classes"][dominant]
    hbm, hbm_src = peaks()
    roof = None
    if cls["timed_launches"] > 0 and cls["timed_ms"] > 0:
        avg_s = cls["timed_ms"] / cls["timed_launches"] / 1e3
        bpl = cls["timed_bytes"] / cls["timed_launches"]
        fpl = cls["timed_flops"] / cls["timed_launches"]
        gbs = bpl / avg_s / 1e9
        tfl = fpl / avg_s / 1e12
        fp64_kernel = dominant in FP64_CLASSES or vcycle == "fp64"
        if fp64_kernel:
            roof = {"bound": "alu", "achieved": round(tfl, 4), "peak": round(FP64_PEAK_TFLOPS, 4), "unit": "TFLOP/s",
                    "frac": round(tfl / FP64_PEAK_TFLOPS, 4),
                    "peak_source": "FP64 FMA: 152 SMs x 2/clk x 2 flop x 2.07 GHz (nominal 1.25 TFLOP/s)"}
        else:
            roof = {"bound": "hbm", "achieved": round(gbs, 1), "peak": hbm, "unit": "GB/s", "frac": round(gbs / hbm, 4),
                    "peak_source": f"{hbm_src} (MEASURED_PEAKS.json hbm_gbs)"}
        rec = ncu_traffic(dominant, wl.name) or {}
        roof.update({"kernel": dominant, "traffic": rec.get("bytes_per_launch_full_size"),
                     "ncu_fp64_pipe_active_pct": rec.get("fp64_pipe_active_pct"), "launches": cls["timed_launches"],
                     "timing": "CUDA events on the library stream around each launch, replay of the K timed steps",
                     "avg_launch_us": round(avg_s * 1e6, 2), "algorithmic_bytes_per_launch": round(bpl),
                     "algorithmic_flops_per_launch": round(fpl), "achieved_gbs": round(gbs, 1),
                     "hbm_frac_of_measured": round(gbs / hbm, 4)})

    out = {
        "metric": METRIC,
        "value": round(steps_per_s, 4),
        "unit": "time-steps/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": round(ms / args.steps, 3),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f64" if vcycle == "fp64" else f"f64 outer / {vcycle} V-cycles",
        "data": "synthetic",
        "config": {"workload": wl.name, "mesh": "x".join([str(wl.N)] * wl.dim) + " Q1", "dofs": dof, "stages": s,
                   "tableau": tab_label(tab), "dt": wl.dt,
                   "kappa": ("lognormal sigma=0.5 seed %s" % wl.kappa_seed) if wl.kappa_seed is not None else "1",
                   "precond": precond, "splitting": SPLIT_LABEL[args.splitting], "vcycle": vcycle,
                   "levels": wl.levels, "rtol": wl.rtol, "orth": args.orth,
                   "restart": args.restart,
                   "parallelism": f"replicas x{world}" if world > 1 else "1 GPU",
                   "l2_policy": "working set > L2: Krylov basis of ~its x %.0f MB stage vectors per step"
                                % (dof * s * 8 / 1e6)},
        "dof_stage_per_s": round(steps_per_s * dof * s, 1),
        "fgmres_its_per_step": round(sum(its) / len(its), 2),
        "vcycles_per_step": round(sum(st["vcycles"] for st in stats) / len(stats), 2),
        "final_rel_resid_max": max(st["rel_resid"] for st in stats),
        "gpu_launches": launches,
        "roofline": roof,
        "kernel_ms_one_step": shares,
        "class_rooflines": class_rates,
        "clocks": clk,
    }
    if rank == 0 and not args.no_e2e:
        out["e2e"] = e2e_leg(sv, tab, wl, u0, args)
    sv.close()
    if rank == 0 and not args.no_variants:
        out["variants"] = variants_leg(wl, u5.cpu().numpy(), args, vcycle, precond)
    if rank == 0 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline_leg(wl, precond, args.splitting if precond not in ("upper", "monolithic") else "ai")
    out["final_u_norm"] = float(torch.linalg.vector_norm(u_final).item())
    return out


def tab_label(tab) -> str:
    return tab.name


def e2e_leg(sv, tab, wl, u0, args):
    """Same metric through the C ABI with pinned host buffers (copies inside the call)."""
    import torch

    nn = (wl.N + 1) ** wl.dim
    uh = u0.cpu().pin_memory()
    fh = torch.from_numpy(W.sine_load_space(wl.dim, wl.N)).pin_memory()
    out = torch.empty(nn, dtype=torch.float64).pin_memory()
    K = max(1, min(args.steps, 10))
    for n in range(1):  # warm the staging buffers
        coef = [W.sine_load_time(wl.dim, c * wl.dt) for c in tab.c]
        sv.step(uh, out, f_space=fh, f_coef=coef)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for n in range(K):
        coef = [W.sine_load_time(wl.dim, (n + c) * wl.dt) for c in tab.c]
        sv.step(uh, out, f_space=fh, f_coef=coef)
        uh, out = out, uh
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    return {"value": round(K / dt, 4), "unit": "time-steps/s", "steps": K, "h2d_bytes_per_step": 2 * nn * 8,
            "d2h_bytes_per_step": nn * 8, "buffers": "pinned host (torch pin_memory), host pointers to irk_step"}


def variants_leg(wl, u5_ref, args, vcycle0, precond0):
    """Other forms / preconditioners / V-cycle precisions / tableaux on the same workload (5 steps each)."""
    import torch

    res = {}
    nsteps = min(5, args.steps)
    alex = ("Alexander", 3)
    if wl.dim == 2:
        runs = [("lower", "fp64", "cgs2", None, "ia"), ("diag", "fp64", "cgs2", None, "ia"),
                ("rana_ld", "fp64", "cgs2", None, "ia"), ("lower", "fp32", "cgs2", None, "ia"),
                ("lower", "bf16", "cgs2", None, "ia"), ("rana_ld", "fp32", "cgs2", None, "ia"),
                ("lower", "fp64", "dgks", None, "ia"), ("lower", "fp64", "cgs", None, "ia"),
                ("lower", "fp32", "cgs", None, "ia"), ("rana_ld", "fp32", "cgs", None, "ia"),
                ("lower", "fp64", "cgs2", None, "ia"), ("lower", "fp32", "cgs2", None, "ia"),
                ("rana_ld", "fp64", "cgs", None, "ia"), ("lower", "bf16", "cgs", None, "ia"),
                ("monolithic", "fp64", "cgs", None, "ai"), ("monolithic", "fp32", "cgs", None, "ai"),
                ("lower", "fp64", "cgs2", None, "ai"), ("diag", "fp64", "cgs2", None, "ai"),
                ("rana_ld", "fp64", "cgs2", None, "ai"), ("lower", "fp32", "cgs2", None, "ai"),
                ("lower", "bf16", "cgs2", None, "ai"),
                ("lower", "fp64", "cgs2", alex, "ai"), ("lower", "fp32", "cgs2", alex, "ai")]
    else:
        runs = [("lower", "fp64", "cgs2", None, "ia"), ("lower", "fp32", "cgs2", None, "ia"),
                ("lower", "bf16", "cgs2", None, "ia"), ("rana_ld", "fp32", "cgs2", None, "ia"),
                ("lower", "fp32", "cgs2", None, "ai"), ("lower", "fp64", "cgs2", None, "ai"),
                ("lower", "fp32", "cgs2", ("GaussLegendre", 2), "ia"),
                ("lower", "fp32", "cgs2", ("GaussLegendre", 4), "ia"),
                ("lower", "bf16", "cgs2", ("GaussLegendre", 4), "ia")]
    for precond, vcycle, orth, tabo, split in runs:
        if (precond, vcycle, orth, tabo, split) == (precond0, vcycle0, args.orth, None, args.splitting):
            continue
        sv, tab = make_solver(wl, precond, vcycle, orth, tabo, split)
        u0 = torch.from_numpy(W.sine_initial(wl.dim, wl.N)).cuda()
        f = torch.from_numpy(W.sine_load_space(wl.dim, wl.N)).cuda()
        u = u0.clone()
        run_steps(sv, tab, wl, u, f, 0, 1)
        u.copy_(u0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        stats = run_steps(sv, tab, wl, u, f, 0, nsteps)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        un = u.cpu().numpy()
        key = f"{split.upper()}/{precond}/{vcycle}/{orth}" + (f"/{tab.name}" if tabo else "")
        entry = {"steps_per_s": round(nsteps / dt, 4), "ms_per_step": round(dt * 1e3 / nsteps, 3),
                 "krylov_its_per_step": round(sum(s["fgmres_its"] for s in stats) / nsteps, 2)}
        if tabo is None:
            entry["rel_l2_vs_headline_after_5_steps"] = float(np.linalg.norm(un - u5_ref) / np.linalg.norm(u5_ref))
        else:
            entry["note"] = "different tableau: a different time discretisation, not compared with the headline state"
        res[key] = entry
        sv.close()
    return res


def oracle_stepper(wl, N, levels, kind, split):
    """The oracle's FGMRES + sparse V-cycle restatement of one RK step (AI or IA form) on an N^dim mesh.
    Returns (one(u, n) -> (u_next, its), u0)."""
    from oracle import fem, krylov, mg, rk
    from oracle import tableaux as OT

    kap = W.lognormal_kappa(wl.dim, N, 0.5, wl.kappa_seed) if wl.kappa_seed is not None else None
    d = fem.Discretisation(wl.dim, N, kap)
    h = mg.Hierarchy(d, levels)
    ot = OT.by_name(wl.tableau, wl.s)
    Ap = krylov.rana_ld(ot.A) if kind == "rana_ld" else ot.A
    if kind == "monolithic":  # AI form only
        S = rk.kronecker_operator(d.M, d.K, ot.A, wl.dt)
        P = mg.MonolithicVCycle(h, ot.A, wl.dt)
        Ainv = np.eye(wl.s)
    elif split == "ia":
        T = np.diag(np.diag(Ap)) if kind == "diag" else np.tril(Ap)
        solves = [mg.VCycle(h, wl.dt * T[i, i]) for i in range(wl.s)]
        S = krylov.ia_operator(d.M, d.K, ot.A, wl.dt)
        P = krylov.IABlockPreconditioner(T, d.M, wl.dt, solves, diagonal_only=(kind == "diag"))
        Ainv = np.linalg.inv(ot.A)
    else:
        solves = [mg.VCycle(h, wl.dt * Ap[i, i]) for i in range(wl.s)]
        S = rk.kronecker_operator(d.M, d.K, ot.A, wl.dt)
        P = krylov.BlockPreconditioner("lower" if kind == "rana_ld" else kind, Ap, d.K, wl.dt, solves)
        Ainv = np.eye(wl.s)
    Fs = d.to_interior(W.sine_load_space(wl.dim, N))

    def one(u, n):
        r = np.stack([W.sine_load_time(wl.dim, (n + c) * wl.dt) * Fs for c in ot.c]) - (d.K @ u)[None, :]
        w, its, _, _ = krylov.fgmres(lambda v: S @ v, r.reshape(-1), P, rtol=wl.rtol)
        k = Ainv @ w.reshape(wl.s, -1)
        return u + wl.dt * (ot.b @ k), its

    return one, d.to_interior(W.sine_initial(wl.dim, N))


def cpu_baseline_leg(wl, precond, split):
    """One time step of the same workload through the oracle's FGMRES + V-cycle restatement
    (3D: on a 64^3 sample, scaled to the full DOF count)."""
    N = wl.N if wl.dim == 2 else min(wl.N, 64)
    levels = wl.levels - int(round(np.log2(wl.N // N)))
    one, u0 = oracle_stepper(wl, N, levels, precond, split)
    t0 = time.perf_counter()
    u1, its = one(u0, 0)
    dt = time.perf_counter() - t0
    scale = ((N + 1) / (wl.N + 1)) ** wl.dim
    where = "at full size" if N == wl.N else f"on a {N}^{wl.dim} sample, steps/s scaled by the DOF ratio {scale:.4f}"
    return {"value": round(scale / dt, 6), "unit": "time-steps/s", "cores": 1, "kind": "oracle",
            "sample": f"1 time step of {wl.name} {where} (oracle FGMRES + sparse V-cycle, {split.upper()} form, "
                      f"{precond}, FP64; {its} its; setup excluded)", "seconds": round(dt, 2),
            "u_norm": float(np.linalg.norm(u1))}


# ----------------------------------------------------------------------------
# reference arm: the FP64 CPU oracle
# ----------------------------------------------------------------------------
def reference_arm(args):
    wl = W.WORKLOADS[args.workload]
    # bounded sample: the same workload on a mesh with 1/4 of the nodes (one fewer level), so that
    # every step is a few seconds of CPU work; throughput is scaled to the full DOF count
    Ns = max(wl.N // 2, 32) if wl.dim == 2 else min(wl.N, 64)
    lv = max(1, wl.levels - int(round(np.log2(wl.N // Ns))))
    split = args.splitting if args.precond not in ("upper", "monolithic") else "ai"
    one, u0 = oracle_stepper(wl, Ns, lv, args.precond, split)

    u = u0.copy()
    for n in range(args.warmup):
        u, _ = one(u, n)
    u = u0.copy()
    t0 = time.perf_counter()
    its = []
    for n in range(args.steps):
        u, it = one(u, n)
        its.append(it)
    dt = time.perf_counter() - t0
    scale = ((Ns + 1) ** wl.dim) / ((wl.N + 1) ** wl.dim)
    value = args.steps / dt * scale
    sample = (f"each step: one RK step of {wl.name} on a {Ns}^{wl.dim} mesh ({lv} levels), oracle FGMRES + sparse "
              f"V-cycle, {split.upper()} form, {args.precond}, FP64; steps/s scaled by the DOF ratio {scale:.4f}")
    return {
        "impl": "reference",
        "metric": METRIC,
        "value": round(value, 6),
        "unit": "time-steps/s",
        "n_gpus": args.gpus,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": round(dt * 1e3 / args.steps, 2),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": wl.name, "mesh": "x".join([str(wl.N)] * wl.dim) + " Q1", "precond": args.precond,
                   "splitting": SPLIT_LABEL[split], "sample_mesh": Ns},
        "fgmres_its_per_step": round(sum(its) / len(its), 2),
        "cpu_baseline": {"value": round(value, 6), "unit": "time-steps/s", "cores": 1, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": round(value, 6), "unit": "time-steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


# ----------------------------------------------------------------------------
# long-horizon study: time-to-solution at equal final L2 error
# ----------------------------------------------------------------------------
def study_long_horizon(args):
    """2048^2 Q1, lognormal kappa (seed 0), integrated to T = 1 with Alexander's 3-stage SDIRK (sequential
    per-stage V-cycle-preconditioned CG) and RadauIIA(3) (FGMRES with P_L in the IA and AI forms, or monolithic
    multigrid), each with FP64 and FP32 V-cycles,
    over a sweep of step sizes.  The error is ||u_N - u_ref||_M / ||u_ref||_M against RadauIIA(4) at
    dt = 1/200 (order 7; its own error is estimated from the same scheme at dt = 1/100).  Time is the
    wall time of the step loop (setup reported apart); at a target error, each form's time is
    interpolated log-log between the two sweep points that bracket it."""
    import torch

    from paper_2403_08084_gb300 import Solver
    from paper_2403_08084_gb300 import tableaux as PT

    wl = W.WORKLOADS["heat2d-2048-long"]
    N, T = wl.N, 1.0
    kap = W.lognormal_kappa(2, N, 0.5, wl.kappa_seed)
    u0 = torch.from_numpy(W.sine_initial(2, N)).cuda()
    f = torch.from_numpy(W.sine_load_space(2, N)).cuda()

    def integrate(tab, nsteps, vcycle, solver, rtol, split="ai", precond="lower"):
        dt = T / nsteps
        t0 = time.perf_counter()
        sv = Solver(N, tab, dt, kappa=kap, levels=wl.levels, precond=precond, vcycle=vcycle, rtol=rtol,
                    solver=solver, restart=RESTART, maxit=2000, splitting=split)
        torch.cuda.synchronize()
        setup = time.perf_counter() - t0
        u = u0.clone()
        for n in range(min(2, nsteps)):  # warm-up: CUDA-graph capture of the first iterations
            sv.step(u, u, f_space=f, f_coef=[W.sine_load_time(2, (n + c) * dt) for c in tab.c])
        u.copy_(u0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        its = 0
        for n in range(nsteps):
            its += sv.step(u, u, f_space=f, f_coef=[W.sine_load_time(2, (n + c) * dt) for c in tab.c])["fgmres_its"]
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        sv.close()
        return u, wall, setup, its / nsteps

    mass = Solver(N, PT.radau_iia(1), 1.0, levels=wl.levels)

    def mnorm(x):
        y = torch.empty_like(x)
        mass.apply_mass(x, y)
        return math.sqrt(float(torch.dot(x, y).item()))

    ref, ref_wall, _, ref_its = integrate(PT.radau_iia(4), 200, "fp64", "fgmres", 1e-13, "ia")
    ref2, _, _, _ = integrate(PT.radau_iia(4), 100, "fp64", "fgmres", 1e-13, "ia")
    ref_norm = mnorm(ref)
    ref_err_est = mnorm(ref2 - ref) / ref_norm / (2**7 - 1)

    forms = [("RadauIIA(3) IA", PT.radau_iia(3), "fgmres", (2, 4, 8, 16, 32, 64), "ia", "lower"),
             ("RadauIIA(3) AI", PT.radau_iia(3), "fgmres", (2, 4, 8, 16, 32, 64), "ai", "lower"),
             ("RadauIIA(3) monolithic MG", PT.radau_iia(3), "fgmres", (2, 4, 8, 16, 32, 64), "ai", "monolithic"),
             ("Alexander SDIRK", PT.alexander(), "dirk_cg", (10, 25, 50, 100, 200, 400), "ai", "lower")]
    rows = []
    for label, tab, solver, sweep, split, precond in forms:
        for vcycle in ("fp64", "fp32"):
            for nsteps in sweep:
                u, wall, setup, its = integrate(tab, nsteps, vcycle, solver, wl.rtol, split, precond)
                rows.append({"scheme": label, "vcycle": vcycle, "dt": 1 / nsteps, "steps": nsteps,
                             "loop_s": round(wall, 4), "setup_s": round(setup, 3), "its_per_step": round(its, 2),
                             "rel_l2_err": mnorm(u - ref) / ref_norm})
    mass.close()

    def time_at(label, vcycle, target):
        pts = sorted((r["rel_l2_err"], r["loop_s"]) for r in rows if r["scheme"] == label and r["vcycle"] == vcycle)
        for (e_lo, t_lo), (e_hi, t_hi) in zip(pts, pts[1:]):
            if e_lo <= target <= e_hi:
                w = (math.log(target) - math.log(e_lo)) / (math.log(e_hi) - math.log(e_lo))
                return round(math.exp((1 - w) * math.log(t_lo) + w * math.log(t_hi)), 4)
        return None

    matched = []
    for target in (1e-4, 1e-5, 1e-6, 1e-7, 1e-8, 1e-9):
        entry = {"target_rel_l2_err": target}
        for label, _, _, _, _, _ in forms:
            for vcycle in ("fp64", "fp32"):
                entry[f"{label} {vcycle}"] = time_at(label, vcycle, target)
        matched.append(entry)
    return {"study": "long-horizon time-to-solution at equal final L2 error",
            "workload": wl.name, "mesh": f"{N}x{N} Q1", "dofs": (N + 1) ** 2, "T": T, "rtol": wl.rtol,
            "levels": wl.levels, "precond": "P_L (RadauIIA, IA and AI forms) or monolithic MG; per-stage V(2,2)-PCG (SDIRK)",
            "reference": {"scheme": "RadauIIA(4), IA form", "dt": 1 / 200, "rtol": 1e-13, "loop_s": round(ref_wall, 2),
                          "its_per_step": round(ref_its, 2), "est_rel_err": ref_err_est},
            "runs": rows, "loop_seconds_at_matched_error": matched}


def main():
    global RESTART
    args = parse()
    RESTART = args.restart
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if args.impl == "reference":
        if rank != 0:
            return 0
        print(json.dumps(reference_arm(args)))
        return 0
    import torch

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if args.study:
        if rank == 0:
            print(json.dumps(study_long_horizon(args)))
        return 0
    if world > 1:
        import torch.distributed as td

        td.init_process_group("nccl", device_id=torch.device("cuda", local))
    out = gpu_arm(args, rank, world)
    if rank == 0:
        print(json.dumps(out))
    if world > 1:
        import torch.distributed as td

        td.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
