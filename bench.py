#!/usr/bin/env python
"""Benchmark of one RK time step of the stage-coupled heat solver on GB300.

Workload (default ``heat2d-2048-long``, the largest single-GPU configuration):
2D heat equation u_t = div(kappa grad u) + f on the unit square, Q1 on 2048 x 2048
quads (4,198,401 nodes), per-cell lognormal kappa (sigma = 0.5 in log, seed 0),
RadauIIA(3), dt = 1/100, FP64 FGMRES (rtol 1e-10) with the block-lower-triangular
stage preconditioner in the IA form, one V(2,2) weighted-Jacobi (omega = 2/3)
V-cycle per block on 7 levels.  Forcing and initial state are the sine
manufactured solution.  A bench "step" is one full time step: right-hand side,
FGMRES solve with V-cycle preconditioning, RK update.

``python bench.py --gpus N --steps K --warmup W`` prints one JSON line.  Besides
the timed steps it reports the end-to-end rate with host buffers, variants of the
solver on the same workload, the 1024^2, 128^3 and adjoint workloads, and the
oracle's step on the host cores with the element-wise error of the GPU states
against it.  ``--impl reference`` times the FP64 CPU oracle instead (rank 0 only).
"""
from __future__ import annotations

import os

# the oracle's timing on the host is reported for one core: keep NumPy's BLAS single-threaded
for _v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_v, "1")

import argparse  # noqa: E402
import hashlib  # noqa: E402
import json  # noqa: E402
import math  # noqa: E402
import statistics  # noqa: E402
import subprocess  # noqa: E402
import sys  # noqa: E402
import tempfile  # noqa: E402
import time  # noqa: E402

import numpy as np  # noqa: E402

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
    ap.add_argument("--workload", default="heat2d-2048-long", choices=sorted(W.WORKLOADS))
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
    ap.add_argument("--no-configs", action="store_true",
                    help="skip the 1024^2, 128^3 and adjoint workloads reported beside the headline")
    ap.add_argument("--repeats", type=int, default=5, help="extra timed runs of the K steps, for their spread")
    ap.add_argument("--study", default=None, choices=["long-horizon"],
                    help="instead of the benchmark line: time-to-solution at equal final L2 error on the "
                         "2048^2 long-horizon workload (SDIRK vs RadauIIA, FP64 vs FP32 V-cycles)")
    args = ap.parse_args()
    args.tab_override = None
    if args.tableau:
        name, _, s_ = args.tableau.partition(":")
        args.tab_override = (name, int(s_ or 3))
    return args


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


# host-only sources (no device code): a change there leaves every kernel's DRAM traffic as it was
HOST_SOURCES = ("api.cu", "hierarchy.cpp", "hierarchy.h")


def source_hash() -> str:
    """Hash of the device-code sources (kernels, their launch shapes and the headers they include)."""
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_2403_08084_gb300", "csrc")
    for f in sorted(os.listdir(d)):
        if f in HOST_SOURCES:
            continue
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
# workload description shared by both arms
# ----------------------------------------------------------------------------
RESTART = 50


def tableau_of(wl, override=None):
    return override or (wl.tableau, wl.s)


def workload_config(wl, args, vcycle, precond, split, world):
    """The ``config`` object of the JSON line; the reference arm prints the same one."""
    name, s = tableau_of(wl, getattr(args, "tab_override", None))
    dof = (wl.N + 1) ** wl.dim
    return {"workload": wl.name, "mesh": "x".join([str(wl.N)] * wl.dim) + " Q1", "dofs": dof, "stages": s,
            "tableau": f"{name}({s})", "dt": wl.dt,
            "kappa": ("lognormal sigma=0.5 seed %s" % wl.kappa_seed) if wl.kappa_seed is not None else "1",
            "precond": precond, "splitting": SPLIT_LABEL[split], "vcycle": vcycle, "levels": wl.levels,
            "rtol": wl.rtol, "orth": args.orth, "restart": args.restart,
            "parallelism": f"replicas x{world}" if world > 1 else "1 GPU",
            "l2_policy": "working set > L2: Krylov basis of ~its x %.0f MB stage vectors per step"
                         % (dof * s * 8 / 1e6)}


# ----------------------------------------------------------------------------
# GPU arm
# ----------------------------------------------------------------------------
def make_solver(wl, precond, vcycle, orth="cgs2", tableau=None, splitting="ai", rtol=None, warm=False):
    from paper_2403_08084_gb300 import Solver
    from paper_2403_08084_gb300 import tableaux as PT

    name, s = tableau_of(wl, tableau)
    tab = PT.by_name(name, s)
    kap = W.lognormal_kappa(wl.dim, wl.N, 0.5, wl.kappa_seed) if wl.kappa_seed is not None else None
    solver = "dirk_cg" if name.lower() == "alexander" else "fgmres"
    sv = Solver(wl.N, tab, wl.dt, dim=wl.dim, kappa=kap, levels=wl.levels, precond=precond, vcycle=vcycle,
                rtol=wl.rtol if rtol is None else rtol, orth=orth, solver=solver, restart=RESTART,
                splitting=splitting, warm_start=warm)
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


def first_step(sv, tab, wl, u0, f):
    """u_1 and the stages k (node-major) of one step from u0, on the host."""
    import torch

    u1 = torch.empty_like(u0)
    k = torch.empty(sv.n_nodes * sv.s, dtype=torch.float64, device=u0.device)
    coef = [W.sine_load_time(wl.dim, c * wl.dt) for c in tab.c]
    sv.step(u0, u1, f_space=f, f_coef=coef, stages_out=k)
    return u1.cpu().numpy(), k.cpu().numpy()


def timed_steps(sv, tab, wl, u0, f, steps, warmup):
    """CUDA-event time of ``steps`` steps from t = 0 after ``warmup`` untimed ones; returns (ms, stats, u)."""
    import torch

    u = u0.clone()
    run_steps(sv, tab, wl, u, f, 0, warmup)
    u.copy_(u0)
    sv.reset_initial_guess()  # a warm-started solver must not start step 0 from the warm-up's own stages
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    stats = run_steps(sv, tab, wl, u, f, 0, steps)
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1), stats, u


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
    if precond == "monolithic":  # monolithic multigrid is built for the AI form
        args.splitting = "ai"
    sv, tab = make_solver(wl, precond, vcycle, args.orth, args.tab_override, args.splitting)
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
    sv.perf_select([])
    # the K steps repeated (each run from u0), for the spread of the step time
    repeats = [timed_steps(sv, tab, wl, u0, f, args.steps, 0)[0] / args.steps for _ in range(args.repeats)]
    # one step from u0 with its stages, for the comparison with the oracle; the state after 5 steps
    # for the variants' agreement check
    u1_k1 = first_step(sv, tab, wl, u0, f) if rank == 0 else None
    u5 = u0.clone()
    run_steps(sv, tab, wl, u5, f, 0, min(5, args.steps))

    steps_per_s = aggregate(world, args.steps, ms)
    s = sv.s
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
        "config": workload_config(wl, args, vcycle, precond, args.splitting, world),
        "dof_stage_per_s": round(steps_per_s * dof * s, 1),
        "fgmres_its_per_step": round(sum(its) / len(its), 2),
        "vcycles_per_step": round(sum(st["vcycles"] for st in stats) / len(stats), 2),
        "final_rel_resid_max": max(st["rel_resid"] for st in stats),
        "gpu_launches": launches,
        "repeats": {"runs": len(repeats), "ms_per_step_median": round(statistics.median(repeats), 3) if repeats else None,
                    "ms_per_step_min": round(min(repeats), 3) if repeats else None,
                    "ms_per_step_max": round(max(repeats), 3) if repeats else None,
                    "note": "the K steps run again from u0 after the timed region, each run timed with CUDA events"},
        "roofline": roof,
        "kernel_ms_one_step": shares,
        "class_rooflines": class_rates,
        "clocks": clk,
    }
    if rank == 0 and not args.no_e2e:
        out["e2e"] = e2e_leg(sv, tab, wl, u0, args)
    sv.close()
    checks = {}  # GPU states compared with the oracle in the cpu_baseline leg
    if rank == 0:
        checks[f"{args.splitting.upper()}/{precond}/{vcycle}/{args.orth} (headline)"] = u1_k1
    if rank == 0 and not args.no_variants:
        out["variants"], vchecks = variants_leg(wl, u5.cpu().numpy(), u0, f, args, vcycle, precond)
        checks.update(vchecks)
    del u5
    extra_checks = {}
    if rank == 0 and not args.no_configs and wl.name == "heat2d-2048-long" and args.tab_override is None:
        out["config2"], extra_checks["config2"] = config2_leg(args)
        out["config3"], extra_checks["config3"] = config3_leg(args)
        out["config4"] = config4_leg(args)
    if rank == 0 and not args.no_cpu_baseline:
        split = args.splitting if precond not in ("upper", "monolithic") else "ai"
        out["cpu_baseline"], out["l2_vs_oracle"] = cpu_baseline_leg(wl, precond, split, checks, extra_checks,
                                                                    args.tab_override)
    elif rank == 0:
        out["l2_vs_oracle"] = None
    out["final_u_norm"] = float(torch.linalg.vector_norm(u_final).item())
    return out


def e2e_leg(sv, tab, wl, u0, args):
    """Same metric and step count as the timed region, through the C ABI with pinned host buffers (the
    copies of u_n and the load in, u_{n+1} out run inside every call)."""
    import torch

    nn = (wl.N + 1) ** wl.dim
    uh = u0.cpu().pin_memory()
    fh = torch.from_numpy(W.sine_load_space(wl.dim, wl.N)).pin_memory()
    out = torch.empty(nn, dtype=torch.float64).pin_memory()
    K = args.steps
    coef = [W.sine_load_time(wl.dim, c * wl.dt) for c in tab.c]
    sv.step(uh, out, f_space=fh, f_coef=coef)  # warm the staging buffers
    uh = u0.cpu().pin_memory()
    sv.reset_initial_guess()
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


def variants_leg(wl, u5_ref, u0, f, args, vcycle0, precond0):
    """Other forms / preconditioners / V-cycle precisions / tableaux on the same workload (5 steps each).
    Returns (results, {label: (u_1, k_1)}) with each same-tableau variant's first step for the oracle check."""
    import torch

    res, checks = {}, {}
    nsteps = min(5, args.steps)
    alex = ("Alexander", 3)
    if wl.dim == 2:
        runs = [("lower", "fp32", "cgs", None, "ia"), ("lower", "bf16", "cgs", None, "ia"),
                ("rana_ld", "fp64", "cgs", None, "ia"), ("rana_ld", "fp32", "cgs", None, "ia"),
                ("diag", "fp64", "cgs", None, "ia"), ("lower", "fp64", "cgs2", None, "ia"),
                ("monolithic", "fp64", "cgs", None, "ai"), ("monolithic", "fp32", "cgs", None, "ai"),
                ("lower", "fp64", "cgs2", None, "ai"), ("diag", "fp64", "cgs2", None, "ai"),
                ("lower", "fp32", "cgs2", None, "ai"),
                ("lower", "fp64", "cgs2", alex, "ai"), ("lower", "fp32", "cgs2", alex, "ai"),
                ("lower", "fp64", "cgs", None, "ia", "warm"), ("lower", "fp32", "cgs", None, "ia", "warm")]
    else:
        runs = [("lower", "fp64", "cgs2", None, "ia"), ("lower", "fp32", "cgs2", None, "ia"),
                ("lower", "bf16", "cgs2", None, "ia"), ("rana_ld", "fp32", "cgs2", None, "ia"),
                ("lower", "fp32", "cgs2", None, "ai"), ("lower", "fp64", "cgs2", None, "ai")]
    for precond, vcycle, orth, tabo, split, *warm in runs:
        if (precond, vcycle, orth, tabo, split, *warm) == (precond0, vcycle0, args.orth, None, args.splitting):
            continue
        sv, tab = make_solver(wl, precond, vcycle, orth, tabo, split, warm=bool(warm))
        key = f"{split.upper()}/{precond}/{vcycle}/{orth}" + (f"/{tab.name}" if tabo else "") + (
            "/warm-start" if warm else "")
        if tabo is None:
            checks[key] = first_step(sv, tab, wl, u0, f)
        ms, stats, u = timed_steps(sv, tab, wl, u0, f, nsteps, 1)
        un = u.cpu().numpy()
        entry = {"steps_per_s": round(nsteps / (ms / 1e3), 4), "ms_per_step": round(ms / nsteps, 3),
                 "krylov_its_per_step": round(sum(s["fgmres_its"] for s in stats) / nsteps, 2)}
        if tabo is None:
            entry["rel_l2_vs_headline_after_5_steps"] = float(np.linalg.norm(un - u5_ref) / np.linalg.norm(u5_ref))
        else:
            entry["note"] = "different tableau: a different time discretisation, not compared with the headline state"
        res[key] = entry
        sv.close()
    return res, checks


def config2_leg(args):
    """The 1024^2 workload (lognormal kappa seed 0, RadauIIA(3), dt 1/256, 6 levels): P_L vs P_D, FP64 and
    FP32 V-cycles, 20 timed steps each; first steps kept for the oracle check."""
    import torch

    wl = W.WORKLOADS["heat2d-1024-radau3"]
    u0 = torch.from_numpy(W.sine_initial(2, wl.N)).cuda()
    f = torch.from_numpy(W.sine_load_space(2, wl.N)).cuda()
    res, checks = {"workload": wl.name, "mesh": f"{wl.N}x{wl.N} Q1", "dt": wl.dt, "levels": wl.levels,
                   "tableau": "RadauIIA(3)", "rtol": wl.rtol, "steps": wl.steps, "runs": {}}, {}
    for precond, vcycle, orth, split in (("lower", "fp64", "cgs", "ia"), ("diag", "fp64", "cgs", "ia"),
                                         ("lower", "fp32", "cgs", "ia"), ("lower", "fp64", "cgs2", "ai"),
                                         ("diag", "fp64", "cgs2", "ai")):
        sv, tab = make_solver(wl, precond, vcycle, orth, None, split)
        key = f"{split.upper()}/{precond}/{vcycle}/{orth}"
        checks[key] = first_step(sv, tab, wl, u0, f)
        ms, stats, _ = timed_steps(sv, tab, wl, u0, f, wl.steps, 3)
        res["runs"][key] = {"steps_per_s": round(wl.steps / (ms / 1e3), 4), "ms_per_step": round(ms / wl.steps, 3),
                            "fgmres_its_per_step": round(sum(s["fgmres_its"] for s in stats) / wl.steps, 2)}
        sv.close()
    return res, checks


def config3_leg(args):
    """The 128^3 workload (kappa = 1, dt 1/64, 5 levels, 10 steps, P_L, IA form): RadauIIA(3) with FP64,
    FP32 and BF16 V-cycles, Gauss-Legendre(2) and (4); final states kept for the eigenmode check."""
    import torch

    wl = W.WORKLOADS["heat3d-128"]
    u0 = torch.from_numpy(W.sine_initial(3, wl.N)).cuda()
    f = torch.from_numpy(W.sine_load_space(3, wl.N)).cuda()
    res, finals = {"workload": wl.name, "mesh": f"{wl.N}^3 Q1", "dt": wl.dt, "levels": wl.levels, "rtol": wl.rtol,
                   "steps": wl.steps, "runs": {}}, {}
    for tabo, vcycle in ((("RadauIIA", 3), "fp64"), (("RadauIIA", 3), "fp32"), (("RadauIIA", 3), "bf16"),
                         (("GaussLegendre", 2), "fp32"), (("GaussLegendre", 4), "fp32"),
                         (("GaussLegendre", 4), "bf16")):
        sv, tab = make_solver(wl, "lower", vcycle, "cgs", tabo, "ia")
        ms, stats, u = timed_steps(sv, tab, wl, u0, f, wl.steps, 2)
        key = f"{tab.name}/IA/lower/{vcycle}/cgs"
        res["runs"][key] = {"steps_per_s": round(wl.steps / (ms / 1e3), 4), "ms_per_step": round(ms / wl.steps, 3),
                            "fgmres_its_per_step": round(sum(s["fgmres_its"] for s in stats) / wl.steps, 2)}
        finals[key] = (tabo, u.cpu().numpy())
        sv.close()
    return res, finals


def config4_leg(args):
    """The adjoint workload: 512^2 Q1, lognormal kappa seed 1, RadauIIA(3), dt 1/100, 50 steps, checkpoints
    every 10 steps, FP32 V-cycles inside FP64 FGMRES.  Times the forward loop alone and the forward loop
    plus the checkpointed adjoint (J = 1/2 ||u_N - u*||_M^2, gradient in log kappa)."""
    import torch

    from paper_2403_08084_gb300 import adjoint as AD

    wl = W.WORKLOADS["adjoint2d-512"]
    sv, tab = make_solver(wl, "lower", wl.vcycle, "cgs2", None, "ai")
    u0 = torch.from_numpy(W.sine_initial(2, wl.N)).cuda()
    f = torch.from_numpy(W.sine_load_space(2, wl.N)).cuda()
    kap = W.lognormal_kappa(2, wl.N, 0.5, wl.kappa_seed)
    theta0 = torch.from_numpy(np.log(kap)).cuda()

    def coef(n):
        return [W.sine_load_time(2, (n + c) * wl.dt) for c in tab.c]

    ut = torch.zeros_like(u0)  # target: the final state with kappa = 1
    sv.set_kappa(np.ones(wl.N * wl.N))
    ut.copy_(u0)
    run_steps(sv, tab, wl, ut, f, 0, wl.steps)
    sv.set_kappa(kap)
    fwd_ms, fstats, _ = timed_steps(sv, tab, wl, u0, f, wl.steps, 2)

    def fwd_bwd():
        th = theta0.clone().requires_grad_(True)
        J = AD.mass_norm2(sv, AD.trajectory(sv, th, u0, wl.steps, f_space=f, f_coef=coef, checkpoint=10) - ut)
        J.backward()
        return th.grad

    fwd_bwd()  # warm-up (CUDA graphs of the transposed iterations)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    g = fwd_bwd()
    torch.cuda.synchronize()
    fb_s = time.perf_counter() - t0
    adj_its = list(sv.adjoint_its)
    sv.close()
    return {"workload": wl.name, "mesh": f"{wl.N}x{wl.N} Q1", "dt": wl.dt, "steps": wl.steps, "levels": wl.levels,
            "checkpoint": 10, "vcycle": wl.vcycle, "rtol": wl.rtol, "precond": "lower (AI form; P_L^T in the adjoint)",
            "forward_steps_per_s": round(wl.steps / (fwd_ms / 1e3), 3),
            "forward_fgmres_its_per_step": round(sum(s["fgmres_its"] for s in fstats) / wl.steps, 2),
            "forward_plus_adjoint_s": round(fb_s, 4),
            "forward_plus_adjoint_steps_per_s": round(wl.steps / fb_s, 3),
            "adjoint_fgmres_its_per_step": round(sum(adj_its) / max(len(adj_its), 1), 2),
            "adjoint_share": round(1.0 - 2.0 * (fwd_ms / 1e3) / fb_s, 3),
            "timing": "forward: CUDA events; forward + adjoint: wall clock around J.backward() (forward with "
                      "checkpoints, recomputation of each segment, reverse sweep)",
            "grad_norm": float(torch.linalg.vector_norm(g).item())}


# ----------------------------------------------------------------------------
# the oracle side: CPU baseline timing and the L2 comparison with the GPU states
# ----------------------------------------------------------------------------
def oracle_stepper(wl, N, levels, kind, split, tableau=None):
    """The oracle's FGMRES + sparse V-cycle restatement of one RK step (AI or IA form) on an N^dim mesh.
    Returns (one, u0, disc) with one(u, n, rtol, x0=None) -> (u_next, k (s, n), w, its); rtol is relative
    to the right-hand side's norm also when FGMRES starts from x0 (a refinement of an earlier solve)."""
    from oracle import fem, krylov, mg, rk
    from oracle import tableaux as OT

    name, s = tableau_of(wl, tableau)
    kap = W.lognormal_kappa(wl.dim, N, 0.5, wl.kappa_seed) if wl.kappa_seed is not None else None
    d = fem.Discretisation(wl.dim, N, kap)
    h = mg.Hierarchy(d, levels)
    ot = OT.by_name(name, s)
    Ap = krylov.rana_ld(ot.A) if kind == "rana_ld" else ot.A
    if kind == "monolithic":  # AI form only
        S = rk.kronecker_operator(d.M, d.K, ot.A, wl.dt)
        P = mg.MonolithicVCycle(h, ot.A, wl.dt)
        Ainv = np.eye(s)
    elif split == "ia":
        T = np.diag(np.diag(Ap)) if kind == "diag" else np.tril(Ap)
        solves = [mg.VCycle(h, wl.dt * T[i, i]) for i in range(s)]
        S = krylov.ia_operator(d.M, d.K, ot.A, wl.dt)
        P = krylov.IABlockPreconditioner(T, d.M, wl.dt, solves, diagonal_only=(kind == "diag"))
        Ainv = np.linalg.inv(ot.A)
    else:
        solves = [mg.VCycle(h, wl.dt * Ap[i, i]) for i in range(s)]
        S = rk.kronecker_operator(d.M, d.K, ot.A, wl.dt)
        P = krylov.BlockPreconditioner("lower" if kind == "rana_ld" else kind, Ap, d.K, wl.dt, solves)
        Ainv = np.eye(s)
    Fs = d.to_interior(W.sine_load_space(wl.dim, N))

    def one(u, n, rtol, x0=None):
        r = (np.stack([W.sine_load_time(wl.dim, (n + c) * wl.dt) * Fs for c in ot.c])
             - (d.K @ u)[None, :]).reshape(-1)
        rt = rtol
        if x0 is not None:
            r0 = np.linalg.norm(r - S @ x0)
            rt = rtol * np.linalg.norm(r) / r0 if r0 > 0 else 1.0
        w, its, _, _ = krylov.fgmres(lambda v: S @ v, r, P, rtol=min(rt, 1.0), x0=x0)
        k = Ainv @ w.reshape(s, -1)
        return u + wl.dt * (ot.b @ k), k, w, its

    return one, d.to_interior(W.sine_initial(wl.dim, N)), d


def compare(d, s, ref_u, ref_k, gpu):
    """Element-wise comparison of a GPU step (u_1 and node-major k on the full grid) with the oracle's."""
    ug, kg = gpu
    e = d.to_interior(ug) - ref_u
    mref = float(ref_u @ (d.M @ ref_u))
    out = {"u1_rel_l2_M": math.sqrt(max(float(e @ (d.M @ e)), 0.0) / mref),
           "u1_max_abs": float(np.abs(e).max()), "u1_max_abs_rel": float(np.abs(e).max() / np.abs(ref_u).max())}
    if kg is not None:
        ki = d.to_interior(kg, s)  # (s, n)
        ek = ki - ref_k
        out["k_rel_l2"] = float(np.linalg.norm(ek) / np.linalg.norm(ref_k))
        out["k_max_abs_rel"] = float(np.abs(ek).max() / np.abs(ref_k).max())
    return out


def cpu_baseline_leg(wl, precond, split, checks, extra_checks, tableau=None):
    """One time step of the workload at full size through the oracle's FGMRES + V-cycle restatement, timed
    on one host core at the workload's rtol; then the same solve continued to rtol 1e-12, which is the
    reference state every GPU first step (headline and variants) is compared with, element by element.
    3D: the timing runs on a 64^3 sample; the eigenmode closed form checks the 128^3 states."""
    from oracle import fem
    from oracle import manufactured as MF
    from oracle import tableaux as OT

    N = wl.N if wl.dim == 2 else min(wl.N, 64)
    levels = wl.levels - int(round(np.log2(wl.N // N)))
    t0 = time.perf_counter()
    one, u0, d = oracle_stepper(wl, N, levels, precond, split, tableau)
    setup = time.perf_counter() - t0
    t0 = time.perf_counter()
    u1, k1, w1, its = one(u0, 0, wl.rtol)
    dt = time.perf_counter() - t0
    scale = ((N + 1) / (wl.N + 1)) ** wl.dim
    where = "at full size" if N == wl.N else f"on a {N}^{wl.dim} sample, steps/s scaled by the DOF ratio {scale:.4f}"
    name, s = tableau_of(wl, tableau)
    base = {"value": round(scale / dt, 6), "unit": "time-steps/s", "cores": 1, "kind": "oracle",
            "sample": f"1 time step of {wl.name} {where} (oracle FGMRES + sparse V-cycle, {split.upper()} form, "
                      f"{precond}, FP64, rtol {wl.rtol:g}; {its} its; setup {setup:.1f} s excluded)",
            "seconds": round(dt, 2), "setup_s": round(setup, 2)}
    l2 = {"reference": "the oracle's FGMRES continued from its timed solve to ||r|| <= 1e-12 ||r_0|| (FP64, CPU), "
                       "one step from the same u_0; GPU runs at the workload's rtol",
          "norms": "u1_rel_l2_M = ||u_gpu - u_ref||_M / ||u_ref||_M over interior nodes; max-abs element-wise"}
    if N == wl.N:
        u1r, k1r, _, its2 = one(u0, 0, 1e-12, x0=w1)
        l2["oracle_extra_its"] = its2
        l2["runs"] = {key: compare(d, s, u1r, k1r, val) for key, val in checks.items() if val is not None}
    if "config2" in extra_checks:
        wl2 = W.WORKLOADS["heat2d-1024-radau3"]
        one2, u02, d2 = oracle_stepper(wl2, wl2.N, wl2.levels, "lower", "ia")
        u1a, _, w1a, _ = one2(u02, 0, wl2.rtol)
        u1r2, k1r2, _, _ = one2(u02, 0, 1e-12, x0=w1a)
        l2["config2"] = {key: compare(d2, wl2.s, u1r2, k1r2, val) for key, val in extra_checks["config2"].items()}
    if "config3" in extra_checks:
        wl3 = W.WORKLOADS["heat3d-128"]
        S3 = W.sine_initial(3, wl3.N)
        res3 = {}
        for key, ((tname, ts), u) in extra_checks["config3"].items():
            ot = OT.by_name(tname, ts)
            a = MF.scalar_rk_amplitudes(3, wl3.N, ot.A, ot.b, ot.c, wl3.dt, wl3.steps)
            ex = a[-1] * S3
            res3[key] = {"u_final_rel_l2": float(np.linalg.norm(u - ex) / np.linalg.norm(ex)),
                         "u_final_max_abs_rel": float(np.abs(u - ex).max() / np.abs(ex).max())}
        l2["config3"] = {"reference": "exact discrete solution a_N S (the sine eigenmode stays an eigenmode; a_N "
                                      "from the oracle's scalar RK recursion), after all 10 steps", "runs": res3}
    _ = fem
    return base, l2


# ----------------------------------------------------------------------------
# reference arm: the FP64 CPU oracle
# ----------------------------------------------------------------------------
def reference_arm(args):
    wl = W.WORKLOADS[args.workload]
    # bounded sample: the same workload on a mesh of at most 513^2 nodes (65^3 in 3D), fewer levels, so that
    # every step is about a second of CPU work; throughput is scaled to the full DOF count
    Ns = min(wl.N, 512) if wl.dim == 2 else min(wl.N, 64)
    lv = max(1, wl.levels - int(round(np.log2(wl.N // Ns))))
    split = args.splitting if args.precond not in ("upper", "monolithic") else "ai"
    vcycle = args.vcycle or wl.vcycle
    if vcycle == "exact":
        vcycle = "fp64"
    one, u0, _ = oracle_stepper(wl, Ns, lv, args.precond, split, args.tab_override)

    u = u0.copy()
    for n in range(args.warmup):
        u = one(u, n, wl.rtol)[0]
    u = u0.copy()
    t0 = time.perf_counter()
    its = []
    for n in range(args.steps):
        u, _, _, it = one(u, n, wl.rtol)
        its.append(it)
    dt = time.perf_counter() - t0
    scale = ((Ns + 1) ** wl.dim) / ((wl.N + 1) ** wl.dim)
    value = args.steps / dt * scale
    sample = (f"each step: one RK step of {wl.name} on a {Ns}^{wl.dim} mesh ({lv} levels), oracle FGMRES + sparse "
              f"V-cycle, {split.upper()} form, {args.precond}, FP64 throughout; steps/s scaled by the DOF ratio "
              f"{scale:.4f}")
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
        "config": workload_config(wl, args, vcycle, args.precond, split, args.gpus),
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
    multigrid; the IA and monolithic forms also warm-started), each with FP64 and FP32 V-cycles,
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

    def integrate(tab, nsteps, vcycle, solver, rtol, split="ai", precond="lower", warm=False):
        dt = T / nsteps
        t0 = time.perf_counter()
        sv = Solver(N, tab, dt, kappa=kap, levels=wl.levels, precond=precond, vcycle=vcycle, rtol=rtol,
                    solver=solver, restart=RESTART, maxit=2000, splitting=split, warm_start=warm)
        torch.cuda.synchronize()
        setup = time.perf_counter() - t0
        u = u0.clone()
        for n in range(min(2, nsteps)):  # warm-up: CUDA-graph capture of the first iterations
            sv.step(u, u, f_space=f, f_coef=[W.sine_load_time(2, (n + c) * dt) for c in tab.c])
        u.copy_(u0)
        sv.reset_initial_guess()
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

    sweep = (2, 4, 8, 16, 32, 64)
    forms = [("RadauIIA(3) IA", PT.radau_iia(3), "fgmres", sweep, "ia", "lower", False),
             ("RadauIIA(3) AI", PT.radau_iia(3), "fgmres", sweep, "ai", "lower", False),
             ("RadauIIA(3) monolithic MG", PT.radau_iia(3), "fgmres", sweep, "ai", "monolithic", False),
             ("RadauIIA(3) IA warm start", PT.radau_iia(3), "fgmres", sweep, "ia", "lower", True),
             ("RadauIIA(3) monolithic MG warm start", PT.radau_iia(3), "fgmres", sweep, "ai", "monolithic", True),
             ("Alexander SDIRK", PT.alexander(), "dirk_cg", (10, 25, 50, 100, 200, 400), "ai", "lower", False)]
    rows = []
    for label, tab, solver, sweep, split, precond, warm in forms:
        for vcycle in ("fp64", "fp32"):
            for nsteps in sweep:
                u, wall, setup, its = integrate(tab, nsteps, vcycle, solver, wl.rtol, split, precond, warm)
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
        for label, *_ in forms:
            for vcycle in ("fp64", "fp32"):
                entry[f"{label} {vcycle}"] = time_at(label, vcycle, target)
        matched.append(entry)
    return {"study": "long-horizon time-to-solution at equal final L2 error",
            "workload": wl.name, "mesh": f"{N}x{N} Q1", "dofs": (N + 1) ** 2, "T": T, "rtol": wl.rtol,
            "levels": wl.levels, "precond": "P_L (RadauIIA, IA and AI forms) or monolithic MG; per-stage V(2,2)-PCG (SDIRK)",
            "warm_start": "FGMRES starts from the previous step's stages (stopping test still relative to the step's "
                          "right-hand side); the other forms start from zero",
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
