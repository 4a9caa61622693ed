#!/usr/bin/env python
"""Solve throughput of the structured multigrid solver on one GB300.

Workload (default): the quarter annulus r in [1/2, 1] mapped from [0,1]^2,
4097 x 4097 nodes (16,769,025 interior DoF), kappa = exp(g) with g a
64-mode random-Fourier Gaussian field (sigma 1, correlation length 0.05,
seed 1), f ~ U[-1,1].  One step = one solve of A x = f from x0 = 0 to a
verified relative residual of 1e-10 (FP32 V(1,1)-cycle preconditioner,
FP64 flexible CG); the hierarchy is built once, before timing.  The plain
FP64 V-cycle solve is timed the same way and reported beside it.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Prints one JSON line (rank 0).  With N > 1 (torchrun), every rank solves
its own replica (no data-path collective): weak scaling.
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
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "DoF/s to 1e-10 rel. residual, FP32-precond vs FP64 on same GB300; % HBM peak"
UNIT = "DoF/s"
TOL = 1e-10
# the sources of the roofline kernels (the streaming V-cycle kernels): the
# committed DRAM traffic is used only while these are unchanged
KERNEL_FILES = ["paper_2509_08109_gb300/csrc/fused2d.cu", "paper_2509_08109_gb300/csrc/fused2d.cuh",
                "paper_2509_08109_gb300/csrc/mbar.cuh", "paper_2509_08109_gb300/csrc/common.cuh"]


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="own", choices=["own", "reference"])
    ap.add_argument("--n", type=int, default=4097)
    ap.add_argument("--cpu-sample-n", type=int, default=1025)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-table", action="store_true",
                    help="time the oracle (plain C, FP64 PCG to 1e-10) on the host cores for every configuration, "
                         "single-threaded and on all cores of the affinity set; prints one JSON line, no GPU work")
    ap.add_argument("--variants", default="all", choices=["all", "fp64"],
                    help="fp64: time only the plain FP64 solve of the annulus workload (a short line for "
                         "profiling the FP64 kernels)")
    ap.add_argument("--shell-n", type=int, default=257,
                    help="nodes per side of the shell workload (smaller values for profiling captures)")
    ap.add_argument("--batch-count", type=int, default=512,
                    help="problems of the batch workload (512 is the configuration; fewer: the first problems of "
                         "the same stream, for profiling captures on a small device footprint)")
    ap.add_argument("--no-configs", action="store_true",
                    help="skip the compact runs of the other configurations (65^2 annulus, 257^3 shell, "
                         "512-problem batch, 1025^2 adjoint batch) that the default line carries")
    ap.add_argument("--no-autotune", action="store_true",
                    help="keep the occupancy-model tile shapes instead of the device-timed ones")
    ap.add_argument("--no-graphs", action="store_true",
                    help="launch every kernel on the stream instead of replaying the per-iteration CUDA graphs "
                         "(for profilers that replay single kernels)")
    ap.add_argument("--workload", default="annulus", choices=["annulus", "annulus65", "shell", "batch", "adjoint", "aux"],
                    help="annulus: the 4097^2 quarter annulus (default, the headline); annulus65: 65^2 plain; "
                         "shell: 257^3 spherical-shell octant; batch: 512 bump-map problems x 4 rhs; "
                         "adjoint: 1025^2 annulus, batch 8, forward + adjoint; aux: the auxiliary-space two-grid "
                         "method on a 1.07 M-vertex P1 mesh of the annulus with the 513^2 grid as coarse level")
    return ap.parse_args()


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def config_for(n: int, graphs: bool = True) -> dict:
    stencil_mb = 5 * 8 * n * n / 1e6
    return {"workload": f"quarter_annulus_lognormal_kappa_n{n}", "nodes_per_side": n, "dof": (n - 2) ** 2,
            "map": "x=(1/2+s/2)cos(pi t/2), y=(1/2+s/2)sin(pi t/2)",
            "kappa": "exp(64-mode Gaussian field, sigma 1, corr 0.05, seed 1)", "rhs": "U[-1,1] seed 1",
            "cycle": "V(1,1), 4-colour GS, operator-induced P, Galerkin RAP, coarsest 3x3",
            "outer": "FP32 V-cycle preconditioner with FP64 residual: iterative refinement (FP32 inner CG) or "
                     "FP64 flexible CG, the faster is the headline (headline_variant); plain FP64 CG + FP64 "
                     "V-cycle in the fp64 field",
            "tol": TOL, "l2": f"inputs larger than L2 (FP64 stencil {stencil_mb:.0f} MB > 129 MB), no flush",
            "launch": "per-iteration CUDA graphs" if graphs else "stream launches (no graphs)"}


# ---------------------------------------------------------------- clocks
class Clocks:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None
        self.result = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self) -> dict | None:
        if self.proc is None:
            return None
        time.sleep(0.12)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = max(smax, float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------- helpers
def kernel_hash() -> str:
    h = hashlib.sha1()
    for f in KERNEL_FILES:
        p = os.path.join(ROOT, f)
        if os.path.exists(p):
            h.update(open(p, "rb").read())
    return h.hexdigest()[:12]


def traffic_for(kernel: str, n: int):
    """DRAM bytes per launch of `kernel` from the committed ncu summary, if
    it was taken on the current kernel sources (else None)."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return None
    try:
        d = json.load(open(path))
    except ValueError:
        return None
    if d.get("kernel_hash") != kernel_hash():
        return None
    ent = d.get("kernels", {}).get(kernel)
    if not ent or ent.get("n") != n:
        return None
    return ent.get("dram_bytes_per_launch")


def cpu_model() -> str:
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    return "unknown"


def cpu_baseline(n_sample: int, n_full: int) -> dict:
    """The oracle (plain FP64 C) on the host cores: one PCG solve to 1e-10
    of the full workload on every core of the process's affinity set (the
    OpenMP build, whose results are bitwise the plain build's), and, beside
    it, the single-threaded build on a sample of the same recipe at n_sample
    nodes per side (hierarchies built beforehand, outside the timings)."""
    import oracle
    from paper_2509_08109_gb300 import inputs
    cores = len(os.sched_getaffinity(0))
    oracle.threads(cores)
    p = inputs.annulus_lognormal(n_full)
    H = oracle.Hierarchy(oracle.assemble(p.coords, p.kappa), omp=True)
    t = time.perf_counter()
    x, it, hist, trr, st = H.pcg(p.rhs, tol=TOL, maxit=500)
    dt = time.perf_counter() - t
    assert st == 0 and trr <= TOL, (st, trr)
    del H, x, p
    q = inputs.annulus_lognormal(n_sample)
    H1 = oracle.Hierarchy(oracle.assemble(q.coords, q.kappa))
    t = time.perf_counter()
    x1, it1, _, trr1, st1 = H1.pcg(q.rhs, tol=TOL, maxit=500)
    dt1 = time.perf_counter() - t
    assert st1 == 0 and trr1 <= TOL
    dof = (n_full - 2) ** 2
    return {"value": dof / dt, "unit": UNIT, "cores": cores, "kind": "oracle", "cpu": cpu_model(),
            "sample": f"one PCG solve to 1e-10 of the full workload (n={n_full}, {dof} DoF, {it} iterations, "
                      f"{dt:.2f} s) on {cores} cores, OpenMP build of the C oracle (bitwise the plain build)",
            "single_thread": {"value": q.unknowns / dt1, "cores": 1,
                              "sample": f"plain single-threaded oracle, same recipe at n={n_sample} "
                                        f"({q.unknowns} DoF, {it1} iterations, {dt1:.2f} s)"}}


def cpu_table(args) -> dict:
    """The oracle on the host cores for every configuration: the OpenMP build
    on every core of the affinity set (bitwise the plain build's results)
    and the plain single-threaded build, each solving to a verified 1e-10
    with FP64 PCG. The solve times exclude assembly and hierarchy setup,
    which are reported beside them, except for the adjoint workload, whose
    metric counts each member's assembly, setup, forward solve, adjoint
    solve and contraction, as the library's timing of it does. Where a
    single-threaded run of the full workload would take many minutes, it is
    timed on a named sample of the same recipe and says so."""
    import oracle
    from paper_2509_08109_gb300 import inputs
    cores = len(os.sched_getaffinity(0))
    oracle.threads(cores)
    out = {"cpu": cpu_model(), "cores": cores, "unit": UNIT, "tol": TOL}

    def solve(p, omp, reps=1, maxit=500):
        t = time.perf_counter()
        H = oracle.Hierarchy(oracle.assemble(p.coords, p.kappa), omp=omp)
        setup = time.perf_counter() - t
        times = []
        for _ in range(reps):
            t = time.perf_counter()
            x, it, _, trr, st = H.pcg(p.rhs, tol=TOL, maxit=maxit)
            times.append(time.perf_counter() - t)
            assert st == 0 and trr <= TOL, (p.name, st, trr)
        dt = statistics.median(times)
        return {"value": p.unknowns / dt, "solve_s": dt, "iterations": it, "setup_s": setup, "dof": p.unknowns,
                "workload": p.name}

    p1 = inputs.annulus_plain(65)
    out["annulus65_plain"] = {"all_cores": solve(p1, True, reps=5), "single_thread": solve(p1, False, reps=5)}
    p2 = inputs.annulus_lognormal(4097)
    out["annulus4097_lognormal"] = {"all_cores": solve(p2, True)}
    del p2
    s2 = solve(inputs.annulus_lognormal(1025), False)
    s2["sample"] = "same recipe at n=1025"
    out["annulus4097_lognormal"]["single_thread"] = s2
    # the full 257^3 solve (508 iterations) would take about ten minutes on
    # all cores of the GPU machine's host: the all-core leg solves the 129^3
    # sample of the same recipe
    p3 = inputs.shell_two_layer(129)
    s3a = solve(p3, True, maxit=4000)
    s3a["sample"] = "same recipe at n=129 (iterations double per refinement on this map)"
    out["shell257"] = {"all_cores": s3a}
    del p3
    s3 = solve(inputs.shell_two_layer(65), False, maxit=4000)
    s3["sample"] = "same recipe at n=65 (iterations double per refinement on this map)"
    out["shell257"]["single_thread"] = s3

    probs = inputs.bump_batch(count=512, nrhs=4, limit=32)
    for key, omp in (("all_cores", True), ("single_thread", False)):
        dof = 0
        solve_s = setup_s = 0.0
        its = []
        for p in probs:
            t = time.perf_counter()
            H = oracle.Hierarchy(oracle.assemble(p.coords, p.kappa), omp=omp)
            setup_s += time.perf_counter() - t
            for r in range(p.rhs.shape[0]):
                t = time.perf_counter()
                x, it, _, trr, st = H.pcg(p.rhs[r], tol=TOL, maxit=500)
                solve_s += time.perf_counter() - t
                assert st == 0 and trr <= TOL
                its.append(it)
                dof += p.unknowns
            del H
        out.setdefault("batch_first32x4", {})[key] = {
            "value": dof / solve_s, "solve_s": solve_s, "setup_s": setup_s, "dof_rhs": dof,
            "iterations_min_max": [min(its), max(its)],
            "workload": "problems 0-31 of the 512-problem bump batch, 4 rhs each, solved one by one (no extrapolation)"}

    members = inputs.annulus_adjoint(1025, batch=8)
    for key, omp, mem in (("all_cores", True, members), ("single_thread", False, members[:1])):
        its = []
        t = time.perf_counter()
        for p in mem:
            H = oracle.Hierarchy(oracle.assemble(p.coords, p.kappa), omp=omp)
            u, iu, _, tru, stu = H.pcg(p.rhs, tol=TOL, maxit=1000)
            lam, il, _, trl, stl = H.pcg(u - p.extra["u_obs"], tol=TOL, maxit=1000)
            assert stu == 0 and stl == 0 and tru <= TOL and trl <= TOL
            g = p.kappa * oracle.adjoint_grad(p.coords, u, lam)
            assert all(map(math.isfinite, g.ravel().tolist()))
            its.append([iu, il])
            del H
        dt = time.perf_counter() - t
        d = {"value": len(mem) * 1023 ** 2 / dt, "wall_s": dt, "members": len(mem), "iterations": its,
             "workload": "1025^2 annulus adjoint: per member assembly, setup, forward solve, adjoint solve, "
                         "gradient contraction"}
        if len(mem) < len(members):
            d["sample"] = f"member 0 of {len(members)}"
        out.setdefault("adjoint1025x8", {})[key] = d
    return out


# ---------------------------------------------------------------- replicas
def whole_job_throughput(local_ms: float, dof_per_rank: int, steps: int, world: int, reduce_max) -> tuple:
    """Weak-scaling replicas: every rank solves its own copy; the job's time
    is the slowest rank's, and the job's throughput counts every rank's
    unknowns.  reduce_max(v) returns the maximum of v over the ranks."""
    ms = reduce_max(local_ms)
    return world * dof_per_rank * steps / (ms * 1e-3), ms


# ---------------------------------------------------------------- own arm
def run_own(args):
    import torch
    import torch.distributed as dist

    from paper_2509_08109_gb300 import binding, inputs

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)

    def barrier():
        if world > 1:
            dist.barrier()

    def max_over_ranks(v: float) -> float:
        if world == 1:
            return v
        t = torch.tensor([v], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())

    n = args.n
    dof = (n - 2) ** 2
    coords, kappa, f = inputs.annulus_lognormal_device(n, dev)
    stream = torch.cuda.current_stream(dev)
    if args.variants == "fp64":
        # only the plain FP64 solve (for profiling its kernels): a short line
        s = binding.Solver(2, n, precision="fp64", outer="cg", device=dev, graphs=not args.no_graphs)
        s.assemble(coords, kappa).setup()
        if not args.no_autotune:
            s.autotune(reps=3)
        ms, launches, infos = _timed_solves(torch, s, f, args.steps, args.warmup)
        assert all(i.true_relres <= TOL for i in infos)
        if rank == 0:
            print(json.dumps({"metric": METRIC, "value": dof / (ms * 1e-3), "unit": UNIT, "n_gpus": world,
                              "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "dtype": "f64",
                              "variants": "fp64 only", "iterations": infos[-1].iterations,
                              "config": config_for(n, not args.no_graphs)}), flush=True)
        return

    def build(prec, outer=None):
        s = binding.Solver(2, n, precision=prec, outer=outer, device=dev, graphs=not args.no_graphs)
        e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        e0.record(stream)
        s.assemble(coords, kappa)
        e1.record(stream)
        s.setup()
        e2.record(stream)
        torch.cuda.synchronize(dev)
        if not args.no_autotune:
            s.autotune(reps=3)     # device-timed tile shapes, outside the timed region
        return s, e0.elapsed_time(e1), e1.elapsed_time(e2)

    sir, asmir, setir = build("fp32", "refine")
    s32, asm32, set32 = build("fp32", "flexible")
    s64, asm64, set64 = build("fp64", "cg")
    x = torch.zeros_like(f)

    def timed(s, k, profile=False, clocks=None):
        for _ in range(args.warmup):
            s.solve(f, tol=TOL, out=x)
        if profile:
            s.profile(True)
        l0 = s.launches
        barrier()
        torch.cuda.synchronize(dev)
        if clocks:
            clocks.start()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        infos = []
        torch.cuda.nvtx.range_push(f"timed_{s.precision}_{s.outer}")
        a.record(stream)
        for _ in range(k):
            _, info = s.solve(f, tol=TOL, out=x)
            infos.append(info)
        b.record(stream)
        torch.cuda.synchronize(dev)
        torch.cuda.nvtx.range_pop()
        barrier()
        ck = clocks.stop() if clocks else None
        ms = a.elapsed_time(b)
        prof = s.profile_read() if profile else {}
        if profile:
            s.profile(False)
        return max_over_ranks(ms), s.launches - l0, infos, prof, ck

    clk = Clocks(local)
    msir, launchesir, infosir, _, ckir = timed(sir, args.steps, clocks=clk)
    msf, launchesf, infosf, _, ckf = timed(s32, args.steps, clocks=Clocks(local))
    ms64, launches64, infos64, _, _ = timed(s64, args.steps)
    # kernel-class durations: a second pass over the same workload with CUDA
    # events around every finest-level launch (launched directly, not from the
    # iteration graphs, so each launch can be bracketed)
    _, _, _, profir, _ = timed(sir, args.steps, profile=True)
    _, _, _, proff, _ = timed(s32, args.steps, profile=True)
    _, _, _, prof64, _ = timed(s64, max(1, min(args.steps, 3)), profile=True)
    assert all(i.true_relres <= TOL for i in infosir + infosf + infos64)
    variants = {"refine": (msir, launchesir, infosir, profir, ckir, sir),
                "flexible": (msf, launchesf, infosf, proff, ckf, s32)}
    head = min(variants, key=lambda k: variants[k][0])
    ms32, launches32, infos32, prof32, ck, shead = variants[head]
    t32 = ms32 / args.steps
    t64 = ms64 / args.steps
    value, _ = whole_job_throughput(t32, dof, 1, world, lambda v: v)   # ms32 is already the max over ranks

    # end to end through the public API with host (pinned) buffers
    fh = f.cpu().pin_memory()
    xh = torch.zeros_like(fh).pin_memory()
    for _ in range(args.warmup):
        shead.solve(fh, tol=TOL, out=xh)
    barrier()
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        xh.zero_()
        shead.solve(fh, tol=TOL, out=xh)
    torch.cuda.synchronize(dev)
    e2e_s = max_over_ranks(time.perf_counter() - t0)
    e2e = {"value": world * dof * args.steps / e2e_s, "unit": UNIT,
           "h2d_bytes_per_step": 2 * fh.numel() * 8, "d2h_bytes_per_step": xh.numel() * 8}

    # roofline of the dominant kernel class of the finest level
    hbm, peak_kind = peaks()
    dom = max(prof32.items(), key=lambda kv: kv[1][0]) if prof32 else None
    roof = None
    if dom:
        name, (kms, nl, kbytes) = dom
        achieved = kbytes / (kms * 1e-3) / 1e9
        roof = {"bound": "hbm", "kernel": name, "achieved": round(achieved, 1), "peak": hbm,
                "peak_source": f"{peak_kind} hbm_gbs", "unit": "GB/s", "frac": round(achieved / hbm, 4),
                "traffic": traffic_for(name, n), "launches": nl, "avg_launch_ms": round(kms / nl, 4),
                "algorithmic_bytes_per_launch": kbytes / nl,
                "share_of_step": round(kms / ms32, 4),
                "measured_in": "profiled pass of the same workload (CUDA events on the library stream)"}
    kclasses = {k: {"ms_per_step": round(v[0] / args.steps, 4), "launches_per_step": v[1] / args.steps,
                    "GB/s": round(v[2] / (v[0] * 1e-3) / 1e9, 1)} for k, v in prof32.items()}

    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": t32, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f32 V-cycle / f64 residual", "data": "synthetic",
           "config": dict(config_for(n, not args.no_graphs),
                          tiles=("autotuned" if not args.no_autotune else "occupancy model") +
                          ", finest level wc x hc (down, up) = {} x ({}, {})".format(*sir.tiles()[0])),
           "e2e": e2e, "gpu_launches": launches32,
           "headline_variant": head,
           "iterations": infos32[-1].iterations, "true_relres": infos32[-1].true_relres,
           "fp32_variants": {k: {"value": world * dof / (v[0] / args.steps * 1e-3), "ms_per_step": v[0] / args.steps,
                                 "iterations": v[2][-1].iterations, "refinements": v[2][-1].refinements,
                                 "true_relres": v[2][-1].true_relres, "gpu_launches": v[1]}
                             for k, v in variants.items()},
           "fp64": {"value": world * dof / (t64 * 1e-3), "ms_per_step": t64, "iterations": infos64[-1].iterations,
                    "gpu_launches": launches64, "true_relres": infos64[-1].true_relres},
           "fp32_over_fp64": t64 / t32,
           "setup_ms": {"fp32_refine": {"assemble": asmir, "setup": setir},
                        "fp32_flexible": {"assemble": asm32, "setup": set32},
                        "fp64": {"assemble": asm64, "setup": set64}},
           "roofline": roof, "kernel_classes_finest_level": kclasses, "clocks": ck}
    out["fp64"]["roofline"] = fp64_roofline(prof64, max(1, min(args.steps, 3)), dof)
    del sir, s32, s64
    torch.cuda.empty_cache()
    if rank == 0 and world == 1 and not args.no_configs:
        out["configs"] = other_configs(args)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(args.cpu_sample_n, n)
    if rank == 0:
        print(json.dumps(out), flush=True)
    if world > 1:
        dist.destroy_process_group()


# FP64 floating-point operations per interior node of one launch of each
# finest-level class of the plain FP64 solve, counted by ncu
# (smsp__sass_thread_inst_executed_op_{dfma,dmul,dadd}_pred_on, an FMA as two)
# on the 2049^2 annulus: profiles/vdown64_annulus2049_fp64.md.  The FP64
# kernels of this path are bound by the FP64 rate rather than by HBM; their
# roofline is the FP64 peak.
FP64_FLOPS_PER_NODE = {"vdown": 36.81, "vup": 39.28, "spmv": 19.45, "update": 6.52}
# GB300 FP64 (non-tensor) peak, nominal: 1.25 TFLOP/s
FP64_PEAK_GFLOPS = 1250.0


def fp64_roofline(prof, steps, dof):
    """Per finest-level class of the FP64 solve: time per solve, algorithmic
    bytes against the HBM peak and, where the FP64 operation count per node
    was measured, FLOP/s against the FP64 peak; the dominant class names the
    bound that is nearer."""
    if not prof:
        return None
    hbm, kind = peaks()
    classes = {}
    for k, (kms, nl, kbytes) in prof.items():
        gbs = kbytes / (kms * 1e-3) / 1e9
        e = {"ms_per_solve": round(kms / steps, 4), "launches": nl, "GB/s": round(gbs, 1),
             "hbm_frac": round(gbs / hbm, 4)}
        if k in FP64_FLOPS_PER_NODE:
            gfl = FP64_FLOPS_PER_NODE[k] * dof * nl / (kms * 1e-3) / 1e9
            e["GFLOP/s"] = round(gfl, 1)
            e["fp64_frac"] = round(gfl / FP64_PEAK_GFLOPS, 4)
        classes[k] = e
    dom = max(prof, key=lambda k: prof[k][0])
    d = classes[dom]
    if "fp64_frac" in d and d["fp64_frac"] > d["hbm_frac"]:
        roof = {"bound": "alu", "kernel": dom, "achieved": d["GFLOP/s"], "peak": FP64_PEAK_GFLOPS,
                "unit": "GFLOP/s", "frac": d["fp64_frac"], "peak_source": "nominal FP64 rate (1.25 TFLOP/s)"}
    else:
        roof = {"bound": "hbm", "kernel": dom, "achieved": d["GB/s"], "peak": hbm, "unit": "GB/s",
                "frac": d["hbm_frac"], "peak_source": f"{kind} hbm_gbs"}
    roof["classes"] = classes
    return roof


def other_configs(args) -> dict:
    """Compact runs of the other configurations, each with its clocks, so
    that one default bench line carries every configuration's number."""
    from paper_2509_08109_gb300 import inputs as _inp
    out = {}

    def keep(r, extra=()):
        d = {k: r.get(k) for k in ("value", "unit", "ms_per_step", "steps", "warmup", "headline_variant",
                                    "fp32_over_fp64", "clocks", "gpu_launches") if k in r}
        d["workload"] = r["config"]["workload"]
        for k in extra:
            if k in r:
                d[k] = r[k]
        return d

    r1 = run_single(args, 2, 65, _inp.annulus_plain(65), "quarter_annulus_plain_n65", steps=10, warmup=3, emit=False)
    out["annulus65_plain"] = keep(r1)
    out["annulus65_plain"]["variants"] = {k: {"value": v["value"], "ms_per_step": v["ms_per_step"],
                                              "iterations": v["iterations"]} for k, v in r1["variants"].items()}
    r3 = run_single(args, 3, 257, _inp.shell_two_layer(257), "shell_octant_two_layer_n257", steps=1, warmup=1,
                    emit=False)
    out["shell257"] = keep(r3)
    out["shell257"]["variants"] = {k: {"value": v["value"], "ms_per_step": v["ms_per_step"],
                                       "iterations": v["iterations"], "clocks": v["clocks"]}
                                   for k, v in r3["variants"].items()}
    r4 = run_batch(args, steps=2, warmup=1, emit=False)
    out["batch512x4"] = keep(r4, ("e2e", "iterations_min_max", "worst_true_relres"))
    r5 = run_adjoint(args, steps=2, warmup=1, emit=False)
    out["adjoint1025x8"] = keep(r5, ("fp64_serial", "grad_rel_diff_between_legs"))
    out["adjoint1025x8"]["metric"] = r5["metric"]
    return out


# ---------------------------------------------------------------- reference arm
def run_reference(args):
    """The oracle, as it stands, on the host cores: each step is one PCG
    solve to 1e-10 of the full workload (the same n as the own arm), on
    every core of the process's affinity set (OpenMP build of the oracle,
    bitwise the plain build's results); at most one warm-up solve (the CPU
    code has nothing to warm beyond its first pass)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    from paper_2509_08109_gb300 import inputs
    cores = len(os.sched_getaffinity(0))
    oracle.threads(cores)
    p = inputs.annulus_lognormal(args.n)
    H = oracle.Hierarchy(oracle.assemble(p.coords, p.kappa), omp=True)
    for _ in range(min(args.warmup, 1)):
        H.pcg(p.rhs, tol=TOL, maxit=500)
    t = time.perf_counter()
    for _ in range(args.steps):
        x, it, hist, trr, st = H.pcg(p.rhs, tol=TOL, maxit=500)
        assert st == 0
    dt = time.perf_counter() - t
    value = p.unknowns * args.steps / dt
    sample = (f"one PCG solve to 1e-10 of the full workload per step (n={args.n}, {p.unknowns} DoF), "
              f"OpenMP build of the C oracle on {cores} cores ({cpu_model()})")
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
           "steps": args.steps, "warmup": min(args.warmup, 1), "ms_per_step": dt / args.steps * 1e3,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": config_for(args.n),
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


# ---------------------------------------------------------------- other workloads
def _timed_solves(torch, s, f, steps, warmup, tol=TOL, maxit=500, clocks=None):
    x = torch.zeros_like(f)
    for _ in range(warmup):
        s.solve(f, tol=tol, out=x, maxit=maxit)
    torch.cuda.synchronize()
    l0 = s.launches
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    infos = []
    if clocks:
        clocks.start()
    torch.cuda.nvtx.range_push(f"timed_{s.precision}_{s.outer}")
    a.record(s.stream)
    for _ in range(steps):
        _, info = s.solve(f, tol=tol, out=x, maxit=maxit)
        infos.append(info)
    b.record(s.stream)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    if clocks:
        clocks.result = clocks.stop()
    return a.elapsed_time(b) / steps, s.launches - l0, infos


def run_single(args, dim, n, problem, name, steps=None, warmup=None, emit=True):
    """FP32-preconditioned (refinement, flexible CG) against plain FP64 on
    one problem; clocks sampled during each variant's timed solves."""
    import torch
    from paper_2509_08109_gb300 import binding
    torch.cuda.set_device(0)
    steps = args.steps if steps is None else steps
    warmup = args.warmup if warmup is None else warmup
    out = {"metric": METRIC, "unit": UNIT, "n_gpus": 1, "steps": steps, "warmup": warmup,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "data": "synthetic",
           "config": {"workload": name, "nodes_per_side": n, "dim": dim, "dof": (n - 2) ** dim, "tol": TOL,
                      "timing": "CUDA events around the timed solves (mean over steps)"}}
    f = torch.as_tensor(problem.rhs, device="cuda")
    res = {}
    for prec, outer in (("fp32", "refine"), ("fp32", "flexible"), ("fp64", "cg")):
        s = binding.Solver(dim, n, precision=prec, outer=outer, graphs=not args.no_graphs)
        t0 = time.perf_counter()
        s.assemble(torch.as_tensor(problem.coords), torch.as_tensor(problem.kappa)).setup()
        torch.cuda.synchronize()
        setup_s = time.perf_counter() - t0
        # point Gauss-Seidel on the shell octant loses h-independence (cells
        # degenerate at the polar edge): PCG iterations double per refinement
        clk = Clocks(0)
        ms, launches, infos = _timed_solves(torch, s, f, steps, warmup, maxit=500 if dim == 2 else 4000, clocks=clk)
        assert all(i.true_relres <= TOL for i in infos)
        res[f"{prec}_{outer}"] = {"value": (n - 2) ** dim / (ms * 1e-3), "ms_per_step": ms,
                                  "iterations": infos[-1].iterations, "true_relres": infos[-1].true_relres,
                                  "gpu_launches": launches, "setup_s": setup_s, "clocks": clk.result}
        del s
    head = max(("fp32_refine", "fp32_flexible"), key=lambda k: res[k]["value"])
    out.update({"value": res[head]["value"], "ms_per_step": res[head]["ms_per_step"], "headline_variant": head,
                "dtype": "f32 V-cycle / f64 residual", "variants": res, "clocks": res[head]["clocks"],
                "fp32_over_fp64": res["fp64_cg"]["ms_per_step"] / res[head]["ms_per_step"]})
    if emit:
        print(json.dumps(out), flush=True)
    return out


def run_batch(args, steps=None, warmup=None, emit=True):
    """512 independent bump-map problems (n = 2^k+1, k in 6..10), 4 rhs each,
    FP32 V-cycle with FP64 refinement, solved together by the batch engine
    (bmg_batch_solve: size-class persistent kernels over a device work-list,
    the four right-hand sides of a problem sharing each stencil read, one
    CUDA graph per batch iteration, tiles autotuned per size class)."""
    import torch
    from paper_2509_08109_gb300 import binding, inputs
    torch.cuda.set_device(0)
    steps = args.steps if steps is None else steps
    warmup = args.warmup if warmup is None else warmup
    probs = inputs.bump_batch(count=512, nrhs=4, limit=args.batch_count)
    t0 = time.perf_counter()
    solvers = []
    for p in probs:
        s = binding.Solver(2, p.n, precision="fp32", outer="refine")
        s.assemble(torch.as_tensor(p.coords), torch.as_tensor(p.kappa)).setup()
        solvers.append(s)
    torch.cuda.synchronize()
    setup_s = time.perf_counter() - t0
    t1 = time.perf_counter()
    B = binding.Batch(solvers, graphs=not args.no_graphs)
    torch.cuda.synchronize()
    batch_setup_s = time.perf_counter() - t1
    tune_ms = None
    if not args.no_autotune:
        tune_ms = B.autotune(reps=2)
    bs = [[torch.as_tensor(p.rhs[r], device="cuda").contiguous() for r in range(4)] for p in probs]
    xs = [[torch.zeros_like(b) for b in row] for row in bs]
    dof = sum((p.n - 2) ** 2 for p in probs) * 4
    stream = B.stream

    def zero():
        for row in xs:
            for x in row:
                x.zero_()

    for _ in range(warmup):
        zero()
        B.solve(bs, xs, tol=TOL)
    torch.cuda.synchronize()
    clk = Clocks(0)
    clk.start()
    times, infos = [], None
    l0 = B.launches
    torch.cuda.nvtx.range_push("timed_batch")
    for _ in range(steps):
        zero()
        torch.cuda.synchronize()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        infos = B.solve(bs, xs, tol=TOL)
        b.record(stream)
        torch.cuda.synchronize()
        times.append(a.elapsed_time(b))
    torch.cuda.nvtx.range_pop()
    ck = clk.stop()
    launches = (B.launches - l0) // steps
    worst = max(i.true_relres for row in infos for i in row)
    assert worst <= TOL
    its = [i.iterations for row in infos for i in row]
    ms = statistics.median(times)
    # end to end through the same call with pinned host buffers (the copies
    # and the interleaving are inside the call)
    bh = [[t.cpu().pin_memory() for t in row] for row in bs]
    xh = [[torch.zeros_like(t).pin_memory() for t in row] for row in bh]
    for row in xh:
        for x in row:
            x.zero_()
    B.solve(bh, xh, tol=TOL)
    e2e_t = []
    for _ in range(max(1, min(steps, 3))):
        for row in xh:
            for x in row:
                x.zero_()
        torch.cuda.synchronize()
        t = time.perf_counter()
        B.solve(bh, xh, tol=TOL)
        torch.cuda.synchronize()
        e2e_t.append(time.perf_counter() - t)
    e2e_s = statistics.median(e2e_t)
    nbytes = sum(t.numel() * 8 for row in bh for t in row)
    out = {"metric": METRIC, "value": dof / (ms * 1e-3), "unit": UNIT, "n_gpus": 1, "steps": steps,
           "warmup": warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f32 V-cycle / f64 residual", "data": "synthetic",
           "config": {"workload": "bump_batch_512x4" if len(probs) == 512 else f"bump_batch_first{len(probs)}x4",
                      "problems": len(probs), "rhs_per_problem": 4,
                      "dof_total_all_rhs": dof, "sizes": "n=2^k+1, k~U{6..10}, seed 5", "tol": TOL,
                      "engine": "bmg_batch_solve (size-class persistent kernels, 4 rhs per stencil read, "
                                "one graph per batch iteration)" + (" [no graphs]" if args.no_graphs else ""),
                      "tiles": B.tiles() if not args.no_autotune else "occupancy model",
                      "timing": "CUDA events on the batch stream around bmg_batch_solve, median",
                      "l2": "inputs larger than L2 (about 3 GB of FP32 class operators), no flush"},
           "e2e": {"value": dof / e2e_s, "unit": UNIT, "h2d_bytes_per_step": 2 * nbytes,
                   "d2h_bytes_per_step": nbytes},
           "gpu_launches": launches, "iterations_min_max": [min(its), max(its)],
           "worst_true_relres": worst, "setup_s": setup_s, "batch_attach_s": batch_setup_s,
           "autotune_ms": tune_ms, "clocks": ck}
    del B, solvers, bs, xs, bh, xh
    torch.cuda.empty_cache()
    if emit:
        print(json.dumps(out), flush=True)
    return out


def run_adjoint(args, steps=None, warmup=None, emit=True):
    """1025^2 annulus, per-cell m ~ N(0, 0.5^2), kappa = exp(m), batch 8:
    forward solve + adjoint gradient per member through torch.autograd.
    Timed leg: the members run concurrently (one stream and one solver per
    member, FP32 V-cycle inside FP64 refinement, forward and adjoint solves
    through bmg_solve_many).  Second leg, reported beside it: the plain
    FP64 PCG, members one after the other."""
    import torch
    from paper_2509_08109_gb300 import autograd, binding, inputs
    torch.cuda.set_device(0)
    steps = args.steps if steps is None else steps
    warmup = args.warmup if warmup is None else warmup
    probs = inputs.annulus_adjoint(1025, batch=8)
    coords = torch.as_tensor(probs[0].coords, device="cuda")
    ms_ = [torch.as_tensor(p.extra["m"], device="cuda") for p in probs]
    fs = [torch.as_tensor(p.rhs, device="cuda") for p in probs]
    uo = [torch.as_tensor(p.extra["u_obs"], device="cuda") for p in probs]
    conc = [binding.Solver(2, 1025, precision="fp32", outer="refine", stream=torch.cuda.Stream()) for _ in probs]
    serial = [binding.Solver(2, 1025, precision="fp64", outer="cg") for _ in probs]

    def step(solvers):
        ms = [m.clone().requires_grad_(True) for m in ms_]
        us = autograd.solve_batch(ms, fs, coords, solvers, tol=TOL, maxit=1000)
        loss = sum(0.5 * ((u - o) ** 2).sum() for u, o in zip(us, uo))
        loss.backward()
        return [m.grad for m in ms]

    def timed(solvers, steps):
        for _ in range(warmup):
            step(solvers)
        torch.cuda.synchronize()
        times = []
        launches0 = sum(s.launches for s in solvers)
        for _ in range(steps):
            t = time.perf_counter()
            step(solvers)
            torch.cuda.synchronize()
            times.append(time.perf_counter() - t)
        return statistics.median(times) * 1e3, (sum(s.launches for s in solvers) - launches0) // steps

    clk = Clocks(0)
    clk.start()
    ms, launches = timed(conc, steps)
    ck = clk.stop()
    ms64, _ = timed(serial, max(1, min(steps, 3)))
    g_c = step(conc)
    g_s = step(serial)
    # both legs solve to the same FP64 residual; their gradients agree to
    # the solves' tolerance (relative, max over members)
    agree = max((torch.linalg.vector_norm(a - b) / torch.linalg.vector_norm(b)).item() for a, b in zip(g_c, g_s))
    dof = 8 * 1023 ** 2
    out = {"metric": "forward+adjoint DoF/s (batch 8, each member: assemble, setup, solve, adjoint solve, dA/dkappa)",
           "value": dof / (ms * 1e-3), "unit": UNIT, "n_gpus": 1, "steps": steps, "warmup": warmup,
           "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": "f32 V-cycle / f64 residual", "data": "synthetic",
           "config": {"workload": "annulus_adjoint_n1025_batch8", "tol": TOL,
                      "launch": "members concurrent, one stream each (bmg_solve_many + bmg_adjoint_cells)",
                      "timing": "host wall clock around the autograd step (device synchronised), median"},
           "gpu_launches": launches, "clocks": ck,
           "fp64_serial": {"ms_per_step": ms64, "value": dof / (ms64 * 1e-3), "dtype": "f64",
                           "launch": "members one after the other, plain FP64 PCG"},
           "grad_rel_diff_between_legs": agree}
    del conc, serial
    torch.cuda.empty_cache()
    if emit:
        print(json.dumps(out), flush=True)
    return out


def run_aux(args):
    """The auxiliary-space two-grid method (Sec. 2.2-2.3) on a jittered P1
    triangulation of the quarter annulus with about the paper's largest
    physical size (845 x 1262 = 1,066,390 vertices), the 513^2 structured
    grid as its coarse level (interior nodes / physical DoF = 0.25, near the
    paper's coarsening factor 0.28), lumped mass, damped Jacobi 2/3,
    gamma 1, to a 1e-10 relative residual: the paper's stationary iteration
    of cycles, and flexible CG with one cycle as the preconditioner."""
    import torch
    from paper_2509_08109_gb300 import binding, inputs
    torch.cuda.set_device(0)
    m = inputs.annulus_mesh(845, 1262)
    n = 513
    coords = inputs.coords_quarter_annulus(n)
    t0 = time.perf_counter()
    s = binding.Solver(2, n, precision="fp32", outer="refine", graphs=not args.no_graphs)
    s.assemble(torch.as_tensor(coords), torch.ones((n - 1, n - 1), dtype=torch.float64)).setup()
    t1 = time.perf_counter()
    f = torch.as_tensor(m.f, device="cuda")
    dof = int((~m.dirichlet).sum())
    res = {}
    for name, krylov in (("stationary", False), ("flexible_cg", True)):
        t2 = time.perf_counter()
        a = binding.AuxSolver(s, m, krylov=krylov)
        torch.cuda.synchronize()
        setup_s = time.perf_counter() - t2
        for _ in range(args.warmup):
            a.solve(f, tol=TOL)
        torch.cuda.synchronize()
        times, infos = [], []
        torch.cuda.nvtx.range_push(f"aux_{name}")
        for _ in range(args.steps):
            ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            ev0.record()
            u, info = a.solve(f, tol=TOL)
            ev1.record()
            torch.cuda.synchronize()
            times.append(ev0.elapsed_time(ev1))
            infos.append(info)
        torch.cuda.nvtx.range_pop()
        ms = statistics.median(times)
        assert all(i.status == 0 and i.true_relres <= 1.01 * TOL for i in infos)
        res[name] = {"value": dof / (ms * 1e-3), "ms_per_step": ms, "iterations": infos[-1].iterations,
                     "true_relres": infos[-1].true_relres, "setup_s": setup_s}
        del a
    # coarse-grid scaling (Sec. 2.4): k = 12 generalized Lanczos steps, each
    # one P^T A_p P product and one coarse PCG solve
    a = binding.AuxSolver(s, m)
    a.estimate_gamma(k=12)
    torch.cuda.synchronize()
    t3 = time.perf_counter()
    gamma, alpha, _ = a.estimate_gamma(k=12)
    torch.cuda.synchronize()
    gamma_ms = (time.perf_counter() - t3) * 1e3
    del a
    head = max(res, key=lambda k: res[k]["value"])
    out = {"metric": "physical DoF/s to 1e-10 rel. residual (auxiliary-space two-grid, BoxMG coarse level)",
           "value": res[head]["value"], "unit": UNIT, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": res[head]["ms_per_step"], "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64 (physical level) / f32 V-cycle (coarse level)", "data": "synthetic",
           "config": {"workload": "aux_annulus_p1_845x1262_coarse513", "physical_dof": dof,
                      "coarse_dof": (n - 2) ** 2, "triangles": int(m.tri.shape[0]), "tol": TOL,
                      "relaxation": "damped Jacobi 2/3, one pre and one post", "mass": "lumped", "gamma": 1.0,
                      "timing": "CUDA events around bmg_aux_solve (host loop, scalars read every iteration)"},
           "headline_variant": head, "variants": res, "coarse_setup_s": t1 - t0,
           "gamma_estimate": {"k": 12, "gamma": gamma, "lanczos_alpha_min_max": [float(min(alpha)), float(max(alpha))],
                              "ms": gamma_ms, "timing": "host wall clock, device synchronised"}}
    print(json.dumps(out), flush=True)


if __name__ == "__main__":
    a = parse()
    if a.impl == "reference":
        run_reference(a)
    elif a.cpu_table:
        print(json.dumps({"cpu_table": cpu_table(a)}), flush=True)
    elif a.workload == "annulus":
        run_own(a)
    elif a.workload == "annulus65":
        from paper_2509_08109_gb300 import inputs as _inp
        run_single(a, 2, 65, _inp.annulus_plain(65), "quarter_annulus_plain_n65")
    elif a.workload == "shell":
        from paper_2509_08109_gb300 import inputs as _inp
        run_single(a, 3, a.shell_n, _inp.shell_two_layer(a.shell_n), f"shell_octant_two_layer_n{a.shell_n}")
    elif a.workload == "batch":
        run_batch(a)
    elif a.workload == "aux":
        run_aux(a)
    else:
        run_adjoint(a)
