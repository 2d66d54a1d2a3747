#!/usr/bin/env python3
"""Benchmark of the MatExPre hot path on GB300.

One step = one full solve of the 2D layered workload (1024^2 interior + 32-cell
PML = 1088^2 unknowns, layered 1.5-4.5 medium times a +-15% Gaussian random
field, 8 points per slowest wavelength, Gaussian point source at the centre):
outer FGMRES(30) in complex128 to a true relative residual of 1e-6, with the
MatExPre apply (Algorithm 1: psi_1 action + inner GMRES on the exp action) in
the chosen precision (complex64 by default).  Inputs are resident in HBM when
the timed region starts; L2 is flushed (256 MiB write) before every step.

value = grid-point updates per second of the whole solve: every stencil sweep
touches every unknown once, pt_updates = sweeps x unknowns, divided by the
device time of the solves (CUDA events on the solve stream), summed over ranks
and divided by the slowest rank's time.

--impl reference times the fp64 CPU oracle (the only reference this work has)
on a bounded sample of the same workload on the host cores.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "MatExPre-apply Gpts/s, HBM % of peak; time to 1e-6 residual vs plain FP64"
UNIT = "Gpts/s"
L2_FLUSH_BYTES = 256 << 20
# algorithmic bytes per unknown of one exp-action Horner sweep: read p, y, kappa; write p
BYTES_PER_PT = {"c128": 16 + 16 + 8 + 16, "c64": 8 + 8 + 4 + 8, "bf16s": 4 + 4 + 4 + 4}
# Algorithmic real flops of one point update (one SpMV row inside the Horner
# recurrence): about 24 in the 2D interior (28 in 3D), where the neighbour
# coefficients are the real 1/h^2, and about 70 in PML cells, where they are
# complex.  A grid's figure weights the two by its PML and interior cell counts.
ALG_FLOPS_INTERIOR = {2: 24.0, 3: 28.0}
ALG_FLOPS_PML = 70.0
# floating-point operations the persistent / fused float kernels execute per
# point update (one code path for every cell): 20 FMA for the complex five-point
# stencil, 2 for the diagonal, 2 for y + i tau q, 2 flops each
EXEC_FLOPS_PER_PT = 48
# FP32 pipe from unit counts and clock, for context: 152 SMs x 128 lanes x 2 x 2.07 GHz
FP32_DERIVED_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12


def alg_flops_per_update(grid):
    """Algorithmic flops per point update of a grid, weighted by its PML and
    interior cell counts."""
    import math
    n = grid.n_total
    n_int = math.prod(grid.ni)
    return (ALG_FLOPS_INTERIOR[grid.dim] * n_int + ALG_FLOPS_PML * (n - n_int)) / n


def nvtx_range(name):
    """Open (name) or close (None) an NVTX range, where torch has NVTX."""
    import torch
    try:
        if name is None:
            torch.cuda.nvtx.range_pop()
        else:
            torch.cuda.nvtx.range_push(name)
    except Exception:
        pass


def plan_for(prec, args):
    """Taylor plan (exp_tol, theta_max) of the actions of one precision."""
    return dict(exp_tol=args.exp_tol, theta_max=args.theta_bf16s if prec == "bf16s" else args.theta)


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--prec", choices=["c64", "bf16s", "c128"], default="c64")
    ap.add_argument("--exp-tol", type=float, default=1e-3,
                    help="truncation bound of the Taylor plan of every exp / psi_1 action (all "
                         "precisions, the FP64 comparison included)")
    ap.add_argument("--theta", type=float, default=6.0,
                    help="largest sub-step norm of the Taylor plan (complex64 and FP64 actions)")
    ap.add_argument("--theta-bf16s", type=float, default=4.0,
                    help="largest sub-step norm of the Taylor plan of the bf16-storage actions "
                         "(their rounding grows with the sub-step norm: at 5 the 1088^2 solve "
                         "needs 85 outer iterations, at 4 it needs 19)")
    ap.add_argument("--no-fp64-compare", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--solve-only", action="store_true",
                    help="timed solves only (no e2e, roofline, 3D, fp64 or CPU legs)")
    ap.add_argument("--profile-case", choices=["2d", "3d", "cnn"], default=None,
                    help="run two exp actions of the 2D (1088^2) or 3D (288^3) workload with the "
                         "benchmark's Taylor plan, or two training steps of the learned stage's "
                         "network on 32 crops of 64 x 64 (cnn), and exit; a small command for ncu")
    ap.add_argument("--record-traffic", nargs=3, metavar=("KERNEL", "PREC", "NCU_CSV"), default=None,
                    help="parse an ncu --csv --print-units base log of dram__bytes_read/write.sum "
                         "for KERNEL (persist2d, fused2d or horner_step) and store the DRAM bytes per "
                         "launch with the kernel source hash in profiles/traffic.json; then exit")
    ap.add_argument("--experiment", choices=["precond", "marmousi", "fused3d", "solve3d", "c3",
                                             "precision", "oracle", "c4", "plan"], default=None,
                    help="run one of the side measurements (one JSON line per case) and exit: "
                         "precond = Algorithm 1 vs P_N vs the psi_2 variant on the 1088^2 "
                         "workload; marmousi = mixed boundary conditions on a Marmousi-shaped "
                         "grid vs a PML grid of the same size; fused3d = 3D sweep kernels; "
                         "c3 = 288^3 solves in FP64, complex64 and bf16 storage; precision = "
                         "errors of the low-precision solves against the FP64 oracle (c1) and "
                         "the FP64 GPU path (c2); oracle = timed oracle runs on the host cores; "
                         "c4 = the multi-source batch (64 sources on 8 mixed 2D media in one grouped "
                         "call, then 8 sources on 432^3 in waves); plan = Taylor plans (exp_tol, "
                         "theta_max) on the 1088^2 workload: sweeps, action errors, solve time")
    ap.add_argument("--c4-3d-waves", type=int, default=2,
                    help="with --experiment c4: waves of the 8 3D sources (0 skips the 3D part)")
    ap.add_argument("--persist-cfg", type=int, default=None,
                    help="with --profile-case 2d: force this persistent-kernel configuration "
                         "(skips the autotuner's other candidates)")
    return ap.parse_args()


def dist_env():
    from paper_2506_03617_gb300 import dist as D
    return D.env()


def workload():
    from paper_2506_03617_gb300 import inputs as I
    grid, c, p = I.config_2d_layered()
    b = I.rhs_from_source(I.gaussian_source(grid)).ravel()
    return grid, c, p, b


def config_dict(grid, prec, rtol, exp_tol=None, theta=None):
    plan = "" if exp_tol is None else f", Taylor plan exp_tol {exp_tol:g} theta_max {theta:g}"
    return {"workload": "2d_layered_1088",
            "grid": f"{grid.ni[0]}x{grid.ni[1]} interior + {grid.npml}-cell PML = "
                    f"{grid.n[0]}x{grid.n[1]} unknowns",
            "medium": "layered 1.5-4.5 x (1 + 0.15 GRF, corr. 20 cells), seeded",
            "source": "Gaussian sigma=h at centre", "ppw": 8,
            "method": f"FGMRES(30) fp64, MatExPre apply in {prec}, fprtol 0.08, t=40h^2, s=1/freq{plan}",
            "rtol": rtol, "l2": "flushed (256 MiB write) before every timed step",
            "parallelism": "medium replicated, sources split across GPUs (one source per GPU: "
                           "the centre source on rank 0, seeded positions on the others; weak scaling)"}


# ----------------------------------------------------------------- oracle sample

def oracle_sample(grid, c, p, frac_t=1.0 / 16.0, seed=1):
    """Time the fp64 CPU oracle's exp action on the full workload grid and medium
    with the time length reduced to t/16 (so it takes seconds); returns
    (pt-updates, seconds, threads)."""
    import oracle
    from paper_2506_03617_gb300 import inputs as I
    P = oracle.Problem(grid.dim, grid.ni, grid.npml, c, p.omega, p.shift, p.t * frac_t,
                       p.cpml, grid.h)
    x = I.random_complex(grid.n_total, seed)
    t0 = time.perf_counter()
    _, spmv = P.phi(0, x)
    dt = time.perf_counter() - t0
    threads = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    return spmv * grid.n_total, dt, threads


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    os.environ.setdefault("OMP_NUM_THREADS", str(os.cpu_count() or 1))
    import oracle
    oracle.build()
    grid, c, p, _ = workload()
    for _ in range(args.warmup):
        oracle_sample(grid, c, p)
    pts, secs, threads = 0, 0.0, 1
    for _ in range(args.steps):
        a, b, threads = oracle_sample(grid, c, p)
        pts += a
        secs += b
    value = pts / secs / 1e9
    sample = ("fp64 C oracle exp(i t' A_s) v, t' = t/16, on the full 1088^2 layered grid "
              "(OpenMP); pt-updates = operator applications x unknowns")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * secs / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "c128", "data": "synthetic",
            "config": config_dict(grid, "fp64 (oracle)", 1e-6),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ----------------------------------------------------------------- clocks

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as fh:
            for ln in fh:
                parts = [x.strip() for x in ln.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    smax.append(float(parts[2]))
                except ValueError:
                    continue
                for nm, v in zip(names, parts[5:9]):
                    if v.lower().startswith("active"):
                        reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax),
                "reasons": sorted(reasons), "samples": len(sm)}


# ----------------------------------------------------------------- ours

KERNEL_SOURCES = {"horner_step": "stencil.cu", "fused2d": "fused2d.cu", "persist2d": "persist2d.cu"}


def kernel_hash(kernel):
    h = hashlib.sha256()
    with open(os.path.join(ROOT, "paper_2506_03617_gb300", "csrc", KERNEL_SOURCES[kernel]), "rb") as fh:
        h.update(fh.read())
    return h.hexdigest()[:16]


def measured_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            return float(json.load(fh)["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def recorded_traffic(kernel, prec):
    """dram bytes per launch from a committed ncu capture, if taken on the
    current kernel source."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as fh:
            rec = json.load(fh)
        e = rec.get(f"{kernel}:{prec}")
        if e and e.get("kernel_sha") == kernel_hash(kernel):
            return float(e["dram_bytes_per_launch"])
    except Exception:
        pass
    return None


KERNEL_NAMES = {"horner_step": "k_step", "fused2d": "k_fused2d", "persist2d": "k_persist2d"}


def record_traffic(kernel, prec, csv_path, out_path=None):
    """DRAM bytes per launch of `kernel` from an ncu CSV log (one row per
    launch and metric), stored with the hash of the kernel's source file in
    out_path (default profiles/traffic.json)."""
    import csv
    per_launch = {}
    with open(csv_path, newline="") as fh:
        rows = [r for r in csv.reader(fh) if r]
    head = next(i for i, r in enumerate(rows) if "Metric Name" in r)
    cols = rows[head]
    iid, iname, imet, iunit, ival = (cols.index("ID"), cols.index("Kernel Name"),
                                     cols.index("Metric Name"), cols.index("Metric Unit"),
                                     cols.index("Metric Value"))
    for r in rows[head + 1:]:
        if len(r) <= ival or KERNEL_NAMES[kernel] not in r[iname]:
            continue
        if r[imet] in ("dram__bytes_read.sum", "dram__bytes_write.sum"):
            if r[iunit] != "byte":
                raise SystemExit(f"expected byte units (ncu --print-units base), got {r[iunit]}")
            per_launch[r[iid]] = per_launch.get(r[iid], 0.0) + float(r[ival].replace(",", ""))
    if not per_launch:
        raise SystemExit(f"no {KERNEL_NAMES[kernel]} launches with DRAM metrics in {csv_path}")
    path = out_path or os.path.join(ROOT, "profiles", "traffic.json")
    rec = {}
    if os.path.exists(path):
        with open(path) as fh:
            rec = json.load(fh)
    rec[f"{kernel}:{prec}"] = {"dram_bytes_per_launch": sum(per_launch.values()) / len(per_launch),
                               "launches": len(per_launch), "kernel_sha": kernel_hash(kernel),
                               "source": os.path.basename(csv_path)}
    with open(path, "w") as fh:
        json.dump(rec, fh, indent=1, sort_keys=True)
    print(json.dumps(rec[f"{kernel}:{prec}"]))
    return 0


def run_ours(args):
    import numpy as np
    import torch
    import torch.distributed as dist
    rank, world, local = dist_env()
    if world > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", init_method="env://")
    dev = torch.cuda.current_device()
    from paper_2506_03617_gb300 import native as N

    grid, c, p, b_centre = workload()
    n = grid.n_total
    # the job's sources: the centre source, then seeded positions, one per GPU;
    # each rank solves its own share (the medium is replicated)
    from paper_2506_03617_gb300 import dist as D
    from paper_2506_03617_gb300 import inputs as I
    sources = [b_centre] + [I.rhs_from_source(I.gaussian_source(grid, center=ctr)).ravel()
                            for ctr in I.random_centers(grid, world - 1, seed=I.SEED_BASE + 1500)]
    mine = D.shard(range(len(sources)), rank, world)
    b_host = sources[mine[0]]
    prob = N.Problem.from_grid(grid, c, p, device=dev)
    plan = plan_for(args.prec, args)
    prob.set_params(prec=args.prec, **plan)
    stream = prob.stream
    b = torch.from_numpy(b_host).to(f"cuda:{dev}")
    x = prob.empty()
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=f"cuda:{dev}")
    rtol = 1e-6

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    for _ in range(args.warmup):
        prob.solve(b, x, rtol=rtol, maxit=300)
    barrier()
    sampler = ClockSampler(dev)
    sampler.start()
    launches0 = N.kernel_launch_count()
    times, pts, stats = [], 0, []
    nvtx_range("timed")          # marks the timed solves for a profiler's range filter
    with torch.cuda.stream(stream):
        for _ in range(args.steps):
            flush.fill_(1.0)
            ev0 = torch.cuda.Event(enable_timing=True)
            ev1 = torch.cuda.Event(enable_timing=True)
            ev0.record(stream)
            _, st = prob.solve(b, x, rtol=rtol, maxit=300)
            ev1.record(stream)
            ev1.synchronize()
            times.append(ev0.elapsed_time(ev1) / 1e3)
            pts += st["pt_updates"]
            stats.append(st)
    barrier()
    nvtx_range(None)
    launches = N.kernel_launch_count() - launches0
    clocks = sampler.stop()
    total = sum(times)
    total_max, pts_all = D.reduce_job(total, float(pts), device=f"cuda:{dev}")
    per_source = D.gather_by_index({mine[0]: {"outer": stats[0]["outer_iters"],
                                              "inner": stats[0]["inner_iters_total"],
                                              "true_relres": max(q["true_relres"] for q in stats),
                                              "seconds_per_solve": total / args.steps}}, len(sources))
    value = pts_all / total_max / 1e9

    if args.solve_only:
        if rank == 0:
            print(json.dumps({"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
                              "steps": args.steps, "ms_per_step": 1e3 * total_max / args.steps,
                              "gpu_launches": int(launches), "clocks": clocks,
                              "partial": "solve-only run"}), flush=True)
        return 0

    # ---- end to end: host buffers through mxp_solve_host (copies inside the timing)
    b_pin = torch.from_numpy(b_host).pin_memory().numpy()
    x_pin = torch.empty(n, dtype=torch.complex128).pin_memory().numpy()
    e2e_steps = max(1, min(args.steps, 3))
    e_pts, e_t = 0, 0.0
    for _ in range(e2e_steps):
        flush.fill_(2.0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        st = prob.solve_host(b_pin, x_pin, rtol=rtol, maxit=300)
        e_t += time.perf_counter() - t0
        e_pts += st["pt_updates"]
    e2e = {"value": e_pts / e_t / 1e9 * world, "unit": UNIT, "h2d_bytes_per_step": 16 * n,
           "d2h_bytes_per_step": 16 * n,
           "note": "mxp_solve_host: pinned host b -> device, solve, device x -> pinned host"}

    # ---- roofline of the dominant kernel: the exp-action sweeps (>= 90% of the
    # solve's sweeps); timed live here with CUDA events on the solve stream
    fp32_peak, fp64_peak = (v / 1e12 for v in N.measure_fma_peak(dev))
    xr = torch.from_numpy(np.random.default_rng(3).standard_normal(n) + 0j).to(f"cuda:{dev}")
    yr = prob.empty()
    pcfg, ptiles = prob.persist_config()
    tcfg, tk = prob.tile_config()
    pgeo = prob.persist_geometry()
    alg_fpu = alg_flops_per_update(grid)
    with torch.cuda.stream(stream):
        prob.apply_phi(0, xr, out=yr)
        torch.cuda.synchronize()
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        reps, passes = 3, 0
        ev0.record(stream)
        for _ in range(reps):
            passes += prob.apply_phi(0, xr, out=yr)[1]
        ev1.record(stream)
        ev1.synchronize()
    t_act = ev0.elapsed_time(ev1) / 1e3 / reps
    passes //= reps
    peak, peak_kind = measured_peak()
    if pcfg >= 0 or tcfg >= 0:
        # persistent (one launch per action) or fused (K steps per launch) sweeps
        # keep the 1088^2 vectors on chip / in L2: bound by the SM, not by HBM
        nlaunch = 1 if pcfg >= 0 else max(1, passes // max(tk, 1))
        flops_launch = alg_fpu * n * passes / nlaunch
        achieved = flops_launch / (t_act / nlaunch) / 1e12
        executed = None
        if pcfg >= 0 and pgeo:
            txo, tyo, ntx, nty, kk = pgeo
            upd = ntx * nty * (txo + 2 * kk) * (tyo + 2 * kk) * passes
            executed = {"flops_per_update": EXEC_FLOPS_PER_PT, "updates_per_launch": upd,
                        "useful_updates_per_launch": n * passes,
                        "redundant_ring_fraction": 1.0 - n * passes / upd,
                        "tflops": EXEC_FLOPS_PER_PT * upd / t_act / 1e12,
                        "tiles": [txo, tyo, ntx, nty], "k": kk}
        roofline = {"bound": "alu", "achieved": achieved, "peak": fp32_peak,
                    "unit": "TFLOP/s", "frac": achieved / fp32_peak,
                    "traffic": recorded_traffic("persist2d" if pcfg >= 0 else "fused2d", args.prec),
                    "kernel": (f"k_persist2d cfg {pcfg} ({ptiles} tiles, one launch per exp action)"
                               if pcfg >= 0 else f"k_fused2d cfg {tcfg} (K={tk} steps per launch)"),
                    "alg_flops_per_update": alg_fpu, "flops_per_launch": flops_launch,
                    "launch_us": t_act / nlaunch * 1e6,
                    "peak_kind": "measured FP32 FMA throughput (mxp_measure_fma_peak), of measured",
                    "peak_derived": FP32_DERIVED_TFLOPS, "executed": executed,
                    "hbm_equivalent_gbs": BYTES_PER_PT[args.prec] * n * passes / t_act / 1e9,
                    "note": "algorithmic flops: 24 per interior and 70 per PML point update, "
                            "weighted over the grid; the 1088^2 working set is L2/SM resident, "
                            "so the HBM roofline applies to the 3D line"}
    else:
        bytes_launch = BYTES_PER_PT[args.prec] * n
        achieved = bytes_launch / (t_act / passes) / 1e9
        roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                    "frac": achieved / peak, "traffic": recorded_traffic("horner_step", args.prec),
                    "kernel": f"k_step<{args.prec}> (one Taylor-Horner sweep)",
                    "bytes_per_launch": bytes_launch, "launch_us": t_act / passes * 1e6,
                    "peak_kind": f"{peak_kind} (copy bandwidth)"}

    extra = {}
    if world == 1 and rank == 0:
        # HBM-resident case: 3D 288^3 exp action sweep throughput
        from paper_2506_03617_gb300 import inputs as I
        g3, c3, p3 = I.config_3d_homogeneous()
        del flush
        P3 = N.Problem.from_grid(g3, c3, p3, device=dev)
        P3.set_params(prec=args.prec, **plan)
        x3 = torch.ones(g3.n_total, dtype=torch.complex128, device=f"cuda:{dev}")
        y3 = P3.empty()
        with torch.cuda.stream(P3.stream):
            P3.apply_phi(0, x3, out=y3)
            torch.cuda.synchronize()
            ev0 = torch.cuda.Event(enable_timing=True)
            ev1 = torch.cuda.Event(enable_timing=True)
            ev0.record(P3.stream)
            ps3 = P3.apply_phi(0, x3, out=y3)[1]
            ev1.record(P3.stream)
            ev1.synchronize()
        t3 = ev0.elapsed_time(ev1) / 1e3
        sw3 = t3 / ps3
        a3 = BYTES_PER_PT[args.prec] * g3.n_total / sw3 / 1e9
        # one whole MatExPre apply (psi_1 action, inner GMRES on exp actions, the
        # FP64 Krylov vectors) and one solve of the 288^3 point-source problem
        b3 = torch.from_numpy(I.rhs_from_source(I.gaussian_source(g3)).ravel()).to(f"cuda:{dev}")
        r3 = b3 / torch.linalg.vector_norm(b3)
        with torch.cuda.stream(P3.stream):
            P3.apply_matexpre(r3, out=y3)
            torch.cuda.synchronize()
            ev0.record(P3.stream)
            _, ast = P3.apply_matexpre(r3, out=y3)
            ev1.record(P3.stream)
            ev1.synchronize()
        tm3 = ev0.elapsed_time(ev1) / 1e3
        am3 = BYTES_PER_PT[args.prec] * g3.n_total * ast["stencil_passes"] / tm3 / 1e9
        row3 = _timed_solve(P3, b3, maxit=300)
        extra["hbm_resident_3d"] = {
            "workload": "3d_homogeneous_288 (256^3 + 16-cell PML)",
            "exp_action": {"gpts": g3.n_total * ps3 / t3 / 1e9, "sweeps": ps3, "achieved_gbs": a3,
                           "frac": a3 / peak},
            "matexpre_apply": {"seconds": tm3, "sweeps": ast["stencil_passes"],
                               "inner_iters": ast["inner_iters"],
                               "gpts": g3.n_total * ast["stencil_passes"] / tm3 / 1e9,
                               "sweep_bytes_gbs": am3, "frac": am3 / peak,
                               "note": "sweep bytes (28 B per c64 point update) over the whole "
                                       "apply's time, Krylov work included in the time"},
            "solve": row3, "kernel": P3.sweep_kernel()}
        del P3, x3, y3, b3, r3
        torch.cuda.empty_cache()
        # many sources per medium in lockstep (one sweep launch per pass for the batch)
        gb_ = I.Grid(2, (512, 512), 16)
        cb_ = I.layered_grf(gb_, I.SEED_BASE + 3000 + 512)
        pb_ = I.paper_params(gb_, cb_, ppw=8.0)
        PB = N.Problem.from_grid(gb_, cb_, pb_, device=dev)
        PB.set_params(prec=args.prec, **plan)
        bsrc = [torch.from_numpy(I.rhs_from_source(I.gaussian_source(gb_, center=ctr)).ravel())
                .to(f"cuda:{dev}") for ctr in I.random_centers(gb_, 8, seed=I.SEED_BASE + 3612)]
        xsb = [PB.empty() for _ in bsrc]
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        seq_pts = sum(PB.solve(bb, xx, rtol=rtol, maxit=300)[1]["pt_updates"] for bb, xx in zip(bsrc, xsb))
        torch.cuda.synchronize()
        t_seq = time.perf_counter() - t0
        N.solve_batch([PB], [0] * 8, bsrc, xsb, rtol=rtol, maxit=300)     # captures graphs
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        bst = N.solve_batch([PB], [0] * 8, bsrc, xsb, rtol=rtol, maxit=300)
        torch.cuda.synchronize()
        t_bat = time.perf_counter() - t0
        extra["batched_sources"] = {
            "workload": "8 seeded Gaussian sources on a 512^2 + 16-PML layered medium",
            "sequential_s": t_seq, "batched_s": t_bat,
            "sequential_gpts": seq_pts / t_seq / 1e9,
            "batched_gpts": sum(q["pt_updates"] for q in bst) / t_bat / 1e9,
            "all_converged": all(q["converged"] for q in bst),
            "max_true_relres": max(q["true_relres"] for q in bst)}
        del PB
        if not args.no_fp64_compare and args.prec != "c128":
            # the plain FP64 path on the same problem, and the other low-precision
            # storage; errors of the low-precision solutions against the FP64 one
            x_lo = x.clone()
            prob.set_params(prec="c128", **plan)
            x64 = prob.empty()
            torch.cuda.synchronize()
            ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            ev0.record(stream)
            _, st64 = prob.solve(b, x64, rtol=rtol, maxit=300)
            ev1.record(stream)
            ev1.synchronize()
            t64 = ev0.elapsed_time(ev1) / 1e3
            pts64 = st64["pt_updates"]
            fl64 = alg_fpu * pts64 / t64 / 1e12
            nrm64 = float(torch.linalg.vector_norm(x64))
            extra["fp64_solve"] = {"seconds": t64,
                                   "outer": st64["outer_iters"],
                                   "inner": st64["inner_iters_total"],
                                   "true_relres": st64["true_relres"],
                                   "pt_updates": pts64, "gpts": pts64 / t64 / 1e9,
                                   "alg_tflops": fl64, "dfma_peak_tflops": fp64_peak,
                                   "frac_of_dfma_peak": fl64 / fp64_peak,
                                   "roofline_note": "FP64 sweeps on an L2-resident grid: bound by "
                                                    "the FP64 pipe (measured DFMA throughput, of measured)",
                                   "speedup_of_this_precision": t64 / (total_max / args.steps),
                                   f"{args.prec}_solution_rel_err":
                                       float(torch.linalg.vector_norm(x_lo - x64)) / nrm64}
            other = "bf16s" if args.prec == "c64" else "c64"
            prob.set_params(prec=other, **plan_for(other, args))
            xo = prob.empty()
            prob.solve(b, xo, rtol=rtol, maxit=300)                # tuning and first launches
            torch.cuda.synchronize()
            ev0.record(stream)
            _, sto = prob.solve(b, xo, rtol=rtol, maxit=300)
            ev1.record(stream)
            ev1.synchronize()
            to = ev0.elapsed_time(ev1) / 1e3
            extra[f"{other}_solve"] = {"seconds": to, "plan": plan_for(other, args), "outer": sto["outer_iters"],
                                       "inner": sto["inner_iters_total"],
                                       "true_relres": sto["true_relres"],
                                       "gpts": sto["pt_updates"] / to / 1e9,
                                       "speedup_over_fp64": t64 / to,
                                       "solution_rel_err_vs_fp64":
                                           float(torch.linalg.vector_norm(xo - x64)) / nrm64}
            del x64, xo, x_lo
            prob.set_params(prec=args.prec, **plan)

    cpu = None
    if world == 1 and rank == 0 and not args.no_cpu_baseline:
        os.environ.setdefault("OMP_NUM_THREADS", str(os.cpu_count() or 1))
        import oracle
        oracle.build()
        cp, cs, ct_ = oracle_sample(grid, c, p)
        cpu = {"value": cp / cs / 1e9, "unit": UNIT, "cores": ct_, "kind": "oracle",
               "sample": "fp64 C oracle exp(i t' A_s) v with t' = t/16 on the full 1088^2 "
                         f"layered grid, {cs:.1f} s"}

    if rank == 0:
        st0 = stats[0]
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": 1e3 * total_max / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": args.prec,
                "data": "synthetic", "config": config_dict(grid, args.prec, rtol, args.exp_tol, plan_for(args.prec, args)["theta_max"]),
                "time_to_1e-6_s": total_max / args.steps,
                "solve": {"outer": st0["outer_iters"], "inner_total": st0["inner_iters_total"],
                          "true_relres": max(s["true_relres"] for s in stats),
                          "sweeps": st0["stencil_passes"]},
                "e2e": e2e, "roofline": roofline, "cpu_baseline": cpu,
                "gpu_launches": int(launches), "clocks": clocks}
        if world > 1:
            line["sources"] = per_source
        line.update(extra)
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


def run_profile_case(args):
    import torch
    from paper_2506_03617_gb300 import inputs as I
    from paper_2506_03617_gb300 import native as N
    if args.profile_case == "cnn":
        import numpy as np
        rng = np.random.default_rng(0)
        net = N.Cnn(32, 64, 64)
        net.set_params(I.cnn_initial_params(I.SEED_BASE + 7000))
        x = torch.from_numpy(rng.standard_normal((32, 3, 64, 64)).astype(np.float32)).cuda()
        t = torch.from_numpy(rng.standard_normal((32, 2, 64, 64)).astype(np.float32)).cuda()
        losses = [net.train_step(x, t, 1e-3) for _ in range(2)]
        torch.cuda.synchronize()
        print(json.dumps({"profile_case": "cnn", "batch": 32, "size": 64, "loss": losses}))
        return 0
    if args.profile_case == "3d":
        g, c, p = I.config_3d_homogeneous()
    else:
        g, c, p, _ = workload()
    prob = N.Problem.from_grid(g, c, p)
    kw = {} if args.persist_cfg is None else {"persist_cfg": args.persist_cfg}
    prob.set_params(prec=args.prec, **plan_for(args.prec, args), **kw)
    x = torch.ones(g.n_total, dtype=torch.complex128, device="cuda")
    y = prob.empty()
    for _ in range(2):
        prob.apply_phi(0, x, out=y)
    torch.cuda.synchronize()
    print(json.dumps({"profile_case": args.profile_case, "prec": args.prec,
                      "unknowns": g.n_total}))
    return 0


def _timed_solve(prob, b, rtol=1e-6, maxit=300, x=None):
    """One solve timed with CUDA events on the problem's stream; the true
    relative residual is recomputed with the FP64 operator."""
    import torch
    x = prob.empty() if x is None else x
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(prob.stream)
    _, st = prob.solve(b, x, rtol=rtol, maxit=maxit, check=False)
    ev1.record(prob.stream)
    ev1.synchronize()
    r = b - prob.apply_operator(x)
    relres = float(torch.linalg.vector_norm(r) / torch.linalg.vector_norm(b))
    return {"seconds": ev0.elapsed_time(ev1) / 1e3, "outer": st["outer_iters"],
            "inner_total": st["inner_iters_total"], "sweeps": st["stencil_passes"],
            "converged": bool(st["converged"]), "true_relres": relres}


def run_experiment(args):
    import torch
    from paper_2506_03617_gb300 import inputs as I
    from paper_2506_03617_gb300 import native as N
    prec = args.prec
    tol = 1e-12 if prec == "c128" else 1e-6
    if args.experiment == "precond":
        grid, c, p, bh = workload()
        b = torch.from_numpy(bh).cuda()
        prob = N.Problem.from_grid(grid, c, p)
        cases = [("alg1", dict(precond=0)), ("psi2_variant", dict(precond=2))]
        cases += [(f"PN{n}", dict(precond=1, neumann_n=n)) for n in (4, 8, 16, 32)]
        for name, kw in cases:
            prob.set_params(prec=prec, exp_tol=tol, **kw)
            _timed_solve(prob, b, maxit=20)                       # warm-up (tuning, first launches)
            row = _timed_solve(prob, b, maxit=400)
            print(json.dumps({"experiment": "precond", "workload": "2d_layered_1088", "prec": prec,
                              "preconditioner": name, **row}), flush=True)
    elif args.experiment == "marmousi":
        g, c, p = I.config_2d_marmousi_like(nx=1700)
        src = I.rhs_from_source(I.gaussian_source(g, center=(0.5, 2.5 * g.h))).ravel()
        gp = I.Grid(2, g.ni, 32)                                  # same interior with a PML
        cp = I.marmousi_like(gp, I.SEED_BASE + 8000)
        pp = I.paper_params(gp, cp, ppw=10.0)
        srcp = I.rhs_from_source(I.gaussian_source(gp, center=(0.5, 2.5 * gp.h))).ravel()
        for name, grid, med, par, bh, bc in (("mixed_bc", g, c, p, src, I.MARMOUSI_BC),
                                            ("pml", gp, cp, pp, srcp, None)):
            prob = N.Problem.from_grid(grid, med, par)
            prob.set_params(prec=prec, exp_tol=tol)
            if bc:
                prob.set_boundary(bc)
            b = torch.from_numpy(bh).cuda()
            _timed_solve(prob, b, maxit=2)
            row = _timed_solve(prob, b, maxit=400)
            print(json.dumps({"experiment": "marmousi", "case": name, "prec": prec,
                              "grid": list(grid.n), "boundary": list(bc) if bc else "PML 32",
                              "tuned": {"tile": prob.tile_config(), "persist": prob.persist_config()},
                              "inner_per_outer": row["inner_total"] / max(row["outer"], 1),
                              **row}), flush=True)
            prob.close()
    elif args.experiment == "c3":
        # 256^3 + 16 PML (288^3 unknowns), homogeneous and converging lens, point
        # source at the centre: FP64, complex64 and bf16-storage actions inside
        # FP64 FGMRES; low-precision solutions against the FP64 one
        for name, (g, c, p) in (("3d_homogeneous_288", I.config_3d_homogeneous()),
                                ("3d_lens_288", I.config_3d_lens())):
            b = torch.from_numpy(I.rhs_from_source(I.gaussian_source(g)).ravel()).cuda()
            prob = N.Problem.from_grid(g, c, p)
            sols = {}
            for pr in ("c64", "bf16s", "c128"):
                prob.set_params(prec=pr, **plan_for(pr, args))
                if pr != "c128":
                    _timed_solve(prob, b, maxit=2)
                x = prob.empty()
                row = _timed_solve(prob, b, maxit=400, x=x)
                sols[pr] = x
                row["kernel"] = prob.sweep_kernel()
                row["gpts"] = g.n_total * row["sweeps"] / row["seconds"] / 1e9
                print(json.dumps({"experiment": "c3", "workload": name, "prec": pr,
                                  "unknowns": g.n_total, **row}), flush=True)
            ref = sols["c128"]
            nr = float(torch.linalg.vector_norm(ref))
            for pr in ("c64", "bf16s"):
                print(json.dumps({"experiment": "c3", "workload": name, "prec": pr,
                                  "solution_rel_err_vs_fp64_gpu":
                                      float(torch.linalg.vector_norm(sols[pr] - ref)) / nr}), flush=True)
            del prob, sols, ref, b
            torch.cuda.empty_cache()
    elif args.experiment == "precision":
        # pattern (1): error of each precision's solution against the FP64
        # oracle's (c1, where the oracle solves in seconds) and against the FP64
        # GPU solution (c2, whose own parity with the oracle is tested at 1e-8 on
        # smaller grids)
        import oracle
        import numpy as np
        g, c, p = I.config_2d_homogeneous()
        bh = I.rhs_from_source(I.gaussian_source(g)).ravel()
        u_ref, info = oracle.Problem.from_grid(g, c, p).fgmres(bh, rtol=1e-6)
        b = torch.from_numpy(bh).cuda()
        prob = N.Problem.from_grid(g, c, p)
        for pr in ("c128", "c64", "bf16s"):
            prob.set_params(prec=pr, exp_tol=1e-12 if pr == "c128" else 1e-6)
            x = prob.empty()
            row = _timed_solve(prob, b, maxit=400, x=x)
            xh = x.cpu().numpy()
            print(json.dumps({"experiment": "precision", "workload": "2d_homogeneous_160 (c1)",
                              "prec": pr, **row, "oracle_outer": info["outer_iters"],
                              "rel_err_vs_fp64_oracle": float(np.linalg.norm(xh - u_ref) / np.linalg.norm(u_ref)),
                              "max_err_vs_fp64_oracle": float(np.max(np.abs(xh - u_ref)) / np.max(np.abs(u_ref)))}),
                  flush=True)
        g, c, p, bh = workload()
        b = torch.from_numpy(bh).cuda()
        prob = N.Problem.from_grid(g, c, p)
        sols = {}
        for pr in ("c128", "c64", "bf16s"):
            prob.set_params(prec=pr, exp_tol=1e-12 if pr == "c128" else 1e-6)
            if pr != "c128":
                _timed_solve(prob, b, maxit=2)
            x = prob.empty()
            row = _timed_solve(prob, b, maxit=400, x=x)
            sols[pr] = x
            err = {}
            if pr != "c128":
                ref = sols["c128"]
                err = {"rel_err_vs_fp64_gpu": float(torch.linalg.vector_norm(x - ref) / torch.linalg.vector_norm(ref)),
                       "max_err_vs_fp64_gpu": float((x - ref).abs().max() / ref.abs().max())}
            print(json.dumps({"experiment": "precision", "workload": "2d_layered_1088 (c2)", "prec": pr,
                              **row, **err}), flush=True)
    elif args.experiment == "oracle":
        # the fp64 C oracle on this machine's host cores: the full c1 solve with
        # all cores, and one exp action of c1 and of the c2 sample single-threaded
        import oracle
        ncores = os.cpu_count() or 1
        g, c, p = I.config_2d_homogeneous()
        P = oracle.Problem.from_grid(g, c, p)
        bh = I.rhs_from_source(I.gaussian_source(g)).ravel()
        os.environ["OMP_NUM_THREADS"] = str(ncores)
        t0 = time.perf_counter()
        _, info = P.fgmres(bh, rtol=1e-6)
        ts = time.perf_counter() - t0
        print(json.dumps({"experiment": "oracle", "case": "c1 full FGMRES solve", "threads": ncores,
                          "seconds": ts, "outer": info["outer_iters"], "spmv": info["spmv"],
                          "gpts": info["spmv"] * g.n_total / ts / 1e9}), flush=True)
        x = I.random_complex(g.n_total, 1)
        for threads in (1, ncores):
            oracle.set_threads(threads)
            t0 = time.perf_counter()
            _, spmv = P.phi(0, x)
            ta = time.perf_counter() - t0
            print(json.dumps({"experiment": "oracle", "case": "c1 exp action", "threads": threads,
                              "seconds": ta, "spmv": spmv, "gpts": spmv * g.n_total / ta / 1e9}), flush=True)
        g2, c2, p2, _ = workload()
        for threads in (1, ncores):
            oracle.set_threads(threads)
            pts, secs, _ = oracle_sample(g2, c2, p2)
            print(json.dumps({"experiment": "oracle", "case": "c2 exp action at t/16", "threads": threads,
                              "seconds": secs, "gpts": pts / secs / 1e9}), flush=True)
        oracle.set_threads(ncores)
    elif args.experiment == "c4":
        # 2D: 64 sources on 8 media (3 x 288^2, 3 x 544^2, 2 x 1088^2 unknowns) in
        # one mxp_solve_batch call (the small media in one lockstep group, the
        # 1088^2 media source by source); then the first source of every medium
        # solved with FP64 actions, and the batched solution's error against it
        media = I.config_batched_2d()
        probs, pofr, bs, xs, meta = [], [], [], [], []
        for k, (g, c, p, centres) in enumerate(media):
            G = N.Problem.from_grid(g, c, p)
            G.set_params(prec=prec, **plan_for(prec, args))
            probs.append(G)
            for j, ctr in enumerate(centres):
                bs.append(torch.from_numpy(I.rhs_from_source(I.gaussian_source(g, center=ctr)).ravel()).cuda())
                xs.append(G.empty())
                pofr.append(k)
                meta.append((k, j, list(g.n)))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        st = N.solve_batch(probs, pofr, bs, xs, rtol=1e-6, maxit=300)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        for (k, j, n), q in zip(meta, st):
            print(json.dumps({"experiment": "c4", "part": "2d", "medium": k, "source": j, "unknowns": n,
                              "outer": q["outer_iters"], "inner": q["inner_iters_total"],
                              "true_relres": q["true_relres"], "converged": q["converged"],
                              "time_to_1e-6_s": q["seconds"]}), flush=True)
        pts = sum(q["pt_updates"] for q in st)
        print(json.dumps({"experiment": "c4", "part": "2d summary", "prec": prec, "sources": len(st),
                          "wall_s": wall, "pt_updates": pts, "gpts": pts / wall / 1e9,
                          "all_converged": all(q["converged"] for q in st),
                          "max_true_relres": max(q["true_relres"] for q in st),
                          "max_time_to_1e-6_s": max(q["seconds"] for q in st)}), flush=True)
        for k, G in enumerate(probs):
            i = next(r for r, kk in enumerate(pofr) if kk == k)
            G.set_params(prec="c128", **plan_for("c128", args))
            x64 = G.empty()
            _, s64 = G.solve(bs[i], x64, rtol=1e-6, maxit=300)
            print(json.dumps({"experiment": "c4", "part": "2d fp64 check", "medium": k, "source": 0,
                              "unknowns": meta[i][2], "fp64_outer": s64["outer_iters"],
                              "fp64_seconds": s64["seconds"],
                              "solution_rel_err_vs_fp64_gpu":
                                  float(torch.linalg.vector_norm(xs[i] - x64) / torch.linalg.vector_norm(x64))}),
                  flush=True)
            G.set_params(prec=prec, **plan_for(prec, args))
            del x64
        del probs, bs, xs
        torch.cuda.empty_cache()
        if args.c4_3d_waves > 0:
            # 3D: 8 sources on a 432^3 layered medium, batched in waves that fit
            # HBM, FGMRES restart 8 and inner restart 8
            g, c, p, centres = I.config_batched_3d()
            G = N.Problem.from_grid(g, c, p)
            G.set_params(prec=prec, **plan_for(prec, args), inner_restart=8)
            per = (len(centres) + args.c4_3d_waves - 1) // args.c4_3d_waves
            t0 = time.perf_counter()
            pts = 0
            rows = []
            for w0 in range(0, len(centres), per):
                wave = centres[w0:w0 + per]
                bw = [torch.from_numpy(I.rhs_from_source(I.gaussian_source(g, center=ctr)).ravel()).cuda()
                      for ctr in wave]
                xw = [G.empty() for _ in wave]
                tw = time.perf_counter()
                stw = N.solve_batch([G], [0] * len(wave), bw, xw, rtol=1e-6, restart=8, maxit=300)
                torch.cuda.synchronize()
                for j, q in enumerate(stw):
                    rows.append(q)
                    pts += q["pt_updates"]
                    print(json.dumps({"experiment": "c4", "part": "3d", "source": w0 + j, "unknowns": list(g.n),
                                      "wave": w0 // per, "outer": q["outer_iters"],
                                      "inner": q["inner_iters_total"], "true_relres": q["true_relres"],
                                      "converged": q["converged"],
                                      "wave_time_s": time.perf_counter() - tw}), flush=True)
                del bw, xw
                torch.cuda.empty_cache()
            wall = time.perf_counter() - t0
            print(json.dumps({"experiment": "c4", "part": "3d summary", "prec": prec, "sources": len(rows),
                              "waves": args.c4_3d_waves, "wall_s": wall, "pt_updates": pts,
                              "gpts": pts / wall / 1e9, "all_converged": all(q["converged"] for q in rows),
                              "max_true_relres": max(q["true_relres"] for q in rows)}), flush=True)
    elif args.experiment == "plan":
        # Taylor plans of the low-precision actions on the 1088^2 workload: sweeps
        # per exp action, the action's error against the FP64 action (exp_tol
        # 1e-12), and the time and iteration counts of the solve to 1e-6
        grid, c, p, bh = workload()
        b = torch.from_numpy(bh).cuda()
        prob = N.Problem.from_grid(grid, c, p)
        xv = torch.from_numpy(I.random_complex(grid.n_total, 5)).cuda()
        prob.set_params(prec="c128", exp_tol=1e-12)
        e128, s128 = prob.apply_phi(0, xv)[0], prob.apply_phi(1, xv)[0]

        def rel(a, r):
            return float(torch.linalg.vector_norm(a - r) / torch.linalg.vector_norm(r))

        plans = ([(1e-6, 4), (1e-5, 6), (1e-4, 6), (1e-3, 6), (1e-3, 8), (1e-4, 10)] if prec != "bf16s" else
                 [(1e-6, 4), (1e-4, 4), (1e-3, 4), (1e-3, 3), (1e-6, 3), (1e-3, 5)])
        for tol, th in plans:
            prob.set_params(prec=prec, exp_tol=tol, theta_max=th)
            e, ps = prob.apply_phi(0, xv)
            s1 = prob.apply_phi(1, xv)[0]
            _timed_solve(prob, b, maxit=2)
            row = _timed_solve(prob, b, maxit=400)
            print(json.dumps({"experiment": "plan", "workload": "2d_layered_1088", "prec": prec,
                              "exp_tol": tol, "theta_max": th, "sweeps_per_exp_action": ps,
                              "exp_err_l2": rel(e, e128),
                              "exp_err_max": float((e - e128).abs().max() / e128.abs().max()),
                              "psi1_err_l2": rel(s1, s128), **row}), flush=True)
    elif args.experiment == "solve3d":
        # converging-lens medium of Sec. 4 on 128^3 + 16 PML, point-like source at the centre
        g, c, p = I.config_3d_lens(n_interior=128, npml=16)
        b = torch.from_numpy(I.rhs_from_source(I.gaussian_source(g)).ravel()).cuda()
        prob = N.Problem.from_grid(g, c, p)
        for pr in ("c64", "bf16s"):
            prob.set_params(prec=pr, exp_tol=1e-6)
            _timed_solve(prob, b, maxit=2)
            row = _timed_solve(prob, b, maxit=400)
            print(json.dumps({"experiment": "solve3d", "workload": "3d_lens_160", "prec": pr,
                              "kernel": prob.sweep_kernel(), "unknowns": g.n_total, **row}), flush=True)
    else:
        g, c, p = I.config_3d_homogeneous()
        prob = N.Problem.from_grid(g, c, p)
        x = torch.ones(g.n_total, dtype=torch.complex128, device="cuda")
        y = prob.empty()
        cfgs = [("unfused", dict(fuse_k=1))] + [(f"fused3d_cfg{k}", dict(fuse_k=0, tile_cfg=k))
                                                for k in range(4)]
        for pr in ("c64", "bf16s"):
            for name, kw in cfgs:
                prob.set_params(prec=pr, exp_tol=1e-6, **kw)
                prob.apply_phi(0, x, out=y)
                torch.cuda.synchronize()
                best, passes = 1e30, 0
                for _ in range(2):
                    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    ev0.record(prob.stream)
                    passes = prob.apply_phi(0, x, out=y)[1]
                    ev1.record(prob.stream)
                    ev1.synchronize()
                    best = min(best, ev0.elapsed_time(ev1) / 1e3)
                print(json.dumps({"experiment": "fused3d", "workload": "3d_homogeneous_288", "prec": pr,
                                  "kernel": name, "sweeps": passes, "ms": best * 1e3,
                                  "gpts": g.n_total * passes / best / 1e9}), flush=True)
    return 0


def main():
    args = parse_args()
    if args.record_traffic:
        return record_traffic(*args.record_traffic)
    if args.experiment:
        return run_experiment(args)
    if args.profile_case:
        return run_profile_case(args)
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
