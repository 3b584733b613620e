#!/usr/bin/env python
"""Benchmark of the partitioned poro-elastic fault solver on GB300.

One "step" = one backward-Euler implicit step of the workload: Newton with the
fault return map, each Jacobian system solved by Prevost's partitioned CG with
inner PCG solves (every row of the hot path: bulk/fault operator applies, return
map, residual, preconditioners, CG vector work).

Default workload (the configuration the metric is quoted on): 160^3 Q1 hexes
on a grid sheared so that the fault node plane dips 60 degrees, per-element
log-normal permeability (log10 k ~ N(-15, 0.5)) and E ~ U[10, 30] GPa from a
seeded generator, friction 0.6, constant injection at the fault centre, tied
lip pressures, 5 s steps; Newton to a 1e-8 scaled residual.  The headline runs
the FP32-refined solver (FP32 operators and preconditioners inside the FP64
Newton / refinement loop; residuals, dots, return map in FP64); the plain FP64
solver runs the first --fp64-steps of the same timed steps from the same state
and the speed-up compares the two over that identical window.
(--config slipfront64: the 64^3 slip-front set-up of Sec. 4.2.)

value = mesh DoF x implicit steps / time  (GDoF/s; s per implicit step is
ms_per_step / 1000).  The operator-apply throughputs (coupled Jacobian, K_T,
K_b, A22; FP32 and FP64) are in "apply", the dominant kernel's roofline in
"roofline".

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
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
sys.path.insert(0, ROOT)

METRIC = "operator-apply GDoF/s & s per implicit step, FP32-refined vs FP64, at 1e-8 resid"
NEWTON_RTOL = 1e-8
# inexact Newton: inner PCG and outer partitioned-CG tolerances of both arms
# (the FP64 Newton loop refines; Newton iterations are set by the fault law)
INNER_RTOL, OUTER_RTOL = 1e-2, 1e-1
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "ncu_traffic.json")
FALLBACK_HBM = 6800.0
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12     # SMs x FP32 lanes x 2 x max SM clock
FP64_PEAK_TFLOPS = 1.25                               # nominal GB300 FP64


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=8)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gm", choices=["gm", "reference"])
    ap.add_argument("--config", default="inclined160", choices=["inclined160", "slipfront64"])
    ap.add_argument("--fp64-steps", type=int, default=2,
                    help="the first steps of the timed window, run again by the plain FP64 solver")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-tet", action="store_true", help="skip the timed tetrahedral lines")
    ap.add_argument("--mesh", type=int, default=0, metavar="N",
                    help="run the workload on an N^3 grid instead of its own size (profiling runs)")
    ap.add_argument("--apply-profile", type=int, default=0, metavar="N",
                    help="only run one K_b, K_T, J and A22 apply in FP32 and FP64 on the N^3 grid "
                         "of the workload, for kernel profiling; prints their times")
    return ap.parse_args()


def run_apply_profile(n, config):
    """Small fixed sequence of operator applies (the bulk kernels) for ncu:
    K_b (one bulk launch), K_T, the coupled Jacobian and A22, FP32 then FP64, on
    the n^3 version of the workload."""
    import torch

    import __graft_entry__ as ge
    ge.build()
    import paper_2410_17133_gb300 as gm
    prob = sample_workload(config, n)
    s = gm.Solver.from_problem(prob)
    s.timestep(prob.dts[0])
    N = s.N
    out = {"nodes": N, "elements": s.n_el}
    for name, dt in (("fp32", torch.float32), ("fp64", torch.float64)):
        for which, shp in (("KB", (3, N)), ("KT", (3, N)), ("J", (4, N)), ("A22", (N,))):
            x = (torch.randn(shp, dtype=torch.float64, device="cuda") * 1e-6).to(dt)
            y = torch.empty_like(x)
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record()
            s.apply(which, x, y)
            b.record()
            b.synchronize()
            out[f"{which}_{name}_ms"] = a.elapsed_time(b)
    print(json.dumps(out))


def workload(name, steps=20, n=0):
    import workloads as W
    if name == "inclined160":
        n = n or 160
        return W.inclined_lognormal(n=n, steps=steps), {
            "workload": f"inclined-fault {n}^3 Q1 hexes ({4 * (n + 1) ** 2 * (n + 2) / 1e6:.1f} M DoF), 60 deg "
                        "fault, lognormal k (log10 N(-15, 0.5)), E ~ U[10, 30] GPa, constant injection, 5 s steps",
            "mesh": [n, n, n], "seed": 3}
    n = n or 64
    return W.slip_front(n=n, steps=max(steps, 50)), {
        "workload": f"slip-front {n}^3 Q1 (Table 1 fault, ratio 0.99, T=0.1)", "mesh": [n, n, n]}


def sample_workload(name, n, steps=20):
    """Same physics on a smaller grid: the bounded sample the CPU oracle runs."""
    import workloads as W
    if name == "inclined160":
        return W.inclined_lognormal(n=n, steps=steps)
    return W.slip_front(n=n, steps=max(steps, 50))


# ---------------------------------------------------------------------------
# clocks
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None

    def __enter__(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                                       "--format=csv,noheader,nounits", "-lms", "50"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None
        return self

    def __exit__(self, *a):
        if self.p is not None:
            self.p.terminate()
            try:
                self.p.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.p.kill()

    def summary(self):
        self.f.flush()
        rows = []
        try:
            with open(self.f.name) as fh:
                for line in fh:
                    parts = [x.strip() for x in line.split(",")]
                    if len(parts) >= 9:
                        rows.append(parts)
        finally:
            os.unlink(self.f.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons, "samples": len(rows)}


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------
def kernel_source_hash():
    h = hashlib.sha256()
    for f in ("gm_bulk32.cuh", "gm_apply.cuh"):
        with open(os.path.join(ROOT, "paper_2410_17133_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


# entries of the parity-basis elasticity operator multiplied per element (the
# cell pattern of gm_make_parpat): box, cell sheared in x-z, general cell
K_PATTERN = {0: 45, 1: 73, 2: 109}


def bulk_flops_per_element(cls):
    """FP32 operations per element of the K_b bulk kernel (FMA = 2): xy
    transform 7 per field (the shared row is transformed once for two faces), z
    transform 21, pattern products 2 x nnz, inverse z with the element scale 42,
    inverse xy and node sums 11 per field."""
    return 3 * 7 + 21 + 2 * K_PATTERN[cls] + 42 + 3 * 11


def log(*a):
    print("[bench]", *a, file=sys.stderr, flush=True)


def max_over_ranks(ms, dist, device):
    """Largest per-rank timed-region duration (all ranks get it)."""
    if dist is None:
        return float(ms)
    import torch
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_value(ndof_per_rank, steps, world, max_ms):
    """GDoF/s of the whole job: every rank solves its own replica of the
    workload (weak scaling), so the work is world x ndof x steps."""
    return ndof_per_rank * steps * world / (max_ms * 1e-3) / 1e9


def run_gm(args, rank, world, local_rank):
    import numpy as np
    import torch

    import __graft_entry__ as ge
    ge.build()
    import paper_2410_17133_gb300 as gm

    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    W, K, F = args.warmup, args.steps, min(args.fp64_steps, args.steps)
    KE = min(K, 2)
    prob, cfg = workload(args.config, steps=W + K + KE + 4, n=args.mesh)
    s = gm.Solver.from_problem(prob, device=local_rank)
    N = s.N
    ndof = 4 * N
    stream = torch.cuda.current_stream()
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    def timed_steps(solver, ks, precision):
        """Per-step device time with CUDA events on the launching stream; L2
        flushed between steps, outside the timed events."""
        ms = []
        reps = []
        for k in ks:
            flush.fill_(float(k))
            barrier()
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            rep = solver.step(prob.dts[k], newton_rtol=NEWTON_RTOL, precision=precision, inner_rtol=INNER_RTOL,
                              outer_rtol=OUTER_RTOL, stream=stream)
            b.record(stream)
            b.synchronize()
            ms.append(a.elapsed_time(b))
            reps.append(rep)
        return ms, reps

    # warm-up (FP32-refined headline solver)
    timed_steps(s, range(W), gm.F32)
    log("warm-up done")
    a_w = s.get_state()
    l0, ap0 = s.counters()
    with ClockSampler(local_rank) as clk:
        barrier()
        t_wall0 = time.perf_counter()
        torch.cuda.nvtx.range_push("timed_steps")    # lets a profiler select these launches
        ms, reps = timed_steps(s, range(W, W + K), gm.F32)
        torch.cuda.nvtx.range_pop()
        t_wall = time.perf_counter() - t_wall0
    clocks = clk.summary()
    l1, ap1 = s.counters()
    launches = l1 - l0
    log("timed steps", ms)
    total_ms = max_over_ranks(sum(ms), dist, "cuda")
    value = whole_job_value(ndof, K, world, total_ms)

    # plain FP64 solver on the first F timed steps, from the same warmed-up state
    fp64 = None
    if F > 0:
        s64 = gm.Solver.from_problem(prob, device=local_rank)
        s64.set_state(u=a_w["u"], p=a_w["p"], dlie=a_w["dlie"], flags=a_w["flags"])
        m64, r64 = timed_steps(s64, range(W, W + F), gm.F64)
        log("fp64 steps", m64)
        b64 = s64.get_state()
        del s64
        # the FP32-refined solver over the same steps from the same state, for
        # the agreement of the two converged solutions
        s_chk = gm.Solver.from_problem(prob, device=local_rank)
        s_chk.set_state(u=a_w["u"], p=a_w["p"], dlie=a_w["dlie"], flags=a_w["flags"])
        timed_steps(s_chk, range(W, W + F), gm.F32)
        c32 = s_chk.get_state()
        del s_chk
        du = float(np.linalg.norm(c32["u"] - b64["u"]) / max(np.linalg.norm(b64["u"]), 1e-300))
        dp = float(np.linalg.norm(c32["p"] - b64["p"]) / max(np.linalg.norm(b64["p"]), 1e-300))
        ms32_same = sum(ms[:F]) / F
        fp64 = {"ms_per_step": sum(m64) / F, "steps": f"{W}..{W + F - 1} (the first {F} of the timed steps)",
                "value": ndof * F / (sum(m64) * 1e-3) / 1e9,
                "fp32_refined_ms_per_step_same_steps": ms32_same,
                "speedup_fp32_refined": (sum(m64) / F) / ms32_same,
                "newton": [r["newton"] for r in r64], "inner_k": [r["inner_k"] for r in r64],
                "inner_a": [r["inner_a"] for r in r64],
                "rel_l2_u_vs_fp32_refined": du, "rel_l2_p_vs_fp32_refined": dp,
                "flags_equal": bool(np.array_equal(c32["flags"], b64["flags"])),
                "preconditioners": "same as the FP32-refined solver (multigrid K_T, Jacobi A22), in FP64",
                "tolerances": f"the same as the FP32-refined solver: inner {INNER_RTOL}, outer {OUTER_RTOL}, Newton {NEWTON_RTOL}"}

    # operator applies: median of 20 launches each, L2 flushed between them
    def apply_time(which, x, y, reps=20):
        s.apply(which, x, y, stream=stream)
        ts = []
        for _ in range(reps):
            flush.fill_(1.0)
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            s.apply(which, x, y, stream=stream)
            b.record(stream)
            b.synchronize()
            ts.append(a.elapsed_time(b))
        return statistics.median(ts) * 1e-3

    log("applies")
    s.timestep(prob.dts[W])
    apply = {}
    t_app = {}
    for which, nf in (("KB", 3), ("KT", 3), ("J", 4), ("A22", 1)):
        for tag, dt in (("fp32", torch.float32), ("fp64", torch.float64)):
            shp = (nf, N) if nf > 1 else (N,)
            x = (torch.randn(shp, dtype=torch.float64, device="cuda") * 1e-6).to(dt)
            y = torch.empty_like(x)
            t = apply_time(which, x, y)
            t_app[(which, tag)] = t
            apply[f"{which}_{tag}_us"] = t * 1e6
            apply[f"{which}_{tag}_gdofs"] = nf * N / t / 1e9
    cls = 0 if prob.shear == (0.0, 0.0) else (1 if prob.shear[1] == 0.0 else 2)
    n_el = s.n_el
    t32 = t_app[("KB", "fp32")]
    flops = bulk_flops_per_element(cls) * n_el
    bytes32 = 28.0 * N            # u read + y write (3 x 4 B each) + E (4 B per element ~ per node)
    apply["J_fp32_GBs_40B_per_node"] = 40.0 * N / t_app[("J", "fp32")] / 1e9
    apply["J_fp64_GBs_80B_per_node"] = 80.0 * N / t_app[("J", "fp64")] / 1e9
    apply["KB_fp64_alu_frac_nominal"] = flops / t_app[("KB", "fp64")] / 1e12 / FP64_PEAK_TFLOPS
    apply["notes"] = ("KB: bulk kernel alone (one launch); KT adds the fault kernel; J: the coupled "
                      "Jacobian (4 DoF per node; FP32 and FP64 run the generic coupled bulk kernel); "
                      "GDoF/s = field DoF of the product / launch time")
    peaks = {}
    if os.path.exists(PEAKS_FILE):
        with open(PEAKS_FILE) as fh:
            peaks = json.load(fh)
    hbm_peak = peaks.get("hbm_gbs", FALLBACK_HBM)
    peak_src = "measured (MEASURED_PEAKS.json hbm_gbs)" if "hbm_gbs" in peaks else "fallback 6.8 TB/s"
    traffic = None
    if os.path.exists(TRAFFIC_FILE):
        with open(TRAFFIC_FILE) as fh:
            tr = json.load(fh)
        if tr.get("source_hash") == kernel_source_hash() and tr.get("config") == args.config:
            traffic = tr.get("dram_bytes_per_launch")
    ach_gbs = bytes32 / t32 / 1e9
    ach_tf = flops / t32 / 1e12
    roof = {"bound": "hbm", "achieved": ach_gbs, "peak": hbm_peak, "unit": "GB/s",
            "frac": ach_gbs / hbm_peak, "traffic": traffic, "peak_source": peak_src,
            "alt_alu": {"achieved": ach_tf, "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s",
                        "frac": ach_tf / FP32_PEAK_TFLOPS,
                        "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2 x 2.07 GHz"},
            "kernel": "gm_bulk32_kernel (K_b, FP32): the bulk elasticity product of the inner K_T "
                      "solves and the multigrid smoother",
            "bytes_per_launch": bytes32, "launch_us": t32 * 1e6}

    # end to end through the public API with host buffers: each step uploads
    # the state from pinned host memory, steps, downloads state and flags
    a = s.get_state()
    pin = {k: torch.from_numpy(np.ascontiguousarray(v)).pin_memory() for k, v in a.items()}
    h2d = sum(pin[k].numel() * pin[k].element_size() for k in ("u", "p", "dlie", "flags"))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for k in range(W + K, W + K + KE):
        s.set_state(u=pin["u"].numpy(), p=pin["p"].numpy(), dlie=pin["dlie"].numpy(), flags=pin["flags"].numpy())
        s.step(prob.dts[k], newton_rtol=NEWTON_RTOL, precision=gm.F32, inner_rtol=INNER_RTOL, outer_rtol=OUTER_RTOL,
               stream=stream)
        a = s.get_state()
    torch.cuda.synchronize()
    te = time.perf_counter() - t0
    d2h = sum(a[k].nbytes for k in ("u", "p", "slip", "dlie", "flags"))
    e2e = {"value": ndof * KE * world / te / 1e9, "unit": "GDoF/s", "h2d_bytes_per_step": int(h2d),
           "d2h_bytes_per_step": int(d2h), "ms_per_step": te / KE * 1e3, "steps": KE}
    log("e2e done")

    tet = None
    if rank == 0 and not args.no_tet:
        tet = tet_lines()
        log("tet lines done")

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(args.config)

    if rank == 0:
        out = {
            "metric": METRIC, "value": value, "unit": "GDoF/s", "n_gpus": world, "steps": K,
            "warmup": W, "ms_per_step": total_ms / K, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32-refined (f32 operators/preconditioners; f64 residual, dots, return map)",
            "data": "synthetic (seeded workload restating the paper's set-up; no paper meshes)",
            "config": dict(cfg, dofs=ndof, newton_rtol=NEWTON_RTOL, inner_rtol=INNER_RTOL, outer_rtol=OUTER_RTOL,
                           steps_timed=f"{W}..{W + K - 1} of the schedule",
                           l2="flushed (512 MB write) between timed steps and between timed applies",
                           inner_solvers="K_T: PCG with a geometric multigrid V-cycle (degree-2 Chebyshev "
                                         "smoothing with nodal / lip-pair block Jacobi, coarsest grid of at least "
                                         "10 cells per direction with a degree-24 polynomial); A22: Jacobi PCG; "
                                         "the FP64 comparison uses the same preconditioners in FP64",
                           parallelism=f"replicas{world}" if world > 1 else "single"),
            "roofline": roof, "apply": apply, "fp64": fp64, "cpu_baseline": cpu, "e2e": e2e, "tet": tet,
            "clocks": clocks, "gpu_launches": int(launches),
            "launches_per_step": launches / K, "bulk_applies_per_step": (ap1 - ap0) / K,
            "per_step": [{"ms": m, "newton": r["newton"], "outer": r["outer"], "inner_k": r["inner_k"],
                          "inner_a": r["inner_a"], "slip": r["n_slip"], "open": r["n_open"]}
                         for m, r in zip(ms, reps)],
            "wall_s_timed": t_wall,
        }
        print(json.dumps(out))
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()


# ---------------------------------------------------------------------------
# Tetrahedral path (P1 tets): timed Cryer steps and fault steps
# ---------------------------------------------------------------------------
def tet_lines(n_cryer=16, n_fault=8, fault_steps=2):
    """Per-step times of the tetrahedral path: Cryer's octant (Sec. 4.1, FP64
    partitioned CG) and the faulted cube of tets (Sec. 3.1, Newton with the
    return map), the latter in FP64 and FP32-refined over the same steps."""
    import numpy as np
    import torch
    import paper_2410_17133_gb300 as gm
    import workloads as W
    out = {}
    prob = W.cryer_octant(n=n_cryer, steps=8)
    s = gm.TetSolver.from_problem(prob)
    u = torch.zeros((3, s.N), dtype=torch.float64, device="cuda")
    p = torch.zeros(s.N, dtype=torch.float64, device="cuda")
    s.step(prob.dts[0], u, p, rtol=1e-10)           # warm-up (preconditioner set-up)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    its = [s.step(dt, u, p, rtol=1e-10)["iterations"] for dt in prob.dts[1:]]
    torch.cuda.synchronize()
    out["cryer"] = {"mesh": f"octant, {n_cryer}^3 cells x 6 tets", "nodes": s.N, "tets": s.M,
                    "ms_per_step": (time.perf_counter() - t0) / len(its) * 1e3, "steps": len(its),
                    "outer_per_step": float(np.mean(its)), "rtol": 1e-10, "precision": "f64"}
    del s
    fprob = W.tetrahedralize(W.fault_small(n_fault, steps=fault_steps + 1))
    res = {}
    for tag, prec in (("fp64", gm.F64), ("fp32_refined", gm.F32)):
        s = gm.TetFaultSolver.from_problem(fprob)
        u = torch.zeros((3, s.N), dtype=torch.float64, device="cuda")
        p = torch.zeros(s.N, dtype=torch.float64, device="cuda")
        s.fault_step(fprob.dts[0], u, p, newton_rtol=1e-10, precision=prec)     # warm-up step
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        reps = [s.fault_step(dt, u, p, newton_rtol=1e-10, precision=prec) for dt in fprob.dts[1:fault_steps + 1]]
        torch.cuda.synchronize()
        res[tag] = {"ms_per_step": (time.perf_counter() - t0) / fault_steps * 1e3,
                    "newton": [r["newton"] for r in reps], "outer": [r["outer"] for r in reps],
                    "inner_k": [r["inner_k"] for r in reps], "slip": [r["n_slip"] for r in reps],
                    "u": u.cpu().numpy(), "p": p.cpu().numpy()}
        del s
    a, b = res["fp64"], res["fp32_refined"]
    agree_u = float(np.linalg.norm(b["u"] - a["u"]) / max(np.linalg.norm(a["u"]), 1e-300))
    agree_p = float(np.linalg.norm(b["p"] - a["p"]) / max(np.linalg.norm(a["p"]), 1e-300))
    for r in res.values():
        r.pop("u")
        r.pop("p")
    out["fault"] = dict(mesh=f"faulted cube, {n_fault}^3 hexes x 6 tets", newton_rtol=1e-10,
                        steps=f"1..{fault_steps} of the schedule", **res,
                        speedup_fp32_refined=a["ms_per_step"] / b["ms_per_step"],
                        rel_diff_u=agree_u, rel_diff_p=agree_p)
    return out


# ---------------------------------------------------------------------------
# CPU oracle (baseline leg and reference arm)
# ---------------------------------------------------------------------------
def oracle_steps(config, n, steps):
    from oracle import solve as osolve
    from oracle.fem import Model
    prob = sample_workload(config, n, steps=max(steps, 20))
    model = Model(prob)
    st = osolve.initial_state(model)
    times = []
    for k in range(steps):
        t0 = time.perf_counter()
        osolve.implicit_step(model, st, prob.dts[k], rtol=NEWTON_RTOL, solver="sparse")
        times.append(time.perf_counter() - t0)
    return 4 * model.N, times


def oracle_spmv(config, n, reps=5):
    """The oracle's assembled coupled Jacobian [K_b, -A_pu; A_up, S + dt C] (CSR)
    times a vector, on one thread and on all host cores (row blocks on threads:
    scipy's CSR product releases the GIL).  Returns GDoF/s both ways."""
    import numpy as np
    import scipy.sparse as sp
    from concurrent.futures import ThreadPoolExecutor
    from oracle.fem import Model
    prob = sample_workload(config, n)
    m = Model(prob)
    J = sp.bmat([[m.Kb, -m.Apu], [m.Apu.T, m.A22(prob.dts[0])]]).tocsr()
    x = np.random.default_rng(0).standard_normal(J.shape[1])
    t0 = time.perf_counter()
    for _ in range(reps):
        y1 = J @ x
    t1 = (time.perf_counter() - t0) / reps
    nt = os.cpu_count() or 1
    cut = np.linspace(0, J.shape[0], nt + 1).astype(int)
    parts = [J[cut[i]:cut[i + 1]] for i in range(nt)]
    y = np.empty(J.shape[0])

    def work(i):
        y[cut[i]:cut[i + 1]] = parts[i] @ x

    with ThreadPoolExecutor(nt) as ex:
        list(ex.map(work, range(nt)))
        t0 = time.perf_counter()
        for _ in range(reps):
            list(ex.map(work, range(nt)))
        tn = (time.perf_counter() - t0) / reps
    assert np.allclose(y, y1)
    return J.shape[0], J.nnz, J.shape[0] / t1 / 1e9, J.shape[0] / tn / 1e9, nt


def cpu_baseline(config, n_step=12, n_spmv=32):
    """The oracle on the machine's host cores, bounded: implicit steps of the same
    workload on an n_step^3 grid (sparse direct solves, one thread) and its
    assembled coupled-Jacobian SpMV on an n_spmv^3 grid (one thread and all
    cores)."""
    ndof, times = oracle_steps(config, n_step, 2)
    nrow, nnz, g1, gn, nt = oracle_spmv(config, n_spmv)
    return {"value": ndof * len(times) / sum(times) / 1e9, "unit": "GDoF/s", "cores": 1, "kind": "oracle",
            "sample": f"first {len(times)} implicit steps of the same workload on a {n_step}^3 grid "
                      f"({ndof} DoF; scipy SuperLU direct solves, one thread), {sum(times):.1f} s",
            "s_per_step": sum(times) / len(times),
            "spmv_gdofs_all_cores": gn, "spmv_cores": nt, "spmv_gdofs_1_core": g1,
            "spmv_sample": f"assembled coupled Jacobian of the same workload on a {n_spmv}^3 grid "
                           f"({nrow} rows, {nnz} nonzeros, FP64 CSR), y = J x; all cores = row blocks "
                           f"on {nt} threads"}


def run_reference(args, rank, world):
    if rank != 0:
        return
    n = 12
    W, K = args.warmup, args.steps
    ndof, times = oracle_steps(args.config, n, W + K)
    t = times[W:]
    value = ndof * K / sum(t) / 1e9
    _, cfg = workload(args.config)
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": "GDoF/s", "n_gpus": world,
           "steps": K, "warmup": W, "ms_per_step": sum(t) / K * 1e3, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": dict(cfg, sample_grid=[n, n, n]),
           "cpu_baseline": {"value": value, "unit": "GDoF/s", "cores": 1, "kind": "oracle",
                            "sample": f"steps {W}..{W + K - 1} of the workload on a {n}^3 grid ({ndof} DoF)"},
           "e2e": {"value": value, "unit": "GDoF/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


def main():
    args = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.apply_profile:
        run_apply_profile(args.apply_profile, args.config)
        return
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    run_gm(args, rank, world, local_rank)


if __name__ == "__main__":
    main()
