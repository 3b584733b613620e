#!/usr/bin/env python
"""Benchmark of the partitioned poro-elastic fault solver on GB300.

One "step" = one backward-Euler implicit step of the workload: Newton with the
fault return map, each Jacobian system solved by Prevost's partitioned CG with
inner PCG solves (every row of the hot path: bulk/fault operator applies, return
map, residual, preconditioners, CG vector work).

Default workload: the slip-front set-up (Sec. 4.2, Table 1) on 64^3 Q1 hexes,
40 m cube, horizontal fault at mid-height, tied fault pressures, constant
centre injection, geometric time steps; Newton to a 1e-8 scaled residual.
(--config inclined160: 160^3 sheared grid with a 60-degree fault and seeded
lognormal permeability.)  The headline
runs the FP32-refined solver (FP32 operators + preconditioners inside the FP64
Newton / refinement loop; residuals, dots, return map in FP64); the plain FP64
solver is timed beside it on the same steps.

value = mesh DoF x implicit steps / time  (GDoF/s; s per implicit step is
ms_per_step / 1000).  The operator-apply throughput of the dominant kernel is in
"roofline" and "apply".

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
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "ncu_traffic.json")
FALLBACK_HBM = 6800.0
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12     # SMs x FP32 lanes x 2 x max SM clock
FP64_PEAK_TFLOPS = 1.25                               # nominal GB300 FP64


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gm", choices=["gm", "reference"])
    ap.add_argument("--config", default="slipfront64", choices=["inclined160", "slipfront64"])
    ap.add_argument("--fp64-steps", type=int, default=3,
                    help="steps of the plain FP64 solver timed beside the headline")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--apply-profile", type=int, default=0, metavar="N",
                    help="only run K_T applies (FP32 twice, FP64 twice) on the N^3 slip-front "
                         "grid, for kernel profiling; prints their times")
    return ap.parse_args()


def run_apply_profile(n):
    """Small fixed sequence of bulk K_T applies (the dominant kernel) for ncu."""
    import torch

    import __graft_entry__ as ge
    ge.build()
    import paper_2410_17133_gb300 as gm
    import workloads as W
    prob = W.slip_front(n=n)
    s = gm.Solver.from_problem(prob)
    N = s.N
    out = {"nodes": N, "elements": s.n_el}
    for name, dt in (("fp32", torch.float32), ("fp64", torch.float64)):
        x = (torch.randn(3, N, dtype=torch.float64, device="cuda") * 1e-6).to(dt)
        y = torch.empty_like(x)
        ms = []
        for _ in range(2):
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record()
            s.apply("KT", x, y)
            b.record()
            b.synchronize()
            ms.append(a.elapsed_time(b))
        out[name + "_ms"] = ms
    print(json.dumps(out))


def workload(name):
    import workloads as W
    if name == "inclined160":
        return W.inclined_lognormal(n=160), {"workload": "inclined-fault 160^3 Q1, lognormal k, E~U[10,30] GPa, 60 deg fault, tied lip pressures",
                                             "mesh": [160, 160, 160], "seed": 3}
    return W.slip_front(n=64), {"workload": "slip-front 64^3 Q1 (Table 1 fault, ratio 0.99, T=0.1)", "mesh": [64, 64, 64]}


def sample_workload(name, n):
    """Same physics on a smaller grid: the bounded sample the CPU oracle runs."""
    import workloads as W
    if name == "inclined160":
        p = W.inclined_lognormal(n=n)
        return p
    return W.slip_front(n=n)


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
    for f in ("gm_bulk.cuh", "gm_apply.cuh"):
        with open(os.path.join(ROOT, "paper_2410_17133_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def bulk_flops_per_element(cls_nb, mode):
    """FP operations per element of the parity-basis bulk kernel (FMA = 2).
    K mode: xy transform 8/field/plane, z stage 8/field, block products
    nb*bu^2 FMAs + 24 scalings, ob/ot accumulation 2/output, inverse xy 12/field,
    node gather 3/field."""
    bu = 24 // cls_nb
    if mode == "K":
        nf = 3
        return nf * 8 + nf * 8 + 2 * cls_nb * bu * bu + 24 + 2 * 24 + nf * 12 + nf * 3
    raise ValueError(mode)


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

    prob, cfg = workload(args.config)
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
            rep = solver.step(prob.dts[k], newton_rtol=NEWTON_RTOL, precision=precision, stream=stream)
            b.record(stream)
            b.synchronize()
            ms.append(a.elapsed_time(b))
            reps.append(rep)
        return ms, reps

    # warm-up (FP32-refined headline solver)
    W, K = args.warmup, args.steps
    timed_steps(s, range(W), gm.F32)
    log("warm-up done")
    a_w = s.get_state()
    l0, _ = s.counters()
    with ClockSampler(local_rank) as clk:
        barrier()
        t_wall0 = time.perf_counter()
        torch.cuda.nvtx.range_push("timed_steps")    # lets a profiler select these launches
        ms, reps = timed_steps(s, range(W, W + K), gm.F32)
        torch.cuda.nvtx.range_pop()
        t_wall = time.perf_counter() - t_wall0
    clocks = clk.summary()
    l1, _ = s.counters()
    launches = l1 - l0
    log("timed steps", ms)
    total_ms = max_over_ranks(sum(ms), dist, "cuda")
    value = whole_job_value(ndof, K, world, total_ms)

    # plain FP64 solver on the same steps (fresh state advanced by the same warm-up)
    fp64 = None
    if args.fp64_steps > 0:
        # the FP64 solver starts from the warmed-up state and runs the same steps
        a = a_w
        s64 = gm.Solver.from_problem(prob, device=local_rank)
        s64.set_state(u=a["u"], p=a["p"], dlie=a["dlie"], flags=a["flags"])
        m64, r64 = timed_steps(s64, range(W, W + args.fp64_steps), gm.F64)
        log("fp64 steps", m64)
        b64 = s64.get_state()
        # agreement of the two solvers after the same step (both converged to 1e-8)
        s_chk = gm.Solver.from_problem(prob, device=local_rank)
        s_chk.set_state(u=a["u"], p=a["p"], dlie=a["dlie"], flags=a["flags"])
        timed_steps(s_chk, range(W, W + args.fp64_steps), gm.F32)
        c32 = s_chk.get_state()
        du = float(np.linalg.norm(c32["u"] - b64["u"]) / max(np.linalg.norm(b64["u"]), 1e-300))
        dp = float(np.linalg.norm(c32["p"] - b64["p"]) / max(np.linalg.norm(b64["p"]), 1e-300))
        fp64 = {"ms_per_step": sum(m64) / len(m64), "steps": args.fp64_steps,
                "value": ndof * len(m64) / (sum(m64) * 1e-3) / 1e9,
                "speedup_fp32_refined": (sum(m64) / len(m64)) / (total_ms / K),
                "newton": [r["newton"] for r in r64], "inner_k": [r["inner_k"] for r in r64],
                "rel_l2_u_vs_fp32_refined": du, "rel_l2_p_vs_fp32_refined": dp,
                "flags_equal": bool(np.array_equal(c32["flags"], b64["flags"]))}
        del s64, s_chk

    # dominant kernel: bulk K_T apply in the inner PCG (FP32 for the headline)
    x32 = torch.randn(3, N, dtype=torch.float32, device="cuda") * 1e-6
    y32 = torch.empty_like(x32)
    x64 = x32.double()
    y64 = torch.empty_like(x64)

    def apply_time(x, y, reps=20):
        s.apply("KT", x, y, stream=stream)
        ts = []
        for _ in range(reps):
            flush.fill_(1.0)
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            s.apply("KT", x, y, stream=stream)
            b.record(stream)
            b.synchronize()
            ts.append(a.elapsed_time(b))
        return statistics.mean(ts)

    log("applies")
    t32 = apply_time(x32, y32) * 1e-3
    t64 = apply_time(x64, y64) * 1e-3
    nb = 8 if prob.shear == (0.0, 0.0) else (4 if prob.shear[1] == 0.0 else 2)
    n_el = s.n_el
    flops = bulk_flops_per_element(nb, "K") * n_el
    bytes32 = 28.0 * N            # u read + y write (3 x 4 B each) + E (4 B) per node
    peaks = {}
    if os.path.exists(PEAKS_FILE):
        with open(PEAKS_FILE) as fh:
            peaks = json.load(fh)
    hbm_peak = peaks.get("hbm_gbs", FALLBACK_HBM)
    peak_src = "measured" if "hbm_gbs" in peaks else "fallback"
    traffic = None
    if os.path.exists(TRAFFIC_FILE):
        with open(TRAFFIC_FILE) as fh:
            tr = json.load(fh)
        if tr.get("source_hash") == kernel_source_hash() and tr.get("config") == args.config:
            traffic = tr.get("dram_bytes_per_launch")
    ach_gbs = bytes32 / t32 / 1e9
    ach_tf = flops / t32 / 1e12
    frac_hbm = ach_gbs / hbm_peak
    frac_alu = ach_tf / FP32_PEAK_TFLOPS
    if frac_hbm >= frac_alu:
        roof = {"bound": "hbm", "achieved": ach_gbs, "peak": hbm_peak, "unit": "GB/s",
                "frac": frac_hbm, "traffic": traffic, "peak_source": peak_src,
                "alt_alu": {"achieved": ach_tf, "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s", "frac": frac_alu}}
    else:
        roof = {"bound": "alu", "achieved": ach_tf, "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s",
                "frac": frac_alu, "traffic": traffic, "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2 x 2.07 GHz",
                "alt_hbm": {"achieved": ach_gbs, "peak": hbm_peak, "unit": "GB/s", "frac": frac_hbm}}
    roof["kernel"] = "gm_bulk_apply_kernel<float,K> (+ fault kernel): the K_T product on the finest grid, the largest per-launch cost; the multigrid smoother, summed over all grid levels, has the larger share of launches"
    roof["launch_ms"] = t32 * 1e3
    apply = {"KT_fp32_gdofs": 3 * N / t32 / 1e9, "KT_fp64_gdofs": 3 * N / t64 / 1e9,
             "KT_fp32_ms": t32 * 1e3, "KT_fp64_ms": t64 * 1e3,
             "KT_fp64_alu_frac": flops / t64 / 1e12 / FP64_PEAK_TFLOPS,
             "fp64_peak_tflops_nominal": FP64_PEAK_TFLOPS}

    # end to end through the public API with host buffers: upload state, step,
    # download state + flags every step
    e2e = None
    if True:
        a = s.get_state()
        h2d = a["u"].nbytes + a["p"].nbytes + a["dlie"].nbytes + a["flags"].nbytes
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ke = 0
        for k in range(W + K, W + 2 * K):
            s.set_state(u=a["u"], p=a["p"], dlie=a["dlie"], flags=a["flags"])
            s.step(prob.dts[k], newton_rtol=NEWTON_RTOL, precision=gm.F32, stream=stream)
            a = s.get_state()
            ke += 1
        torch.cuda.synchronize()
        te = time.perf_counter() - t0
        d2h = a["u"].nbytes + a["p"].nbytes + a["slip"].nbytes + a["dlie"].nbytes + a["flags"].nbytes
        e2e = {"value": ndof * ke * world / te / 1e9, "unit": "GDoF/s", "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": int(d2h), "ms_per_step": te / ke * 1e3}

    log("e2e done")
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(args.config, budget_s=20.0)

    if rank == 0:
        out = {
            "metric": METRIC, "value": value, "unit": "GDoF/s", "n_gpus": world, "steps": K,
            "warmup": W, "ms_per_step": total_ms / K, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32-refined(f64 residual/dots/return map)",
            "data": "synthetic (seeded workload restating the paper's set-up; no paper meshes)",
            "config": dict(cfg, dofs=ndof, newton_rtol=NEWTON_RTOL,
                           steps_timed=f"{W}..{W + K - 1} of the schedule",
                           l2="flushed (512 MB write) between timed steps and between timed applies",
                           inner_solvers="FP32 K_T: PCG with a multigrid V-cycle; A22: Jacobi PCG; "
                                         "FP64 comparison: PCG with nodal/lip-pair block Jacobi",
                           parallelism=f"replicas{world}" if world > 1 else "single"),
            "roofline": roof, "apply": apply, "fp64": fp64, "cpu_baseline": cpu, "e2e": e2e,
            "clocks": clocks, "gpu_launches": int(launches),
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
# CPU oracle (baseline leg and reference arm)
# ---------------------------------------------------------------------------
def oracle_steps(config, n, steps):
    from oracle import solve as osolve
    from oracle.fem import Model
    prob = sample_workload(config, n)
    model = Model(prob)
    st = osolve.initial_state(model)
    times = []
    for k in range(steps):
        t0 = time.perf_counter()
        osolve.implicit_step(model, st, prob.dts[k], rtol=NEWTON_RTOL, solver="sparse")
        times.append(time.perf_counter() - t0)
    return 4 * model.N, times


def cpu_baseline(config, budget_s=20.0):
    n = 12
    ndof, times = oracle_steps(config, n, 2)
    return {"value": ndof * len(times) / sum(times) / 1e9, "unit": "GDoF/s", "cores": 1,
            "kind": "oracle",
            "sample": f"first {len(times)} implicit steps of the same workload on a {n}^3 grid "
                      f"({ndof} DoF), scipy SuperLU direct solves (single thread), {sum(times):.1f} s"}


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
        run_apply_profile(args.apply_profile)
        return
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    run_gm(args, rank, world, local_rank)


if __name__ == "__main__":
    main()
