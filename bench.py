"""Benchmark of the GB300 matrix-free Poisson multigrid solver.

Workload (default): continuous Q4 and SIPG DG_Q4 on 32^3 cells of the curved
mesh x -> x + 0.1 sin(pi x) sin(pi y) sin(pi z), float64 throughout,
manufactured sine right-hand side.  One step = one V-cycle preconditioned
CG solve to 1e-10 relative residual of each discretization (every stage of
the hot path: cell and face kernels, Jacobi-Chebyshev smoothing, transfer,
coarse solve, fused CG updates and reductions).  `value` = dofs solved per
second over both solves (float64); the JSON line also carries the operator
apply throughput (MDoF/s) in float64 and float32 and the mixed-precision
solve rate.

python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = ("MDoF/s operator apply; solve DoF/s to 1e-10 rel. residual, "
          "FP64 vs mixed")
N_CELLS, DEGREE, AMP = 32, 4, 0.1
RTOL = 1e-10


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cells", type=int, default=N_CELLS)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", default="solve",
                    choices=["solve", "latency", "sweep", "batched",
                             "gradient"],
                    help="solve: the default contract line; the others print "
                         "their own lines for the remaining configurations")
    ap.add_argument("--degrees", default="1,2,3,4,5,6,7,8")
    return ap.parse_args()


def aggregate(ms_local, dofs_local, dist=None):
    """Whole-job figures of one timed region: the step time is the maximum
    over ranks, the dofs the sum over ranks (independent replicas)."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return ms_local, dofs_local, dofs_local / (ms_local * 1e-3)
    import torch
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([ms_local], dtype=torch.float64, device=dev)
    d = torch.tensor([float(dofs_local)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(d, op=dist.ReduceOp.SUM)
    ms, dofs = float(t.item()), float(d.item())
    return ms, dofs, dofs / (ms * 1e-3)


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


# ---------------------------------------------------------------------------
# clocks sampled during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,"
             "clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.samples = []
        self._stop = threading.Event()
        self._t = None

    def _run(self):
        while not self._stop.is_set():
            try:
                out = subprocess.run(
                    ["nvidia-smi", "-i", str(self.idx),
                     "--query-gpu=" + self.QUERY,
                     "--format=csv,noheader,nounits"],
                    capture_output=True, text=True, timeout=5).stdout
                for line in out.strip().splitlines():
                    f = [x.strip() for x in line.split(",")]
                    if len(f) >= 9:
                        self.samples.append(f)
            except Exception:
                pass
            self._stop.wait(0.2)

    def __enter__(self):
        self._t = threading.Thread(target=self._run, daemon=True)
        self._t.start()
        return self

    def __exit__(self, *a):
        self._stop.set()
        if self._t:
            self._t.join(timeout=10)

    def summary(self):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = sorted(float(s[1]) for s in self.samples if s[1].replace(
            ".", "").isdigit())
        mx = max(float(s[2]) for s in self.samples if s[2].replace(
            ".", "").isdigit())
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown",
                 "sw_power_cap"]
        reasons = set()
        for s in self.samples:
            for nm, v in zip(names, s[5:9]):
                if "Active" in v and "Not" not in v:
                    reasons.add(nm)
        return {"sm_mhz": sm[len(sm) // 2] if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(self.samples)}


# ---------------------------------------------------------------------------
# algorithmic work of one operator application
# ---------------------------------------------------------------------------
def apply_flops(disc, k, ncells, curved):
    """Floating-point operations of one apply, counted from the algorithm
    (FMA = 2): 12 sum-factorization sweeps of p^4 FMAs per cell, the
    quadrature-point operation (21 flops curved, 5 Cartesian), the two
    transposed accumulations and, for SIPG, each face once (3 per cell):
    per side the normal slope on the nodes (p^3 FMAs), the interpolation of
    value and slope to the face points (4 p^3), their transposes (4 p^3) and
    the normal-slope test distribution (p^3), plus for curved cells the
    tangential slopes and their fold (4 p^3); the flux arithmetic is 20
    flops per face point (40 curved)."""
    p = k + 1
    cell = 2 * 12 * p ** 4 + (21 if curved else 5) * p ** 3 + 2 * p ** 3
    if disc == "dg":
        side = (14 if curved else 10) * p ** 3
        face = 2 * 2 * side + (40 if curved else 20) * p * p
        cell += 3 * face
    return float(cell) * ncells


# One float64 multiply-add (2 flops) is one double-float multiply-accumulate
# on the FP32 pipe: FMUL + 3 FFMA + 8 FADD/FSUB = 14 flops (FFMA = 2).
DF_FLOPS_PER_FP64_FLOP = 7


def apply_flops_df(disc, k, ncells, curved):
    """Algorithmic FP32-pipe work of one double-float apply: the method's
    float64 flops (apply_flops) at 14 FP32-pipe flops per multiply-add.
    It does not depend on how the kernel organizes the work."""
    return DF_FLOPS_PER_FP64_FLOP * apply_flops(disc, k, ncells, curved)


def hdg_flops(k, ncells):
    """Flops of one HDG mixed apply as implemented (k_hdg.cu): per cell
    30 N p + 36 p^3 multiply-adds (S sweeps of four fields in three
    directions each way, the divergence / gradient lines, six faces), per
    face 8 p^3 for the trace; about three faces per cell."""
    p = k + 1
    N = p ** 3
    return 2.0 * ncells * (30 * N * p + 36 * p ** 3 + 3 * 8 * p ** 3)


def apply_bytes(disc, k, n, curved, word=8):
    """Compulsory DRAM bytes of one apply: source read, destination written
    (CG: plus the zero fill), stored geometry (6 words per cell point) and,
    for curved SIPG, 7 words per face point plus one per face."""
    p = k + 1
    ncells = n ** 3
    ndofs = (n * k + 1) ** 3 if disc == "cg" else ncells * p ** 3
    b = 2 * ndofs * word + (ndofs * word if disc == "cg" else 0)
    if curved:
        b += 6 * ncells * p ** 3 * word
        if disc == "dg":
            nf = 3 * n * n * (n + 1)
            b += (7 * p * p + 1) * nf * word
    return float(b)


# FP64 pipe peak of the GB300 from its unit counts: 152 SMs x 2 DFMA per
# clock per SM x 2 flop x 2.07 GHz = 1258.6 GFLOP/s (a DFMA-chain probe on
# this pool measured 1254.6).  FP32: 152 x 128 FFMA x 2 x 2.07 GHz.
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12  # probe measured 73.2

# DRAM traffic (read + write) per launch of the dominant kernel from one ncu
# capture, keyed by a hash of the sources it was compiled from; a kernel
# changed since its capture reports null.
TRAFFIC = {"dee6cd16a4158dcf": 431.08e6}  # ncu, Q4 32^3 curved, 1 launch


def kernel_hash():
    import hashlib
    h = hashlib.sha256()
    for f in ("k_apply_df.cuh", "df.cuh", "dev_tables.cuh",
              "apply_dg_df_lo.cu"):
        h.update(open(os.path.join(ROOT, "paper_1611_03029_gb300", "csrc",
                                   f), "rb").read())
    return h.hexdigest()[:16]


def load_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


# ---------------------------------------------------------------------------
# oracle (CPU baseline / reference arm): bounded sample of the workload
# ---------------------------------------------------------------------------
def oracle_sample_setup(n=8):
    from oracle import fem, mg
    out = []
    for disc in ("cg", "dg"):
        P = fem.Problem(n, n, n, DEGREE, disc=disc, mapping="sine", amp=AMP)
        V = mg.VCycle(P)
        b = fem.load_vector(P, fem.sine_forcing)
        out.append((P, V, b))
    return out


def oracle_sample_solve(setup):
    from oracle import mg
    dofs = 0
    its = []
    for P, V, b in setup:
        x, it, rr = mg.pcg(V.levels[-1].A, b, V.apply, rtol=RTOL)
        dofs += P.n_dofs
        its.append(it)
    return dofs, its


def cpu_baseline(n=8):
    t0 = time.time()
    setup = oracle_sample_setup(n)
    t_setup = time.time() - t0
    t0 = time.time()
    dofs, its = oracle_sample_solve(setup)
    t = time.time() - t0
    return {"value": dofs / t, "unit": "DoF/s", "cores": 1, "kind": "oracle",
            "sample": "oracle assembled-matrix V-cycle PCG to 1e-10, CG and "
                      "SIPG Q4 on the same curved map with %d^3 cells "
                      "(%d dofs, its %s); solve time only (setup %.1f s "
                      "excluded, as on the GPU); scipy sparse products run "
                      "on one thread" % (n, dofs, its, t_setup)}


def run_reference(args):
    rank, world, local = dist_env()
    if world > 1 and rank != 0:
        return
    setup = oracle_sample_setup(8)
    for _ in range(args.warmup):
        oracle_sample_solve(setup)
    times = []
    dofs = 0
    for _ in range(args.steps):
        t0 = time.time()
        dofs, its = oracle_sample_solve(setup)
        times.append(time.time() - t0)
    tm = sum(times) / len(times)
    v = dofs / tm
    line = {"metric": METRIC, "value": v, "unit": "DoF/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": tm * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "impl": "reference",
            "config": {"workload": "Q4 CG + SIPG DG_Q4, curved sine map, "
                       "8^3-cell bounded sample of the 32^3 workload",
                       "cells": 8, "degree": DEGREE, "rtol": RTOL},
            "cpu_baseline": {"value": v, "unit": "DoF/s", "cores": 1,
                             "kind": "oracle",
                             "sample": "8^3 cells CG+SIPG Q4 curved, "
                                       "solve only"},
            "e2e": {"value": v, "unit": "DoF/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------
def run_ours(args):
    import torch
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist_mod
        dist_mod.init_process_group("nccl")
        dist = dist_mod
    from paper_1611_03029_gb300 import build
    if rank == 0 or world == 1:
        build.build()
    if dist:
        dist.barrier()
    from paper_1611_03029_gb300 import mfpoisson as M

    n = args.cells
    stream = torch.cuda.current_stream()
    ops = {}
    for disc in ("cg", "dg"):
        ops[disc] = M.Poisson(n, n, n, DEGREE, disc=disc, mapping="sine",
                              map_param=AMP)
    mixed = {disc: M.Poisson(n, n, n, DEGREE, disc=disc, mapping="sine",
                             map_param=AMP, mg_precision="fp32")
             for disc in ("cg", "dg")}
    tuned = {}
    for d in ("cg", "dg"):
        tuned["f64_" + d] = ops[d].autotune(prec="fp64")[0]
        tuned["f32_" + d] = mixed[d].autotune(prec="fp32")[0]
    b = {d: ops[d].rhs(0) for d in ops}
    x = {d: torch.empty_like(b[d]) for d in ops}
    N = {d: ops[d].n_dofs() for d in ops}
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32,
                        device="cuda")

    def step(opset):
        its = {}
        for d in ("cg", "dg"):
            _, it, rel = opset[d].solve(b[d], x[d], rtol=RTOL, max_it=200)
            its[d] = (it[0], rel[0])
        return its

    for _ in range(args.warmup):
        step(ops)
    # --- timed region: K steps, L2 flushed before each -------------------
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    _, _, l0 = ops["cg"].counters()
    with ClockSampler(local) as clk:
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        step_ms = []
        for i in range(args.steps):
            flush.fill_(float(i))
            starts[i].record(stream)
            torch.cuda.nvtx.range_push("timed_step")  # launch-list window
            its = step(ops)
            torch.cuda.nvtx.range_pop()
            ends[i].record(stream)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
    _, _, l1 = ops["cg"].counters()
    step_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    dofs_step = N["cg"] + N["dg"]
    ms, _, value = aggregate(sum(step_ms) / len(step_ms), dofs_step, dist)

    # --- mixed-precision solve rate (same workload, float32 V-cycle) -----
    for _ in range(2):
        step(mixed)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(
        enable_timing=True)
    e0.record(stream)
    its_mixed = step(mixed)
    e1.record(stream)
    torch.cuda.synchronize()
    mixed_ms = e0.elapsed_time(e1)

    # --- operator apply throughput, per kernel, CUDA events ---------------
    apply = {}
    for prec, opset, dt in (("f64", ops, torch.float64),
                            ("f32", mixed, torch.float32)):
        for d in ("cg", "dg"):
            src = torch.randn(N[d], dtype=dt, device="cuda")
            dst = torch.empty_like(src)
            for _ in range(3):
                opset[d].apply(src, dst)
            reps = 20 if prec == "f64" else 50
            a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(
                enable_timing=True)
            flush.fill_(1.0)
            a0.record(stream)
            for _ in range(reps):
                opset[d].apply(src, dst)
            a1.record(stream)
            torch.cuda.synchronize()
            t = a0.elapsed_time(a1) / reps * 1e-3
            equiv = n ** 3 * DEGREE ** 3
            apply[prec + "_" + d] = {
                "ms": t * 1e3, "MDoF_s": N[d] / t / 1e6,
                "equiv_MDoF_s": equiv / t / 1e6,
                "GFLOP_s": apply_flops(d, DEGREE, n ** 3, True) / t / 1e9,
                "fp32_pipe_GFLOP_s": (apply_flops_df(d, DEGREE, n ** 3, True)
                                      / t / 1e9 if prec == "f64" else None),
                "GB_s": apply_bytes(d, DEGREE, n, True,
                                    8 if prec == "f64" else 4) / t / 1e9}

    # --- end to end through the C ABI with host buffers ------------------
    hb = {d: b[d].cpu().pin_memory() for d in ops}
    hx = {d: torch.empty(N[d], dtype=torch.float64).pin_memory() for d in ops}
    db = {d: torch.empty_like(b[d]) for d in ops}
    torch.cuda.synchronize()
    e0.record(stream)
    for d in ("cg", "dg"):
        db[d].copy_(hb[d], non_blocking=True)
        ops[d].solve(db[d], x[d], rtol=RTOL, max_it=200)
        hx[d].copy_(x[d], non_blocking=True)
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = e0.elapsed_time(e1)

    # --- HDG mixed operator on (q, u), Cartesian cells, float64 -----------
    try:
        oph = M.Poisson(n, n, n, DEGREE, disc="dg", n_levels=1)
        nu = oph.n_dofs()
        hsrc = torch.randn(4 * nu, dtype=torch.float64, device="cuda")
        hdst = torch.empty_like(hsrc)
        for _ in range(3):
            oph.hdg_apply(hsrc, hdst)
        reps = 10
        h0, h1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(
            enable_timing=True)
        flush.fill_(2.0)
        h0.record(stream)
        for _ in range(reps):
            oph.hdg_apply(hsrc, hdst)
        h1.record(stream)
        torch.cuda.synchronize()
        t = h0.elapsed_time(h1) / reps * 1e-3
        apply["hdg_f64_cartesian"] = {
            "ms": t * 1e3, "MDoF_s": nu / t / 1e6,
            "unknowns_per_s": 4 * nu / t,
            "GFLOP_s": hdg_flops(DEGREE, n ** 3) / t / 1e9,
            "GB_s": 2 * 4 * nu * 8 / t / 1e9}
        del oph, hsrc, hdst
    except Exception as exc:  # reported, never fatal to the contract line
        apply["hdg_f64_cartesian"] = {"error": str(exc)[:200]}

    # --- the paper's smooth example (Sec. 5): three Gaussians on (-1, 1)^3,
    # Neumann data on x_e = -1, 32^3 cells Q4 (its 32768-cell row) --------
    paper_cube = {}
    try:
        s3 = (1.0 / (0.2 * math.sqrt(2.0 * math.pi))) ** 3
        gauss = [[-0.5, 0.5, 0.25, 0.2, s3], [-0.6, -0.5, -0.125, 0.2, s3],
                 [0.5, -0.5, 0.5, 0.2, s3]]
        for d, pf in (("cg", 1.0), ("dg", 3.0)):
            opc = M.Poisson(n, n, n, DEGREE, disc=d, neumann_sides=(0, 2, 4),
                            box=(-1.0, 1.0), penalty_factor=pf)
            bc = opc.rhs(2, gauss)
            xc = torch.empty_like(bc)
            opc.solve(bc, xc, rtol=RTOL, max_it=200)
            c0, c1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(
                enable_timing=True)
            flush.fill_(3.0)
            c0.record(stream)
            _, itc, relc = opc.solve(bc, xc, rtol=RTOL, max_it=200)
            c1.record(stream)
            torch.cuda.synchronize()
            tc = c0.elapsed_time(c1)
            paper_cube[d] = {"ms": tc, "iterations": itc[0],
                             "relres": relc[0],
                             "dofs": opc.n_dofs(),
                             "DoF_s": opc.n_dofs() / (tc * 1e-3)}
            del opc, bc, xc
    except Exception as exc:  # reported, never fatal to the contract line
        paper_cube["error"] = str(exc)[:200]

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return
    peaks = load_peaks()
    # dominant kernel: the float64 SIPG apply (largest share of the step in
    # the launch list), double-float arithmetic, bound by the FP32 pipe.
    dom = apply["f64_dg"]
    ach = dom["fp32_pipe_GFLOP_s"] / 1e3
    roof = {"kernel": "k_apply_df<P=5,DG,curved>", "bound": "alu",
            "achieved": ach, "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s",
            "frac": ach / FP32_PEAK_TFLOPS,
            "traffic": TRAFFIC.get(kernel_hash()),
            "algorithmic_bytes": apply_bytes("dg", DEGREE, n, True),
            "work": "the method's float64 flops (bench.apply_flops) at 14 "
                    "FP32-pipe flops per double-float multiply-add "
                    "(bench.apply_flops_df)",
            "fp64_equivalent_TFLOP_s": dom["GFLOP_s"] / 1e3,
            "fp64_pipe_peak": FP64_PEAK_TFLOPS,
            "peak_source": "FP32 pipe from unit counts (152 SMs x 128 FFMA/clk "
                           "x 2 x 2.07 GHz); FFMA probe measured 73.2 TFLOP/s",
            "kernel_source_hash": kernel_hash()}
    line = {
        "metric": METRIC, "value": value, "unit": "DoF/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic",
        "config": {"workload": "CG Q4 + SIPG DG_Q4 V-cycle PCG solves to "
                   "1e-10, 32^3 cells, curved map amplitude 0.1",
                   "cells": n, "degree": DEGREE, "dofs_cg": N["cg"],
                   "dofs_dg": N["dg"], "rtol": RTOL,
                   "l2": "flushed (256 MB write) before every timed step",
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "iterations": {d: its[d][0] for d in its},
        "solve_ms": None,
        "mixed": {"ms_per_step": mixed_ms,
                  "value": dofs_step / (mixed_ms * 1e-3),
                  "iterations": {d: its_mixed[d][0] for d in its_mixed},
                  "speedup_vs_fp64": ms / mixed_ms},
        "apply": apply,
        "paper_cube": paper_cube,
        "cells_per_block": tuned,
        "roofline": roof,
        "e2e": {"value": dofs_step / (e2e_ms * 1e-3), "unit": "DoF/s",
                "h2d_bytes_per_step": 8 * dofs_step,
                "d2h_bytes_per_step": 8 * dofs_step},
        "gpu_launches": int((l1 - l0) // max(args.steps, 1)),
        "gpu_launches_scope": "per timed step",
        "clocks": clk.summary(),
        "peaks": {"hbm_gbs": peaks.get("hbm_gbs")},
    }
    if not args.no_cpu_baseline and world == 1:
        line["cpu_baseline"] = cpu_baseline(8)
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


# ---------------------------------------------------------------------------
# Further configurations (one JSON line each, not the contract line)
# ---------------------------------------------------------------------------
def _timed(fn, stream):
    import torch
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    out = fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1), out


def run_latency(args):
    """8^3 cells, continuous Q2 (17^3 = 4913 dofs), Cartesian, FP64: time to
    1e-10 with the V-cycle replayed from a CUDA graph and eagerly, and the
    latency of one operator apply."""
    import torch
    from paper_1611_03029_gb300 import build
    build.build()
    from paper_1611_03029_gb300 import mfpoisson as M
    st = torch.cuda.current_stream()
    op = M.Poisson(8, 8, 8, 2, disc="cg")
    b = op.rhs(0)
    x = torch.empty_like(b)
    res = {}
    for mode in ("graph", "eager"):
        os.environ["MFP_CUDA_GRAPHS"] = "1" if mode == "graph" else "0"
        for _ in range(args.warmup):
            op.solve(b, x, rtol=RTOL)
        ts = []
        for _ in range(args.steps):
            t, (_, it, rel) = _timed(lambda: op.solve(b, x, rtol=RTOL), st)
            ts.append(t)
        res[mode] = {"ms": min(ts), "median_ms": sorted(ts)[len(ts) // 2],
                     "iterations": it[0], "relres": rel[0]}
    os.environ["MFP_CUDA_GRAPHS"] = "1"
    src = torch.randn(op.n_dofs(), dtype=torch.float64, device="cuda")
    dst = torch.empty_like(src)
    t, _ = _timed(lambda: [op.apply(src, dst) for _ in range(200)], st)
    print(json.dumps({"workload": "latency: CG Q2 8^3 cells (4913 dofs), "
                      "Cartesian, FP64, 3 levels", "solve": res,
                      "apply_us": t / 200 * 1e3,
                      "dofs": op.n_dofs()}), flush=True)


SWEEP = {  # degree: (cells per axis CG, cells per axis SIPG)
    1: (256, 128), 2: (128, 96), 3: (96, 64), 4: (64, 64),
    5: (56, 48), 6: (48, 40), 7: (40, 32), 8: (32, 32)}


def run_sweep(args):
    """Degree sweep on Cartesian meshes of 16-33M dofs: FP64 V-cycle versus
    FP32 V-cycle inside the float64 CG, time to 1e-10, iterations and the
    difference of the two solutions."""
    import torch
    from paper_1611_03029_gb300 import build
    build.build()
    from paper_1611_03029_gb300 import mfpoisson as M
    st = torch.cuda.current_stream()
    for k in [int(v) for v in args.degrees.split(",")]:
        for disc, n in (("cg", SWEEP[k][0]), ("dg", SWEEP[k][1])):
            out = {"workload": "sweep", "disc": disc, "degree": k,
                   "cells": n}
            xs = {}
            for prec in ("fp64", "fp32"):
                op = M.Poisson(n, n, n, k, disc=disc, mg_precision=prec)
                b = op.rhs(0)
                x = torch.empty_like(b)
                op.solve(b, x, rtol=RTOL, max_it=200)
                t, (_, it, rel) = _timed(
                    lambda: op.solve(b, x, rtol=RTOL, max_it=200), st)
                out["dofs"] = op.n_dofs()
                out[prec] = {"ms": t, "iterations": it[0], "relres": rel[0],
                             "dofs_per_s": op.n_dofs() / (t * 1e-3)}
                xs[prec] = x.clone()
                del op
                torch.cuda.empty_cache()
            out["mixed_vs_fp64_rel_diff"] = float(
                (xs["fp32"] - xs["fp64"]).norm() / xs["fp64"].norm())
            out["mixed_speedup"] = out["fp64"]["ms"] / out["fp32"]["ms"]
            print(json.dumps(out), flush=True)


def run_batched(args):
    """16 right-hand sides (sums of 8 Gaussians), continuous Q3 on 48^3
    Cartesian cells (3,048,625 dofs each): one batched mixed-precision solve
    (one launch per operator apply, graph-captured V-cycle) versus 16
    sequential float64 solves."""
    import torch
    from paper_1611_03029_gb300 import build, synthetic
    build.build()
    from paper_1611_03029_gb300 import mfpoisson as M
    st = torch.cuda.current_stream()
    R, n, k = 16, 48, 3
    mixed = M.Poisson(n, n, n, k, disc="cg", mg_precision="fp32")
    fp64 = M.Poisson(n, n, n, k, disc="cg")
    N = mixed.n_dofs()
    B = torch.empty(N * R, dtype=torch.float64, device="cuda")
    for r in range(R):
        mixed.rhs(1, synthetic.gaussian_terms(1000 + r), out=B[r:], stride=R)
    X = torch.empty_like(B)
    tuned = mixed.autotune(prec="fp64", n_rhs=R)[0]
    mixed.solve(B, X, n_rhs=R, rtol=RTOL)
    t_b, (_, its_b, rel_b) = _timed(
        lambda: mixed.solve(B, X, n_rhs=R, rtol=RTOL), st)
    cols = [B[r::R].contiguous() for r in range(R)]
    x1 = torch.empty(N, dtype=torch.float64, device="cuda")
    fp64.solve(cols[0], x1, rtol=RTOL)

    def seq():
        its = []
        for r in range(R):
            _, it, _ = fp64.solve(cols[r], x1, rtol=RTOL)
            its.append(it[0])
        return its
    t_s, its_s = _timed(seq, st)
    print(json.dumps({"workload": "batched: 16 RHS, CG Q3 48^3 Cartesian",
                      "dofs_per_rhs": N, "batched_mixed_ms": t_b,
                      "batched_iterations": its_b,
                      "batched_max_relres": max(rel_b),
                      "sequential_fp64_ms": t_s,
                      "sequential_iterations": its_s,
                      "speedup": t_s / t_b,
                      "cells_per_block_fp64_R16": tuned,
                      "dofs_per_s_batched": N * R / (t_b * 1e-3)}),
          flush=True)


def run_gradient(args):
    """-div(a grad u) = f, a = exp(g) at every quadrature point, SIPG Q3 on
    32^3 Cartesian cells: forward solve, adjoint solve and the dL/da kernel,
    with the directional finite-difference check of the gradient."""
    import numpy as np
    import torch
    from paper_1611_03029_gb300 import build, synthetic
    build.build()
    from paper_1611_03029_gb300 import mfpoisson as M
    st = torch.cuda.current_stream()
    n, k = 32, 3
    op = M.Poisson(n, n, n, k, disc="dg")
    a_c, a_f = synthetic.log_coefficient((n, n, n), k + 1, seed=7)
    ac = torch.from_numpy(a_c).cuda()
    af = torch.from_numpy(a_f).cuda()
    t_set, _ = _timed(lambda: op.set_coefficient(ac, af), st)
    b = op.rhs(0)
    u, _, _ = op.solve(b, rtol=1e-13, max_it=300)
    ut = torch.from_numpy(
        synthetic.random_vector(op.n_dofs(), 8)).cuda() * u.norm() / \
        np.sqrt(op.n_dofs())

    def fwd_adj_grad():
        u, itf, _ = op.solve(b, rtol=1e-13, max_it=300)
        lam, ita, _ = op.solve((u - ut).contiguous(), rtol=1e-13, max_it=300)
        gc, gf = op.gradient(u, lam)
        return u, lam, gc, gf, itf[0], ita[0]
    t, (u, lam, gc, gf, itf, ita) = _timed(fwd_adj_grad, st)
    t_g, _ = _timed(lambda: op.gradient(u, lam), st)

    def loss(dc, df, eps):
        op.set_coefficient((ac + eps * dc).contiguous(),
                           (af + eps * df).contiguous())
        uu, _, _ = op.solve(b, rtol=1e-13, max_it=300)
        return 0.5 * float(((uu - ut) ** 2).sum())
    rng = np.random.default_rng(11)
    eps = 1e-4 * float(ac.abs().max())
    checks = []
    for _ in range(3):
        dc = torch.from_numpy(rng.standard_normal(a_c.shape)).cuda()
        df = torch.from_numpy(rng.standard_normal(a_f.shape)).cuda()
        dc /= dc.norm()
        df /= df.norm()
        # fourth-order central difference
        fd = (8 * (loss(dc, df, eps) - loss(dc, df, -eps))
              - (loss(dc, df, 2 * eps) - loss(dc, df, -2 * eps))) / (12 * eps)
        an = float((gc * dc).sum() + (gf * df).sum())
        checks.append(abs(fd - an) / abs(an))
    op.set_coefficient(ac, af)
    print(json.dumps({"workload": "gradient: SIPG Q3 32^3, a = exp(g)",
                      "dofs": op.n_dofs(), "cell_points": a_c.size,
                      "face_points": a_f.size,
                      "forward_adjoint_gradient_ms": t,
                      "gradient_kernel_ms": t_g,
                      "set_coefficient_ms": t_set,
                      "iterations": {"forward": itf, "adjoint": ita},
                      "fd_rel_errors": checks}), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "solve":
        run_ours(args)
    else:
        {"latency": run_latency, "sweep": run_sweep, "batched": run_batched,
         "gradient": run_gradient}[args.workload](args)


if __name__ == "__main__":
    main()
