"""Benchmark of the GB300 matrix-free Poisson multigrid solver.

Workload (default): continuous Q4 and SIPG DG_Q4 on 32^3 cells of the curved
mesh x -> x + 0.1 sin(pi x) sin(pi y) sin(pi z), manufactured sine
right-hand side.  One step = one V-cycle preconditioned CG solve to 1e-10
relative residual of each discretization (every stage of the hot path: cell
and face kernels, Jacobi-Chebyshev smoothing, transfer, coarse solve, fused
CG updates and reductions); the two solves run at once on two streams.
`value` = dofs solved per second over both solves, with float64 vectors and
double-float operator arithmetic (key "arith"); the line also carries the
same solves with a float32 V-cycle ("mixed") and with IEEE float64 applies
("fp64_native"), every apply's throughput with its HBM and pipe fractions,
the paper's smooth example, and the other workloads ("configs": latency,
degree sweep, 16 batched right-hand sides, adjoint gradient).

python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
import argparse
import concurrent.futures as cf
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
    ap.add_argument("--launch-list", default="fp64", choices=["fp64", "mixed"],
                    help="the step that the NVTX range timed_step marks (the "
                         "timed FP64 steps, or one mixed-precision step), for "
                         "a launch list under ncu --nvtx-include")
    ap.add_argument("--no-extras", action="store_true",
                    help="leave the other workloads out of the contract line")
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
    """Algorithmic DRAM bytes of one apply: source read once, destination
    written once, stored geometry (6 words per cell point) and, for curved
    SIPG, 7 words per face point plus one per face (the per-dof figures of
    the algorithmic-work table: curved Q4 110 B/dof CG and 98 B/dof SIPG in
    float64).  Index arrays are not needed (structured brick) and the CG
    destination's zero fill is an implementation cost, not counted."""
    p = k + 1
    ncells = n ** 3
    ndofs = (n * k + 1) ** 3 if disc == "cg" else ncells * p ** 3
    b = 2 * ndofs * word
    if curved:
        b += 6 * ncells * p ** 3 * word
        if disc == "dg":
            nf = 3 * n * n * (n + 1)
            b += (7 * p * p + 1) * nf * word
    return float(b)


# Float64 flops per dof of the SIPG apply in the algorithmic-work table of
# the scope (12 sweeps of p^4 multiply-adds per cell, about 15 flops per
# point, faces at the Cartesian cost); apply_flops also counts the curved
# tangential face terms, so the line reports the fraction at both counts.
SCOPE_DG_FLOPS_PER_DOF = {1: 156, 2: 165, 3: 182, 4: 201, 6: 244, 8: 289}


def fp32_pipe_peak_tflops(sm_count, sm_mhz):
    """FP32-pipe peak from the unit counts: SMs x 128 FFMA per clock x 2 flop
    x the maximum SM clock (GB300: 152 x 128 x 2 x 2.07 GHz = 80.5 TFLOP/s;
    an FFMA-chain probe on this GPU measured 73.2)."""
    return sm_count * 128 * 2 * sm_mhz * 1e6 / 1e12


def fp64_pipe_peak_tflops(sm_count, sm_mhz):
    """FP64-pipe peak: SMs x 2 DFMA per clock x 2 flop x clock (GB300:
    1.26 TFLOP/s; a DFMA-chain probe measured 1.25)."""
    return sm_count * 2 * 2 * sm_mhz * 1e6 / 1e12


# DRAM traffic (read + write) per launch of the dominant kernel from one ncu
# capture, keyed by a hash of the sources it was compiled from; a kernel
# changed since its capture reports null.
TRAFFIC = {"4e61a7c9b224f910": 499.1e6}  # ncu, Q4 32^3 curved: k_apply_df + k_dg_face_add


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
            "host_cpus": os.cpu_count(), "cpu_model": cpu_model(),
            "sample": "oracle assembled-matrix V-cycle PCG to 1e-10, CG and "
                      "SIPG Q4 on the same curved map with %d^3 cells "
                      "(%d dofs, its %s); solve time only (setup %.1f s "
                      "excluded, as on the GPU); the oracle's scipy sparse "
                      "products run on one thread of the %s host CPUs"
                      % (n, dofs, its, t_setup, os.cpu_count())}


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
                             "kind": "oracle", "host_cpus": os.cpu_count(),
                             "cpu_model": cpu_model(),
                             "sample": "8^3 cells CG+SIPG Q4 curved, "
                                       "solve only"},
            "e2e": {"value": v, "unit": "DoF/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------
def _events():
    import torch
    return (torch.cuda.Event(enable_timing=True),
            torch.cuda.Event(enable_timing=True))


def timed_runs(fn, stream, n, flush=None):
    """n runs of fn, each between its own pair of CUDA events recorded on
    `stream` (the stream the library launches on), the L2 flushed by a
    256 MB write before each run; returns the per-run milliseconds."""
    out = []
    for i in range(n):
        if flush is not None:
            flush.fill_(float(i))
        e0, e1 = _events()
        e0.record(stream)
        fn()
        e1.record(stream)
        e1.synchronize()
        out.append(e0.elapsed_time(e1))
    return out


def stats(ts):
    s = sorted(ts)
    return {"min_ms": s[0], "median_ms": s[len(s) // 2],
            "mean_ms": sum(s) / len(s), "runs": len(s)}


def cpu_model():
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu model")):
                return line.split(":", 1)[1].strip()
        out = subprocess.run(["lscpu"], capture_output=True, text=True,
                             timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    return "unknown"


ARITH = ("double-float: vectors float64 in HBM; the operator applies (cell, "
         "face, diagonal, gradient kernels) carry every intermediate as an "
         "unevaluated pair of floats on the FP32 pipes (error-free TwoSum and "
         "FMA TwoProd, about 2^-46 relative per operation); CG updates, dot "
         "products, Chebyshev updates and transfers in IEEE float64. "
         "fp64_native holds the same solve with IEEE float64 (DFMA) applies")


def measure_applies(M, ops, native, mixed, N, n, stream, flush, reps,
                    hbm_gbs, sm_count, sm_mhz):
    """Per-launch CUDA-event timing of every fine-level apply (L2 flushed
    before each launch) with its HBM and pipe fractions."""
    import torch
    res = {}
    p32 = fp32_pipe_peak_tflops(sm_count, sm_mhz)
    p64 = fp64_pipe_peak_tflops(sm_count, sm_mhz)
    for tag, opset, dt in (("f64", ops, torch.float64),
                           ("f64_native", native, torch.float64),
                           ("f32", mixed, torch.float32)):
        word = 4 if dt == torch.float32 else 8
        for d in ("cg", "dg"):
            src = torch.randn(N[d], dtype=dt, device="cuda")
            dst = torch.empty_like(src)
            for _ in range(3):
                opset[d].apply(src, dst)
            ts = timed_runs(lambda: opset[d].apply(src, dst), stream,
                            reps, flush)
            st_ = stats(ts)
            t = st_["mean_ms"] * 1e-3
            fl = apply_flops(d, DEGREE, n ** 3, True)
            by = apply_bytes(d, DEGREE, n, True, word)
            e = {"launch": stats(ts), "MDoF_s": N[d] / t / 1e6,
                 "equiv_MDoF_s": n ** 3 * DEGREE ** 3 / t / 1e6,
                 "GFLOP_s": fl / t / 1e9,
                 "algorithmic_bytes": by, "GB_s": by / t / 1e9,
                 "hbm_frac": by / t / 1e9 / hbm_gbs}
            if tag == "f64":
                e["fp32_pipe_TFLOP_s"] = DF_FLOPS_PER_FP64_FLOP * fl / t / 1e12
                e["fp32_pipe_frac"] = e["fp32_pipe_TFLOP_s"] / p32
            elif tag == "f64_native":
                e["fp64_pipe_frac"] = fl / t / 1e12 / p64
            else:
                e["fp32_pipe_frac"] = fl / t / 1e12 / p32
            res[tag + "_" + d] = e
            del src, dst
    return res


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
    peaks = load_peaks()
    hbm_gbs = float(peaks.get("hbm_gbs") or 6800.0)
    sm_mhz = float(peaks.get("sm_max_mhz") or 2070.0)
    sm_count = torch.cuda.get_device_properties(local).multi_processor_count

    def make(disc, **kw):
        return M.Poisson(n, n, n, DEGREE, disc=disc, mapping="sine",
                         map_param=AMP, **kw)
    ops = {d: make(d) for d in ("cg", "dg")}
    mixed = {d: make(d, mg_precision="fp32") for d in ("cg", "dg")}
    native = {d: make(d, fp64_arith="native") for d in ("cg", "dg")}
    # cells per block of every level's applies (the coarse levels are
    # latency-bound and may prefer other shapes than the finest)
    tuned = {}
    for d in ("cg", "dg"):
        for tag, opx, pr in (("f64_", ops[d], "fp64"),
                             ("f64_native_", native[d], "fp64"),
                             ("f32_", mixed[d], "fp32")):
            tuned[tag + d] = [opx.autotune(level=lv, prec=pr)[0]
                              for lv in range(opx.n_levels - 1, 0, -1)]
    b = {d: ops[d].rhs(0) for d in ops}
    x = {d: torch.empty_like(b[d]) for d in ops}
    N = {d: ops[d].n_dofs() for d in ops}
    dofs_step = N["cg"] + N["dg"]
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32,
                        device="cuda")

    def step_sequential(opset):
        its = {}
        for d in ("cg", "dg"):
            _, it, rel = opset[d].solve(b[d], x[d], rtol=RTOL, max_it=200)
            its[d] = (it[0], rel[0])
        return its

    # a step: the two independent solves at once, each on its own stream from
    # its own host thread (mfp_solve waits on its stream once per iteration),
    # so that one solve's latency-bound coarse levels overlap the other's
    # fine-level kernels; the timing stream waits for both
    # the SIPG solve is the longer one: its stream gets the higher priority,
    # so the CG solve's kernels fill the gaps rather than delay it
    lo_pri, hi_pri = torch.cuda.Stream.priority_range() \
        if hasattr(torch.cuda.Stream, "priority_range") else (0, -1)
    side = {"cg": torch.cuda.Stream(priority=lo_pri),
            "dg": torch.cuda.Stream(priority=hi_pri)}
    pool = cf.ThreadPoolExecutor(max_workers=2)

    def solve_on(opset, d, start, mark):
        torch.cuda.set_device(local)  # a worker thread's current device
        st_ = side[d]
        st_.wait_event(start)
        if mark:  # NVTX ranges are per thread: the launch-list window
            torch.cuda.nvtx.range_push("timed_step")
        _, it, rel = opset[d].solve(b[d], x[d], rtol=RTOL, max_it=200,
                                    stream=st_)
        if mark:
            torch.cuda.nvtx.range_pop()
        done = torch.cuda.Event()
        done.record(st_)
        return (it[0], rel[0]), done

    def step(opset, mark=False):
        start = torch.cuda.Event()
        start.record(stream)
        futs = {d: pool.submit(solve_on, opset, d, start, mark)
                for d in ("cg", "dg")}
        its = {}
        for d, f in futs.items():
            its[d], done = f.result()
            stream.wait_event(done)
        return its

    for _ in range(args.warmup):  # captures the V-cycle graphs first
        step_sequential(ops)
    for _ in range(2):
        step(ops)
    # --- timed region: K steps, L2 flushed before each -------------------
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    _, _, l0 = ops["cg"].counters()
    with ClockSampler(local) as clk:
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        for i in range(args.steps):
            flush.fill_(float(i))
            starts[i].record(stream)
            its = step(ops, mark=args.launch_list == "fp64")
            ends[i].record(stream)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        _, _, l1 = ops["cg"].counters()
        step_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
        ms, _, value = aggregate(sum(step_ms) / len(step_ms), dofs_step, dist)

        # --- the same solves with a float32 V-cycle (mixed precision) and
        # with IEEE float64 (DFMA) applies: min of 5 and median of 20 ------
        for _ in range(3):
            step_sequential(mixed)
            step_sequential(native)
            step(mixed)
            step(native)
        its_mixed = step(mixed, mark=args.launch_list == "mixed")
        mixed_ts = timed_runs(lambda: step(mixed), stream, 20, flush)
        its_native = step(native)
        native_ts = timed_runs(lambda: step(native), stream, 5, flush)

        # --- operator applies, one event pair per launch -----------------
        apply = measure_applies(M, ops, native, mixed, N, n, stream, flush,
                                20, hbm_gbs, sm_count, sm_mhz)

        # --- end to end through the C ABI with host buffers --------------
        hb = {d: b[d].cpu().pin_memory() for d in ops}
        hx = {d: torch.empty(N[d], dtype=torch.float64).pin_memory()
              for d in ops}
        db = {d: torch.empty_like(b[d]) for d in ops}

        def e2e_one(d, start):
            torch.cuda.set_device(local)
            st_ = side[d]
            st_.wait_event(start)
            with torch.cuda.stream(st_):
                db[d].copy_(hb[d], non_blocking=True)
                ops[d].solve(db[d], x[d], rtol=RTOL, max_it=200, stream=st_)
                hx[d].copy_(x[d], non_blocking=True)
            done = torch.cuda.Event()
            done.record(st_)
            return done

        def e2e_step():  # the step's form, with the host copies
            start = torch.cuda.Event()
            start.record(stream)
            futs = [pool.submit(e2e_one, d, start) for d in ("cg", "dg")]
            for f in futs:
                stream.wait_event(f.result())
        e2e_step()
        e2e_ts = timed_runs(e2e_step, stream, 20, flush)
        # the same FP64 solves one after the other on one stream
        seq_ts = timed_runs(lambda: step_sequential(ops), stream, 5, flush)
    mixed_st, native_st, e2e_st = (stats(mixed_ts), stats(native_ts),
                                   stats(e2e_ts))
    del native
    torch.cuda.empty_cache()

    # --- HDG mixed operator on (q, u), Cartesian cells, float64 -----------
    try:
        oph = M.Poisson(n, n, n, DEGREE, disc="dg", n_levels=1)
        nu = oph.n_dofs()
        hsrc = torch.randn(4 * nu, dtype=torch.float64, device="cuda")
        hdst = torch.empty_like(hsrc)
        for _ in range(3):
            oph.hdg_apply(hsrc, hdst)
        hst = stats(timed_runs(lambda: oph.hdg_apply(hsrc, hdst), stream, 20,
                               flush))
        t = hst["mean_ms"] * 1e-3
        apply["hdg_f64_cartesian"] = {
            "launch": hst, "MDoF_s": nu / t / 1e6,
            "unknowns_per_s": 4 * nu / t,
            "GFLOP_s": hdg_flops(DEGREE, n ** 3) / t / 1e9,
            "GB_s": 2 * 4 * nu * 8 / t / 1e9,
            "hbm_frac": 2 * 4 * nu * 8 / t / 1e9 / hbm_gbs}
        del oph, hsrc, hdst
    except Exception as exc:  # reported, never fatal to the contract line
        apply["hdg_f64_cartesian"] = {"error": str(exc)[:200]}

    # --- the paper's smooth example (Sec. 4.3): three Gaussians on (-1, 1)^3,
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
            _, itc, relc = opc.solve(bc, xc, rtol=RTOL, max_it=200)
            cst = stats(timed_runs(
                lambda: opc.solve(bc, xc, rtol=RTOL, max_it=200), stream, 5,
                flush))
            paper_cube[d] = {"solve": cst, "iterations": itc[0],
                             "relres": relc[0], "dofs": opc.n_dofs(),
                             "DoF_s": opc.n_dofs() / (cst["median_ms"] * 1e-3)}
            del opc, bc, xc
    except Exception as exc:  # reported, never fatal to the contract line
        paper_cube["error"] = str(exc)[:200]

    # --- the other workloads (latency, degree sweep, batched, gradient) ---
    configs = {}
    if not args.no_extras:
        del mixed
        torch.cuda.empty_cache()
        for name, fn in (("latency_cg_q2_8", config_latency),
                         ("sweep_cartesian", config_sweep),
                         ("batched_16rhs_cg_q3_48", config_batched),
                         ("gradient_sipg_q3_32", config_gradient)):
            try:
                configs[name] = fn(M, stream, flush)
            except Exception as exc:  # reported, never fatal
                configs[name] = {"error": str(exc)[:300]}
            torch.cuda.empty_cache()

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return
    # dominant kernel: the float64 SIPG apply (largest share of the step in
    # the launch list), double-float arithmetic, bound by the FP32 pipe.
    dom = apply["f64_dg"]
    p32 = fp32_pipe_peak_tflops(sm_count, sm_mhz)
    t_dom = dom["launch"]["mean_ms"] * 1e-3
    fl = apply_flops("dg", DEGREE, n ** 3, True)
    ach = DF_FLOPS_PER_FP64_FLOP * fl / t_dom / 1e12
    fl_s = SCOPE_DG_FLOPS_PER_DOF[DEGREE] * N["dg"]
    roof = {"kernel": "k_apply_df<P=5,DG,curved> + k_dg_face_add",
            "bound": "alu", "achieved": ach, "peak": p32, "unit": "TFLOP/s",
            "frac": ach / p32,
            "traffic": TRAFFIC.get(kernel_hash()),
            "algorithmic_flops_fp64": fl,
            "flops_per_dof_fp64": fl / N["dg"],
            "work": "float64 flops of the method as counted in "
                    "bench.apply_flops (sweeps, quadrature-point operation, "
                    "each face once with the curved tangential terms) x 7 "
                    "FP32-pipe flops per float64 flop (one double-float "
                    "multiply-add: FMUL + 3 FFMA + 8 FADD = 14 flops)",
            "frac_at_scope_flop_count": (DF_FLOPS_PER_FP64_FLOP * fl_s
                                          / t_dom / 1e12 / p32),
            "algorithmic_bytes": dom["algorithmic_bytes"],
            "hbm_frac": dom["hbm_frac"],
            "launch_mean_ms": dom["launch"]["mean_ms"],
            "peak_source": "FP32 pipe from unit counts: %d SMs (device query) "
                           "x 128 FFMA/clk x 2 flop x %.0f MHz" % (sm_count,
                                                                  sm_mhz),
            "kernel_source_hash": kernel_hash()}
    line = {
        "metric": METRIC, "value": value, "unit": "DoF/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "arith": ARITH, "data": "synthetic",
        "config": {"workload": "CG Q4 + SIPG DG_Q4 V-cycle PCG solves to "
                   "1e-10, 32^3 cells, curved map amplitude 0.1",
                   "cells": n, "degree": DEGREE, "dofs_cg": N["cg"],
                   "dofs_dg": N["dg"], "rtol": RTOL,
                   "l2": "flushed (256 MB write) before every timed step "
                         "and every timed launch",
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "step_ms": stats(step_ms),
        "step_sequential_ms": stats(seq_ts),
        "step_form": "the CG and SIPG solves of a step run at once on two "
                     "streams (one host thread each; the SIPG stream at "
                     "the higher priority); step_sequential_ms times them "
                     "one after the other",
        "iterations": {d: its[d][0] for d in its},
        "mixed": {"solve": mixed_st,
                  "value": dofs_step / (mixed_st["median_ms"] * 1e-3),
                  "iterations": {d: its_mixed[d][0] for d in its_mixed},
                  "speedup_vs_fp64": stats(step_ms)["median_ms"]
                  / mixed_st["median_ms"]},
        "fp64_native": {"solve": native_st,
                        "value": dofs_step / (native_st["median_ms"] * 1e-3),
                        "iterations": {d: its_native[d][0]
                                       for d in its_native},
                        "arith": "IEEE float64 (DFMA) applies"},
        "apply": apply,
        "paper_cube": paper_cube,
        "configs": configs,
        "cells_per_block": tuned,
        "roofline": roof,
        "e2e": {"value": dofs_step / (e2e_st["median_ms"] * 1e-3),
                "unit": "DoF/s", "solve": e2e_st,
                "h2d_bytes_per_step": 8 * dofs_step,
                "d2h_bytes_per_step": 8 * dofs_step},
        "gpu_launches": int((l1 - l0) // max(args.steps, 1)),
        "gpu_launches_scope": "per timed step",
        "clocks": clk.summary(),
        "peaks": {"hbm_gbs": hbm_gbs, "sm_count": sm_count,
                  "sm_max_mhz": sm_mhz,
                  "fp32_pipe_tflops": p32,
                  "fp64_pipe_tflops": fp64_pipe_peak_tflops(sm_count,
                                                            sm_mhz)},
    }
    if not args.no_cpu_baseline and world == 1:
        line["cpu_baseline"] = cpu_baseline(8)
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


# ---------------------------------------------------------------------------
# The other configurations: each returns a dict that the contract line
# carries under "configs" (and --workload prints alone)
# ---------------------------------------------------------------------------
def config_latency(M, stream, flush, runs=20):
    """8^3 cells, continuous Q2 (17^3 = 4913 dofs), Cartesian, FP64, 3
    levels: time to 1e-10 with the V-cycle replayed from a CUDA graph and
    eagerly, and the latency of one operator apply."""
    import torch
    op = M.Poisson(8, 8, 8, 2, disc="cg")
    b = op.rhs(0)
    x = torch.empty_like(b)
    res = {"dofs": op.n_dofs(), "levels": op.n_levels}
    for mode in ("graph", "eager"):
        os.environ["MFP_CUDA_GRAPHS"] = "1" if mode == "graph" else "0"
        for _ in range(3):
            _, it, rel = op.solve(b, x, rtol=RTOL)
        res[mode] = stats(timed_runs(lambda: op.solve(b, x, rtol=RTOL),
                                     stream, runs))
        res[mode].update(iterations=it[0], relres=rel[0])
    os.environ["MFP_CUDA_GRAPHS"] = "1"
    src = torch.randn(op.n_dofs(), dtype=torch.float64, device="cuda")
    dst = torch.empty_like(src)
    ts = timed_runs(lambda: [op.apply(src, dst) for _ in range(100)], stream,
                    5)
    res["apply_us"] = min(ts) / 100 * 1e3
    return res


SWEEP = {  # degree: (cells per axis CG, cells per axis SIPG)
    1: (256, 128), 2: (128, 96), 3: (96, 64), 4: (64, 64),
    5: (56, 48), 6: (48, 40), 7: (40, 32), 8: (32, 32)}


def config_sweep(M, stream, flush, degrees=(2, 4, 8), runs=5):
    """Degree sweep on Cartesian meshes of 16-33M dofs: time to 1e-10 with
    the float64 V-cycle and with the float32 V-cycle inside the float64 CG,
    iterations, and the difference of the two solutions."""
    import torch
    out = {}
    for k in degrees:
        for disc, n in (("cg", SWEEP[k][0]), ("dg", SWEEP[k][1])):
            e = {"cells": n}
            xs = {}
            for prec in ("fp64", "fp32"):
                op = M.Poisson(n, n, n, k, disc=disc, mg_precision=prec)
                b = op.rhs(0)
                x = torch.empty_like(b)
                _, it, rel = op.solve(b, x, rtol=RTOL, max_it=200)
                st_ = stats(timed_runs(
                    lambda: op.solve(b, x, rtol=RTOL, max_it=200), stream,
                    runs, flush))
                e["dofs"] = op.n_dofs()
                st_.update(iterations=it[0], relres=rel[0],
                           dofs_per_s=op.n_dofs() / (st_["median_ms"] * 1e-3))
                e[prec] = st_
                xs[prec] = x.clone()
                del op, b, x
                torch.cuda.empty_cache()
            e["mixed_vs_fp64_rel_diff"] = float(
                (xs["fp32"] - xs["fp64"]).norm() / xs["fp64"].norm())
            e["mixed_speedup"] = (e["fp64"]["median_ms"]
                                  / e["fp32"]["median_ms"])
            out["%s_q%d" % (disc, k)] = e
            del xs
    return out


def config_batched(M, stream, flush, runs=5):
    """16 right-hand sides (sums of 8 Gaussians), continuous Q3 on 48^3
    Cartesian cells (3,048,625 dofs each), time to 1e-10 for all 16:
    batched (one launch per operator apply for all columns, graph-captured
    V-cycle) and sequential, each with the float32 and the float64 V-cycle,
    so that batching and precision show separately."""
    import torch
    from paper_1611_03029_gb300 import synthetic
    R, n, k = 16, 48, 3
    ctx = {"fp32": M.Poisson(n, n, n, k, disc="cg", mg_precision="fp32"),
           "fp64": M.Poisson(n, n, n, k, disc="cg")}
    N = ctx["fp64"].n_dofs()
    B = torch.empty(N * R, dtype=torch.float64, device="cuda")
    for r in range(R):
        ctx["fp64"].rhs(1, synthetic.gaussian_terms(1000 + r), out=B[r:],
                        stride=R)
    X = torch.empty_like(B)
    cols = [B[r::R].contiguous() for r in range(R)]
    x1 = torch.empty(N, dtype=torch.float64, device="cuda")
    out = {"dofs_per_rhs": N, "rhs": R}
    for prec, op in ctx.items():
        vp = "fp32" if prec == "fp32" else "fp64"
        out["cells_per_block_R16_" + prec] = op.autotune(prec=vp, n_rhs=R)[0]
        _, its, rel = op.solve(B, X, n_rhs=R, rtol=RTOL)
        st_ = stats(timed_runs(lambda: op.solve(B, X, n_rhs=R, rtol=RTOL),
                               stream, runs, flush))
        st_.update(iterations=its, max_relres=max(rel),
                   dofs_per_s=N * R / (st_["median_ms"] * 1e-3))
        out["batched_" + prec] = st_

        def seq():
            for r in range(R):
                op.solve(cols[r], x1, rtol=RTOL)
        seq()
        st_ = stats(timed_runs(seq, stream, max(2, runs // 2), flush))
        st_["dofs_per_s"] = N * R / (st_["median_ms"] * 1e-3)
        out["sequential_" + prec] = st_
    t = {kk: v["median_ms"] for kk, v in out.items()
         if isinstance(v, dict) and "median_ms" in v}
    out["speedup_batched_mixed_vs_sequential_fp64"] = (
        t["sequential_fp64"] / t["batched_fp32"])
    out["speedup_batching_fp64"] = t["sequential_fp64"] / t["batched_fp64"]
    out["speedup_batching_mixed"] = t["sequential_fp32"] / t["batched_fp32"]
    out["speedup_precision_sequential"] = (t["sequential_fp64"]
                                           / t["sequential_fp32"])
    return out


def config_gradient(M, stream, flush, runs=5):
    """-div(a grad u) = f, a = exp(g) at every quadrature point, SIPG Q3 on
    32^3 Cartesian cells: forward solve, adjoint solve and the dL/da kernel
    (rtol 1e-13), with the directional fourth-order finite-difference check
    of the gradient along 3 seeded directions with standard normal entries
    (every coefficient value moves by about eps = 1e-4 max a)."""
    import numpy as np
    import torch
    from paper_1611_03029_gb300 import synthetic
    n, k = 32, 3
    op = M.Poisson(n, n, n, k, disc="dg")
    a_c, a_f = synthetic.log_coefficient((n, n, n), k + 1, seed=7)
    ac = torch.from_numpy(a_c).cuda()
    af = torch.from_numpy(a_f).cuda()
    t_set = stats(timed_runs(lambda: op.set_coefficient(ac, af), stream, 2))
    b = op.rhs(0)
    u, _, _ = op.solve(b, rtol=1e-13, max_it=300)
    ut = torch.from_numpy(
        synthetic.random_vector(op.n_dofs(), 8)).cuda() * u.norm() / \
        np.sqrt(op.n_dofs())
    res = {}

    def fwd_adj_grad():
        u, itf, _ = op.solve(b, rtol=1e-13, max_it=300)
        lam, ita, _ = op.solve((u - ut).contiguous(), rtol=1e-13, max_it=300)
        gc, gf = op.gradient(u, lam)
        res.update(u=u, lam=lam, gc=gc, gf=gf, itf=itf[0], ita=ita[0])
    fwd_adj_grad()
    t_all = stats(timed_runs(fwd_adj_grad, stream, runs, flush))
    u, lam, gc, gf = res["u"], res["lam"], res["gc"], res["gf"]
    t_g = stats(timed_runs(lambda: op.gradient(u, lam), stream, 20, flush))

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
        fd = (8 * (loss(dc, df, eps) - loss(dc, df, -eps))
              - (loss(dc, df, 2 * eps) - loss(dc, df, -2 * eps))) / (12 * eps)
        an = float((gc * dc).sum() + (gf * df).sum())
        checks.append(abs(fd - an) / abs(an))
    op.set_coefficient(ac, af)
    return {"dofs": op.n_dofs(), "cell_points": a_c.size,
            "face_points": a_f.size,
            "forward_adjoint_gradient": t_all, "gradient_kernel": t_g,
            "set_coefficient": t_set,
            "iterations": {"forward": res["itf"], "adjoint": res["ita"]},
            "fd_rel_errors": checks}


def run_config(args):
    import torch
    from paper_1611_03029_gb300 import build
    build.build()
    from paper_1611_03029_gb300 import mfpoisson as M
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32,
                        device="cuda")
    fn = {"latency": config_latency, "sweep": config_sweep,
          "batched": config_batched, "gradient": config_gradient}[
        args.workload]
    kw = {}
    if args.workload == "sweep":
        kw["degrees"] = [int(v) for v in args.degrees.split(",")]
    out = fn(M, stream, flush, **kw)
    print(json.dumps({"workload": args.workload, **out}), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "solve":
        run_ours(args)
    else:
        run_config(args)


if __name__ == "__main__":
    main()
