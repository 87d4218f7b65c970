"""Time the operator apply of one configuration with CUDA events.

    python -m paper_1611_03029_gb300.profile_apply --disc dg --cells 32 \
        --degree 4 --curved --prec f64 --reps 20

Builds a single-level context (its setup runs `eig_cg_iters` applies), does
`--warmup` untimed applies, then `--reps` timed ones, and prints one JSON
line with the mean time per apply and dofs per second.  Used for the ncu
captures summarised under profiles/ and for choosing cells per block
(environment variable MFP_CELLS_PER_BLOCK).
"""
import argparse
import json
import os
import sys


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--disc", default="cg", choices=["cg", "dg"])
    ap.add_argument("--cells", type=int, default=32)
    ap.add_argument("--degree", type=int, default=4)
    ap.add_argument("--curved", action="store_true")
    ap.add_argument("--prec", default="f64", choices=["f64", "f32"])
    ap.add_argument("--arith", default="df", choices=["df", "native"],
                    help="float64 arithmetic: double-float or DFMA")
    ap.add_argument("--nrhs", type=int, default=1)
    ap.add_argument("--hdg", action="store_true",
                    help="the HDG mixed operator on (q, u) (SIPG cells, "
                         "float64)")
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--reps", type=int, default=20)
    a = ap.parse_args(argv)

    import torch
    here = os.path.dirname(os.path.abspath(__file__))
    sys.path.insert(0, os.path.dirname(here))
    from paper_1611_03029_gb300 import build, mfpoisson as M
    build.build()
    n = a.cells
    op = M.Poisson(n, n, n, a.degree, disc=a.disc,
                   mapping="sine" if a.curved else "identity",
                   map_param=0.1 if a.curved else 0.0, n_levels=1,
                   mg_precision="fp64" if a.prec == "f64" else "fp32",
                   fp64_arith=a.arith)
    dt = torch.float64 if a.prec == "f64" else torch.float32
    N = op.n_dofs()
    if a.hdg:
        if a.disc != "dg" or a.prec != "f64" or a.nrhs != 1:
            raise SystemExit("--hdg needs --disc dg, f64 and one column")
        src = torch.randn(4 * N, dtype=dt, device="cuda")

        def run(x, y):
            op.hdg_apply(x, y)
    else:
        src = torch.randn(N * a.nrhs, dtype=dt, device="cuda")

        def run(x, y):
            op.apply(x, y, n_rhs=a.nrhs)
    dst = torch.empty_like(src)
    for _ in range(a.warmup):
        run(src, dst)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    for _ in range(a.reps):
        run(src, dst)
    e1.record()
    torch.cuda.synchronize()
    t = e0.elapsed_time(e1) / a.reps * 1e-3
    print(json.dumps({"disc": a.disc, "cells": n, "degree": a.degree,
                      "curved": a.curved, "prec": a.prec, "nrhs": a.nrhs,
                      "arith": a.arith if a.prec == "f64" else "f32",
                      "hdg": a.hdg, "unknowns": src.numel(),
                      "dofs": N, "ms": t * 1e3,
                      "MDoF_s": N * a.nrhs / t / 1e6,
                      "cells_per_block": os.environ.get(
                          "MFP_CELLS_PER_BLOCK", "default")}))


if __name__ == "__main__":
    main()
