"""Launch each of the library's vector, transfer, coarse-solve, gradient and
HDG kernels a few times on one configuration, in a fixed order, for ncu
captures of those kernels (the operator applies have profile_apply).

    python -m paper_1611_03029_gb300.profile_kernels --cells 32 --degree 4

On 32^3 curved Q4 cells (the timed workload's finest level) it runs, after
the contexts' set-up:
  CG context:   one smoother pass from a non-zero start on the finest level
                (k_cheb_first, k_cheb_step after the CG applies), one
                restriction and one prolongation to / from the next level,
                the coarse solve on the coarsest level (k_dense_apply), two
                PCG iterations (k_dot, k_cg_update, k_cg_p and a V-cycle);
  SIPG context: one gradient (k_grad_cells, k_grad_faces);
  SIPG context on Cartesian cells: one HDG mixed apply (k_hdg_trace per
                face direction, k_hdg_cell).
Each step runs inside the NVTX range "profile".  Prints one JSON line with
the wall time of each step.
"""
import argparse
import json
import os
import sys
import time


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--cells", type=int, default=32)
    ap.add_argument("--degree", type=int, default=4)
    a = ap.parse_args(argv)

    import torch
    here = os.path.dirname(os.path.abspath(__file__))
    sys.path.insert(0, os.path.dirname(here))
    from paper_1611_03029_gb300 import build, mfpoisson as M
    build.build()
    n, k = a.cells, a.degree
    cg = M.Poisson(n, n, n, k, disc="cg", mapping="sine", map_param=0.1)
    dg = M.Poisson(n, n, n, k, disc="dg", mapping="sine", map_param=0.1,
                   n_levels=1)
    hd = M.Poisson(n, n, n, k, disc="dg", n_levels=1)
    torch.cuda.synchronize()
    out = {}

    def step(name, fn):
        # each step inside the NVTX range "profile" (ncu --nvtx-include), so
        # that a capture skips the contexts' set-up launches
        t0 = time.time()
        torch.cuda.nvtx.range_push("profile")
        fn()
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
        out[name] = time.time() - t0

    top = cg.n_levels - 1
    N = cg.n_dofs()
    b = torch.randn(N, dtype=torch.float64, device="cuda")
    x = torch.randn(N, dtype=torch.float64, device="cuda")
    step("smooth", lambda: cg.smooth(b, x, level=top))
    xc = cg.restrict(x, top)
    step("restrict", lambda: cg.restrict(x, top))
    step("prolongate", lambda: cg.prolongate(xc, top))
    b0 = torch.randn(cg.n_dofs(0), dtype=torch.float64, device="cuda")
    step("coarse_solve", lambda: cg.smooth(b0, level=0))
    rhs = cg.rhs(0)
    step("pcg_2", lambda: cg.solve(rhs, rtol=1e-10, max_it=2,
                                   raise_on_fail=False))
    Nd = dg.n_dofs()
    u = torch.randn(Nd, dtype=torch.float64, device="cuda")
    lam = torch.randn(Nd, dtype=torch.float64, device="cuda")
    step("gradient", lambda: dg.gradient(u, lam))
    q = torch.randn(4 * hd.n_dofs(), dtype=torch.float64, device="cuda")
    step("hdg_apply", lambda: hd.hdg_apply(q))
    print(json.dumps({"cells": n, "degree": k, "steps_s": out}))


if __name__ == "__main__":
    main()
