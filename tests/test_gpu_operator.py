"""Parity of the CUDA operator apply (Eq. 12 with the SIPG terms of Eq. 6/7)
with the oracle's assembled matrix, element by element.

float64: max |y_gpu - y_oracle| <= 1e-12 max |y_oracle| (the 1e-12 target).
float32: 2e-5 max |y_oracle| (float rounding of O(p) sums of O(1) terms over
about 10 sweeps; the float path only serves inside the preconditioner)."""
import numpy as np
import pytest
import torch

from conftest import rel_err
from oracle import fem, rows
from paper_1611_03029_gb300 import synthetic

pytestmark = pytest.mark.gpu

TOL64 = 1e-12
TOL32 = 2e-5


def cases():
    out = []
    for disc in ("cg", "dg"):
        for mapping in ("identity", "sine"):
            for k in range(1, 9):
                # several blocks of cells and a ragged tail at every degree
                n = (3, 5, 5) if k <= 3 else ((3, 2, 3) if k <= 5 else (3, 2, 1))
                out.append((disc, mapping, k, n))
    return out


@pytest.mark.parametrize("disc,mapping,k,n", cases())
def test_apply_matches_oracle_fp64(mfp, disc, mapping, k, n):
    # both float64 arithmetics: double-float on the FP32 pipes (default) and
    # native DFMA
    amp = 0.1 if mapping == "sine" else 0.0
    P = fem.Problem(*n, k, disc=disc, mapping=mapping, amp=amp)
    A = fem.assemble(P)
    u = synthetic.random_vector(P.n_dofs, seed=100 + k)
    ref = A @ u
    for arith in ("df", "native"):
        op = mfp.Poisson(*n, k, disc=disc, mapping=mapping, map_param=amp,
                         n_levels=1, fp64_arith=arith)
        y = op.apply(torch.from_numpy(u).cuda()).cpu().numpy()
        assert rel_err(y, ref) <= TOL64, arith
    # anisotropic penalty / normals: same with the paper's penalty factor
    if disc == "dg" and k == 2:
        op3 = mfp.Poisson(*n, k, disc=disc, mapping=mapping, map_param=amp,
                          n_levels=1, penalty_factor=3.0)
        P3 = fem.Problem(*n, k, disc=disc, mapping=mapping, amp=amp,
                         penalty_factor=3.0)
        y3 = op3.apply(torch.from_numpy(u).cuda()).cpu().numpy()
        assert rel_err(y3, fem.assemble(P3) @ u) <= TOL64


@pytest.mark.parametrize("disc,mapping,k", [("cg", "identity", 2),
                                            ("cg", "sine", 4),
                                            ("dg", "identity", 3),
                                            ("dg", "sine", 4)])
def test_apply_matches_oracle_fp32(mfp, disc, mapping, k):
    n = (3, 4, 5)
    amp = 0.1 if mapping == "sine" else 0.0
    op = mfp.Poisson(*n, k, disc=disc, mapping=mapping, map_param=amp,
                     n_levels=1, mg_precision="fp32")
    P = fem.Problem(*n, k, disc=disc, mapping=mapping, amp=amp)
    u = synthetic.random_vector(P.n_dofs, seed=7).astype(np.float32)
    y = op.apply(torch.from_numpy(u).cuda()).cpu().numpy()
    ref = fem.assemble(P) @ u.astype(np.float64)
    assert rel_err(y, ref) <= TOL32


@pytest.mark.parametrize("disc", ["cg", "dg"])
@pytest.mark.parametrize("arith", ["df", "native"])
def test_variable_coefficient_apply(mfp, disc, arith):
    n, k = (4, 2, 3), 3
    p = k + 1
    a_cell, a_face = synthetic.log_coefficient(n, p, seed=7)
    op = mfp.Poisson(*n, k, disc=disc, n_levels=1, fp64_arith=arith)
    op.set_coefficient(torch.from_numpy(a_cell).cuda().contiguous(),
                       torch.from_numpy(a_face).cuda().contiguous())
    P = fem.Problem(*n, k, disc=disc, a_cell=a_cell, a_face=a_face)
    u = synthetic.random_vector(P.n_dofs, seed=3)
    y = op.apply(torch.from_numpy(u).cuda()).cpu().numpy()
    assert rel_err(y, fem.assemble(P) @ u) <= TOL64


@pytest.mark.parametrize("disc", ["cg", "dg"])
def test_batched_apply_equals_columns(mfp, disc):
    n, k, R = (3, 2, 4), 2, 5
    op = mfp.Poisson(*n, k, disc=disc, mapping="sine", map_param=0.1,
                     n_levels=1)
    N = op.n_dofs()
    U = synthetic.random_vector(N, seed=9, ncols=R)
    Ut = torch.from_numpy(np.ascontiguousarray(U)).cuda()
    Y = op.apply(Ut.reshape(-1), n_rhs=R).reshape(N, R).cpu().numpy()
    A = fem.assemble(fem.Problem(*n, k, disc=disc, mapping="sine", amp=0.1))
    assert rel_err(Y, A @ U) <= TOL64


@pytest.mark.parametrize("disc", ["cg", "dg"])
@pytest.mark.parametrize("arith", ["df", "native"])
def test_full_size_curved_q4_sampled_rows(mfp, disc, arith):
    # 32^3 cells, Q4, curved: the apply-throughput workload; the oracle
    # evaluates sampled rows one by one.
    n, k = (32, 32, 32), 4
    op = mfp.Poisson(*n, k, disc=disc, mapping="sine", map_param=0.1,
                     n_levels=1, fp64_arith=arith)
    N = op.n_dofs()
    u = synthetic.random_vector(N, seed=21)
    y = op.apply(torch.from_numpy(u).cuda()).cpu().numpy()
    P = fem.Problem(*n, k, disc=disc, mapping="sine", amp=0.1)
    rng = np.random.default_rng(5)
    r = np.concatenate([rng.choice(N, 40, replace=False), [0, N - 1, N // 2]])
    ref = rows.apply_rows(P, u, r)
    scale = np.abs(ref).max()
    assert np.abs(y[r] - ref).max() <= TOL64 * scale


def test_rhs_matches_oracle(mfp):
    for disc, mapping in (("cg", "sine"), ("dg", "identity")):
        n, k = (3, 4, 2), 3
        amp = 0.1 if mapping == "sine" else 0.0
        op = mfp.Poisson(*n, k, disc=disc, mapping=mapping, map_param=amp,
                         n_levels=1)
        P = fem.Problem(*n, k, disc=disc, mapping=mapping, amp=amp)
        b = op.rhs(0).cpu().numpy()
        assert rel_err(b, fem.load_vector(P, fem.sine_forcing)) <= 1e-12
        g = synthetic.gaussian_terms(1000)
        b = op.rhs(1, g).cpu().numpy()
        ref = fem.load_vector(P, synthetic.gaussian_forcing(g))
        assert rel_err(b, ref) <= 1e-12


@pytest.mark.parametrize("mapping", ["identity", "sine"])
@pytest.mark.parametrize("k", [1, 2, 3, 4])
def test_warp_per_cell_cg_float(mfp, mapping, k, monkeypatch):
    # the float CG kernel that gives each cell one warp (k <= 4), selected by
    # the cells-per-block override 1000, on a mesh with several warps' worth
    # of cells and a ragged tail; also through a V-cycle of the float
    # hierarchy (every level)
    amp = 0.1 if mapping == "sine" else 0.0
    n = (5, 3, 4)
    P = fem.Problem(*n, k, mapping=mapping, amp=amp)
    u = synthetic.random_vector(P.n_dofs, seed=300 + k)
    op = mfp.Poisson(*n, k, mapping=mapping, map_param=amp, n_levels=1,
                     mg_precision="fp32")
    ref = fem.assemble(P) @ u
    y0 = op.apply(torch.from_numpy(u).float().cuda()).cpu().numpy()
    monkeypatch.setenv("MFP_CELLS_PER_BLOCK", "1000")
    y = op.apply(torch.from_numpy(u).float().cuda()).cpu().numpy()
    assert rel_err(y, ref) <= TOL32
    assert rel_err(y, y0) <= TOL32
    monkeypatch.delenv("MFP_CELLS_PER_BLOCK")
    cells, ms = op.autotune(prec="fp32")
    assert cells >= 0 and ms > 0
    y1 = op.apply(torch.from_numpy(u).float().cuda()).cpu().numpy()
    assert rel_err(y1, ref) <= TOL32
