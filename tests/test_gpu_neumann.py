"""Neumann sides, the box domain and the boundary-data right-hand side
(f_kind 2) against the oracle, and the paper's smooth three-dimensional
example (Sec. 4.3: three Gaussians on (-1, 1)^3, Neumann data on x_e = -1,
Dirichlet data on x_e = +1) solved on the GPU against the L2 errors the
paper prints.

Tolerances as for the all-Dirichlet operator: float64 applies 1e-12 of the
largest entry, float32 2e-5.  The right-hand side of f_kind 2 holds the
lifted Dirichlet data (CG: sums of p^6 products per cell that cancel to the
size of the other terms) and penalty-weighted data (SIPG), so it gets 1e-11.
"""
import numpy as np
import pytest
import torch

from conftest import rel_err
from oracle import adjoint, cube, fem, mg
from paper_1611_03029_gb300 import synthetic

pytestmark = pytest.mark.gpu

BOX = (-1.0, 1.0)
SIDES = [(0, 2, 4), (1,), (3, 4, 5)]


def cuda(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def cube_params():
    """The paper's three Gaussians as f_kind 2 parameter blocks."""
    return np.array([[c[0], c[1], c[2], cube.ALPHA, cube.SCALE]
                     for c in cube.CENTERS])


def problem(disc, mapping, k, n, sides, penalty_factor=1.0, kappa=1.0):
    amp = 0.1 if mapping == "sine" else 0.0
    return fem.Problem(*n, k, disc=disc, mapping=mapping, amp=amp, box=BOX,
                       neumann_sides=sides, penalty_factor=penalty_factor,
                       kappa=kappa)


def pair(mfp, disc, mapping, k, n, sides, **kw):
    amp = 0.1 if mapping == "sine" else 0.0
    op = mfp.Poisson(*n, k, disc=disc, mapping=mapping, map_param=amp,
                     neumann_sides=sides, box=BOX, **kw)
    P = problem(disc, mapping, k, n, sides,
                penalty_factor=kw.get("penalty_factor", 1.0),
                kappa=kw.get("kappa", 1.0))
    return op, P


@pytest.mark.parametrize("disc", ["cg", "dg"])
@pytest.mark.parametrize("mapping", ["identity", "sine"])
@pytest.mark.parametrize("k,n", [(2, (3, 4, 2)), (4, (3, 2, 2))])
@pytest.mark.parametrize("sides", SIDES)
def test_apply_with_neumann_sides(mfp, disc, mapping, k, n, sides):
    P = problem(disc, mapping, k, n, sides)
    A = fem.assemble(P)
    u = synthetic.random_vector(P.n_dofs, seed=40 + k)
    ref = A @ u
    for arith in ("df", "native"):
        op2, _ = pair(mfp, disc, mapping, k, n, sides, n_levels=1,
                      fp64_arith=arith)
        y = op2.apply(cuda(u)).cpu().numpy()
        assert rel_err(y, ref) <= 1e-12, arith
    op32, _ = pair(mfp, disc, mapping, k, n, sides, n_levels=1,
                   mg_precision="fp32")
    u32 = u.astype(np.float32)
    y32 = op32.apply(cuda(u32)).cpu().numpy()
    assert rel_err(y32, A @ u32.astype(np.float64)) <= 2e-5


@pytest.mark.parametrize("disc,mapping,k", [("cg", "identity", 2),
                                            ("cg", "sine", 3),
                                            ("dg", "identity", 2),
                                            ("dg", "sine", 1)])
def test_multigrid_pieces_with_neumann_sides(mfp, disc, mapping, k):
    n, sides = (4, 4, 4), (0, 2, 4)
    op, P = pair(mfp, disc, mapping, k, n, sides)
    V = mg.VCycle(P)
    probs = mg.hierarchy(P)
    for lv, L in enumerate(V.levels):
        assert rel_err(op.inverse_diagonal(lv).cpu().numpy(), L.dinv) <= 1e-12
        info = op.level_info(lv)
        assert abs(info["lam_max"] - L.lam_max) <= 1e-9 * L.lam_max
    for lv in range(1, len(probs)):
        Pm = mg.prolongation(probs[lv], probs[lv - 1])
        xc = synthetic.random_vector(probs[lv - 1].n_dofs, seed=lv)
        xf = synthetic.random_vector(probs[lv].n_dofs, seed=10 + lv)
        assert rel_err(op.prolongate(cuda(xc), lv).cpu().numpy(),
                       Pm @ xc) <= 1e-13
        assert rel_err(op.restrict(cuda(xf), lv).cpu().numpy(),
                       Pm.T @ xf) <= 1e-13
    r = synthetic.random_vector(P.n_dofs, seed=3)
    r[P.constrained()] = 0.0
    assert rel_err(op.vcycle(cuda(r)).cpu().numpy(), V.apply(r)) <= 1e-9


@pytest.mark.parametrize("disc,mapping,k,n,sides,kappa", [
    ("cg", "identity", 2, (3, 4, 2), (0, 2, 4), 1.0),
    ("cg", "sine", 3, (2, 3, 2), (1, 3), 2.5),
    ("dg", "identity", 2, (3, 4, 2), (0, 2, 4), 1.0),
    ("dg", "sine", 3, (2, 3, 2), (5,), 2.5)])
def test_boundary_data_rhs(mfp, disc, mapping, k, n, sides, kappa):
    op, P = pair(mfp, disc, mapping, k, n, sides, n_levels=1, kappa=kappa,
                 penalty_factor=3.0)
    b = op.rhs(2, cube_params()).cpu().numpy()
    ref = fem.manufactured_rhs(P, lambda x: kappa * cube.f(x), cube.u,
                               cube.grad_u)
    assert rel_err(b, ref) <= 1e-11
    # a column of a batch (stride) gets the same values; CG rows are sums
    # of atomic adds in arbitrary order, equal up to rounding
    R = 3
    out = torch.zeros(P.n_dofs * R, dtype=torch.float64, device="cuda")
    op.rhs(2, cube_params(), out=out[1:], stride=R)
    col = out.reshape(-1, R)[:, 1].cpu().numpy()
    if disc == "dg":
        assert np.array_equal(col, b)
    else:
        assert rel_err(col, b) <= 1e-14


@pytest.mark.parametrize("disc,k,n,limit", [("cg", 2, (8, 8, 8), 20),
                                            ("dg", 2, (8, 8, 8), 40)])
def test_solve_with_boundary_data(mfp, disc, k, n, limit):
    pf = 3.0 if disc == "dg" else 1.0
    op, P = pair(mfp, disc, "sine", k, n, (0, 2, 4), penalty_factor=pf)
    b = op.rhs(2, cube_params())
    x, its, _ = op.solve(b, rtol=1e-10, max_it=200)
    A = fem.assemble(P)
    bh, xh = b.cpu().numpy(), x.cpu().numpy()
    assert np.linalg.norm(bh - A @ xh) / np.linalg.norm(bh) <= 1.05e-10
    assert its[0] <= limit
    xd = fem.solve_manufactured(P, cube.f, cube.u, cube.grad_u)
    assert rel_err(xh, xd) <= 1e-7
    # the mixed-precision solve (float V-cycle) reaches the same solution
    opm, _ = pair(mfp, disc, "sine", k, n, (0, 2, 4), penalty_factor=pf,
                  mg_precision="fp32")
    xm, _, _ = opm.solve(opm.rhs(2, cube_params()), rtol=1e-10, max_it=200)
    assert rel_err(xm.cpu().numpy(), xd) <= 1e-7


# rows of the paper's error table that the GPU solves here (n^3 cells)
PAPER_ROWS = [("cg", 1, 8, 4.241e-01), ("cg", 3, 8, 1.491e-02),
              ("cg", 4, 4, 5.924e-02), ("cg", 5, 4, 2.366e-02),
              ("dg", 1, 8, 3.759e-01), ("dg", 2, 8, 1.264e-01),
              ("dg", 3, 4, 2.481e-01)]


@pytest.mark.parametrize("disc,k,n,paper", PAPER_ROWS)
def test_paper_cube_l2_error(mfp, disc, k, n, paper):
    # SIPG with the paper's penalty (k+1)^2 d / h, d = 3
    pf = 3.0 if disc == "dg" else 1.0
    op = mfp.Poisson(n, n, n, k, disc=disc, neumann_sides=(0, 2, 4), box=BOX,
                     penalty_factor=pf)
    x, _, rel = op.solve(op.rhs(2, cube_params()), rtol=1e-10, max_it=300)
    assert rel[0] <= 1e-10
    P = cube.problem(n, k, disc, penalty_factor=pf)
    err = fem.l2_error(P, x.cpu().numpy(), cube.u)
    assert abs(err / paper - 1.0) <= 5e-3, (err, paper)


@pytest.mark.parametrize("disc", ["cg", "dg"])
def test_gradient_with_neumann_sides(mfp, disc):
    n, k, sides = (3, 2, 4), 3, (1, 2)
    op, P = pair(mfp, disc, "sine", k, n, sides, n_levels=1)
    u = synthetic.random_vector(P.n_dofs, 1)
    lam = synthetic.random_vector(P.n_dofs, 2)
    gc, gf = op.gradient(cuda(u), cuda(lam))
    rc, rf = adjoint.gradient(P, u, lam)
    assert rel_err(gc.cpu().numpy(), rc) <= 1e-12
    if disc == "dg":
        assert rel_err(gf.cpu().numpy(), rf) <= 1e-12


# ---------------------------------------------------------------------------
# Strongly varying coefficient (the paper's shell diffusivity on the brick
# (-1, 1)^3, contrast 10^6; synthetic.strong_coefficient): the GPU hierarchy
# takes the same V-cycle as the oracle's, so PCG needs the oracle's
# iteration count, and the solution meets the residual on the oracle's
# matrix.
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("disc,k,n", [("cg", 2, 8), ("dg", 2, 8),
                                      ("cg", 3, 8), ("dg", 1, 8)])
def test_strong_coefficient_solve(mfp, disc, k, n):
    N3 = (n, n, n)
    a_cell, a_face = synthetic.strong_coefficient(N3, k + 1, box=BOX)
    op = mfp.Poisson(*N3, k, disc=disc, box=BOX)
    op.set_coefficient(cuda(a_cell), cuda(a_face))
    P = fem.Problem(*N3, k, disc=disc, box=BOX, a_cell=a_cell, a_face=a_face)
    b = op.rhs(0)
    x, its, _ = op.solve(b, rtol=1e-10, max_it=300)
    V = mg.VCycle(P)
    A = V.levels[-1].A
    bh, xh = b.cpu().numpy(), x.cpu().numpy()
    assert rel_err(bh, fem.load_vector(P, fem.sine_forcing)) <= 1e-12
    assert np.linalg.norm(bh - A @ xh) / np.linalg.norm(bh) <= 1.05e-10
    _, its_oracle = mg.pcg(A, bh, V.apply, rtol=1e-10, max_it=300)[:2]
    assert its[0] <= its_oracle + 1, (its, its_oracle)


@pytest.mark.parametrize("disc", ["cg", "dg"])
def test_full_size_neumann_sampled_rows(mfp, disc):
    # 32^3 cells, Q4, curved, the timed size, on (-1, 1)^3 with the Neumann
    # sides of the paper's example; rows sampled on those sides, on the
    # Dirichlet sides and inside
    from oracle import rows
    n, k, sides = (32, 32, 32), 4, (0, 2, 4)
    op = mfp.Poisson(*n, k, disc=disc, mapping="sine", map_param=0.1,
                     n_levels=1, neumann_sides=sides, box=BOX)
    N = op.n_dofs()
    u = synthetic.random_vector(N, seed=22)
    y = op.apply(cuda(u)).cpu().numpy()
    P = problem(disc, "sine", k, n, sides)
    rng = np.random.default_rng(7)
    r = np.concatenate([rng.choice(N, 30, replace=False),
                        [0, N - 1, N // 2, 1, N - 2]])
    ref = rows.apply_rows(P, u, r)
    assert np.abs(y[r] - ref).max() <= 1e-12 * np.abs(ref).max()
