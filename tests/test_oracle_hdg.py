"""Pins of the HDG oracle (Sec. 2.3; the mixed operator of Sec. 3, "HDG mixed
matrix-free"): the L2 errors the paper prints for the HDG solution and its
post-processing on the smooth 3D example, exact reproduction of a quadratic
solution, and the mixed form agreeing with the statically condensed one."""
import os

import numpy as np
import pytest
import scipy.sparse.linalg as spla

from oracle import cube, fem, hdg

HERE = os.path.dirname(os.path.abspath(__file__))


def golden():
    out = []
    for line in open(os.path.join(HERE, "golden",
                                  "paper_cube_hdg_l2_errors.txt")):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        k, cells, e, ep = line.split()
        n = round(int(cells) ** (1.0 / 3.0))
        assert n ** 3 == int(cells)
        out.append((int(k), n, float(e), float(ep)))
    return out


def cube_problem(n, k, mapping="identity", sides=(0, 2, 4)):
    return fem.Problem(n, n, n, k, disc="dg", mapping=mapping,
                       amp=0.1 if mapping == "sine" else 0.0,
                       box=(-1.0, 1.0), neumann_sides=sides)


@pytest.mark.parametrize("k,n,paper,paper_post", golden())
def test_hdg_l2_errors_match_paper(k, n, paper, paper_post):
    P = cube_problem(n, k)
    sol = hdg.solve(P, cube.f, cube.u, cube.grad_u)
    err = fem.l2_error(P, sol.U, cube.u)
    assert abs(err / paper - 1.0) <= 2e-3, (err, paper)
    ust, P2 = hdg.postprocess(P, sol)
    errp = fem.l2_error(P2, ust, cube.u)
    assert abs(errp / paper_post - 1.0) <= 1e-2, (errp, paper_post)


def _quad_u(x):
    X, Y, Z = x[..., 0], x[..., 1], x[..., 2]
    return 1.0 + X - 2.0 * Y + 0.5 * Z + X * Y - Z * Z + 0.3 * Y * Z


def _quad_grad(x):
    X, Y, Z = x[..., 0], x[..., 1], x[..., 2]
    return np.stack([1.0 + Y, -2.0 + X + 0.3 * Z, 0.5 - 2.0 * Z + 0.3 * Y], -1)


def _quad_f(x):
    return np.full(x.shape[:-1], 2.0)


@pytest.mark.parametrize("sides", [(0, 2, 4), (1, 3), ()])
def test_hdg_reproduces_quadratics(sides):
    # u in Q_2 and q = -grad u in Q_1^3: the HDG solution is exact (a
    # consistent method with every integral exact on affine cells)
    P = cube_problem(2, 2, sides=sides)
    sol = hdg.solve(P, _quad_f, _quad_u, _quad_grad)
    assert np.abs(sol.U - fem.interpolate(P, _quad_u)).max() < 1e-11
    X = P.node_points()
    qx = -_quad_grad(X)                                 # [ndofs, 3]
    q = sol.Q.transpose(0, 2, 1).reshape(-1, 3)         # node-major
    assert np.abs(q - qx).max() < 1e-10


def test_hdg_wrong_flux_sign_is_not_exact():
    # flipping the Neumann flux (the sign the printed weak form suggests)
    P = cube_problem(2, 2, sides=(0, 3))
    sol = hdg.solve(P, _quad_f, _quad_u, lambda x: -_quad_grad(x))
    assert np.abs(sol.U - fem.interpolate(P, _quad_u)).max() > 1e-2


@pytest.mark.parametrize("mapping,sides", [("identity", (0, 2, 4)),
                                           ("sine", (1,)), ("sine", ())])
def test_mixed_form_equals_condensed_solution(mapping, sides):
    # [A B^T; B D] + [C^T; G^T] H^-1 [C G] (symmetric) solved directly gives
    # the statically condensed solution
    P = fem.Problem(2, 3, 2, 2, disc="dg", mapping=mapping,
                    amp=0.1 if mapping == "sine" else 0.0, box=(-1.0, 1.0),
                    neumann_sides=sides)
    sol = hdg.solve(P, cube.f, cube.u, cube.grad_u)
    A = hdg.mixed_operator(P)
    assert abs(A - A.T).max() <= 1e-14 * abs(A).max()
    X = spla.spsolve(A.tocsc(), hdg.mixed_rhs(P, cube.f, cube.u, cube.grad_u))
    assert np.abs(X - sol.X).max() <= 1e-11 * np.abs(sol.X).max()


def _sine_grad(x):
    s, c = np.sin(np.pi * x), np.cos(np.pi * x)
    return np.pi * np.stack([c[..., 0] * s[..., 1] * s[..., 2],
                             s[..., 0] * c[..., 1] * s[..., 2],
                             s[..., 0] * s[..., 1] * c[..., 2]], -1)


def test_hdg_converges_at_k_plus_1_and_post_at_k_plus_2():
    # optimal rates (Sec. 4.3: k+1 for u_h, k+2 after post-processing), Q2 on
    # 2^3 and 4^3 affine cells
    errs, post = [], []
    for n in (2, 4):
        P = fem.Problem(n, n, n, 2, disc="dg")
        sol = hdg.solve(P, fem.sine_forcing, fem.sine_solution, _sine_grad)
        errs.append(fem.l2_error(P, sol.U, fem.sine_solution))
        ust, P2 = hdg.postprocess(P, sol)
        post.append(fem.l2_error(P2, ust, fem.sine_solution))
    assert np.log2(errs[0] / errs[1]) > 3 - 0.3, errs
    assert np.log2(post[0] / post[1]) > 4 - 0.3, post


@pytest.mark.parametrize("mapping,sides", [("identity", (0, 2, 4)),
                                           ("sine", (5,))])
def test_mixed_rows_of_listed_cells(mapping, sides):
    # the per-cell evaluation used at sizes too large to assemble agrees
    # with the assembled mixed operator
    P = fem.Problem(3, 2, 3, 2, disc="dg", mapping=mapping,
                    amp=0.1 if mapping == "sine" else 0.0, box=(-1.0, 1.0),
                    neumann_sides=sides)
    A = hdg.mixed_operator(P)
    x = np.random.default_rng(5).standard_normal(A.shape[0])
    ref = (A @ x).reshape(P.ncells, -1)
    cells = np.array([0, 4, P.ncells - 1, 7])
    got = hdg.mixed_apply_cells(P, x, cells)
    assert np.abs(got - ref[cells]).max() <= 1e-13 * np.abs(ref).max()
