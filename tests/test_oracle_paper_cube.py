"""Pins of the oracle against values the paper prints: the L2 errors of its
three-dimensional example with a smooth solution (Sec. 4.3; three Gaussians on
(-1, 1)^3 with Neumann data on x_e = -1 and Dirichlet data on x_e = +1).

These check the oracle's cell integrals under the isoparametric map, the
(k+1)-point Gauss load vector, the Neumann and Dirichlet data (lifted
Dirichlet values for CG, the extension of Eq. 7 for SIPG), the SIPG face
terms with the paper's penalty (k+1)^2 d / h (penalty_factor = d = 3) and the
L2 error.  A dropped term, a wrong sign or the other penalty moves the
errors by several percent; the printed values have four digits."""
import os

import numpy as np
import pytest

from oracle import cube, fem

HERE = os.path.dirname(os.path.abspath(__file__))


def golden():
    out = []
    for line in open(os.path.join(HERE, "golden", "paper_cube_l2_errors.txt")):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        disc, k, cells, err = line.split()
        n = round(int(cells) ** (1.0 / 3.0))
        assert n ** 3 == int(cells)
        out.append((disc, int(k), n, float(err)))
    return out


@pytest.mark.parametrize("disc,k,n,paper", golden())
def test_l2_error_matches_paper(disc, k, n, paper):
    pf = 3.0 if disc == "dg" else 1.0
    err = cube.l2_error(n, k, disc, penalty_factor=pf)
    assert abs(err / paper - 1.0) <= 5e-3, (err, paper)


def test_sipg_penalty_reading():
    # the workload's penalty (k+1)^2 / h (factor 1) does not reproduce the
    # printed SIPG error: the paper's own results use (k+1)^2 d / h
    err1 = cube.l2_error(8, 1, "dg", penalty_factor=1.0)
    assert abs(err1 / 3.759e-01 - 1.0) > 0.1


def test_boundary_data_are_consistent():
    # the exact solution's own data: f = -Laplace(u) by a second-order
    # finite difference, and the Neumann side only carries natural data
    rng = np.random.default_rng(3)
    x = rng.uniform(-0.9, 0.9, (20, 3))
    h = 1e-3
    lap = sum((cube.u(x + h * e) - 2 * cube.u(x) + cube.u(x - h * e)) / h ** 2
              for e in np.eye(3))
    assert np.allclose(-lap, cube.f(x), rtol=1e-3, atol=1e-3)
    g = np.stack([(cube.u(x + h * e) - cube.u(x - h * e)) / (2 * h)
                  for e in np.eye(3)], -1)
    assert np.allclose(g, cube.grad_u(x), rtol=1e-4, atol=1e-6)
    P = cube.problem(2, 1)
    c = P.constrained()
    pts = P.node_points()
    # Dirichlet exactly on the nodes with some coordinate at +1
    assert np.array_equal(c, np.any(np.isclose(pts, 1.0), axis=1))


# ---------------------------------------------------------------------------
# Exactness: a quadratic u lies in Q_k (k >= 2) and every integrand on affine
# cells is a polynomial the (k+1)-point Gauss rule integrates exactly, so
# CG (interpolated Dirichlet data, Sec. 2.1) and SIPG (Eq. 6 / Eq. 7, a
# consistent method) both return u itself, whatever the Neumann sides.
# ---------------------------------------------------------------------------
def _quad_u(x):
    X, Y, Z = x[..., 0], x[..., 1], x[..., 2]
    return 1.0 + X - 2.0 * Y + 0.5 * Z + X * Y - Z * Z + 0.3 * Y * Z


def _quad_grad(x):
    X, Y, Z = x[..., 0], x[..., 1], x[..., 2]
    return np.stack([1.0 + Y, -2.0 + X + 0.3 * Z, 0.5 - 2.0 * Z + 0.3 * Y], -1)


def _quad_f(x):
    return np.full(x.shape[:-1], 2.0)      # -Laplace(u)


@pytest.mark.parametrize("disc", ["cg", "dg"])
@pytest.mark.parametrize("sides,box", [((0, 2, 4), (-1.0, 1.0)),
                                       ((1, 3), (0.0, 1.0)),
                                       ((5,), (-0.5, 2.0)),
                                       ((), (-1.0, 1.0))])
def test_boundary_data_reproduce_quadratics(disc, sides, box):
    P = fem.Problem(2, 3, 2, 2, disc=disc, box=box, neumann_sides=sides,
                    penalty_factor=3.0)
    x = fem.solve_manufactured(P, _quad_f, _quad_u, _quad_grad)
    assert np.abs(x - fem.interpolate(P, _quad_u)).max() < 1e-11


def test_neumann_term_sign_matters():
    # flipping the Neumann data (a wrong normal orientation) breaks exactness
    P = fem.Problem(2, 2, 2, 2, box=(-1.0, 1.0), neumann_sides=(0, 3))
    x = fem.solve_manufactured(P, _quad_f, _quad_u, lambda y: -_quad_grad(y))
    assert np.abs(x - fem.interpolate(P, _quad_u)).max() > 1e-3
