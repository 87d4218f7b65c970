"""Pins of the oracle against values the paper prints: the L2 errors of its
three-dimensional example with a smooth solution (Sec. 5; three Gaussians on
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
