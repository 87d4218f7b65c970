"""The paper's three-dimensional example with a smooth solution (Sec. 4.3,
"Three-dimensional example with smooth solution"): u is a sum of three
Gaussians of width alpha = 1/5 on the cube (-1, 1)^3, with Neumann data on
the sides x_e = -1 and Dirichlet data on the sides x_e = +1, kappa = 1.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).  Used to pin the oracle's
assembly, load vector, boundary data and L2 error against the L2 errors the
paper prints for this example."""
import numpy as np

from oracle import fem

ALPHA = 0.2
CENTERS = np.array([[-0.5, 0.5, 0.25],
                    [-0.6, -0.5, -0.125],
                    [0.5, -0.5, 0.5]])
SCALE = (1.0 / (ALPHA * np.sqrt(2.0 * np.pi))) ** 3


def _gauss_terms(x):
    x = np.asarray(x, float)
    d = x[..., None, :] - CENTERS                       # [..., 3 centers, 3]
    r2 = np.sum(d * d, axis=-1)
    return d, r2, np.exp(-r2 / ALPHA ** 2)


def u(x):
    """u(x) = (1 / (alpha sqrt(2 pi)))^3 sum_j exp(-|x - x_j|^2 / alpha^2)."""
    _, _, e = _gauss_terms(x)
    return SCALE * e.sum(-1)


def grad_u(x):
    d, _, e = _gauss_terms(x)
    return SCALE * np.sum((-2.0 / ALPHA ** 2) * d * e[..., None], axis=-2)


def f(x):
    """f = -Laplace(u): Laplace exp(-r^2/a^2) = exp(-r^2/a^2)(4 r^2/a^4 -
    6/a^2) in three dimensions."""
    _, r2, e = _gauss_terms(x)
    return -SCALE * np.sum(e * (4.0 * r2 / ALPHA ** 4 - 6.0 / ALPHA ** 2),
                           axis=-1)


def problem(n, k, disc="cg", penalty_factor=1.0):
    """n^3 cells on (-1, 1)^3; Neumann on x_e = -1 (sides 0, 2, 4),
    Dirichlet on x_e = +1."""
    return fem.Problem(n, n, n, k, disc=disc, box=(-1.0, 1.0),
                       neumann_sides=(0, 2, 4),
                       penalty_factor=penalty_factor)


def l2_error(n, k, disc="cg", penalty_factor=1.0):
    """||u_h - u||_L2 of the discrete solution on n^3 cells."""
    P = problem(n, k, disc, penalty_factor)
    x = fem.solve_manufactured(P, f, u, grad_u)
    return fem.l2_error(P, x, u)
