"""Pins of the oracle's multigrid pieces (Sec. 4.1) against closed forms
(Q1 spectrum, Chebyshev polynomials), library routines and invariants."""
import numpy as np
import pytest
import scipy.linalg as sla
from numpy.polynomial import chebyshev as npcheb

from oracle import fem, mg


def q1_spectrum(n):
    """Eigenvalues of the Dirichlet Q1 stiffness on an n^3 Cartesian mesh of
    the unit cube: sum over axes of a(t_d) prod_{e != d} m(t_e) with
    a(t) = (2 - 2 cos t)/h, m(t) = h (4 + 2 cos t)/6, t = j pi / n."""
    h = 1.0 / n
    t = np.arange(1, n) * np.pi / n
    a = (2 - 2 * np.cos(t)) / h
    m = h * (4 + 2 * np.cos(t)) / 6
    A = np.einsum("i,j,k->ijk", a, m, m)
    return (A + A.transpose(1, 0, 2) + A.transpose(1, 2, 0)).ravel()


def test_q1_spectrum_closed_form():
    n = 4
    P = fem.Problem(n, n, n, 1)
    ev = np.sort(np.linalg.eigvalsh(fem.assemble(P).toarray()))
    nb = P.constrained().sum()
    ref = np.sort(np.concatenate([q1_spectrum(n), np.ones(nb)]))
    assert np.allclose(ev, ref, atol=1e-13)


def test_eigen_estimate_q1_cartesian():
    n = 8
    P = fem.Problem(n, n, n, 1)
    L = mg.Level(P)
    exact = q1_spectrum(n).max() * 3.0 / (8.0 / n)        # D = 8h/3
    assert 0.9 * exact <= L.lam_max <= exact * (1 + 1e-12)


def test_lanczos_exact_on_small_spd():
    rng = np.random.default_rng(5)
    B = rng.standard_normal((9, 9))
    A = B @ B.T + 9 * np.eye(9)
    d = np.diag(A).copy()
    diag, off = mg.lanczos_from_cg(A, 1 / d, rng.standard_normal(9), 15)
    ev = sla.eigh(A, np.diag(d), eigvals_only=True)
    assert abs(mg.tridiag_extreme(diag, off, "max") - ev.max()) < 1e-9
    assert abs(mg.tridiag_extreme(diag, off, "min") - ev.min()) < 1e-9


def test_sturm_bisection_matches_library():
    rng = np.random.default_rng(6)
    dg, of = rng.uniform(1, 3, 12), rng.uniform(-1, 1, 11)
    ev = sla.eigvalsh_tridiagonal(dg, of)
    assert abs(mg.tridiag_extreme(dg, of, "max") - ev.max()) < 1e-11
    assert abs(mg.tridiag_extreme(dg, of, "min") - ev.min()) < 1e-11


@pytest.mark.parametrize("m", [1, 2, 5, 9])
@pytest.mark.parametrize("zero_start", [True, False])
def test_chebyshev_closed_form(m, zero_start):
    # On A = diag(lam), D = I the error after m updates is
    # T_m((theta - lam)/delta) / T_m(theta/delta) times the initial error.
    lam = np.linspace(0.05, 2.5, 40)
    lo, hi = 0.1, 2.4
    A = np.diag(lam)
    xs = np.random.default_rng(m).standard_normal(40)
    b = lam * xs
    x0 = None if zero_start else np.cos(np.arange(40.0))
    x, napp = mg.chebyshev(A, np.ones(40), b, x0, lo, hi, m)
    th, de = 0.5 * (hi + lo), 0.5 * (hi - lo)
    Tm = np.zeros(m + 1)
    Tm[m] = 1
    R = npcheb.chebval((th - lam) / de, Tm) / npcheb.chebval(th / de, Tm)
    e0 = xs - (0 if zero_start else x0)
    assert np.allclose(xs - x, R * e0, atol=1e-12)
    assert napp == (m - 1 if zero_start else m)


def test_coarse_degree_bound():
    lo, hi = 0.02, 2.0
    m = mg.coarse_degree(lo, hi)
    th, de = 0.5 * (hi + lo), 0.5 * (hi - lo)
    c = np.zeros(m + 1)
    c[m] = 1
    assert 1 / npcheb.chebval(th / de, c) < 1e-3
    c = np.zeros(m)
    c[m - 1] = 1
    assert 1 / npcheb.chebval(th / de, c) >= 1e-3


@pytest.mark.parametrize("k", range(1, 9))
def test_prolongation_1d_exact_on_polynomials(k):
    nc = 3
    P = mg.prolongation_1d_cg(nc, k)
    xc = (np.arange(nc)[:, None] + 0.5 * (fem.gll_points(k)[None, :-1] + 1))
    xc = np.append(xc.ravel(), nc) / nc
    nf = 2 * nc
    xf = (np.arange(nf)[:, None] + 0.5 * (fem.gll_points(k)[None, :-1] + 1))
    xf = np.append(xf.ravel(), nf) / nf
    for m in range(k + 1):
        assert np.allclose(P @ xc ** m, xf ** m, atol=1e-12)


@pytest.mark.parametrize("disc,k", [("cg", 2), ("cg", 3), ("dg", 1),
                                    ("dg", 3)])
def test_prolongation_exact_on_qk(disc, k):
    fine = fem.Problem(4, 2, 4, k, disc=disc)
    coarse = mg.coarsen_problem(fine)
    rng = np.random.default_rng(k)
    c = rng.standard_normal((3, k + 1))

    def q(x):
        v = np.ones(x.shape[:-1])
        for d in range(3):
            t = x[..., d]
            v = v * np.polynomial.polynomial.polyval(t, c[d])
            if disc == "cg":
                v = v * t * (1 - t) if k >= 2 else v
        return v
    if disc == "cg" and k < 2:
        pytest.skip("no nonzero Q1 function vanishes on the boundary")
    if disc == "cg":            # keep the degree <= k per axis
        c[:, k - 1:] = 0
    P = mg.prolongation(fine, coarse)
    assert np.abs(P @ fem.interpolate(coarse, q)
                  - fem.interpolate(fine, q)).max() < 1e-12


@pytest.mark.parametrize("disc", ["cg", "dg"])
def test_vcycle_symmetric(disc):
    P = fem.Problem(4, 4, 4, 2, disc=disc, mapping="sine", amp=0.1)
    V = mg.VCycle(P)
    rng = np.random.default_rng(7)
    x, y = rng.standard_normal((2, P.n_dofs))
    x[P.constrained()] = 0
    y[P.constrained()] = 0
    a, b = V.apply(x) @ y, x @ V.apply(y)
    assert abs(a - b) <= 1e-13 * abs(a)


@pytest.mark.parametrize("disc,limit", [("cg", 8), ("dg", 16)])
def test_iteration_counts_near_paper(disc, limit):
    # Sec. 4.3, Table "tab:solver_times_3d": 4-5 (CG) and 10-14 (DG-SIP)
    # iterations at 1e-9 for the same recipe on a different problem.
    P = fem.Problem(8, 8, 8, 2, disc=disc)
    V = mg.VCycle(P)
    b = fem.load_vector(P, fem.sine_forcing)
    x, it, rr = mg.pcg(V.levels[-1].A, b, V.apply, rtol=1e-10)
    assert rr <= 1e-10 and it <= limit
    # the PCG solution solves the assembled system
    r = b - V.levels[-1].A @ x
    assert np.linalg.norm(r) <= 1.0000001e-10 * np.linalg.norm(b)


def test_coarsened_coefficient_constant_is_preserved():
    P = fem.Problem(4, 4, 2, 2, disc="dg", a_cell=np.full((32, 27), 2.5),
                    a_face=np.full((fem.Problem(4, 4, 2, 2).n_faces, 9), 2.5))
    C = mg.coarsen_problem(P)
    assert np.allclose(C.a_cell, 2.5) and np.allclose(C.a_face, 2.5)
    assert C.a_face.shape[0] == C.n_faces
