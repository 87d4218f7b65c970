"""Pins of the oracle's assembled operator (Eq. 4, Eq. 6, Eq. 7, Eq. 12):
closed-form element matrices, symmetry, definiteness, kernels, polynomial
reproduction and O(h^{k+1}) convergence (Sec. 4.3 reports optimal rates)."""
import numpy as np
import pytest
import scipy.sparse.linalg as sla

from oracle import fem, mg, rows


def q1_closed_form(h):
    """Trilinear stiffness matrix of a cube of side h: h/3 on the diagonal,
    0 for nodes sharing an edge, -h/12 across a face or the body diagonal."""
    K = np.zeros((8, 8))
    for a in range(8):
        for b in range(8):
            diff = bin(a ^ b).count("1")
            K[a, b] = {0: 4.0, 1: 0.0, 2: -1.0, 3: -1.0}[diff] * h / 12.0
    return K


def test_q1_element_closed_form():
    for n in (1, 3):
        P = fem.Problem(n, n, n, 1, dirichlet=False)
        K = fem.cell_matrices(P, [0])[0]
        assert np.allclose(K, q1_closed_form(1.0 / n), atol=1e-15)


def test_q2_element_closed_form():
    # 1D quadratic stiffness / mass on [0, h] with nodes 0, h/2, h
    n = 2
    h = 1.0 / n
    K1 = np.array([[7, -8, 1], [-8, 16, -8], [1, -8, 7]]) / (3 * h)
    M1 = np.array([[4, 2, -1], [2, 16, 2], [-1, 2, 4]]) * h / 30
    ref = (np.kron(M1, np.kron(M1, K1)) + np.kron(M1, np.kron(K1, M1))
           + np.kron(K1, np.kron(M1, M1)))
    P = fem.Problem(n, n, n, 2, dirichlet=False)
    K = fem.cell_matrices(P, [5])[0]
    assert np.allclose(K, ref, atol=1e-14)


def test_anisotropic_q1_scaling():
    # box hx x hy x hz: the x-part of the stiffness scales as hy hz / hx
    P = fem.Problem(2, 1, 4, 1, dirichlet=False)
    hx, hy, hz = P.h
    K = fem.cell_matrices(P, [0])[0]
    K1 = lambda h: np.array([[1, -1], [-1, 1]]) / h
    M1 = lambda h: np.array([[2, 1], [1, 2]]) * h / 6
    ref = (np.kron(M1(hz), np.kron(M1(hy), K1(hx)))
           + np.kron(M1(hz), np.kron(K1(hy), M1(hx)))
           + np.kron(K1(hz), np.kron(M1(hy), M1(hx))))
    assert np.allclose(K, ref, atol=1e-14)


@pytest.mark.parametrize("disc", ["cg", "dg"])
@pytest.mark.parametrize("mapping", ["identity", "sine"])
@pytest.mark.parametrize("k", [1, 2, 3])
def test_symmetric_positive_definite(disc, mapping, k):
    P = fem.Problem(2, 1, 3, k, disc=disc, mapping=mapping, amp=0.1)
    A = fem.assemble(P).toarray()
    assert np.abs(A - A.T).max() <= 1e-13 * np.abs(A).max()
    assert np.linalg.eigvalsh(A).min() > 0


@pytest.mark.parametrize("disc", ["cg", "dg"])
def test_constants_in_kernel_without_boundary(disc):
    P = fem.Problem(2, 3, 2, 3, disc=disc, mapping="sine", amp=0.1,
                    dirichlet=False)
    A = fem.assemble(P)
    assert np.abs(A @ np.ones(P.n_dofs)).max() < 1e-12


def test_sipg_paper_penalty_factor_also_coercive():
    P = fem.Problem(2, 2, 2, 2, disc="dg", penalty_factor=3.0)
    assert np.linalg.eigvalsh(fem.assemble(P).toarray()).min() > 0


def _poly(x):
    X, Y, Z = x[..., 0], x[..., 1], x[..., 2]
    return X * (1 - X) * Y * (1 - Y) * Z * (1 - Z)


def _poly_f(x):
    X, Y, Z = x[..., 0], x[..., 1], x[..., 2]
    return 2 * (Y * (1 - Y) * Z * (1 - Z) + X * (1 - X) * Z * (1 - Z)
                + X * (1 - X) * Y * (1 - Y))


@pytest.mark.parametrize("disc", ["cg", "dg"])
@pytest.mark.parametrize("k", [2, 3])
def test_polynomial_reproduction(disc, k):
    # u in Q_2 is in the discrete space, quadrature is exact on Cartesian
    # cells and both methods are consistent: the discrete solution is u.
    P = fem.Problem(2, 3, 2, k, disc=disc)
    A = fem.assemble(P)
    b = fem.load_vector(P, _poly_f)
    u = sla.spsolve(A.tocsc(), b)
    assert np.abs(u - fem.interpolate(P, _poly)).max() < 1e-12


@pytest.mark.parametrize("disc,mapping,k,meshes", [
    ("cg", "identity", 1, (2, 4, 8)), ("cg", "sine", 2, (2, 4, 8)),
    ("cg", "identity", 3, (2, 4)), ("dg", "identity", 2, (2, 4)),
    ("dg", "sine", 1, (2, 4, 8)), ("dg", "sine", 3, (2, 4))])
def test_convergence_rate(disc, mapping, k, meshes):
    errs = []
    for n in meshes:
        P = fem.Problem(n, n, n, k, disc=disc, mapping=mapping, amp=0.1)
        A = fem.assemble(P)
        u = sla.spsolve(A.tocsc(), fem.load_vector(P, fem.sine_forcing))
        errs.append(fem.l2_error(P, u, fem.sine_solution))
    rate = np.log2(errs[-2] / errs[-1])
    assert rate > k + 1 - 0.25, (errs, rate)


@pytest.mark.parametrize("disc", ["cg", "dg"])
def test_cg_equals_dense_solve(disc):
    P = fem.Problem(2, 2, 2, 2, disc=disc, mapping="sine", amp=0.1)
    A = fem.assemble(P)
    b = fem.load_vector(P, fem.sine_forcing)
    x, it, rr = mg.cg(A, b, rtol=1e-13)
    xd = np.linalg.solve(A.toarray(), b)
    assert rr <= 1e-13
    assert np.abs(x - xd).max() <= 1e-10 * np.abs(xd).max()


@pytest.mark.parametrize("disc", ["cg", "dg"])
def test_sampled_rows_match_assembly(disc):
    P = fem.Problem(3, 2, 2, 2, disc=disc, mapping="sine", amp=0.1)
    rng = np.random.default_rng(3)
    u = rng.standard_normal(P.n_dofs)
    r = rng.choice(P.n_dofs, 25, replace=False)
    assert np.allclose(rows.apply_rows(P, u, r), (fem.assemble(P) @ u)[r],
                       rtol=0, atol=1e-13)


def test_paper_dof_counts():
    import os
    path = os.path.join(os.path.dirname(__file__), "golden",
                        "paper_dof_counts.txt")
    for line in open(path):
        if line.startswith("#") or not line.strip():
            continue
        disc, k, cells, dofs = line.split()
        n = round(int(cells) ** (1 / 3))
        assert n ** 3 == int(cells)
        P = fem.Problem(n, n, n, int(k), disc=disc)
        assert P.n_dofs == int(dofs)


def test_mapping_is_invertible_and_fixes_boundary():
    P = fem.Problem(4, 4, 4, 3, mapping="sine", amp=0.1)
    x = P.node_points()
    logical = fem.Problem(4, 4, 4, 3).node_points()
    bnd = P.constrained()
    assert np.abs(x[bnd] - logical[bnd]).max() < 1e-15
    assert np.abs(x[~bnd] - logical[~bnd]).max() > 0.05


def _sipg_1d_q1(n, sigma_factor=1.0):
    """Textbook 1D SIPG matrix (Q1, n cells on [0, 1], homogeneous Dirichlet
    by the mirror state) and the block-diagonal DG mass matrix, written out
    from phi_0 = 1 - s, phi_1 = s on each cell."""
    h = 1.0 / n
    sig = sigma_factor * 4.0 / h                        # (k+1)^2 / h
    A = np.zeros((2 * n, 2 * n))
    M = np.zeros((2 * n, 2 * n))
    for c in range(n):
        i = [2 * c, 2 * c + 1]
        A[np.ix_(i, i)] += np.array([[1, -1], [-1, 1]]) / h
        M[np.ix_(i, i)] += np.array([[2, 1], [1, 2]]) * h / 6
    dphi = np.array([-1.0, 1.0]) / h                    # derivatives on a cell
    for f in range(1, n):                               # interior points
        L, R = [2 * f - 2, 2 * f - 1], [2 * f, 2 * f + 1]
        jump = np.zeros(2 * n)
        avg = np.zeros(2 * n)
        jump[L[1]], jump[R[0]] = 1.0, -1.0
        avg[L] += 0.5 * dphi
        avg[R] += 0.5 * dphi
        A += (-np.outer(jump, avg) - np.outer(avg, jump)
              + sig * np.outer(jump, jump))
    for node, nrm, cell in ((0, -1.0, [0, 1]), (2 * n - 1, 1.0,
                                                [2 * n - 2, 2 * n - 1])):
        v = np.zeros(2 * n)
        g = np.zeros(2 * n)
        v[node] = 1.0
        g[cell] = nrm * dphi
        A += -np.outer(v, g) - np.outer(g, v) + 2 * sig * np.outer(v, v)
    return A, M


def test_sipg_cartesian_is_kronecker_sum_of_1d():
    # On a Cartesian mesh the Q1 SIPG operator separates:
    # A = A_x (x) M_y (x) M_z + M_x (x) A_y (x) M_z + M_x (x) M_y (x) A_z,
    # with each axis using its own h in the penalty.
    n = (3, 2, 4)
    P = fem.Problem(*n, 1, disc="dg")
    A = fem.assemble(P).toarray()
    Ax, Mx = _sipg_1d_q1(n[0])
    Ay, My = _sipg_1d_q1(n[1])
    Az, Mz = _sipg_1d_q1(n[2])
    ref = (np.kron(Mz, np.kron(My, Ax)) + np.kron(Mz, np.kron(Ay, Mx))
           + np.kron(Az, np.kron(My, Mx)))
    g = np.arange(P.n_dofs)
    c, a = g // 8, g % 8
    cx, cy, cz = P.cell_coords(c)
    ix, iy, iz = 2 * cx + a % 2, 2 * cy + (a // 2) % 2, 2 * cz + a // 4
    kidx = ix + 2 * n[0] * (iy + 2 * n[1] * iz)
    assert np.allclose(A, ref[np.ix_(kidx, kidx)], atol=1e-13)
