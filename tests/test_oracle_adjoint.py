"""Pin of the oracle's adjoint gradient against central finite differences
of the loss through full solves."""
import numpy as np
import pytest
import scipy.sparse.linalg as sla

from oracle import adjoint, fem


@pytest.mark.parametrize("disc,sides", [("cg", ()), ("dg", ()),
                                        ("cg", (1, 2)), ("dg", (1, 2))])
def test_gradient_matches_finite_differences(disc, sides):
    rng = np.random.default_rng(11)
    shape = fem.Problem(2, 2, 1, 2, disc=disc)
    a_c = np.exp(0.3 * rng.standard_normal((shape.ncells, 27)))
    a_f = np.exp(0.3 * rng.standard_normal((shape.n_faces, 9)))
    ut = rng.standard_normal(shape.n_dofs)

    def solve(ac, af):
        P = fem.Problem(2, 2, 1, 2, disc=disc, mapping="sine", amp=0.1,
                        a_cell=ac, a_face=af, neumann_sides=sides)
        A = fem.assemble(P)
        u = sla.spsolve(A.tocsc(), fem.load_vector(P, fem.sine_forcing))
        return P, A, u

    P, A, u = solve(a_c, a_f)
    lam = sla.spsolve(A.tocsc(), u - ut)
    gc, gf = adjoint.gradient(P, u, lam)
    eps = 1e-5
    for _ in range(3):
        dc = rng.standard_normal(a_c.shape)
        df = rng.standard_normal(a_f.shape) if disc == "dg" else 0 * a_f
        lp = adjoint.loss(solve(a_c + eps * dc, a_f + eps * df)[2], ut)
        lm = adjoint.loss(solve(a_c - eps * dc, a_f - eps * df)[2], ut)
        fd = (lp - lm) / (2 * eps)
        an = np.sum(gc * dc) + np.sum(gf * df)
        assert abs(fd - an) <= 1e-6 * abs(an)
    if disc == "cg":
        assert np.all(gf == 0)
    else:
        # faces on Neumann sides carry no term of the form (Eq. 7)
        for side in sides:
            d, s = side // 2, side % 2
            fid, left, right = fem.face_cells(P, d)
            bnd = fid[(right < 0) if s else (left < 0)]
            assert np.all(gf[bnd] == 0)
