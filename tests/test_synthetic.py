"""The seeded input generators place coefficient samples at the same
points and in the same order as the oracle's quadrature points."""
import numpy as np

from oracle import fem
from paper_1611_03029_gb300 import synthetic


def test_cell_points_match_oracle_quadrature():
    P = fem.Problem(3, 2, 4, 2)
    gq, _ = fem.gauss_rule(3)
    x, _, _, _ = P.geometry(np.arange(P.ncells), fem.tensor_points(gq))
    assert np.abs(x - synthetic.cell_points(P.n, 3)).max() < 1e-15


def test_face_points_match_oracle_faces():
    P = fem.Problem(3, 2, 4, 2)
    pts = synthetic.face_points(P.n, 3)
    assert pts.shape[0] == P.n_faces
    for d in range(3):
        fid, L, R = fem.face_cells(P, d)
        for side, cells in ((1.0, L), (-1.0, R)):
            sel = cells >= 0
            sd = fem._side_data(P, cells[sel], d, side)
            assert np.abs(sd["x"] - pts[fid[sel]]).max() < 1e-15


def test_seeds_are_reproducible():
    a = synthetic.gaussian_terms(1000)
    b = synthetic.gaussian_terms(1000)
    assert np.array_equal(a, b) and a.shape == (8, 5)
    assert np.all((a[:, 3] >= 0.05) & (a[:, 3] <= 0.2))
