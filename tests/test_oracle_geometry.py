"""Pins of the oracle's curved-cell geometry and of its coefficient
coarsening, from invariants of the mapping and of linear fields.

The sine map x -> x + a sin(pi x) sin(pi y) sin(pi z) (1, 1, 1) is the
identity on the boundary of the unit cube, and the isoparametric cells
through its Gauss-Lobatto support points tile the cube (neighbours share
their face nodes).  So the cell volumes |K| (the integrals of det J that
enter the penalty of Sec. 2.2 through h_F) sum to the cube's volume, the
boundary face areas |F| (det J |J^{-T} n| by the face rule) sum to its
surface area, and both sides of an interior face see the same area element
with opposite normals.  A wrong area element, a dropped det J or a flipped
orientation breaks one of these.

Coefficient coarsening (the quadrature-weighted child mean of reading R16):
a linear field's weighted mean over a Cartesian cell or face is its value at
the centroid (the Gauss rule is exact for linear functions), so the coarse
value must equal the field at the coarse centroid, which checks the child
index bookkeeping of every face direction."""
import numpy as np
import pytest

from oracle import fem, mg
from paper_1611_03029_gb300 import synthetic


@pytest.mark.parametrize("k", [1, 2, 3, 4, 6])
@pytest.mark.parametrize("box", [(0.0, 1.0), (-1.0, 1.0)])
def test_volumes_and_boundary_areas_of_sine_map(k, box):
    P = fem.Problem(3, 2, 4, k, mapping="sine", amp=0.1, box=box)
    L = box[1] - box[0]
    vol = fem.cell_volumes(P, np.arange(P.ncells))
    assert abs(vol.sum() - L ** 3) <= 1e-13 * L ** 3
    # curved cells: the volumes differ from cell to cell
    assert vol.max() - vol.min() > 1e-3 * vol.mean()
    area = 0.0
    for d in range(3):
        for s in (-1, 1):
            _, sd = fem._boundary_side(P, d, s)
            area += sd["dA"].sum()
    assert abs(area - 6 * L ** 2) <= 1e-13 * 6 * L ** 2


@pytest.mark.parametrize("k", [1, 3, 4])
@pytest.mark.parametrize("d", [0, 1, 2])
def test_interior_faces_agree_from_both_sides(k, d):
    P = fem.Problem(3, 3, 2, k, mapping="sine", amp=0.1)
    _, left, right = fem.face_cells(P, d)
    m = (left >= 0) & (right >= 0)
    sl = fem._side_data(P, left[m], d, 1.0)
    sr = fem._side_data(P, right[m], d, -1.0)
    assert np.abs(sl["x"] - sr["x"]).max() <= 1e-15
    assert np.abs(sl["dA"] - sr["dA"]).max() <= 1e-15
    assert np.abs(sl["n"] + sr["n"]).max() <= 1e-15
    # the face is curved: its normal is not the axis everywhere
    assert np.abs(np.abs(sl["n"][..., d]) - 1).max() > 1e-4


def _linear(x):
    return 1.0 + 0.3 * x[..., 0] - 0.2 * x[..., 1] + 0.5 * x[..., 2]


@pytest.mark.parametrize("k", [1, 2, 3])
def test_coarsened_linear_coefficient_is_centroid_value(k):
    n, p = (4, 6, 2), k + 1
    a_cell = _linear(synthetic.cell_points(n, p))
    a_face = _linear(synthetic.face_points(n, p))
    P = fem.Problem(*n, k, disc="dg", a_cell=a_cell, a_face=a_face)
    nc = tuple(m // 2 for m in n)
    c_cell, c_face = mg.coarsen_coefficient(P, nc)
    cent = synthetic.cell_points(nc, p).mean(axis=1)
    assert np.abs(c_cell - _linear(cent)[:, None]).max() <= 1e-14
    fcent = synthetic.face_points(nc, p).mean(axis=1)
    assert c_face.shape == (fcent.shape[0], p * p)
    assert np.abs(c_face - _linear(fcent)[:, None]).max() <= 1e-14


@pytest.mark.parametrize("disc", ["cg", "dg"])
@pytest.mark.parametrize("mapping", ["identity", "sine"])
def test_given_nodes_reproduce_the_mapping(disc, mapping):
    # support points handed over as nodes give the same operator
    n, k = (2, 3, 2), 2
    P = fem.Problem(*n, k, disc=disc, mapping=mapping, amp=0.1)
    Q = fem.Problem(*n, k, disc=disc, mapping="nodes",
                    map_nodes=P.support_points(np.arange(P.ncells)))
    A, B = fem.assemble(P), fem.assemble(Q)
    assert abs(A - B).max() <= 1e-14 * abs(A).max()


def _quadratic_map(x):
    y = x.copy()
    for d in range(3):
        e = (d + 1) % 3
        y[..., d] += 0.05 * x[..., e] * (1.0 - x[..., e])
    return y


@pytest.mark.parametrize("k", [2, 3])
def test_coarse_nodes_reproduce_a_polynomial_map(k):
    # the fine isoparametric map of a degree-2 map is the map itself, so the
    # coarse nodes (the fine map at the coarse Gauss-Lobatto points) are the
    # map's values there; this checks the child and the reference point
    n = (4, 2, 6)
    I = fem.Problem(*n, k)
    nodes = _quadratic_map(I.support_points(np.arange(I.ncells)))
    P = fem.Problem(*n, k, mapping="nodes", map_nodes=nodes)
    nc = (2, 1, 3)
    Ic = fem.Problem(*nc, k)
    got = mg.coarsen_nodes(P, nc)
    ref = _quadratic_map(Ic.support_points(np.arange(Ic.ncells)))
    assert np.abs(got - ref).max() <= 1e-14


@pytest.mark.parametrize("disc", ["cg", "dg"])
@pytest.mark.parametrize("k", [1, 2, 4])
def test_perturbed_lattice_mesh_is_valid(disc, k):
    # the generator's meshes are conforming and invertible, and their
    # operator is symmetric positive definite (P1) on every level
    n = (4, 4, 2)
    nodes = synthetic.perturbed_lattice_nodes(n, k, seed=3)
    P = fem.Problem(*n, k, disc=disc, mapping="nodes", map_nodes=nodes)
    for Q in mg.hierarchy(P, 2):
        A = fem.assemble(Q).toarray()
        assert np.abs(A - A.T).max() <= 1e-13 * np.abs(A).max()
        np.linalg.cholesky(A)
    # the boundary points stay on the cube's faces, so the cells fill it;
    # det J has degree 3k - 1 per axis, which the (k+1)-point Gauss rule
    # integrates exactly for k <= 2 only
    vol = fem.cell_volumes(P, np.arange(P.ncells))
    assert abs(vol.sum() - 1.0) <= (1e-13 if k <= 2 else 1e-5)
    # neighbours share their face nodes: the CG node positions agree
    Q = fem.Problem(*n, k, mapping="nodes", map_nodes=nodes)
    dm = Q.dof_map()
    X = np.zeros((Q.n_dofs, 3))
    X[dm.ravel()] = nodes.reshape(-1, 3)
    assert np.abs(X[dm] - nodes).max() == 0.0
