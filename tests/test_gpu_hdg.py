"""The HDG mixed matrix-free operator (Sec. 3, "HDG mixed matrix-free") of
the CUDA library against the oracle's assembled mixed operator, element by
element, 1e-12 of the largest entry (the tolerance of the other float64
applies), in the default double-float arithmetic and in IEEE float64."""
import numpy as np
import pytest
import torch

from conftest import rel_err
from oracle import hdg, fem
from paper_1611_03029_gb300 import synthetic

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("k,n,sides,box,kappa", [
    (1, (3, 2, 4), (), (0.0, 1.0), 1.0),
    (2, (3, 2, 4), (0, 2, 4), (-1.0, 1.0), 1.0),
    (3, (2, 3, 2), (1, 5), (-0.5, 2.0), 2.0),
    (4, (2, 2, 3), (0, 2, 4), (-1.0, 1.0), 1.0),
    # 9 cells: the last block of 4 cells (and of 8 faces) is ragged
    (4, (3, 1, 3), (1,), (0.0, 1.0), 1.5),
    (6, (2, 1, 2), (3,), (0.0, 1.0), 0.5),
    (8, (1, 2, 1), (), (0.0, 1.0), 1.0)])
def test_hdg_apply_matches_oracle(mfp, k, n, sides, box, kappa):
    op = mfp.Poisson(*n, k, disc="dg", n_levels=1, neumann_sides=sides,
                     box=box, kappa=kappa)
    P = fem.Problem(*n, k, disc="dg", box=box, neumann_sides=sides,
                    kappa=kappa)
    A = hdg.mixed_operator(P)
    x = synthetic.random_vector(A.shape[0], seed=60 + k)
    y = op.hdg_apply(torch.from_numpy(x).cuda()).cpu().numpy()
    assert rel_err(y, A @ x) <= 1e-12
    # repeated applies are identical (no atomics)
    y2 = op.hdg_apply(torch.from_numpy(x).cuda()).cpu().numpy()
    assert np.array_equal(y, y2)


@pytest.mark.parametrize("k,mapping", [(2, "identity"), (4, "sine")])
def test_hdg_apply_native_fp64(mfp, k, mapping):
    # the IEEE float64 (DFMA) kernels of a native context; the default
    # contexts above run the double-float ones
    n, sides = (2, 3, 2), (0, 2, 4)
    amp = 0.1 if mapping == "sine" else 0.0
    op = mfp.Poisson(*n, k, disc="dg", n_levels=1, neumann_sides=sides,
                     mapping=mapping, map_param=amp, fp64_arith="native")
    P = fem.Problem(*n, k, disc="dg", neumann_sides=sides, mapping=mapping,
                    amp=amp)
    A = hdg.mixed_operator(P)
    x = synthetic.random_vector(A.shape[0], seed=90 + k)
    y = op.hdg_apply(torch.from_numpy(x).cuda()).cpu().numpy()
    assert rel_err(y, A @ x) <= 1e-12


def test_hdg_apply_full_size_sampled_cells(mfp):
    # 32^3 cells, Q4, Cartesian: the size bench.py times; the oracle
    # evaluates the rows of sampled cells (corners, faces, interior) one by
    # one
    n, k = 32, 4
    op = mfp.Poisson(n, n, n, k, disc="dg", n_levels=1)
    P = fem.Problem(n, n, n, k, disc="dg")
    x = synthetic.random_vector(4 * op.n_dofs(), seed=81)
    y = op.hdg_apply(torch.from_numpy(x).cuda()).cpu().numpy()
    rng = np.random.default_rng(6)
    cells = np.concatenate([[0, n - 1, n * n - 1, P.ncells - 1,
                             P.ncells // 2 + n // 2],
                            rng.choice(P.ncells, 15, replace=False)])
    ref = hdg.mixed_apply_cells(P, x, cells)
    got = y.reshape(P.ncells, -1)[cells]
    assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("k,n,sides,mapping", [
    (1, (3, 2, 2), (), "sine"),
    (2, (2, 3, 2), (0, 2, 4), "sine"),
    (3, (2, 2, 3), (1,), "nodes"),
    (4, (2, 2, 2), (0, 3), "sine"),
    (4, (3, 2, 1), (2,), "nodes"),
    (5, (2, 1, 2), (), "nodes")])
def test_hdg_apply_curved_variable_coefficient(mfp, k, n, sides, mapping):
    # curved cells (w det J and J^{-1} per point, dA and the normal per face
    # point) with a per-point coefficient a = exp(g) on cells and faces (tau
    # from the largest face value)
    kw = {}
    if mapping == "nodes":
        kw["map_nodes"] = synthetic.perturbed_lattice_nodes(n, k, seed=9)
    else:
        kw["amp"] = 0.1
    a_c, a_f = synthetic.log_coefficient(n, k + 1, seed=7)
    op = mfp.Poisson(*n, k, disc="dg", n_levels=1, neumann_sides=sides,
                     mapping=mapping, map_param=kw.get("amp", 0.0),
                     map_nodes=kw.get("map_nodes"))
    op.set_coefficient(torch.from_numpy(a_c).cuda(),
                       torch.from_numpy(a_f).cuda())
    P = fem.Problem(*n, k, disc="dg", neumann_sides=sides, mapping=mapping,
                    a_cell=a_c, a_face=a_f, **kw)
    A = hdg.mixed_operator(P)
    x = synthetic.random_vector(A.shape[0], seed=70 + k)
    y = op.hdg_apply(torch.from_numpy(x).cuda()).cpu().numpy()
    assert rel_err(y, A @ x) <= 1e-12


def test_hdg_apply_curved_full_size_sampled_cells(mfp):
    # 32^3 cells Q4 on the curved map: sampled cells' rows by the oracle
    n, k = 32, 4
    op = mfp.Poisson(n, n, n, k, disc="dg", n_levels=1, mapping="sine",
                     map_param=0.1)
    P = fem.Problem(n, n, n, k, disc="dg", mapping="sine", amp=0.1)
    x = synthetic.random_vector(4 * op.n_dofs(), seed=82)
    y = op.hdg_apply(torch.from_numpy(x).cuda()).cpu().numpy()
    rng = np.random.default_rng(7)
    cells = np.concatenate([[0, n - 1, P.ncells - 1],
                            rng.choice(P.ncells, 9, replace=False)])
    ref = hdg.mixed_apply_cells(P, x, cells)
    got = y.reshape(P.ncells, -1)[cells]
    assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()


def test_hdg_apply_rejects_unsupported(mfp):
    x = torch.zeros(4 * 8 * 8, dtype=torch.float64, device="cuda")
    op = mfp.Poisson(2, 2, 2, 1, n_levels=1, disc="cg")
    with pytest.raises(mfp.MfpError):
        op.hdg_apply(x)
