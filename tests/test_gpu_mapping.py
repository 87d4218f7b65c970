"""User-supplied support points (MFP_MAP_NODES; Sec. 2: cells are images of
the reference cube under a degree-k polynomial map through Gauss-Lobatto
support points): the operator on every level, the V-cycle (whose coarse
levels re-interpolate the fine map) and the solve against the oracle built
on the same nodes, on randomly perturbed conforming meshes."""
import numpy as np
import pytest
import torch

from conftest import rel_err
from oracle import fem, mg
from paper_1611_03029_gb300 import synthetic

pytestmark = pytest.mark.gpu

CASES = [("cg", 1, (4, 4, 2)), ("cg", 2, (4, 2, 4)), ("cg", 4, (4, 4, 4)),
         ("dg", 1, (2, 4, 4)), ("dg", 2, (4, 4, 2)), ("dg", 4, (4, 4, 4))]


def pair(mfp, disc, k, n, **kw):
    nodes = synthetic.perturbed_lattice_nodes(n, k, seed=5)
    op = mfp.Poisson(*n, k, disc=disc, mapping="nodes", map_nodes=nodes,
                     **kw)
    P = fem.Problem(*n, k, disc=disc, mapping="nodes", map_nodes=nodes)
    return op, P


@pytest.mark.parametrize("arith", ["df", "native"])
@pytest.mark.parametrize("disc,k,n", CASES)
def test_apply_every_level(mfp, disc, k, n, arith):
    op, P = pair(mfp, disc, k, n, fp64_arith=arith)
    probs = mg.hierarchy(P)
    assert len(probs) == op.n_levels
    for lv, Q in enumerate(probs):
        u = synthetic.random_vector(Q.n_dofs, seed=lv)
        y = op.apply(torch.from_numpy(u).cuda(), level=lv).cpu().numpy()
        assert rel_err(y, fem.assemble(Q) @ u) <= 1e-12, lv


@pytest.mark.parametrize("disc,k,n", CASES[1::2])
def test_apply_float(mfp, disc, k, n):
    op, P = pair(mfp, disc, k, n, mg_precision="fp32")
    u = synthetic.random_vector(P.n_dofs, seed=1)
    y = op.apply(torch.from_numpy(u).float().cuda()).cpu().numpy()
    assert rel_err(y, fem.assemble(P) @ u) <= 2e-5


@pytest.mark.parametrize("disc,k,n", CASES)
def test_vcycle_and_solve(mfp, disc, k, n):
    op, P = pair(mfp, disc, k, n)
    V = mg.VCycle(P)
    r = synthetic.random_vector(P.n_dofs, seed=3)
    r[P.constrained()] = 0.0
    z = op.vcycle(torch.from_numpy(r).cuda()).cpu().numpy()
    assert rel_err(z, V.apply(r)) <= 1e-9
    b = op.rhs(0)
    x, its, rel = op.solve(b, rtol=1e-10, max_it=100)
    A = fem.assemble(P)
    bh = b.cpu().numpy()
    assert rel_err(bh, fem.load_vector(P, fem.sine_forcing)) <= 1e-12
    res = np.linalg.norm(bh - A @ x.cpu().numpy()) / np.linalg.norm(bh)
    assert res <= 1.05e-10, res


def test_folded_mesh_is_rejected(mfp):
    n, k = (2, 2, 2), 2
    nodes = synthetic.perturbed_lattice_nodes(n, k, seed=5, amp=0.0)
    nodes[0, 13] += np.array([0.4, 0.0, 0.0])   # centre node of cell 0
    with pytest.raises(mfp.MfpError) as e:
        mfp.Poisson(*n, k, mapping="nodes", map_nodes=nodes)
    assert e.value.status == mfp.MFP_ERR_ARG


@pytest.mark.parametrize("disc", ["cg", "dg"])
def test_neumann_sides_and_boundary_data(mfp, disc):
    # given nodes with Neumann sides: the operator and the f_kind 2
    # right-hand side (Dirichlet and Neumann data of a Gaussian sum) on the
    # curved faces
    n, k, sides = (3, 2, 3), 2, (0, 3)
    nodes = synthetic.perturbed_lattice_nodes(n, k, seed=11)
    op = mfp.Poisson(*n, k, disc=disc, mapping="nodes", map_nodes=nodes,
                     n_levels=1, neumann_sides=sides)
    P = fem.Problem(*n, k, disc=disc, mapping="nodes", map_nodes=nodes,
                    neumann_sides=sides)
    u = synthetic.random_vector(P.n_dofs, seed=12)
    y = op.apply(torch.from_numpy(u).cuda()).cpu().numpy()
    assert rel_err(y, fem.assemble(P) @ u) <= 1e-12
    g = np.array([[0.3, 0.6, 0.4, 0.3, 1.5], [0.7, 0.2, 0.8, 0.25, -0.5]])
    f = synthetic.gaussian_forcing(g)

    def uex(x):
        return f(x)

    def grad(x):
        out = np.zeros(x.shape)
        for cx, cy, cz, w, a in g:
            d = x - np.array([cx, cy, cz])
            e = a * np.exp(-np.sum(d * d, -1) / w ** 2)
            out += (-2.0 / w ** 2) * d * e[..., None]
        return out

    def lap(x):
        out = np.zeros(x.shape[:-1])
        for cx, cy, cz, w, a in g:
            d = x - np.array([cx, cy, cz])
            r2 = np.sum(d * d, -1)
            out += a * np.exp(-r2 / w ** 2) * (4 * r2 / w ** 4 - 6 / w ** 2)
        return -out
    ref = fem.manufactured_rhs(P, lap, uex, grad)
    got = op.rhs(2, g).cpu().numpy()
    assert rel_err(got, ref) <= 1e-11


def test_batched_apply_columns(mfp):
    n, k, R = (3, 2, 2), 3, 4
    nodes = synthetic.perturbed_lattice_nodes(n, k, seed=13)
    op = mfp.Poisson(*n, k, disc="dg", mapping="nodes", map_nodes=nodes,
                     n_levels=1)
    N = op.n_dofs()
    X = synthetic.random_vector(N, seed=14, ncols=R)
    Y = op.apply(torch.from_numpy(np.ascontiguousarray(X)).cuda().reshape(-1),
                 n_rhs=R).cpu().numpy().reshape(N, R)
    for r in range(R):
        y1 = op.apply(torch.from_numpy(X[:, r].copy()).cuda()).cpu().numpy()
        assert rel_err(Y[:, r], y1) <= 1e-13
