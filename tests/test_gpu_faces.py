"""SIPG face terms (Eq. 6, mirror states of Eq. 7) in the layouts where the
face scheme of the kernels has special cases: each interior face is
evaluated once by the cell below it, the upper neighbour's share goes
through a per-level face buffer, boundary faces are one-sided.  Meshes with
one cell along an axis (every face in that direction on the boundary), a
single cell, batched columns with a face buffer grown and reused at a
smaller column count, in double-float, native float64 and float."""
import numpy as np
import pytest
import torch

from conftest import rel_err
from oracle import fem
from paper_1611_03029_gb300 import synthetic

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("n,k", [((1, 1, 1), 3), ((1, 4, 1), 2),
                                 ((2, 1, 3), 5), ((4, 3, 1), 7)])
@pytest.mark.parametrize("mapping", ["identity", "sine"])
def test_boundary_only_axes(mfp, n, k, mapping):
    amp = 0.1 if mapping == "sine" else 0.0
    P = fem.Problem(*n, k, disc="dg", mapping=mapping, amp=amp)
    A = fem.assemble(P)
    u = synthetic.random_vector(P.n_dofs, seed=31 + k)
    ref = A @ u
    for arith in ("df", "native"):
        op = mfp.Poisson(*n, k, disc="dg", mapping=mapping, map_param=amp,
                         n_levels=1, fp64_arith=arith)
        y = op.apply(torch.from_numpy(u).cuda()).cpu().numpy()
        assert rel_err(y, ref) <= 1e-12, arith
    op32 = mfp.Poisson(*n, k, disc="dg", mapping=mapping, map_param=amp,
                       n_levels=1, mg_precision="fp32")
    y32 = op32.apply(torch.from_numpy(u.astype(np.float32)).cuda())
    assert rel_err(y32.cpu().numpy(), ref) <= 2e-5


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_face_buffer_grown_then_reused(mfp, prec):
    # applies with 7 columns, then 2, then 1: the buffer allocated for 7
    # columns serves the smaller counts with their own stride
    n, k = (3, 2, 2), 3
    dt = np.float64 if prec == "fp64" else np.float32
    tol = 1e-12 if prec == "fp64" else 2e-5
    op = mfp.Poisson(*n, k, disc="dg", mapping="sine", map_param=0.1,
                     n_levels=1, mg_precision=prec)
    A = fem.assemble(fem.Problem(*n, k, disc="dg", mapping="sine", amp=0.1))
    N = op.n_dofs()
    for R in (7, 2, 1):
        U = synthetic.random_vector(N, seed=40 + R, ncols=R).astype(dt)
        U = U.reshape(N, R)
        Ut = torch.from_numpy(np.ascontiguousarray(U)).cuda().reshape(-1)
        Y = op.apply(Ut, n_rhs=R).reshape(N, R).cpu().numpy()
        assert rel_err(Y, A @ U.astype(np.float64)) <= tol, R


def test_apply_is_deterministic(mfp):
    # no atomics in the SIPG apply: repeated applies agree bit for bit
    op = mfp.Poisson(6, 5, 4, 4, disc="dg", mapping="sine", map_param=0.1,
                     n_levels=1)
    u = torch.from_numpy(synthetic.random_vector(op.n_dofs(), seed=2)).cuda()
    y0 = op.apply(u).cpu().numpy()
    for _ in range(3):
        assert np.array_equal(op.apply(u).cpu().numpy(), y0)


@pytest.mark.parametrize("disc", ["cg", "dg"])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_dense_coarse_level_apply(mfp, disc, prec):
    # the coarsest level of a hierarchy (at most 2048 dofs) is applied from
    # its assembled dense matrix; same operator as the oracle's coarse level,
    # single and batched columns
    from oracle import mg
    dt = np.float64 if prec == "fp64" else np.float32
    tol = 1e-12 if prec == "fp64" else 2e-5
    op = mfp.Poisson(4, 4, 4, 3, disc=disc, mapping="sine", map_param=0.1,
                     mg_precision=prec)
    assert op.n_levels == 2
    P0 = mg.hierarchy(fem.Problem(4, 4, 4, 3, disc=disc, mapping="sine",
                                  amp=0.1))[0]
    A0 = fem.assemble(P0)
    N = P0.n_dofs
    assert op.n_dofs(0) == N
    for R in (1, 3):
        U = synthetic.random_vector(N, seed=50 + R, ncols=R).reshape(N, R)
        Ut = torch.from_numpy(np.ascontiguousarray(U.astype(dt))).cuda()
        Y = op.apply(Ut.reshape(-1), level=0, n_rhs=R).reshape(N, R)
        assert rel_err(Y.cpu().numpy(), A0 @ U) <= tol, R
