"""Edge cases and error paths of the C ABI: invalid descriptions, limits,
non-convergence with the last iterate returned, zero right-hand sides, a
single-cell mesh, the largest batch, high degree solves."""
import ctypes

import numpy as np
import pytest
import torch

from conftest import rel_err
from oracle import fem
from paper_1611_03029_gb300 import synthetic

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("kw,match", [
    (dict(nx=0), "cell counts"), (dict(degree=9), "degree"),
    (dict(degree=0), "degree"), (dict(n_levels=3, nx=3), "halved"),
    (dict(kappa=-1.0), "kappa"), (dict(map_param=0.5, mapping="sine"),
                                  "fold")])
def test_invalid_descriptions(mfp, kw, match):
    args = dict(nx=2, ny=2, nz=2, degree=2)
    args.update(kw)
    with pytest.raises(mfp.MfpError) as e:
        mfp.Poisson(args.pop("nx"), args.pop("ny"), args.pop("nz"),
                    args.pop("degree"), **args)
    assert e.value.status == mfp.MFP_ERR_ARG
    assert match in str(e.value)


def test_argument_errors_leave_context_usable(mfp):
    op = mfp.Poisson(4, 4, 4, 2)
    x = torch.zeros(op.n_dofs(), dtype=torch.float64, device="cuda")
    with pytest.raises(mfp.MfpError):
        op.apply(x, x)  # aliasing
    with pytest.raises(mfp.MfpError):
        op.apply(x, level=7)
    with pytest.raises(mfp.MfpError):
        op.apply(torch.zeros(op.n_dofs() * 257, dtype=torch.float64,
                             device="cuda"), n_rhs=257)
    with pytest.raises(mfp.MfpError):  # no float level data
        op.apply(x.float())
    y = op.apply(torch.ones_like(x))
    assert torch.isfinite(y).all()


def test_not_converged_returns_last_iterate(mfp):
    op = mfp.Poisson(8, 8, 8, 2)
    b = op.rhs(0)
    x, its, rel = op.solve(b, max_it=1, rtol=1e-14, raise_on_fail=False)
    assert its == [1] and rel[0] > 1e-14
    # the iterate is the first CG step: its residual matches the report
    r = b - op.apply(x)
    assert abs(float(r.norm() / b.norm()) - rel[0]) <= 1e-6 * rel[0]
    with pytest.raises(mfp.MfpError) as e:
        op.solve(b, max_it=1, rtol=1e-14)
    assert e.value.status == mfp.MFP_ERR_NOT_CONVERGED


def test_zero_rhs_and_batch_with_zero_column(mfp):
    op = mfp.Poisson(4, 4, 4, 3, disc="dg")
    N = op.n_dofs()
    B = torch.zeros(N * 3, dtype=torch.float64, device="cuda")
    op.rhs(0, out=B[1:], stride=3)
    X, its, rel = op.solve(B, n_rhs=3)
    Xh = X.reshape(N, 3).cpu().numpy()
    assert its[0] == 0 and its[2] == 0 and its[1] > 0
    assert np.all(Xh[:, 0] == 0) and np.all(Xh[:, 2] == 0)


def test_single_cell_cg_is_identity_on_boundary(mfp):
    # one Q1 cell: every node is a Dirichlet node, the operator is identity
    op = mfp.Poisson(1, 1, 1, 1)
    x = torch.randn(8, dtype=torch.float64, device="cuda")
    assert torch.equal(op.apply(x), x)
    b = torch.zeros(8, dtype=torch.float64, device="cuda")
    X, its, _ = op.solve(b)
    assert its == [0] and torch.all(X == 0)


def test_largest_batch(mfp):
    op = mfp.Poisson(2, 2, 2, 1, disc="dg", n_levels=1)
    N, R = op.n_dofs(), 256
    U = synthetic.random_vector(N, 5, ncols=R)
    Y = op.apply(torch.from_numpy(np.ascontiguousarray(U)).cuda().reshape(-1),
                 n_rhs=R).reshape(N, R).cpu().numpy()
    A = fem.assemble(fem.Problem(2, 2, 2, 1, disc="dg"))
    assert rel_err(Y, A @ U) <= 1e-12


@pytest.mark.parametrize("disc", ["cg", "dg"])
def test_degree_eight_solve(mfp, disc):
    op = mfp.Poisson(2, 2, 2, 8, disc=disc)
    P = fem.Problem(2, 2, 2, 8, disc=disc)
    b = op.rhs(0)
    x, its, rel = op.solve(b, rtol=1e-10)
    A = fem.assemble(P)
    bh = b.cpu().numpy()
    res = np.linalg.norm(bh - A @ x.cpu().numpy()) / np.linalg.norm(bh)
    assert res <= 1.05e-10


def test_rhs_and_destroy_many_contexts(mfp):
    # creating and destroying contexts repeatedly neither leaks launch
    # state nor changes results
    ref = None
    for _ in range(5):
        op = mfp.Poisson(3, 3, 3, 2, disc="dg", mapping="sine",
                         map_param=0.1)
        b = op.rhs(0).cpu().numpy()
        if ref is None:
            ref = b
        assert np.array_equal(b, ref)
        op.close()
