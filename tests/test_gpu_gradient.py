"""Adjoint gradient (not in the paper): parity with the oracle's assembled
coefficient derivative, and the finite-difference check of the loss
through GPU solves."""
import numpy as np
import pytest
import torch

from conftest import rel_err
from oracle import adjoint, fem
from paper_1611_03029_gb300 import synthetic

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("disc,mapping", [("cg", "identity"), ("cg", "sine"),
                                          ("dg", "identity"), ("dg", "sine")])
def test_gradient_kernel_matches_oracle(mfp, disc, mapping):
    n, k = (3, 2, 4), 3
    amp = 0.1 if mapping == "sine" else 0.0
    op = mfp.Poisson(*n, k, disc=disc, mapping=mapping, map_param=amp,
                     n_levels=1)
    P = fem.Problem(*n, k, disc=disc, mapping=mapping, amp=amp)
    u = synthetic.random_vector(P.n_dofs, 1)
    lam = synthetic.random_vector(P.n_dofs, 2)
    gc, gf = op.gradient(torch.from_numpy(u).cuda(),
                         torch.from_numpy(lam).cuda())
    rc, rf = adjoint.gradient(P, u, lam)
    assert rel_err(gc.cpu().numpy(), rc) <= 1e-12
    if disc == "dg":
        assert rel_err(gf.cpu().numpy(), rf) <= 1e-12


def test_autograd_gradient_matches_finite_differences(mfp):
    from paper_1611_03029_gb300.mfpoisson import MFPSolve
    n, k = (4, 4, 4), 2
    p = k + 1
    a_c, a_f = synthetic.log_coefficient(n, p, seed=7)
    op = mfp.Poisson(*n, k, disc="dg")
    b = op.rhs(0)
    ut = torch.from_numpy(synthetic.random_vector(op.n_dofs(), 8) * 0.01).cuda()
    ac = torch.from_numpy(a_c).cuda().requires_grad_(True)
    af = torch.from_numpy(a_f).cuda().requires_grad_(True)
    u = MFPSolve.apply(ac, af, op, b, 1e-13, 300)
    loss = 0.5 * ((u - ut) ** 2).sum()
    loss.backward()
    rng = np.random.default_rng(11)
    eps = 1e-4 * float(np.abs(a_c).max())
    for _ in range(3):
        dc = torch.from_numpy(rng.standard_normal(a_c.shape)).cuda()
        df = torch.from_numpy(rng.standard_normal(a_f.shape)).cuda()
        def L(e):
            with torch.no_grad():
                return float(0.5 * ((MFPSolve.apply(
                    ac + e * dc, af + e * df, op, b, 1e-13, 300) - ut) ** 2
                ).sum())
        # fourth-order central difference
        fd = (8 * (L(eps) - L(-eps)) - (L(2 * eps) - L(-2 * eps))) / (12 * eps)
        an = float((ac.grad * dc).sum() + (af.grad * df).sum())
        assert abs(fd - an) <= 1e-6 * abs(an), (fd, an)


def test_gradient_full_size_sampled(mfp):
    # 32^3 cells SIPG Q3 with a = exp(g) at every cell and face point (the
    # gradient workload); the oracle evaluates the gradient at sampled cells
    # and faces one by one.
    n, k = (32, 32, 32), 3
    a_c, a_f = synthetic.log_coefficient(n, k + 1, seed=7)
    op = mfp.Poisson(*n, k, disc="dg", n_levels=1)
    op.set_coefficient(torch.from_numpy(a_c).cuda(),
                       torch.from_numpy(a_f).cuda())
    N = op.n_dofs()
    u = synthetic.random_vector(N, 1)
    lam = synthetic.random_vector(N, 2)
    gc, gf = op.gradient(torch.from_numpy(u).cuda(),
                         torch.from_numpy(lam).cuda())
    gc, gf = gc.cpu().numpy(), gf.cpu().numpy()
    P = fem.Problem(*n, k, disc="dg", a_cell=a_c, a_face=a_f)
    rng = np.random.default_rng(4)
    cells = np.concatenate([rng.choice(P.ncells, 12, replace=False),
                            [0, P.ncells - 1]])
    faces = np.concatenate([rng.choice(P.n_faces, 12, replace=False),
                            [0, P.n_faces - 1]])
    rc, rf = adjoint.gradient_sampled(P, u, lam, cells, faces)
    scale = np.abs(gc).max()
    assert np.abs(gc[cells] - rc).max() <= 1e-12 * scale
    fscale = np.abs(gf).max()
    for f, v in rf.items():
        assert np.abs(gf[f] - v).max() <= 1e-12 * fscale


def test_autograd_two_forwards_then_backward(mfp):
    # the context holds one coefficient: a second forward on the same
    # context replaces it, and the first loss's backward must still
    # differentiate at its own coefficient
    from paper_1611_03029_gb300.mfpoisson import MFPSolve
    n, k = (4, 4, 4), 2
    p = k + 1
    a1c, a1f = synthetic.log_coefficient(n, p, seed=7)
    a2c, a2f = synthetic.log_coefficient(n, p, seed=9)
    op = mfp.Poisson(*n, k, disc="dg")
    b = op.rhs(0)

    def grads(first_only):
        ac = torch.from_numpy(a1c).cuda().requires_grad_(True)
        af = torch.from_numpy(a1f).cuda().requires_grad_(True)
        u1 = MFPSolve.apply(ac, af, op, b, 1e-13, 300)
        if not first_only:
            bc = torch.from_numpy(a2c).cuda().requires_grad_(True)
            bf = torch.from_numpy(a2f).cuda().requires_grad_(True)
            MFPSolve.apply(bc, bf, op, b, 1e-13, 300)
        (0.5 * (u1 ** 2).sum()).backward()
        return ac.grad.cpu().numpy(), af.grad.cpu().numpy()

    rc, rf = grads(True)
    gc, gf = grads(False)
    assert rel_err(gc, rc) <= 1e-9
    assert rel_err(gf, rf) <= 1e-9


def test_gradient_fd_full_size(mfp):
    # the gradient workload at its size: SIPG Q3 on 32^3 cells, a = exp(g)
    # at every cell and face point; central differences of the loss through
    # GPU solves at rtol 1e-13 along 3 seeded directions with standard
    # normal entries, so that every coefficient value moves by about eps
    n, k = (32, 32, 32), 3
    a_c, a_f = synthetic.log_coefficient(n, k + 1, seed=7)
    op = mfp.Poisson(*n, k, disc="dg")
    ac = torch.from_numpy(a_c).cuda()
    af = torch.from_numpy(a_f).cuda()
    op.set_coefficient(ac, af)
    b = op.rhs(0)
    u, _, _ = op.solve(b, rtol=1e-13, max_it=300)
    ut = torch.from_numpy(synthetic.random_vector(op.n_dofs(), 8)).cuda() \
        * u.norm() / np.sqrt(op.n_dofs())
    lam, _, _ = op.solve((u - ut).contiguous(), rtol=1e-13, max_it=300)
    gc, gf = op.gradient(u, lam)

    def loss(dc, df, e):
        op.set_coefficient((ac + e * dc).contiguous(),
                           (af + e * df).contiguous())
        uu, _, _ = op.solve(b, rtol=1e-13, max_it=300)
        return 0.5 * float(((uu - ut) ** 2).sum())
    rng = np.random.default_rng(11)
    eps = 1e-4 * float(ac.abs().max())
    for _ in range(3):
        dc = torch.from_numpy(rng.standard_normal(a_c.shape)).cuda()
        df = torch.from_numpy(rng.standard_normal(a_f.shape)).cuda()
        fd = (8 * (loss(dc, df, eps) - loss(dc, df, -eps))
              - (loss(dc, df, 2 * eps) - loss(dc, df, -2 * eps))) / (12 * eps)
        an = float((gc * dc).sum() + (gf * df).sum())
        assert abs(fd - an) <= 1e-6 * abs(an), (fd, an)
