"""Assembled-matrix adjoint gradient of a solve-based loss (not in the
paper; its operator is the one of Eq. 4 / Eq. 6 with a coefficient a(x)
given at every quadrature point).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

With A(a) u = f and L(u) = 0.5 ||u - u_t||_2^2 on the dof vector, the
adjoint lambda solves A^T lambda = A lambda = u - u_t and
  dL/da_q = - lambda^T (dA/da_q) u.
A is linear in every coefficient value a_q, so dA/da_q is the matrix the
assembly produces when the coefficient is the indicator of q.  This module
forms it literally for every quadrature point of every cell and face and
contracts it with lambda and u; Dirichlet-constrained rows and columns do
not depend on a, so those dofs are zeroed first.
"""
import numpy as np

from . import fem


def cell_qp_matrices(prob, cells):
    """dK^e/da_q [c, m, N, N] for the cell quadrature points m (Eq. 12 with
    kappa replaced by the indicator of point m)."""
    cells = np.asarray(cells)
    gq, wq = fem.gauss_rule(prob.p)
    ref = fem.tensor_points(gq)
    w = fem.tensor_weights(wq)
    _, grad = fem.basis3d(prob.k, ref)
    _, _, det, Jinv = prob.geometry(cells, ref)
    pg = np.einsum("cmed,mie->cmid", Jinv, grad)           # physical grads
    return np.einsum("cmid,cmjd->cmij", pg, pg) * (w[None] * det)[..., None,
                                                                  None]


def gradient(prob, u, lam):
    """(dL/da at cell points [ncells, p^3], at face points [nfaces, p^2])."""
    u = np.array(u, float)
    lam = np.array(lam, float)
    cmask = prob.constrained()
    u[cmask] = 0.0
    lam[cmask] = 0.0
    g_cell = np.zeros((prob.ncells, prob.p ** 3))
    chunk = 32
    allc = np.arange(prob.ncells)
    for s in range(0, prob.ncells, chunk):
        cells = allc[s:s + chunk]
        dK = cell_qp_matrices(prob, cells)
        dm = prob.dof_map(cells)
        g_cell[cells] = -np.einsum("ci,cmij,cj->cm", lam[dm], dK, u[dm])
    g_face = np.zeros((prob.n_faces, prob.p ** 2))
    if prob.disc == "dg":
        for d in range(3):
            for g in fem.face_operators(prob, d):
                dm = prob.dof_map(g["cells"].ravel()).reshape(
                    len(g["fid"]), -1)
                ul, ll = u[dm], lam[dm]
                ju = np.einsum("fmj,fj->fm", g["jump_u"], ul)
                au = np.einsum("fmj,fj->fm", g["avg_u"], ul)
                jv = np.einsum("fmi,fi->fm", g["jump_v"], ll)
                av = np.einsum("fmi,fi->fm", g["avg_v"], ll)
                val = g["c"] * (-jv * au - av * ju
                                + g["sigma"][:, None] * jv * ju)
                g_face[g["fid"]] = -val
    return g_cell, g_face


def loss(u, u_target):
    """L = 0.5 ||u - u_t||_2^2 on the dof vector."""
    d = np.asarray(u) - np.asarray(u_target)
    return 0.5 * float(d @ d)


def gradient_sampled(prob, u, lam, cells, faces):
    """dL/da at the points of selected cells and faces only (the same
    assembled derivative as `gradient`), for checking large meshes."""
    u = np.array(u, float)
    lam = np.array(lam, float)
    cmask = prob.constrained()
    u[cmask] = 0.0
    lam[cmask] = 0.0
    cells = np.asarray(cells)
    dK = cell_qp_matrices(prob, cells)
    dm = prob.dof_map(cells)
    g_cell = -np.einsum("ci,cmij,cj->cm", lam[dm], dK, u[dm])
    g_face = {}
    if prob.disc == "dg":
        for d in range(3):
            for g in fem.face_operators(prob, d, faces):
                dmf = prob.dof_map(g["cells"].ravel()).reshape(
                    len(g["fid"]), -1)
                ul, ll = u[dmf], lam[dmf]
                ju = np.einsum("fmj,fj->fm", g["jump_u"], ul)
                au = np.einsum("fmj,fj->fm", g["avg_u"], ul)
                jv = np.einsum("fmi,fi->fm", g["jump_v"], ll)
                av = np.einsum("fmi,fi->fm", g["avg_v"], ll)
                val = g["c"] * (-jv * au - av * ju
                                + g["sigma"][:, None] * jv * ju)
                for t, f in enumerate(g["fid"]):
                    g_face[int(f)] = -val[t]
    return g_cell, g_face
