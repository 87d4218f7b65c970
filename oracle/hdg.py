"""Plain float64 hybridizable DG (HDG) discretization of
-div(kappa grad u) = f (Sec. 2.3, Eq. hdg and its matrix form): the flux
q = -kappa grad u and u in the discontinuous Q_k space of each cell, the
trace lambda in Q_k of each face, the numerical flux
q^ . n = q . n + tau (u - lambda), tau = 5 max kappa on the face (Sec. 4.2).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).  Written from the paper's
weak form, not from the CUDA library.  Used to pin the HDG blocks against
the L2 errors the paper prints for its smooth example (u_h and the
element-by-element post-processed u*), and as the reference of the mixed
HDG operator  [A B^T; B D] + [C^T; G^T] H^{-1} [C G]  (Sec. 3, "HDG mixed
matrix-free").

Signs (a reading: the printed second equation carries the face term with the
sign that makes it inconsistent; written here from the integration by parts
of div q = f):
  (w, kappa^-1 q)_K - (div w, u)_K + <w . n, lambda>_dK            = 0
  (grad v, q)_K - <v, q . n + tau (u - lambda)>_dK                 = -(v, f)_K
  sum_K <mu, q . n + tau (u - lambda)>_dK                          = <mu, q_N . n>
where q_N . n = -kappa grad u . n is the exact flux on Neumann faces and
lambda is the L2 projection of the Dirichlet data on Dirichlet faces.  In
blocks (unknowns Q, U, Lambda):
  A = (w, kappa^-1 q),  B^T = -(div w, u),  C^T = <w . n, lambda>,
  D = -<v, tau u>,      G^T = <v, tau lambda>,  H = sum <mu, tau lambda>,
  [A B^T C^T; B D G^T; -C -G H] [Q; U; Lambda] = [0; -(v, f); -<mu, q_N.n>].
"""
import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from oracle import fem

TAU_FACTOR = 5.0


def face_basis(k):
    """Values [p^2 face points, p^2 trace functions] of the face's Q_k
    Lagrange basis in the Gauss-Lobatto points at its Gauss points, both in
    the order a + p b over the tangential axes a < b."""
    gq, _ = fem.gauss_rule(k + 1)
    S = fem.lagrange_values(fem.gll_points(k), gq)     # [q, m]
    return np.kron(S, S)


def _cell_face_list():
    """The six faces of a cell: (direction d, side s = -1 lower / +1 upper)."""
    return [(d, s) for d in range(3) for s in (-1, 1)]


def cell_face_ids(prob, cells):
    """Global face ids [c, 6] of the faces of `cells` in _cell_face_list
    order (x-normal faces first, each direction lexicographic)."""
    cx, cy, cz = prob.cell_coords(np.asarray(cells))
    out = []
    for d, s in _cell_face_list():
        fc = [cx, cy, cz]
        fc[d] = fc[d] + (1 if s > 0 else 0)
        m = list(prob.n)
        m[d] += 1
        off = sum(prob.n_faces_dir(e) for e in range(d))
        out.append(off + fc[0] + m[0] * (fc[1] + m[1] * fc[2]))
    return np.stack(out, 1)


def face_sides(prob):
    """Boundary side (0..5) of every face, -1 for interior faces."""
    side = np.full(prob.n_faces, -1)
    for d in range(3):
        fid, left, right = fem.face_cells(prob, d)
        side[fid[left < 0]] = 2 * d
        side[fid[right < 0]] = 2 * d + 1
    return side


def tau_faces(prob):
    """tau = TAU_FACTOR max kappa over the points of each face (Sec. 4.2)."""
    return TAU_FACTOR * prob.kappa_face(np.arange(prob.n_faces)).max(1)


def local_blocks(prob, cells, tau):
    """Cell blocks: M = [A B^T; B D] [c, 4N, 4N] with unknowns ordered
    (q_x, q_y, q_z, u), N = p^3 each; Nc = [C^T; G^T] [c, 4N, 6 p^2] on the
    cell's six faces; and the face-side mass tau <mu, lambda> [c, 6, p^2,
    p^2] that builds H."""
    k, p = prob.k, prob.p
    N, F = p ** 3, p * p
    cells = np.asarray(cells)
    nc = cells.size
    gq, wq = fem.gauss_rule(p)
    ref = fem.tensor_points(gq)
    w = fem.tensor_weights(wq)
    val, grad = fem.basis3d(k, ref)
    _, _, det, Jinv = prob.geometry(cells, ref)
    pg = np.einsum("cmed,mie->cmid", Jinv, grad)          # physical gradients
    kap = prob.kappa_cell(cells)
    wd = det * w[None]
    M = np.zeros((nc, 4 * N, 4 * N))
    mass_k = np.einsum("cm,mi,mj->cij", wd / kap, val, val)
    for d in range(3):
        M[:, d * N:(d + 1) * N, d * N:(d + 1) * N] = mass_k
        # B^T: -(div w, u) with w = phi_i e_d
        bt = -np.einsum("cm,cmi,mj->cij", wd, pg[..., d], val)
        M[:, d * N:(d + 1) * N, 3 * N:] = bt
        M[:, 3 * N:, d * N:(d + 1) * N] = np.transpose(bt, (0, 2, 1))
    Nc = np.zeros((nc, 4 * N, 6 * F))
    Hs = np.zeros((nc, 6, F, F))
    psi = face_basis(k)
    fids = cell_face_ids(prob, cells)
    for j, (d, s) in enumerate(_cell_face_list()):
        sd = fem._side_data(prob, cells, d, float(s))
        t = tau[fids[:, j]][:, None]                      # [c, 1]
        dA = sd["dA"]                                     # [c, q]
        v = sd["val"]                                     # [q, N]
        nrm = sd["n"]                                     # [c, q, 3]
        # D: -<v, tau u>
        M[:, 3 * N:, 3 * N:] -= np.einsum("cq,qi,qj->cij", t * dA, v, v)
        cols = slice(j * F, (j + 1) * F)
        for e in range(3):
            Nc[:, e * N:(e + 1) * N, cols] = np.einsum(
                "cq,qi,qm->cim", dA * nrm[..., e], v, psi)
        Nc[:, 3 * N:, cols] = np.einsum("cq,qi,qm->cim", t * dA, v, psi)
        Hs[:, j] = np.einsum("cq,qm,ql->cml", t * dA, psi, psi)
    return M, Nc, Hs, fids


def _face_points(prob, faces):
    """Physical points, outward normal of the lower cell side and area
    element of `faces` (evaluated from one adjacent cell)."""
    out = {}
    for d in range(3):
        fid, left, right = fem.face_cells(prob, d)
        sel = np.isin(fid, faces)
        for f, L, R in zip(fid[sel], left[sel], right[sel]):
            c, s = (L, 1.0) if L >= 0 else (R, -1.0)
            sd = fem._side_data(prob, np.array([c]), d, s)
            out[f] = (sd["x"][0], sd["n"][0], sd["dA"][0])
    return out


class Solution:
    pass


def cell_load(prob, f):
    """Cell right-hand sides [c, 4 p^3]: 0 on the flux rows, -(v, f) on the
    u rows ((k+1)^3 Gauss rule)."""
    k, p = prob.k, prob.p
    N = p ** 3
    gq, wq = fem.gauss_rule(p)
    ref = fem.tensor_points(gq)
    w = fem.tensor_weights(wq)
    val, _ = fem.basis3d(k, ref)
    x, _, det, _ = prob.geometry(np.arange(prob.ncells), ref)
    Fc = np.zeros((prob.ncells, 4 * N))
    Fc[:, 3 * N:] = -(f(x) * det * w[None]) @ val
    return Fc


def trace_data(prob, u_exact, grad_u):
    """Boundary data on the trace unknowns [nfaces * p^2]: R = -<mu, q_N . n>
    on Neumann faces (q_N . n = -kappa grad u . n, outward), and the L2
    projection of u on Dirichlet faces with their mask."""
    F = prob.p ** 2
    nt = prob.n_faces * F
    side = face_sides(prob)
    psi = face_basis(prob.k)
    bfaces = np.nonzero(side >= 0)[0]
    pts = _face_points(prob, bfaces)
    R = np.zeros(nt)
    lam = np.zeros(nt)
    dmask = np.zeros(nt, bool)
    for fce in bfaces:
        xq, nq, dA = pts[fce]
        rows = fce * F + np.arange(F)
        if side[fce] in prob.neumann:
            kap = prob.kappa_face(np.array([fce]))[0]
            qn = -kap * np.einsum("qd,qd->q", grad_u(xq), nq)
            R[rows] = -(dA * qn) @ psi
        else:
            Mf = np.einsum("q,qm,ql->ml", dA, psi, psi)
            lam[rows] = np.linalg.solve(Mf, (dA * u_exact(xq)) @ psi)
            dmask[rows] = True
    return R, lam, dmask


def _ldof(fids, F):
    return (fids[:, :, None] * F + np.arange(F)[None, None]).reshape(
        fids.shape[0], 6 * F)


def solve(prob, f, u_exact, grad_u, tau=None):
    """HDG solution of the problem whose exact solution is u_exact (data on
    the Dirichlet and Neumann sides of `prob`), by static condensation onto
    the trace (Eq. hdg_matrix_condensed) and a sparse direct solve.

    Returns a Solution with U [ncells * p^3] (cell-major, like the SIPG
    vectors), Q [ncells, 3, p^3], Lam [nfaces, p^2]."""
    p = prob.p
    N, F = p ** 3, p * p
    if tau is None:
        tau = tau_faces(prob)
    cells = np.arange(prob.ncells)
    M, Nc, Hs, fids = local_blocks(prob, cells, tau)
    Fc = cell_load(prob, f)
    MiN = np.linalg.solve(M, Nc)                          # [c, 4N, 6F]
    MiF = np.linalg.solve(M, Fc[..., None])[..., 0]       # [c, 4N]
    # condensed matrix K = H + sum N^T M^-1 N, rhs R + sum N^T M^-1 F
    Kc = np.einsum("cai,caj->cij", Nc, MiN)               # [c, 6F, 6F]
    rc = np.einsum("cai,ca->ci", Nc, MiF)                 # [c, 6F]
    ldof = _ldof(fids, F)
    for j in range(6):
        Kc[:, j * F:(j + 1) * F, j * F:(j + 1) * F] += Hs[:, j]
    nt = prob.n_faces * F
    K = sp.coo_matrix((Kc.ravel(), (np.repeat(ldof, 6 * F, 1).ravel(),
                                    np.tile(ldof, (1, 6 * F)).ravel())),
                      shape=(nt, nt)).tocsr()
    R, lam, dmask = trace_data(prob, u_exact, grad_u)
    np.add.at(R, ldof.ravel(), rc.ravel())
    free = ~dmask
    rhs = R[free] - K[free][:, dmask] @ lam[dmask]
    lam[free] = spla.spsolve(K[free][:, free].tocsc(), rhs)
    X = MiF - np.einsum("caj,cj->ca", MiN, lam[ldof])
    out = Solution()
    out.Q = X[:, :3 * N].reshape(prob.ncells, 3, N)
    out.U = X[:, 3 * N:].reshape(-1)
    out.X = X.reshape(-1)
    out.Lam = lam.reshape(prob.n_faces, F)
    return out


def postprocess(prob, sol):
    """Element-by-element post-processing (Sec. 2.3): u* in Q_{k+1}(K) with
    (grad u*, grad w)_K = -(kappa^-1 q_h, grad w)_K for all w in Q_{k+1}(K)
    and (u*, 1)_K = (u_h, 1)_K, with the (k+2)-point Gauss rule.  Returns
    the degree k+1 SIPG-layout vector and its fem.Problem.  u* is defined on
    the cells of `prob`; the returned Problem interpolates the map with
    degree k+1, so it describes the same cells only when they are affine."""
    k = prob.k
    P2 = fem.Problem(*prob.n, k + 1, disc="dg", mapping=prob.mapping,
                     amp=prob.amp, kappa=prob.kappa, a_cell=None,
                     box=prob.box)
    if prob.a_cell is not None:
        raise ValueError("post-processing with a point coefficient")
    gq, wq = fem.gauss_rule(k + 2)
    ref = fem.tensor_points(gq)
    w = fem.tensor_weights(wq)
    v1, _ = fem.basis3d(k, ref)
    v2, g2 = fem.basis3d(k + 1, ref)
    cells = np.arange(prob.ncells)
    _, _, det, Jinv = prob.geometry(cells, ref)
    pg2 = np.einsum("cmed,mie->cmid", Jinv, g2)
    wd = det * w[None]
    S = np.einsum("cm,cmid,cmjd->cij", wd, pg2, pg2)
    qh = np.einsum("mi,cdi->cmd", v1, sol.Q) / prob.kappa  # kappa^-1 q_h
    rhs = -np.einsum("cm,cmid,cmd->ci", wd, pg2, qh)
    mean2 = wd @ v2                                       # (phi_i, 1)
    uh = sol.U.reshape(prob.ncells, -1)
    mean_u = np.einsum("cm,mi,ci->c", wd, v1, uh)
    n2 = v2.shape[1]
    big = np.zeros((prob.ncells, n2 + 1, n2 + 1))
    big[:, :n2, :n2] = S
    big[:, :n2, n2] = mean2
    big[:, n2, :n2] = mean2
    b = np.concatenate([rhs, mean_u[:, None]], 1)
    ust = np.linalg.solve(big, b[..., None])[..., 0][:, :n2]
    return ust.reshape(-1), P2


def mixed_operator(prob, tau=None):
    """The mixed HDG operator [A B^T; B D] + [C^T; G^T] H^{-1} [C G] (Sec. 3,
    "HDG mixed matrix-free") on the cell unknowns (q_x, q_y, q_z, u) of every
    cell (cell-major blocks of 4 p^3), with the Dirichlet traces eliminated
    as known (no H^{-1} coupling through Dirichlet faces): a sparse matrix."""
    F = prob.p ** 2
    if tau is None:
        tau = tau_faces(prob)
    cells = np.arange(prob.ncells)
    M, Nc, Hs, fids = local_blocks(prob, cells, tau)
    n4 = M.shape[1]
    nc = prob.ncells
    rows = [np.repeat(np.arange(n4)[None] + n4 * cells[:, None], n4, 1)]
    cols = [np.tile(np.arange(n4)[None] + n4 * cells[:, None], (1, n4))]
    vals = [M.reshape(nc, -1)]
    # H per face and its inverse
    H = face_H(prob, Hs, fids)
    side = face_sides(prob)
    dir_face = (side >= 0) & ~np.isin(side, list(prob.neumann))
    Hi = np.zeros_like(H)
    Hi[~dir_face] = np.linalg.inv(H[~dir_face])
    # [C^T; G^T] H^-1 [C G]: couples the (one or two) cells of each face
    owner = [[] for _ in range(prob.n_faces)]
    for c in range(nc):
        for j in range(6):
            owner[fids[c, j]].append((c, j))
    for fce in range(prob.n_faces):
        if dir_face[fce]:
            continue
        for (c1, j1) in owner[fce]:
            L = Nc[c1][:, j1 * F:(j1 + 1) * F] @ Hi[fce]
            for (c2, j2) in owner[fce]:
                blk = L @ Nc[c2][:, j2 * F:(j2 + 1) * F].T
                r = np.arange(n4) + n4 * c1
                cc = np.arange(n4) + n4 * c2
                rows.append(np.repeat(r, n4)[None])
                cols.append(np.tile(cc, n4)[None])
                vals.append(blk.reshape(1, -1))
    A = sp.coo_matrix((np.concatenate([v.ravel() for v in vals]),
                       (np.concatenate([r.ravel() for r in rows]),
                        np.concatenate([c.ravel() for c in cols]))),
                      shape=(n4 * nc, n4 * nc)).tocsr()
    A.sum_duplicates()
    return A


def face_H(prob, Hs, fids):
    """H per face [nfaces, p^2, p^2] from the cells' side contributions."""
    F = prob.p ** 2
    H = np.zeros((prob.n_faces, F, F))
    for j in range(6):
        np.add.at(H, fids[:, j], Hs[:, j])
    return H


def mixed_rhs(prob, f, u_exact, grad_u, tau=None):
    """Right-hand side of the mixed system (cell unknowns only, cell-major
    blocks of 4 p^3): [0; -(v, f)] - [C^T; G^T] (H^{-1} R on the other
    faces, the projected data on Dirichlet faces), so that
    mixed_operator(prob) X = mixed_rhs(...) has the HDG solution."""
    F = prob.p ** 2
    if tau is None:
        tau = tau_faces(prob)
    cells = np.arange(prob.ncells)
    _, Nc, Hs, fids = local_blocks(prob, cells, tau)
    H = face_H(prob, Hs, fids)
    R, lam, dmask = trace_data(prob, u_exact, grad_u)
    Rf = R.reshape(prob.n_faces, F)
    dface = dmask.reshape(prob.n_faces, F).any(1)
    lamf = lam.reshape(prob.n_faces, F).copy()
    for fce in np.nonzero(~dface)[0]:
        lamf[fce] = np.linalg.solve(H[fce], Rf[fce])
    Fc = cell_load(prob, f)
    Fc -= np.einsum("caj,cj->ca", Nc, lamf[fids].reshape(prob.ncells, -1))
    return Fc.reshape(-1)



def mixed_apply_cells(prob, x, cells, tau=None):
    """Rows of the mixed operator for the listed cells only (for meshes too
    large to assemble): y_c = M_c x_c + sum over the non-Dirichlet faces f of
    c of N_c,f H_f^{-1} sum over the cells c' of f of N_c',f^T x_c'.
    x is the full cell-major vector; returns [len(cells), 4 p^3]."""
    F = prob.p ** 2
    if tau is None:
        tau = tau_faces(prob)
    cells = np.asarray(cells)
    n4 = 4 * prob.p ** 3
    X = np.asarray(x).reshape(prob.ncells, n4)
    side = face_sides(prob)
    dir_face = (side >= 0) & ~np.isin(side, list(prob.neumann))
    # the listed cells and every cell across one of their faces
    fids_c = cell_face_ids(prob, cells)
    need = set(int(c) for c in cells)
    owners = {}
    for d in range(3):
        fid, left, right = fem.face_cells(prob, d)
        sel = np.isin(fid, fids_c.ravel())
        for f, L, R in zip(fid[sel], left[sel], right[sel]):
            owners[int(f)] = [int(c) for c in (L, R) if c >= 0]
            need.update(owners[int(f)])
    need = np.array(sorted(need))
    M, Nc, Hs, fids = local_blocks(prob, need, tau)
    pos = {int(c): i for i, c in enumerate(need)}
    out = np.zeros((cells.size, n4))
    for r, c in enumerate(cells):
        i = pos[int(c)]
        y = M[i] @ X[c]
        for j in range(6):
            f = int(fids[i, j])
            if dir_face[f]:
                continue
            H = np.zeros((F, F))
            g = np.zeros(F)
            for c2 in owners[f]:
                i2 = pos[c2]
                j2 = int(np.nonzero(fids[i2] == f)[0][0])
                H += Hs[i2, j2]
                g += Nc[i2][:, j2 * F:(j2 + 1) * F].T @ X[c2]
            y += Nc[i][:, j * F:(j + 1) * F] @ np.linalg.solve(H, g)
        out[r] = y
    return out
