"""Plain float64 finite-element assembly for -div(kappa grad u) = f
(Sec. 2, Eq. 1) on a structured hexahedral brick of the unit cube.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).  Written from the paper,
not from the CUDA library: it evaluates every 3D basis function directly as
a product of 1D Lagrange polynomials at every quadrature point and forms the
element matrices as dense sums over quadrature points.  No sum
factorisation, no tensor-product shortcuts.

Conventions (shared with the CUDA library only through the documented
vector layouts):
  * reference cell [-1, 1]^3 (Sec. 2); local node / quadrature point index
    a = ax + p*ay + p*p*az with p = k+1 (x fastest);
  * cells c = cx + nx*(cy + ny*cz) on the unit cube, cell size 1/n per axis;
  * CG vectors: global lexicographic nodes on the (nx*k+1, ny*k+1, nz*k+1)
    grid, x fastest, boundary nodes included; DG vectors: cell-major blocks
    of p^3 values in local order;
  * faces: all x-normal faces, then y-normal, then z-normal; within one
    direction lexicographic with x fastest over (n_x+dx, n_y+dy, n_z+dz)
    where d* = 1 on the normal axis; face quadrature point q = qa + p*qb with
    a < b the two tangential axes.
"""
import numpy as np
import scipy.sparse as sp
from numpy.polynomial import legendre as npleg


# --------------------------------------------------------------------------
# 1D reference element (Sec. 2.1: Lagrange basis in the (k+1) Gauss-Lobatto
# -Legendre nodes; Sec. 3: Gauss-Legendre quadrature with k+1 points)
# --------------------------------------------------------------------------
def gll_points(k):
    """The k+1 Gauss-Lobatto-Legendre nodes on [-1, 1]: the end points and the
    roots of P_k' (Sec. 2.1), sorted ascending."""
    if k < 1:
        raise ValueError("degree must be >= 1")
    if k == 1:
        return np.array([-1.0, 1.0])
    c = np.zeros(k + 1)
    c[k] = 1.0
    dp = npleg.legder(c)
    d2p = npleg.legder(dp)
    r = np.sort(npleg.legroots(dp).real)
    for _ in range(4):  # Newton polish of the roots of P_k'
        r = r - npleg.legval(r, dp) / npleg.legval(r, d2p)
    return np.concatenate([[-1.0], r, [1.0]])


def gauss_rule(n):
    """n-point Gauss-Legendre points and weights on [-1, 1] (Sec. 3)."""
    x, w = npleg.leggauss(n)
    return np.asarray(x, float), np.asarray(w, float)


def lagrange_values(nodes, x):
    """V[m, i] = phi_i(x_m), phi_i the Lagrange polynomial of `nodes`."""
    x = np.asarray(x, float)
    n = len(nodes)
    V = np.ones((x.size, n))
    for i in range(n):
        for j in range(n):
            if j != i:
                V[:, i] *= (x - nodes[j]) / (nodes[i] - nodes[j])
    return V


def lagrange_derivatives(nodes, x):
    """D[m, i] = phi_i'(x_m) by the product rule on the Lagrange product."""
    x = np.asarray(x, float)
    n = len(nodes)
    D = np.zeros((x.size, n))
    for i in range(n):
        for m in range(n):
            if m == i:
                continue
            term = np.full(x.size, 1.0 / (nodes[i] - nodes[m]))
            for j in range(n):
                if j != i and j != m:
                    term = term * (x - nodes[j]) / (nodes[i] - nodes[j])
            D[:, i] += term
    return D


def basis3d(k, pts):
    """Values [M, N] and reference gradients [M, N, 3] of all N=(k+1)^3 nodal
    basis functions phi_a(xi) = phi_ax(xi_1) phi_ay(xi_2) phi_az(xi_3) at the
    reference points pts [M, 3] (Sec. 2.1: tensor-product Q_k)."""
    nodes = gll_points(k)
    p = k + 1
    pts = np.atleast_2d(pts)
    Vd = [lagrange_values(nodes, pts[:, d]) for d in range(3)]
    Dd = [lagrange_derivatives(nodes, pts[:, d]) for d in range(3)]
    ax = np.tile(np.arange(p), p * p)
    ay = np.tile(np.repeat(np.arange(p), p), p)
    az = np.repeat(np.arange(p), p * p)
    val = Vd[0][:, ax] * Vd[1][:, ay] * Vd[2][:, az]
    grad = np.stack([Dd[0][:, ax] * Vd[1][:, ay] * Vd[2][:, az],
                     Vd[0][:, ax] * Dd[1][:, ay] * Vd[2][:, az],
                     Vd[0][:, ax] * Vd[1][:, ay] * Dd[2][:, az]], axis=-1)
    return val, grad


def tensor_points(x1):
    """All points (x1[a], x1[b], x1[c]) in local order a + p b + p^2 c."""
    p = len(x1)
    X = np.empty((p ** 3, 3))
    X[:, 0] = np.tile(x1, p * p)
    X[:, 1] = np.tile(np.repeat(x1, p), p)
    X[:, 2] = np.repeat(x1, p * p)
    return X


def tensor_weights(w1):
    p = len(w1)
    return (np.tile(w1, p * p) * np.tile(np.repeat(w1, p), p)
            * np.repeat(w1, p * p))


# --------------------------------------------------------------------------
# Problem description, mesh and mapping (Sec. 2: cells are images of the
# reference cube under a degree-l polynomial map through Gauss-Lobatto
# support points placed on the manifold; here l = k)
# --------------------------------------------------------------------------
class Problem:
    """Discrete Poisson problem on the unit cube.

    disc          'cg' (Sec. 2.1) or 'dg' (symmetric interior penalty, Sec. 2.2)
    mapping       'identity' or 'sine': x -> x + amp sin(pi x) sin(pi y)
                  sin(pi z) (1,1,1), interpolated isoparametrically; or
                  'nodes': the support points are given (map_nodes)
    map_nodes     mapping 'nodes': physical support points [ncells, p^3, 3]
                  (the images of each cell's Gauss-Lobatto grid, local order
                  a = ax + p ay + p^2 az); the box is not applied to them
    kappa         constant coefficient, used when a_cell / a_face are None
    a_cell        optional [ncells, p^3] coefficient at cell quadrature points
    a_face        optional [nfaces, p^2] coefficient at face quadrature points
    penalty_factor  sigma_F = penalty_factor (k+1)^2 / h_F (Sec. 2.2)
    dirichlet     Dirichlet data on the boundary; False drops the constraints
                  (CG) or the boundary faces (DG), which is only used to test
                  that constants are in the kernel
    box           (lo, hi): the domain is [lo, hi]^3, the image of the unit
                  cube under x -> lo + (hi - lo) x after the mapping above
    neumann_sides boundary sides with Neumann data (natural for CG, no
                  operator terms on the SIPG faces, Eq. 7); side 2d is
                  x_d = lo, side 2d+1 is x_d = hi; the others are Dirichlet
    """

    def __init__(self, nx, ny, nz, k, disc="cg", mapping="identity", amp=0.0,
                 kappa=1.0, a_cell=None, a_face=None, penalty_factor=1.0,
                 dirichlet=True, box=(0.0, 1.0), neumann_sides=(),
                 map_nodes=None):
        if disc not in ("cg", "dg"):
            raise ValueError(disc)
        if mapping not in ("identity", "sine", "nodes"):
            raise ValueError(mapping)
        self.n = (int(nx), int(ny), int(nz))
        self.k = int(k)
        self.p = self.k + 1
        self.disc = disc
        self.mapping = mapping
        self.amp = float(amp) if mapping == "sine" else 0.0
        self.kappa = float(kappa)
        self.a_cell = None if a_cell is None else np.asarray(a_cell, float)
        self.a_face = None if a_face is None else np.asarray(a_face, float)
        self.penalty_factor = float(penalty_factor)
        self.dirichlet = bool(dirichlet)
        self.box = (float(box[0]), float(box[1]))
        if not self.box[1] > self.box[0]:
            raise ValueError("box must have hi > lo")
        self.neumann = frozenset(int(v) for v in neumann_sides)
        if not self.neumann <= set(range(6)):
            raise ValueError("neumann_sides must be in 0..5")
        self.h = tuple(1.0 / n for n in self.n)
        self.ncells = self.n[0] * self.n[1] * self.n[2]
        self.nodes1 = gll_points(self.k)
        self.map_nodes = None
        if mapping == "nodes":
            X = np.asarray(map_nodes, float)
            if X.shape != (self.ncells, self.p ** 3, 3):
                raise ValueError("map_nodes must be [ncells, p^3, 3]")
            self.map_nodes = X

    # ---- sizes -----------------------------------------------------------
    @property
    def grid(self):
        return tuple(n * self.k + 1 for n in self.n)

    @property
    def n_dofs(self):
        if self.disc == "cg":
            g = self.grid
            return g[0] * g[1] * g[2]
        return self.ncells * self.p ** 3

    def n_faces_dir(self, d):
        n = list(self.n)
        n[d] += 1
        return n[0] * n[1] * n[2]

    @property
    def n_faces(self):
        return sum(self.n_faces_dir(d) for d in range(3))

    # ---- geometry --------------------------------------------------------
    def cell_index(self, cx, cy, cz):
        return cx + self.n[0] * (cy + self.n[1] * cz)

    def cell_coords(self, cells):
        cells = np.asarray(cells)
        cx = cells % self.n[0]
        cy = (cells // self.n[0]) % self.n[1]
        cz = cells // (self.n[0] * self.n[1])
        return cx, cy, cz

    def phi_map(self, x):
        """The analytic map of the unit cube (identity or sine), followed by
        the affine map onto the box."""
        x = np.asarray(x, float)
        y = x.copy()
        if self.amp != 0.0:
            s = (np.sin(np.pi * x[..., 0]) * np.sin(np.pi * x[..., 1])
                 * np.sin(np.pi * x[..., 2]))
            y = x + self.amp * s[..., None]
        lo, hi = self.box
        if (lo, hi) != (0.0, 1.0):
            y = lo + (hi - lo) * y
        return y

    def logical_points(self, cells, ref):
        """Unit-cube points of reference coordinates ref [M,3] in `cells`."""
        cx, cy, cz = self.cell_coords(cells)
        org = np.stack([cx * self.h[0], cy * self.h[1], cz * self.h[2]], -1)
        return org[:, None, :] + 0.5 * (np.asarray(ref)[None] + 1.0) * \
            np.asarray(self.h)[None, None, :]

    def support_points(self, cells):
        """Isoparametric support points X[c, a, 3]: the analytic map evaluated
        at the GLL nodes of each cell (Sec. 2), or the given nodes."""
        if self.map_nodes is not None:
            return self.map_nodes[np.asarray(cells)]
        ref = tensor_points(self.nodes1)
        return self.phi_map(self.logical_points(cells, ref))

    def geometry(self, cells, ref):
        """Physical points x, Jacobians J[c,m,d,e] = dx_d/dxi_e, det J and
        J^{-1} at reference points ref [M,3] of the interpolated map."""
        X = self.support_points(cells)
        val, grad = basis3d(self.k, ref)
        x = np.einsum("cad,ma->cmd", X, val)
        J = np.einsum("cad,mae->cmde", X, grad)
        det = np.linalg.det(J)
        if np.any(det <= 0):
            raise ValueError("mapping is not invertible")
        return x, J, det, np.linalg.inv(J)

    # ---- coefficient -----------------------------------------------------
    def kappa_cell(self, cells):
        cells = np.asarray(cells)
        if self.a_cell is not None:
            return self.a_cell[cells]
        return np.full((cells.size, self.p ** 3), self.kappa)

    def kappa_face(self, faces):
        faces = np.asarray(faces)
        if self.a_face is not None:
            return self.a_face[faces]
        return np.full((faces.size, self.p ** 2), self.kappa)

    # ---- dof numbering ---------------------------------------------------
    def dof_map(self, cells=None):
        """Global dof index [c, a] of local node a of cell c."""
        if cells is None:
            cells = np.arange(self.ncells)
        cells = np.asarray(cells)
        p, k = self.p, self.k
        a = np.arange(p ** 3)
        ax, ay, az = a % p, (a // p) % p, a // (p * p)
        if self.disc == "dg":
            return cells[:, None] * p ** 3 + a[None, :]
        cx, cy, cz = self.cell_coords(cells)
        g = self.grid
        ix = cx[:, None] * k + ax[None]
        iy = cy[:, None] * k + ay[None]
        iz = cz[:, None] * k + az[None]
        return ix + g[0] * (iy + g[1] * iz)

    def constrained(self):
        """Boolean mask of Dirichlet-constrained dofs (CG boundary nodes)."""
        N = self.n_dofs
        mask = np.zeros(N, bool)
        if self.disc != "cg" or not self.dirichlet:
            return mask
        g = self.grid
        i = np.arange(N)
        idx = (i % g[0], (i // g[0]) % g[1], i // (g[0] * g[1]))
        for d in range(3):
            if 2 * d not in self.neumann:
                mask |= idx[d] == 0
            if 2 * d + 1 not in self.neumann:
                mask |= idx[d] == g[d] - 1
        return mask

    def node_points(self):
        """Physical location of every dof (the support points)."""
        X = self.support_points(np.arange(self.ncells))
        dm = self.dof_map()
        out = np.empty((self.n_dofs, 3))
        out[dm.ravel()] = X.reshape(-1, 3)
        return out


# --------------------------------------------------------------------------
# Cell integrals (Eq. 4 / Eq. 12): K^e_ij = sum_q w_q det J kappa
#   (J^{-T} grad_xi phi_i) . (J^{-T} grad_xi phi_j)
# --------------------------------------------------------------------------
def cell_matrices(prob, cells):
    cells = np.asarray(cells)
    gq, wq = gauss_rule(prob.p)
    ref = tensor_points(gq)
    w = tensor_weights(wq)
    _, grad = basis3d(prob.k, ref)                       # [M, N, 3]
    _, _, det, Jinv = prob.geometry(cells, ref)
    kap = prob.kappa_cell(cells)
    # G[c,m,e,f] = w_m det J kappa (J^{-1} J^{-T})_{ef}
    G = np.einsum("cmed,cmfd->cmef", Jinv, Jinv) * \
        (w[None, :] * det * kap)[..., None, None]
    M, N = grad.shape[0], grad.shape[1]
    tmp = np.einsum("cmef,mjf->cmej", G, grad).reshape(len(cells), 3 * M, N)
    B = grad.transpose(0, 2, 1).reshape(3 * M, N)          # rows (m, e)
    return np.einsum("ri,crj->cij", B, tmp)


# --------------------------------------------------------------------------
# SIPG face integrals (Eq. 6 with the boundary extension of Eq. 7)
# --------------------------------------------------------------------------
def _face_ref_points(p, d, side):
    """Reference points [p^2, 3] and weights of the face xi_d = side."""
    gq, wq = gauss_rule(p)
    t = [e for e in range(3) if e != d]
    pts = np.empty((p * p, 3))
    pts[:, d] = side
    pts[:, t[0]] = np.tile(gq, p)
    pts[:, t[1]] = np.repeat(gq, p)
    return pts, np.tile(wq, p) * np.repeat(wq, p)


def face_cells(prob, d):
    """For direction d: (face ids, left cell or -1, right cell or -1)."""
    n = list(prob.n)
    m = list(n)
    m[d] += 1
    f = np.arange(m[0] * m[1] * m[2])
    fc = [f % m[0], (f // m[0]) % m[1], f // (m[0] * m[1])]
    off = sum(prob.n_faces_dir(e) for e in range(d))
    lo = list(fc)
    lo[d] = fc[d] - 1
    left = np.where(fc[d] >= 1, prob.cell_index(*lo), -1)
    right = np.where(fc[d] < n[d], prob.cell_index(*fc), -1)
    return f + off, left, right


def cell_volumes(prob, cells):
    gq, wq = gauss_rule(prob.p)
    _, _, det, _ = prob.geometry(cells, tensor_points(gq))
    return det @ tensor_weights(wq)


def _side_data(prob, cells, d, side, normal=None):
    """Basis values, physical gradients, outward normal and area element of
    `cells` on their face xi_d = side at the face Gauss points."""
    pts, wf = _face_ref_points(prob.p, d, side)
    val, grad = basis3d(prob.k, pts)
    x, J, det, Jinv = prob.geometry(cells, pts)
    # physical gradient: J^{-T} grad_xi
    pg = np.einsum("cmed,mie->cmid", Jinv, grad)
    # cofactor normal: det J J^{-T} e_d scaled by the reference orientation
    nvec = side * Jinv[:, :, d, :] * 1.0                  # J^{-T} e_d rows
    nlen = np.linalg.norm(nvec, axis=-1)
    n_out = nvec / nlen[..., None]
    dA = det * nlen * wf[None, :]
    return dict(val=val, pg=pg, n=n_out, dA=dA, x=x)


def face_operators(prob, d, faces=None):
    """Per-quadrature-point jump and average operators of the faces of
    direction d (Eq. 6, boundary extension of Eq. 7).

    Yields groups dict(fid, cells [F, s], jump_u, avg_u, jump_v, avg_v,
    c [F, m] = dA (no coefficient), sigma [F]) with s = 2 (interior: left,
    right) or 1 (boundary).  The operators act on the concatenated local
    dofs of the cells: for interior faces [u] = u- - u+ and
    {d_n u} = (d_n u- + d_n u+)/2 with n the outward normal of the left
    cell; on the boundary the mirror u+ = -u-, grad u+ = grad u- gives
    [u] = 2 u-, {d_n u} = d_n u-, while the test function has no outside
    value, so the test-side operators are v- and d_n v- / 2."""
    fid, left, right = face_cells(prob, d)
    if faces is not None:
        sel = np.isin(fid, faces)
        fid, left, right = fid[sel], left[sel], right[sel]
    pen = prob.penalty_factor * prob.p ** 2
    inner = (left >= 0) & (right >= 0)
    if inner.any():
        fi, L, R = fid[inner], left[inner], right[inner]
        sl = _side_data(prob, L, d, +1.0)
        sr = _side_data(prob, R, d, -1.0)
        n = sl["n"]                                         # n = n^- (left)
        gL = np.einsum("cmid,cmd->cmi", sl["pg"], n)
        gR = np.einsum("cmid,cmd->cmi", sr["pg"], n)
        vL = np.broadcast_to(sl["val"], gL.shape)
        vR = np.broadcast_to(sr["val"], gR.shape)
        area = sl["dA"].sum(1)
        sigma = pen * 0.5 * (area / cell_volumes(prob, L)
                             + area / cell_volumes(prob, R))
        jump = np.concatenate([vL, -vR], axis=2)
        avg = 0.5 * np.concatenate([gL, gR], axis=2)
        yield dict(fid=fi, cells=np.stack([L, R], 1), jump_u=jump,
                   avg_u=avg, jump_v=jump, avg_v=avg, c=sl["dA"],
                   sigma=sigma)
    if prob.dirichlet and (~inner).any():
        fb = fid[~inner]
        cells = np.where(left[~inner] >= 0, left[~inner], right[~inner])
        side = np.where(left[~inner] >= 0, 1.0, -1.0)
        for s in (1.0, -1.0):
            sel = side == s
            if not sel.any() or (2 * d + (s > 0)) in prob.neumann:
                continue
            cs, fs = cells[sel], fb[sel]
            sd = _side_data(prob, cs, d, s)
            g = np.einsum("cmid,cmd->cmi", sd["pg"], sd["n"])
            v = np.broadcast_to(sd["val"], g.shape)
            area = sd["dA"].sum(1)
            sigma = pen * area / cell_volumes(prob, cs)
            yield dict(fid=fs, cells=cs[:, None], jump_u=2.0 * v, avg_u=g,
                       jump_v=v, avg_v=0.5 * g, c=sd["dA"], sigma=sigma)


def face_terms(prob, d, faces=None):
    """Face matrices of direction d: a list of (face id, cells, matrix) with
    matrix = sum_q kappa_q dA_q [ -[v]{d_n u} - {d_n v}[u] + sigma [v][u] ]
    over the local dofs of the listed cells (Eq. 6, 7)."""
    out = []
    for g in face_operators(prob, d, faces):
        c = prob.kappa_face(g["fid"]) * g["c"]
        A = (-np.einsum("fmi,fm,fmj->fij", g["jump_v"], c, g["avg_u"])
             - np.einsum("fmi,fm,fmj->fij", g["avg_v"], c, g["jump_u"])
             + g["sigma"][:, None, None]
             * np.einsum("fmi,fm,fmj->fij", g["jump_v"], c, g["jump_u"]))
        for t in range(len(g["fid"])):
            out.append((g["fid"][t], tuple(g["cells"][t]), A[t]))
    return out


# --------------------------------------------------------------------------
# Global assembly with Dirichlet rows and columns replaced by identity
# (Sec. 2.1: "elimination of Dirichlet rows and columns")
# --------------------------------------------------------------------------
def assemble(prob, chunk=64):
    N = prob.n_dofs
    rows, cols, vals = [], [], []
    allc = np.arange(prob.ncells)
    for s in range(0, prob.ncells, chunk):
        cells = allc[s:s + chunk]
        K = cell_matrices(prob, cells)
        dm = prob.dof_map(cells)
        rows.append(np.repeat(dm, dm.shape[1], axis=1).ravel())
        cols.append(np.tile(dm, (1, dm.shape[1])).ravel())
        vals.append(K.ravel())
    if prob.disc == "dg":
        for d in range(3):
            for _, cells, A in face_terms(prob, d):
                dm = prob.dof_map(np.array(cells)).ravel()
                rows.append(np.repeat(dm, dm.size))
                cols.append(np.tile(dm, dm.size))
                vals.append(A.ravel())
    A = sp.coo_matrix((np.concatenate(vals),
                       (np.concatenate(rows), np.concatenate(cols))),
                      shape=(N, N)).tocsr()
    A.sum_duplicates()
    cmask = prob.constrained()
    if cmask.any():
        keep = sp.diags((~cmask).astype(float))
        A = (keep @ A @ keep + sp.diags(cmask.astype(float))).tocsr()
    return A


# --------------------------------------------------------------------------
# Load vector (Eq. 4 / Eq. 6 right-hand side), interpolation and L2 error
# --------------------------------------------------------------------------
def load_vector(prob, f, chunk=256):
    """b_i = sum_q w_q det J f(x_q) phi_i(xi_q) with the (k+1)^3 Gauss rule;
    zero on Dirichlet-constrained dofs."""
    gq, wq = gauss_rule(prob.p)
    ref = tensor_points(gq)
    w = tensor_weights(wq)
    val, _ = basis3d(prob.k, ref)
    b = np.zeros(prob.n_dofs)
    allc = np.arange(prob.ncells)
    for s in range(0, prob.ncells, chunk):
        cells = allc[s:s + chunk]
        x, _, det, _ = prob.geometry(cells, ref)
        fq = f(x) * det * w[None]
        be = fq @ val                                       # [c, N]
        np.add.at(b, prob.dof_map(cells).ravel(), be.ravel())
    b[prob.constrained()] = 0.0
    return b


def interpolate(prob, fn):
    """Nodal interpolant: value of fn at every support point."""
    return fn(prob.node_points())


def l2_error(prob, u, exact, chunk=256):
    """||u_h - u||_{L2} with a (k+3)-point Gauss rule per direction."""
    gq, wq = gauss_rule(prob.k + 3)
    ref = tensor_points(gq)
    w = tensor_weights(wq)
    val, _ = basis3d(prob.k, ref)
    err2 = 0.0
    allc = np.arange(prob.ncells)
    for s in range(0, prob.ncells, chunk):
        cells = allc[s:s + chunk]
        x, _, det, _ = prob.geometry(cells, ref)
        uh = u[prob.dof_map(cells)] @ val.T
        err2 += np.sum((uh - exact(x)) ** 2 * det * w[None])
    return np.sqrt(err2)


def sine_solution(x):
    """u = sin(pi x) sin(pi y) sin(pi z), the manufactured solution."""
    return (np.sin(np.pi * x[..., 0]) * np.sin(np.pi * x[..., 1])
            * np.sin(np.pi * x[..., 2]))


def sine_forcing(x):
    """f = 3 pi^2 sin sin sin = -Laplace(u) for kappa = 1."""
    return 3.0 * np.pi ** 2 * sine_solution(x)


# --------------------------------------------------------------------------
# Inhomogeneous boundary data (Eq. 7 and its continuous counterpart):
# Dirichlet values g_D and Neumann fluxes g_N = kappa grad u . n (outward)
# of a manufactured solution, moved to the right-hand side
# --------------------------------------------------------------------------
def _boundary_side(prob, d, s):
    """Cells on boundary side x_d = lo (s = -1) or hi (s = +1) and their
    face data at the face Gauss points (values, physical gradients, outward
    normal, area element, points)."""
    cx, cy, cz = prob.cell_coords(np.arange(prob.ncells))
    c = (cx, cy, cz)[d]
    cells = np.nonzero(c == (prob.n[d] - 1 if s > 0 else 0))[0]
    return cells, _side_data(prob, cells, d, float(s))


def neumann_vector(prob, grad_u):
    """b_i = sum over Neumann sides of int kappa grad u . n phi_i ds
    (natural boundary condition; SIPG: the extension of Eq. 7 leaves only
    this data term on a Neumann face)."""
    b = np.zeros(prob.n_dofs)
    for side in sorted(prob.neumann):
        d, s = side // 2, (1 if side % 2 else -1)
        cells, sd = _boundary_side(prob, d, s)
        faces = _boundary_face_ids(prob, d, s, cells)
        kap = prob.kappa_face(faces)
        gn = np.einsum("cmd,cmd->cm", grad_u(sd["x"]), sd["n"])
        be = (kap * gn * sd["dA"]) @ sd["val"]
        np.add.at(b, prob.dof_map(cells).ravel(), be.ravel())
    return b


def _boundary_face_ids(prob, d, s, cells):
    cx, cy, cz = prob.cell_coords(cells)
    fc = [cx, cy, cz]
    fc[d] = fc[d] + (1 if s > 0 else 0)
    m = list(prob.n)
    m[d] += 1
    off = sum(prob.n_faces_dir(e) for e in range(d))
    return off + fc[0] + m[0] * (fc[1] + m[1] * fc[2])


def sipg_dirichlet_vector(prob, u):
    """SIPG data terms of the Dirichlet extension u+ = -u- + 2 g_D, grad u+ =
    grad u- (Eq. 7): with the boundary form of face_terms the known part is
    kappa dA (-d_n v g_D + 2 sigma v g_D), moved to the right-hand side."""
    b = np.zeros(prob.n_dofs)
    pen = prob.penalty_factor * prob.p ** 2
    for d in range(3):
        for s in (-1, 1):
            if (2 * d + (s > 0)) in prob.neumann:
                continue
            cells, sd = _boundary_side(prob, d, s)
            faces = _boundary_face_ids(prob, d, s, cells)
            kap = prob.kappa_face(faces)
            sigma = pen * sd["dA"].sum(1) / cell_volumes(prob, cells)
            gd = u(sd["x"]) * kap * sd["dA"]
            dn = np.einsum("cmid,cmd->cmi", sd["pg"], sd["n"])
            be = (-np.einsum("cm,cmi->ci", gd, dn)
                  + 2.0 * sigma[:, None] * (gd @ sd["val"]))
            np.add.at(b, prob.dof_map(cells).ravel(), be.ravel())
    return b


def manufactured_rhs(prob, f, u, grad_u):
    """Right-hand side for -div(kappa grad u) = f with the Dirichlet data of
    u on the Dirichlet sides and the Neumann flux of u on the Neumann sides,
    for the matrix of `assemble(prob)`: load vector plus Neumann data; SIPG:
    plus the data terms of Eq. 7; CG: the constrained rows hold the
    interpolated Dirichlet values and the free rows have them lifted out,
    b_f - A_fc g_c (Sec. 2.1), so that the system's solution is complete."""
    b = load_vector(prob, f) + neumann_vector(prob, grad_u)
    if prob.disc == "dg":
        return b + sipg_dirichlet_vector(prob, u)
    full = Problem(*prob.n, prob.k, disc="cg", mapping=prob.mapping,
                   amp=prob.amp, kappa=prob.kappa, a_cell=prob.a_cell,
                   a_face=prob.a_face, dirichlet=False, box=prob.box,
                   map_nodes=prob.map_nodes)
    dmask = prob.constrained()
    g = np.zeros(prob.n_dofs)
    g[dmask] = u(prob.node_points()[dmask])
    b = b - assemble(full) @ g
    b[dmask] = g[dmask]
    return b


def solve_manufactured(prob, f, u, grad_u):
    """Discrete solution of the problem of manufactured_rhs by a sparse
    direct solve.  CG: interpolated Dirichlet values (Sec. 2.1); SIPG:
    weakly imposed (Eq. 7)."""
    import scipy.sparse.linalg as spla
    b = manufactured_rhs(prob, f, u, grad_u)
    return spla.spsolve(assemble(prob).tocsc(), b)
