"""Textbook multigrid-preconditioned CG on assembled matrices (Sec. 4.1).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Sec. 4.1 fixes the recipe: CG preconditioned by one geometric V-cycle,
stopped when the residual norm falls below a tolerance times the norm of
the right-hand side; Chebyshev-accelerated point-Jacobi smoothing of degree
five on the interval [0.06, 1.2] x (estimate of the largest eigenvalue of
D^{-1} A); that estimate from 15 CG iterations; transfer by the geometric
embedding; a Chebyshev coarse solve whose a-priori error bound is below
1e-3.  Readings of what the paper leaves open:
  * Chebyshev: the three-term semi-iteration (Saad, Iterative Methods for
    Sparse Linear Systems, 2nd ed., Alg. 12.1) on D^{-1} A with
    theta = (b + a)/2, delta = (b - a)/2.  `degree` counts the updates of
    x; from a zero start the first update needs no operator application.
  * eigenvalue estimate: 15 Jacobi-PCG iterations on A x = s with
    s_i = 1 + 0.1 sin(i) (0 on constrained dofs), then the extreme
    eigenvalues of the Lanczos tridiagonal built from the CG coefficients
    (Saad Sec. 6.7.3), found by Sturm-sequence bisection.
  * coarse solve: Chebyshev on [0.9 lambda_min, 1.2 lambda_max] of the same
    tridiagonal, smallest degree m with 2 rho^m / (1 + rho^{2m}) < 1e-3,
    rho = (sqrt(c) - 1)/(sqrt(c) + 1), c the interval's condition number.
  * transfer: prolongation is the embedding of the coarse Q_k space in the
    fine one on the reference coordinates; restriction its transpose;
    constrained rows / columns removed.
  * levels: halve the cell counts down to 2 (or n_levels levels); the
    operator is rediscretised on every level.  A per-quadrature-point
    coefficient is carried to a coarse level as the quadrature-weighted
    mean over the children of each coarse cell (cells) or coarse face
    (faces).
"""
import numpy as np
import scipy.sparse as sp

from . import fem


# --------------------------------------------------------------------------
# Level hierarchy
# --------------------------------------------------------------------------
def coarsen_problem(prob):
    """Rediscretisation of `prob` on the mesh with half the cells per axis."""
    if any(n % 2 for n in prob.n):
        raise ValueError("cell counts must be even to coarsen")
    nc = tuple(n // 2 for n in prob.n)
    a_cell = a_face = None
    if prob.a_cell is not None:
        a_cell, a_face = coarsen_coefficient(prob, nc)
    nodes = coarsen_nodes(prob, nc) if prob.map_nodes is not None else None
    return fem.Problem(*nc, prob.k, disc=prob.disc, mapping=prob.mapping,
                       amp=prob.amp, kappa=prob.kappa, a_cell=a_cell,
                       a_face=a_face, penalty_factor=prob.penalty_factor,
                       dirichlet=prob.dirichlet, box=prob.box,
                       neumann_sides=tuple(prob.neumann), map_nodes=nodes)


def coarsen_nodes(prob, nc):
    """Support points of the coarse cells of a mesh given by its nodes: the
    fine isoparametric map evaluated at the coarse cells' Gauss-Lobatto
    points (a coarse point on the interface of two children is taken from
    the upper child)."""
    p = prob.p
    r = prob.nodes1                       # coarse GLL nodes on [-1, 1]
    off = np.minimum(np.floor(r + 1.0), 1).astype(int)   # child per axis
    eta = 2.0 * (r + 1.0 - off) - 1.0     # its reference coordinate
    ncc = nc[0] * nc[1] * nc[2]
    C = np.arange(ncc)
    cx, cy, cz = C % nc[0], (C // nc[0]) % nc[1], C // (nc[0] * nc[1])
    out = np.empty((ncc, p ** 3, 3))
    for a in range(p ** 3):
        ax, ay, az = a % p, (a // p) % p, a // (p * p)
        child = prob.cell_index(2 * cx + off[ax], 2 * cy + off[ay],
                                2 * cz + off[az])
        val, _ = fem.basis3d(prob.k, np.array([[eta[ax], eta[ay], eta[az]]]))
        out[:, a] = np.einsum("cbd,b->cd", prob.support_points(child), val[0])
    return out


def coarsen_coefficient(prob, nc):
    """Quadrature-weighted child means of a per-point coefficient."""
    p = prob.p
    _, wq = fem.gauss_rule(p)
    w3 = fem.tensor_weights(wq)
    w2 = np.tile(wq, p) * np.repeat(wq, p)
    n = prob.n
    cm = (prob.a_cell @ w3 / w3.sum()).reshape(n[2], n[1], n[0])
    coarse = cm.reshape(nc[2], 2, nc[1], 2, nc[0], 2).mean(axis=(1, 3, 5))
    a_cell = np.repeat(coarse.reshape(-1, 1), p ** 3, axis=1)
    fmean = prob.a_face @ w2 / w2.sum()
    out = []
    off = 0
    for d in range(3):
        m = list(n)
        m[d] += 1
        cnt = m[0] * m[1] * m[2]
        blk = fmean[off:off + cnt].reshape(m[2], m[1], m[0])
        off += cnt
        for e in range(3):                  # array axis of mesh axis e: 2-e
            ax = 2 - e
            ev = np.take(blk, np.arange(0, blk.shape[ax], 2), axis=ax)
            if e == d:                      # coarse face F is fine face 2F
                blk = ev
            else:                           # mean of the two tangential kids
                od = np.take(blk, np.arange(1, blk.shape[ax], 2), axis=ax)
                blk = 0.5 * (ev + od)
        out.append(blk.reshape(-1))
    fc = np.concatenate(out)
    return a_cell, np.repeat(fc.reshape(-1, 1), p * p, axis=1)


def hierarchy(prob, n_levels=0):
    """Problems from coarsest (index 0) to `prob` (last).  n_levels = 0 means
    halve while every cell count is even and >= 4."""
    levels = [prob]
    while True:
        cur = levels[-1]
        if n_levels and len(levels) >= n_levels:
            break
        if not n_levels and (any(n % 2 for n in cur.n) or min(cur.n) < 4):
            break
        levels.append(coarsen_problem(cur))
    if n_levels and len(levels) < n_levels:
        raise ValueError("mesh cannot be coarsened that often")
    return levels[::-1]


def prolongation_1d_cg(nc, k):
    """1D embedding matrix [(2 nc k + 1), (nc k + 1)]: coarse global Lagrange
    basis evaluated at the fine GLL nodes."""
    nodes = fem.gll_points(k)
    nf = 2 * nc
    P = np.zeros((nf * k + 1, nc * k + 1))
    for I in range(nf * k + 1):
        cf = min(I // k, nf - 1)
        a = I - cf * k
        x = 0.5 * (cf + 0.5 * (nodes[a] + 1.0))            # coarse-cell units
        C = min(int(np.floor(x)), nc - 1)
        xi = 2.0 * (x - C) - 1.0
        P[I, C * k:C * k + k + 1] = fem.lagrange_values(nodes, [xi])[0]
    P[np.abs(P) < 1e-15] = 0.0
    return P


def child_embedding(k, o):
    """E[i, j] = phi_j((xi_i + (2o - 1)) / 2): coarse basis at the GLL nodes
    of child o in {0, 1} (left / right half of the reference interval)."""
    nodes = fem.gll_points(k)
    return fem.lagrange_values(nodes, 0.5 * (nodes + (2 * o - 1)))


def prolongation(fine, coarse):
    """Sparse prolongation coarse -> fine (Sec. 4.1 geometric embedding)."""
    k = fine.k
    if fine.disc == "cg":
        P = sp.csr_matrix(prolongation_1d_cg(coarse.n[0], k))
        for d in (1, 2):
            P = sp.kron(sp.csr_matrix(prolongation_1d_cg(coarse.n[d], k)), P)
        P = P.tocsr()
        keep_f = sp.diags((~fine.constrained()).astype(float))
        keep_c = sp.diags((~coarse.constrained()).astype(float))
        return (keep_f @ P @ keep_c).tocsr()
    p = fine.p
    E = [child_embedding(k, 0), child_embedding(k, 1)]
    rows, cols, vals = [], [], []
    for C in range(coarse.ncells):
        cx, cy, cz = (int(v) for v in coarse.cell_coords(C))
        for oz in (0, 1):
            for oy in (0, 1):
                for ox in (0, 1):
                    F = fine.cell_index(2 * cx + ox, 2 * cy + oy, 2 * cz + oz)
                    B = np.kron(E[oz], np.kron(E[oy], E[ox]))
                    r, c = np.nonzero(np.abs(B) > 0)
                    rows.append(F * p ** 3 + r)
                    cols.append(C * p ** 3 + c)
                    vals.append(B[r, c])
    return sp.csr_matrix((np.concatenate(vals),
                          (np.concatenate(rows), np.concatenate(cols))),
                         shape=(fine.n_dofs, coarse.n_dofs))


# --------------------------------------------------------------------------
# Eigenvalue estimate (Sec. 4.1: 15 CG iterations)
# --------------------------------------------------------------------------
def start_vector(prob):
    s = 1.0 + 0.1 * np.sin(np.arange(prob.n_dofs, dtype=float))
    s[prob.constrained()] = 0.0
    return s


def lanczos_from_cg(A, dinv, s, iters):
    """Run `iters` Jacobi-PCG steps on A x = s from x = 0 and return the
    Lanczos tridiagonal (diag, offdiag) built from the CG coefficients."""
    r = s.copy()
    z = dinv * r
    p = z.copy()
    rz = r @ z
    rz0 = rz
    alphas, betas = [], []
    for _ in range(iters):
        Ap = A @ p
        alpha = rz / (p @ Ap)
        r = r - alpha * Ap
        z = dinv * r
        rz_new = r @ z
        beta = rz_new / rz
        alphas.append(alpha)
        betas.append(beta)
        rz = rz_new
        if rz <= 1e-30 * rz0:
            break
        p = z + beta * p
    m = len(alphas)
    diag = np.empty(m)
    off = np.empty(max(m - 1, 0))
    for j in range(m):
        diag[j] = 1.0 / alphas[j] + (betas[j - 1] / alphas[j - 1] if j else 0.0)
        if j < m - 1:
            off[j] = np.sqrt(betas[j]) / alphas[j]
    return diag, off


def sturm_count(diag, off, x):
    """Number of eigenvalues of the symmetric tridiagonal below x."""
    cnt = 0
    q = 1.0
    for j in range(len(diag)):
        q = diag[j] - x - (off[j - 1] ** 2 / q if j else 0.0)
        if q == 0.0:
            q = -1e-300
        if q < 0:
            cnt += 1
    return cnt


def tridiag_extreme(diag, off, which, rtol=1e-12):
    """Largest ('max') or smallest ('min') eigenvalue by bisection."""
    r = np.zeros(len(diag))
    r[:-1] += np.abs(off)
    r[1:] += np.abs(off)
    lo, hi = np.min(diag - r), np.max(diag + r)
    target = len(diag) - 1 if which == "max" else 0
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if sturm_count(diag, off, mid) > target:
            hi = mid
        else:
            lo = mid
        if hi - lo <= rtol * max(abs(hi), abs(lo)):
            break
    return 0.5 * (lo + hi)


# --------------------------------------------------------------------------
# Chebyshev iteration (Sec. 4.1)
# --------------------------------------------------------------------------
def chebyshev(A, dinv, b, x0, lo, hi, degree):
    """`degree` Chebyshev updates of x for D^{-1} A on [lo, hi]; x0 = None
    means a zero start (first residual is b, no operator application).
    Returns (x, number of applications of A)."""
    theta = 0.5 * (hi + lo)
    delta = 0.5 * (hi - lo)
    sigma = theta / delta
    rho = 1.0 / sigma
    napp = 0
    if x0 is None:
        x = np.zeros_like(b)
        r = b.copy()
    else:
        x = x0.copy()
        r = b - A @ x
        napp += 1
    d = dinv * r / theta
    x = x + d
    for _ in range(degree - 1):
        r = b - A @ x
        napp += 1
        rho_new = 1.0 / (2.0 * sigma - rho)
        d = rho_new * rho * d + 2.0 * rho_new / delta * (dinv * r)
        x = x + d
        rho = rho_new
    return x, napp


def coarse_degree(lmin, lmax, tol=1e-3):
    c = lmax / lmin
    rho = (np.sqrt(c) - 1.0) / (np.sqrt(c) + 1.0)
    m = 1
    while 2.0 * rho ** m / (1.0 + rho ** (2 * m)) >= tol:
        m += 1
    return m


class Level:
    def __init__(self, prob, cheb_degree=5, eig_iters=15, coarse=False):
        self.prob = prob
        self.A = fem.assemble(prob)
        d = self.A.diagonal()
        self.dinv = 1.0 / d
        diag, off = lanczos_from_cg(self.A, self.dinv, start_vector(prob),
                                    eig_iters)
        self.lam_max = tridiag_extreme(diag, off, "max")
        self.lam_min = tridiag_extreme(diag, off, "min")
        self.cheb_degree = cheb_degree
        if coarse:
            self.lo, self.hi = 0.9 * self.lam_min, 1.2 * self.lam_max
            self.degree = coarse_degree(self.lo, self.hi)
        else:
            self.hi = 1.2 * self.lam_max
            self.lo = 0.06 * self.lam_max
            self.degree = cheb_degree


class VCycle:
    """Multigrid V-cycle preconditioner on the rediscretised hierarchy."""

    def __init__(self, prob, n_levels=0, cheb_degree=5, eig_iters=15):
        probs = hierarchy(prob, n_levels)
        self.levels = [Level(q, cheb_degree, eig_iters, coarse=(i == 0))
                       for i, q in enumerate(probs)]
        self.P = [None] + [prolongation(probs[i], probs[i - 1])
                           for i in range(1, len(probs))]
        self.applies = np.zeros(len(probs), int)

    def apply(self, b, level=None):
        if level is None:
            level = len(self.levels) - 1
        L = self.levels[level]
        if level == 0:
            x, n = chebyshev(L.A, L.dinv, b, None, L.lo, L.hi, L.degree)
            self.applies[0] += n
            return x
        x, n1 = chebyshev(L.A, L.dinv, b, None, L.lo, L.hi, L.degree)
        r = b - L.A @ x
        rc = self.P[level].T @ r
        ec = self.apply(rc, level - 1)
        x = x + self.P[level] @ ec
        x, n2 = chebyshev(L.A, L.dinv, b, x, L.lo, L.hi, L.degree)
        self.applies[level] += n1 + 1 + n2
        return x


def pcg(A, b, precond, rtol=1e-10, max_it=1000):
    """CG preconditioned by `precond` from x = 0, stopped when
    ||b - A x||_2 <= rtol ||b||_2 on the recursively updated residual
    (Sec. 4.1).  Returns (x, iterations, relative residual)."""
    x = np.zeros_like(b)
    r = b.copy()
    bn = np.linalg.norm(b)
    if bn == 0.0:
        return x, 0, 0.0
    z = precond(r)
    p = z.copy()
    rz = r @ z
    for it in range(1, max_it + 1):
        Ap = A @ p
        alpha = rz / (p @ Ap)
        x = x + alpha * p
        r = r - alpha * Ap
        rn = np.linalg.norm(r)
        if rn <= rtol * bn:
            return x, it, rn / bn
        z = precond(r)
        rz_new = r @ z
        p = z + (rz_new / rz) * p
        rz = rz_new
    return x, max_it, np.linalg.norm(r) / bn


def cg(A, b, rtol=1e-10, max_it=100000):
    """Unpreconditioned textbook CG."""
    return pcg(A, b, lambda r: r, rtol, max_it)
