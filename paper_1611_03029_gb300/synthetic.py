"""Seeded synthetic inputs shared by the tests, bench.py and the oracle
legs.  Holds none of the method's arithmetic: random vectors, the
Gaussian-sum forcing parameters, the log-coefficient Fourier field and the
strongly varying coefficient sampled at the physical positions of the Gauss
points of a Cartesian mesh.
"""
import numpy as np


def random_vector(n, seed, ncols=1):
    """Standard normal float64 values, shape [n] or [n, ncols]."""
    rng = np.random.default_rng(seed)
    v = rng.standard_normal((n, ncols) if ncols > 1 else n)
    return v


def gaussian_terms(seed, n_terms=8):
    """Forcing f(x) = sum_j A_j exp(-|x - c_j|^2 / w_j^2): rows (c_x, c_y,
    c_z, w, A); centres uniform in the unit cube, widths uniform in
    [0.05, 0.2], amplitudes standard normal, drawn in that order."""
    rng = np.random.default_rng(seed)
    c = rng.uniform(0.0, 1.0, (n_terms, 3))
    w = rng.uniform(0.05, 0.2, n_terms)
    a = rng.standard_normal(n_terms)
    return np.column_stack([c, w, a])


def gaussian_forcing(params):
    """The forcing of `gaussian_terms` as a function of points [..., 3]."""
    params = np.asarray(params)

    def f(x):
        out = np.zeros(x.shape[:-1])
        for cx, cy, cz, w, a in params:
            d2 = ((x[..., 0] - cx) ** 2 + (x[..., 1] - cy) ** 2
                  + (x[..., 2] - cz) ** 2)
            out += a * np.exp(-d2 / w ** 2)
        return out
    return f


def fourier_modes(seed, n_modes=32, kmax=4, amplitude=0.5):
    """g(x) = sum_m c cos(pi k_m . x + phi_m): k_m uniform in {0..kmax}^3
    without 0, phi_m uniform in [0, 2 pi), c = amplitude sqrt(2 / n_modes)
    so that the RMS of g is about `amplitude`."""
    rng = np.random.default_rng(seed)
    ks = []
    while len(ks) < n_modes:
        k = rng.integers(0, kmax + 1, 3)
        if k.any():
            ks.append(k)
    phi = rng.uniform(0.0, 2 * np.pi, n_modes)
    c = amplitude * np.sqrt(2.0 / n_modes)
    return np.array(ks, float), phi, c


def fourier_field(modes, x):
    ks, phi, c = modes
    arg = np.pi * np.tensordot(x, ks.T, axes=([-1], [0])) + phi
    return c * np.cos(arg).sum(-1)


def _gauss01(p):
    g, _ = np.polynomial.legendre.leggauss(p)
    return 0.5 * (g + 1.0)


def cell_points(n, p):
    """Physical Gauss points of every cell of the Cartesian n[0] x n[1] x
    n[2] mesh of the unit cube: [ncells, p^3, 3], local order x fastest."""
    g = _gauss01(p)
    h = [1.0 / m for m in n]
    cz, cy, cx = np.meshgrid(np.arange(n[2]), np.arange(n[1]),
                             np.arange(n[0]), indexing="ij")
    qz, qy, qx = np.meshgrid(g, g, g, indexing="ij")
    X = (cx.reshape(-1, 1) + qx.reshape(1, -1)) * h[0]
    Y = (cy.reshape(-1, 1) + qy.reshape(1, -1)) * h[1]
    Z = (cz.reshape(-1, 1) + qz.reshape(1, -1)) * h[2]
    return np.stack([X, Y, Z], -1)


def face_points(n, p):
    """Physical Gauss points of every face (x-normal, then y-, then z-normal
    faces; each direction lexicographic, x fastest; point qa + p qb over the
    tangential axes a < b): [nfaces, p^2, 3]."""
    g = _gauss01(p)
    h = [1.0 / m for m in n]
    out = []
    for d in range(3):
        m = list(n)
        m[d] += 1
        t = [e for e in range(3) if e != d]
        fz, fy, fx = np.meshgrid(np.arange(m[2]), np.arange(m[1]),
                                 np.arange(m[0]), indexing="ij")
        fc = [fx.reshape(-1), fy.reshape(-1), fz.reshape(-1)]
        qb, qa = np.meshgrid(g, g, indexing="ij")
        q = {t[0]: qa.reshape(-1), t[1]: qb.reshape(-1)}
        pts = np.empty((fc[0].size, p * p, 3))
        for e in range(3):
            if e == d:
                pts[..., e] = (fc[e] * h[e])[:, None]
            else:
                pts[..., e] = (fc[e][:, None] + q[e][None, :]) * h[e]
        out.append(pts)
    return np.concatenate(out, 0)


def log_coefficient(n, p, seed):
    """a = exp(g) at all cell and face Gauss points of the Cartesian mesh,
    g the Fourier field of `fourier_modes(seed)`."""
    modes = fourier_modes(seed)
    a_cell = np.exp(fourier_field(modes, cell_points(n, p)))
    a_face = np.exp(fourier_field(modes, face_points(n, p)))
    return a_cell, a_face


def strong_coefficient_field(x):
    """The strongly varying diffusivity of the paper's shell example (Sec. 4.3),
    1 + 10^6 prod_e cos(2 pi x_e + 0.1 e) for e = 1, 2, 3, read with the
    product in absolute value: as printed it is negative on about half of any
    domain, which no SPD solver accepts; the absolute value keeps its
    contrast (10^6) and its pattern."""
    e = np.arange(1, 4)
    return 1.0 + 1e6 * np.abs(np.prod(np.cos(2.0 * np.pi * x + 0.1 * e), -1))


def strong_coefficient(n, p, box=(-1.0, 1.0)):
    """strong_coefficient_field at all cell and face Gauss points of the
    Cartesian mesh of [box_lo, box_hi]^3."""
    lo, hi = box
    a_cell = strong_coefficient_field(lo + (hi - lo) * cell_points(n, p))
    a_face = strong_coefficient_field(lo + (hi - lo) * face_points(n, p))
    return a_cell, a_face



def perturbed_lattice_nodes(n, k, seed, amp=0.05):
    """Support points [ncells, (k+1)^3, 3] of a conforming mesh of the unit
    cube: the equispaced lattice of (n_e k + 1) points per axis, every
    interior lattice point moved by amp / (n_e k) times a uniform draw in
    [-1, 1]^3 (boundary points stay, so the domain is still the unit cube),
    then handed to each cell as its local nodes a = ax + p ay + p^2 az
    (neighbours share the points of their common face)."""
    rng = np.random.default_rng(seed)
    p = k + 1
    g = [m * k + 1 for m in n]
    iz, iy, ix = np.meshgrid(np.arange(g[2]), np.arange(g[1]),
                             np.arange(g[0]), indexing="ij")
    idx = [ix.reshape(-1), iy.reshape(-1), iz.reshape(-1)]
    pts = np.stack([idx[e] / (g[e] - 1.0) for e in range(3)], -1)
    noise = rng.uniform(-1.0, 1.0, pts.shape)
    interior = np.ones(pts.shape[0], bool)
    for e in range(3):
        interior &= (idx[e] > 0) & (idx[e] < g[e] - 1)
    for e in range(3):
        pts[:, e] += np.where(interior, amp / (g[e] - 1.0) * noise[:, e], 0)
    nc = n[0] * n[1] * n[2]
    c = np.arange(nc)
    cx, cy, cz = c % n[0], (c // n[0]) % n[1], c // (n[0] * n[1])
    a = np.arange(p ** 3)
    ax, ay, az = a % p, (a // p) % p, a // (p * p)
    gi = ((cx[:, None] * k + ax) + g[0] * ((cy[:, None] * k + ay)
                                          + g[1] * (cz[:, None] * k + az)))
    return pts[gi]
