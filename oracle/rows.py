"""Selected entries of y = A u without assembling the global matrix
(Eq. 12: the product is a sum of element contributions), for checking
large meshes at sampled outputs.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).
"""
import numpy as np

from . import fem


def _cells_of_cg_node(prob, node):
    g = prob.grid
    idx = [node % g[0], (node // g[0]) % g[1], node // (g[0] * g[1])]
    cand = []
    for d in range(3):
        i = idx[d]
        c = {min(i // prob.k, prob.n[d] - 1)}
        if i % prob.k == 0 and i > 0:
            c.add(i // prob.k - 1)
        cand.append(sorted(c))
    return [prob.cell_index(a, b, c) for c in cand[2] for b in cand[1]
            for a in cand[0]]


def _faces_of_cell(prob, c):
    cx, cy, cz = (int(v) for v in prob.cell_coords(c))
    n = prob.n
    out = []
    off = 0
    for d in range(3):
        m = list(n)
        m[d] += 1
        cc = [cx, cy, cz]
        for s in (0, 1):
            fc = list(cc)
            fc[d] += s
            out.append(off + fc[0] + m[0] * (fc[1] + m[1] * fc[2]))
        off += m[0] * m[1] * m[2]
    return out


def apply_rows(prob, u, rows):
    """(A u)[rows] with the same Dirichlet treatment as fem.assemble."""
    rows = np.asarray(rows)
    cmask = prob.constrained()
    um = np.array(u, float)
    um[cmask] = 0.0
    out = np.zeros(len(rows))
    if prob.disc == "cg":
        need = sorted({c for r in rows for c in _cells_of_cg_node(prob, r)})
    else:
        need = sorted({int(r) // prob.p ** 3 for r in rows})
    need = np.array(need, int)
    K = fem.cell_matrices(prob, need)
    dm = prob.dof_map(need)
    contrib = {}
    for t, c in enumerate(need):
        ye = K[t] @ um[dm[t]]
        for a, gidx in enumerate(dm[t]):
            contrib[gidx] = contrib.get(gidx, 0.0) + ye[a]
    if prob.disc == "dg":
        faces = sorted({f for c in need for f in _faces_of_cell(prob, c)})
        for d in range(3):
            for _, cells, A in fem.face_terms(prob, d, faces):
                dmf = prob.dof_map(np.array(cells)).ravel()
                ye = A @ um[dmf]
                for a, gidx in enumerate(dmf):
                    contrib[gidx] = contrib.get(gidx, 0.0) + ye[a]
    for i, r in enumerate(rows):
        out[i] = u[r] if cmask[r] else contrib.get(int(r), 0.0)
    return out
