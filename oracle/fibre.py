"""FP64 oracle for the yarn directions from potential flow (Sec. 6).

Test infrastructure (see ``oracle/__init__``).

For every yarn, the Laplace problem grad^2 phi = 0 is solved on the yarn's own
tetrahedra (linear elements, nodes renumbered) with phi = 0 on the nodes at its
lower end along its axis, phi = 1 at its upper end and zero flux on its lateral
surface; the fibre direction of each yarn tetrahedron is grad phi / |grad phi|
(constant per linear element).  Sparse direct solve.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse.linalg as spla

from . import macro as mo


def yarn_potential(xyz, tets, axis):
    """phi at the nodes of one yarn submesh (xyz, tets local) and grad phi per tet."""
    K, _ = mo.assemble(xyz, tets, np.eye(3), 1.0)
    s = xyz[:, axis]
    lo, hi = s.min(), s.max()
    tol = 1e-9 * max(1.0, hi - lo)
    held = (s <= lo + tol) | (s >= hi - tol)
    phi = np.where(s >= hi - tol, 1.0, 0.0)
    free = np.nonzero(~held)[0]
    fixed = np.nonzero(held)[0]
    K = K.tocsr()
    rhs = -K[free][:, fixed] @ phi[fixed]
    phi[free] = spla.splu(K[free][:, free].tocsc()).solve(rhs)
    _, g = mo.p1_geometry(xyz, tets)
    grad = np.einsum("tai,ta->ti", g, phi[tets])
    return phi, grad


def yarn_directions(xyz, tets, yarn_of_tet, axes, dir_in):
    """Unit grad phi for every yarn tetrahedron; matrix tetrahedra keep dir_in."""
    out = np.array(dir_in, float, copy=True)
    for y, axis in enumerate(axes):
        sel = np.nonzero(yarn_of_tet == y)[0]
        if len(sel) == 0:
            continue
        nodes, loc = np.unique(tets[sel], return_inverse=True)
        _, grad = yarn_potential(xyz[nodes], loc.reshape(-1, 4).astype(np.int64), axis)
        n = np.linalg.norm(grad, axis=1)
        ok = n > 0
        out[sel[ok]] = grad[ok] / n[ok, None]
    return out
