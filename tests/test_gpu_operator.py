"""The matrix-free operator itself against the oracle's element matrices, entry
by entry (operator apply vs assembled matvec).

The GPU works in the hierarchic basis (vertex functions lam_a; edge functions
lam_a lam_b for p >= 2; lam_a lam_b (lam_b - lam_a) and face functions
lam_a lam_b lam_c for p = 3, local vertices ordered as rve_mesh_get_dofmap
reports), the oracle in the Lagrange basis of the same P_p space.  Every
hierarchic function is a polynomial of degree <= p, so its Lagrange
interpolant is itself: T_e[l, j] = phi_j(node l).  Then the hierarchic element
matrix is T_e^T K_e T_e, and y = sum_e A_e^T T_e^T K_e T_e A_e x must equal the
GPU's y = K x for any x, on the GPU's own DOF numbering (periodic fold
included)."""
import numpy as np
import pytest

import rve_inputs as ri
from oracle import fem
from oracle import lagrange
from oracle import materials as mt

pytestmark = pytest.mark.gpu

EDGES = ((0, 1), (0, 2), (0, 3), (1, 2), (1, 3), (2, 3))
FACES = ((0, 1, 2), (0, 1, 3), (0, 2, 3), (1, 2, 3))


@pytest.fixture(scope="module")
def rve():
    import paper_1610_03484_gb300 as pkg
    from paper_1610_03484_gb300 import _build
    _build.build()
    pkg.load_library()
    return pkg


def hierarchic_values(p, lam):
    """The hierarchic local functions at barycentric points lam [n, 4] -> [n, ne]."""
    cols = [lam[:, a] for a in range(4)]
    if p >= 2:
        cols += [lam[:, a] * lam[:, b] for a, b in EDGES]
    if p >= 3:
        cols += [lam[:, a] * lam[:, b] * (lam[:, b] - lam[:, a]) for a, b in EDGES]
        cols += [lam[:, a] * lam[:, b] * lam[:, c] for a, b, c in FACES]
    return np.stack(cols, axis=1)


def oracle_apply(xyz, tets, grid, p, Ke_lagr, nc, edofs, lverts, x):
    """y = sum_e A_e^T T_e^T K_e T_e A_e x with the GPU's element DOF map."""
    ms = np.asarray(lagrange.node_multi_indices(p), float) / p       # Lagrange nodes, oracle vertex order
    nt, ne = edofs.shape
    nl = ms.shape[0]
    ncols = x.shape[-1]
    X = x.reshape(-1, nc, ncols)
    Y = np.zeros_like(X)
    for e in range(nt):
        pos = [int(np.nonzero(tets[e] == v)[0][0]) for v in lverts[e]]   # GPU local vertex -> oracle slot
        T = hierarchic_values(p, ms[:, pos])                              # [nl, ne]
        K = Ke_lagr[e].reshape(nl * nc, nl * nc)
        Th = np.kron(T, np.eye(nc))                                       # [nl*nc, ne*nc]
        Kh = Th.T @ K @ Th
        xe = X[edofs[e]].reshape(ne * nc, ncols)
        np.add.at(Y, edofs[e], (Kh @ xe).reshape(ne, nc, ncols))
    return Y.reshape(x.shape)


@pytest.mark.parametrize("p", [1, 2, 3])
@pytest.mark.parametrize("bc", [1, 2])      # periodic (folded DOFs), Neumann (no fold)
def test_operator_matches_oracle_element_matrices(rve, p, bc):
    grid = (3, 3, 2)
    xyz, tets, phase, tangent = ri.weave_rve(*grid)
    # nominal (undegraded) constituents: the batched path applies the degradation
    # as a per-column factor on top of this operator
    D, Kt, Dd = mt.element_tensors(phase, tangent, ri.NOMINAL_MATRIX, ri.NOMINAL_YARN)
    nm = fem.build_nodal_mesh(xyz, tets, grid, p, periodic=False)    # element geometry only
    KeM = fem.element_stiffness_mech(nm, D)
    KeT = fem.element_stiffness_scalar(nm, Kt)
    KeD = fem.element_stiffness_scalar(nm, Dd)
    rng = np.random.default_rng(100 * p + bc)
    with rve.Context(precision=rve.PREC_FP64) as ctx:
        mesh = ctx.mesh_load(xyz, tets, p, phase, tangent)
        mesh.set_materials(ri.NOMINAL_MATRIX, ri.NOMINAL_YARN)
        mesh.set_bc(bc)
        edofs, lverts = mesh.dofmap()
        N = mesh.info()["n_scalar_dofs"]
        assert edofs.min() >= 0 and edofs.max() < N
        for a in range(len(tets)):
            assert sorted(lverts[a]) == sorted(tets[a])
        for field, Ke, nc in ((0, KeM, 3), (1, KeT, 1), (2, KeD, 1)):
            x = rng.standard_normal((N * nc, 6))
            got = mesh.apply_operator(field, x)
            want = oracle_apply(xyz, tets, grid, p, Ke, nc, edofs.astype(np.int64), lverts.astype(np.int64), x)
            assert np.abs(got - want).max() <= 1e-11 * np.abs(want).max(), (field, p, bc)
            # and it is symmetric: x2 . K x1 = x1 . K x2
            x2 = rng.standard_normal((N * nc, 6))
            got2 = mesh.apply_operator(field, x2)
            lhs = np.einsum("rc,rc->c", x2, got)
            rhs = np.einsum("rc,rc->c", x, got2)
            assert np.allclose(lhs, rhs, rtol=1e-11, atol=1e-11 * np.abs(lhs).max())
        mesh.free()
