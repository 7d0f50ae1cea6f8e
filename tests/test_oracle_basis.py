"""Pins for oracle.lagrange and the DOF counts printed in Sec. 7."""
import json
import os

import numpy as np
import pytest

import rve_inputs as ri
from oracle import fem, lagrange


@pytest.mark.parametrize("p", [1, 2, 3])
def test_partition_of_unity_and_kronecker(p):
    ms = np.asarray(lagrange.node_multi_indices(p), float)
    vals = lagrange.evaluate(p, ms / p)
    np.testing.assert_allclose(vals, np.eye(len(ms)), atol=1e-13)
    lam = np.random.default_rng(p).dirichlet(np.ones(4), size=50)
    np.testing.assert_allclose(lagrange.evaluate(p, lam).sum(-1), 1.0, atol=1e-13)


@pytest.mark.parametrize("p", [1, 2, 3])
def test_reference_integrals(p):
    S, G, M0, Fc = lagrange.reference_tables(p)
    # mean of the basis sums to 1 (partition of unity), on faces too
    assert M0.sum() == pytest.approx(1.0)
    np.testing.assert_allclose(Fc.sum(axis=1), 1.0)
    # the basis sums to a polynomial that is symmetric in the barycentric
    # variables, so its derivative is the same along every lam_a: the physical
    # gradient sum_a (d/dlam_a) grad(lam_a) of the partition of unity vanishes
    gs = G.sum(axis=1)
    np.testing.assert_allclose(gs, gs[0], atol=1e-13)
    ss = S.sum(axis=(2, 3))
    np.testing.assert_allclose(ss, ss[0, 0], atol=1e-12)
    # S is symmetric under (a,i) <-> (b,j)
    np.testing.assert_allclose(S, S.transpose(1, 0, 3, 2), atol=1e-15)
    # Monte-Carlo-free check of exactness: P1 gradient mass matrix by hand
    if p == 1:
        np.testing.assert_allclose(S[0, 0], np.diag([1, 0, 0, 0]))


def test_p1_stiffness_textbook():
    # P1 Laplacian on the reference tet: K = |T| G G^T with G the gradient matrix
    xyz = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1.0]])
    tets = np.array([[0, 1, 2, 3]])
    m = fem.build_nodal_mesh(xyz, tets, (1, 1, 1), 1)
    K = fem.element_stiffness_scalar(m, np.eye(3)[None])[0]
    order = m.elem_nodes[0]
    Gm = np.array([[-1, -1, -1], [1, 0, 0], [0, 1, 0], [0, 0, 1.0]])
    np.testing.assert_allclose(K, Gm @ Gm.T / 6.0, atol=1e-15)
    assert sorted(order) == [0, 1, 2, 3]


@pytest.mark.parametrize("grid", [(2, 3, 2), (4, 4, 2), (12, 12, 6)])
@pytest.mark.parametrize("p", [1, 2, 3])
def test_node_count_formula(grid, p):
    xyz, tets = ri.kuhn_grid(*grid)
    m = fem.build_nodal_mesh(xyz, tets, grid, p)
    V, E, F, T = ri.mesh_counts(*grid)
    expect = V + (p - 1) * E + (p - 1) * (p - 2) // 2 * F
    assert fem.n_nodes(m) == expect
    # periodic fold: every image node collapses onto its master
    mp = fem.build_nodal_mesh(xyz, tets, grid, p, periodic=True)
    nx, ny, nz = grid
    Vp = nx * ny * nz
    Ep = 7 * Vp              # 3 axis + 3 face-diagonal + 1 body-diagonal edge per cell
    Fp = 12 * Vp             # torus: V - E + F - T = 0
    assert fem.n_nodes(mp) == Vp + (p - 1) * Ep + (p - 1) * (p - 2) // 2 * Fp


def test_paper_dof_counts_consistent(golden_dir):
    # The printed DOF counts fit V + (p-1)E + (p-1)(p-2)/2 F with the printed
    # number of tetrahedra and the Euler characteristic of a ball.
    with open(os.path.join(golden_dir, "dof_counts.json")) as f:
        g = json.load(f)
    s = {int(k): v for k, v in g["scalar_dofs"].items()}
    V = s[1]
    E = s[2] - V
    F = s[3] - V - 2 * E
    assert V - E + F - g["tets"] == 1
    for p in (1, 2, 3):
        assert g["mechanical_dofs"][str(p)] == 3 * s[p]
