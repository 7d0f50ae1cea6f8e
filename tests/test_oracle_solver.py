"""Pins for oracle.fem.pcg_columns, the Jacobi-preconditioned CG that solves
every oracle cell problem above the direct-solve size (Sec. 2: the cell
problem's Galerkin solution, to a true relative residual of 1e-13).

* closed form: a laminate aligned with the grid planes, periodic BC, solved by
  CG alone (``direct_max=0``) above 4000 DOFs, gives the textbook laminate
  average;
* the sparse-LU route: a plain-weave RVE above 4000 DOFs, Dirichlet and
  periodic, CG against ``splu`` of the same system;
* exact arithmetic facts of CG: termination in k steps when the preconditioned
  matrix has k distinct eigenvalues, the first step's closed form, and the
  true-residual guarantee on an ill-conditioned system;
* planted mistakes (a wrong beta, a stop on the recursive residual alone) fail
  these pins.
"""
import numpy as np
import pytest
import scipy.sparse as sp

import rve_inputs as ri
from oracle import fem
from oracle import materials as mt

from test_oracle_homogenisation import laminate_average, rel, weave_tensors


def _jacobi_system(lams, seed):
    """A = S M S with M = H diag(lams) H^T, H an orthonormal Hadamard matrix,
    S a random positive diagonal.  Every diagonal entry of M is mean(lams), so
    diag(A)^-1 A is similar to M / mean(lams): Jacobi-preconditioned CG on A
    runs exactly as CG on a matrix with the spectrum lams / mean(lams)."""
    from scipy.linalg import hadamard
    n = len(lams)
    H = hadamard(n) / np.sqrt(n)
    M = (H * np.asarray(lams)) @ H.T
    s = np.exp(np.random.default_rng(seed).uniform(-2.0, 2.0, n))
    return sp.csr_matrix(s[:, None] * M * s[None, :])


def test_laminate_closed_form_by_cg_alone():
    grid = (2, 2, 16)
    xyz, tets = ri.kuhn_grid(*grid)
    phase = ri.layered(xyz, tets, [0, 0, 0, 0, 1, 1, 1, 1], nz=16)
    D0 = mt.iso_stiffness(3.5, 0.35)
    D1 = mt.ti_stiffness(45, 12, 5, 0.28, 0.4, [1.0, 0.4, 0.0])
    Dm = np.where(phase[:, None, None] == 0, D0, D1)
    k0 = 0.2 * np.eye(3)
    k1 = mt.transport_tensor(0.6, 0.35, [1.0, 0.4, 0.0])
    km = np.where(phase[:, None, None] == 0, k0, k1)
    p = 3
    m = fem.build_nodal_mesh(xyz, tets, grid, p, periodic=True)
    assert fem.n_nodes(m) * 3 > 4000          # above the direct-solve size
    sm = fem.homogenise_field(xyz, tets, grid, p, fem.BC_PERIODIC, Dm, 3, direct_max=0)
    ss = fem.homogenise_field(xyz, tets, grid, p, fem.BC_PERIODIC, km, 1, direct_max=0)
    C_lam = laminate_average([D0, D1], [0.5, 0.5], [2, 4, 5], [0, 1, 3])
    K_lam = laminate_average([k0, k1], [0.5, 0.5], [2], [0, 1])
    assert rel(sm.tensor, C_lam) < 1e-11
    assert rel(ss.tensor, K_lam) < 1e-11


@pytest.mark.parametrize("bc", [fem.BC_DIRICHLET, fem.BC_PERIODIC])
def test_weave_cg_matches_sparse_lu(bc):
    grid = (8, 8, 4)
    xyz, tets, D, K, _ = weave_tensors(grid)
    m = fem.build_nodal_mesh(xyz, tets, grid, 2, periodic=(bc == fem.BC_PERIODIC))
    assert fem.n_nodes(m) * 3 > 4000
    cg = fem.homogenise_field(xyz, tets, grid, 2, bc, D, 3, direct_max=0)
    lu = fem.homogenise_field(xyz, tets, grid, 2, bc, D, 3, direct_max=10 ** 9)
    assert rel(cg.tensor, lu.tensor) < 1e-11
    assert np.abs(cg.u_tilde - lu.u_tilde).max() <= 1e-9 * np.abs(lu.u_tilde).max()


@pytest.mark.parametrize("k", [1, 2, 4, 8])
def test_terminates_in_k_steps_for_k_distinct_eigenvalues(k):
    # CG's error after j steps is minimal over degree-j polynomials that are 1 at
    # 0; with k distinct eigenvalues the product of (1 - t / lam_i) vanishes on
    # the spectrum, so step k gives the exact solution.
    n = 64
    A = _jacobi_system(np.repeat(np.linspace(0.2, 1.8, k), n // k), 3)
    b = np.random.default_rng(5).normal(size=(n, 3))
    info = {}
    X = fem.pcg_columns(A, b, rtol=1e-12, info=info)
    assert info["iterations"] == k
    np.testing.assert_allclose(X, np.linalg.solve(A.toarray(), b), rtol=0, atol=1e-10 * np.abs(X).max())


def _ill_conditioned():
    n = 64
    A = _jacobi_system(np.logspace(-7, 0, n), 3)
    b = np.random.default_rng(5).normal(size=(n, 2))
    return A, b


def test_returns_only_on_the_true_residual():
    # kappa ~ 1e7 before the diagonal scaling: the recursive residual runs ahead
    # of the true one by about eps * kappa.
    A, b = _ill_conditioned()
    info = {}
    X = fem.pcg_columns(A, b, rtol=1e-9, maxiter=3000, info=info)
    tr = np.linalg.norm(b - A @ X, axis=0) / np.linalg.norm(b, axis=0)
    assert (tr <= 1e-9).all()
    assert info["restarts"] >= 1           # the drift did occur


def test_planted_solver_mistakes_are_caught(monkeypatch):
    # 1. a wrong beta: no finite termination on a 2-point spectrum
    monkeypatch.setattr(fem, "_cg_beta", lambda rz_new, rz: 0.5 * rz_new / rz)
    n = 64
    A = _jacobi_system(np.repeat([0.2, 1.8], n // 2), 3)
    b = np.random.default_rng(5).normal(size=(n, 1))
    info = {}
    fem.pcg_columns(A, b, rtol=1e-12, info=info)
    assert info["iterations"] > 2
    monkeypatch.undo()
    # 2. stopping on the recursive residual alone returns a solution whose true
    #    residual misses the tolerance
    monkeypatch.setattr(fem, "_true_residual_met", lambda A, B, X, rtol, bn: np.ones(B.shape[1], bool))
    A, b = _ill_conditioned()
    X = fem.pcg_columns(A, b, rtol=1e-9, maxiter=3000)
    tr = np.linalg.norm(b - A @ X, axis=0) / np.linalg.norm(b, axis=0)
    assert (tr > 2e-9).any()
