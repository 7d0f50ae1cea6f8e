"""Deterministic mode: element colouring and bit-reproducible cell solves.

The colouring must be proper (no two elements of one colour share a DOF of the
current map, checked here against the DOF map itself), and with
deterministic=1 two independent contexts that make the same calls return
bitwise-identical tensors.  The coloured solve is the same discrete problem, so
it agrees with the one-launch (atomic) solve and with the oracle to the solver
tolerance.
"""
import numpy as np
import pytest

import rve_inputs as ri
from oracle import fem
from oracle import materials as mt

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rve():
    import paper_1610_03484_gb300 as pkg
    from paper_1610_03484_gb300 import _build
    _build.build()
    pkg.load_library()
    return pkg


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(b))


@pytest.mark.parametrize("p,bc", [(1, 0), (2, 1), (3, 1), (2, 2)])
def test_colouring_is_proper(rve, p, bc):
    xyz, tets, phase, tangent = ri.weave_rve(6, 6, 4)
    with rve.Context() as ctx:
        m = ctx.mesh_load(xyz, tets, p, phase, tangent)
        m.set_bc(bc)
        ed, _ = m.dofmap()
        col, n = m.colouring()
        assert n >= 1 and col.min() == 0 and col.max() == n - 1
        # every colour class touches each DOF at most once
        for k in range(n):
            d = ed[col == k].ravel()
            assert len(np.unique(d)) == len(d), k
        # greedy: each element's colour is the smallest one free at its turn, so a
        # colour c > 0 element meets every lower colour among its DOF neighbours
        # (checked on a sample)
        owner = {}
        for e in range(len(ed)):
            for d in ed[e]:
                owner.setdefault(int(d), []).append(e)
        for e in range(0, len(ed), 37):
            nb = {int(col[f]) for d in ed[e] for f in owner[int(d)] if f < e}
            assert all(c in nb for c in range(col[e])), e
        m.free()


def _solve(rve, det, prec, grid, p, bc, states, rtol):
    xyz, tets, phase, tangent = ri.weave_rve(*grid)
    with rve.Context(precision=prec, rtol=rtol, inner_rtol=1e-6,
                     deterministic=det) as ctx:
        m = ctx.mesh_load(xyz, tets, p, phase, tangent)
        m.set_materials(ri.NOMINAL_MATRIX, ri.NOMINAL_YARN)
        m.set_bc(bc)
        T, c, t = states
        Cc, Kk, Dd, st, _, _ = ctx.macro_update([m], T, c, t, np.zeros(len(T), np.int32))
        assert (st == 0).all()
        m.free()
        return Cc, Kk, Dd


@pytest.mark.parametrize("prec", [0, 1])
def test_deterministic_solves_are_bitwise_reproducible(rve, prec):
    """Two contexts, same calls, deterministic=1: identical bits.  Against the
    one-launch solve: equal to the solver tolerance."""
    T, c, t, _, _ = ri.gauss_point_states(12, seed=11)
    states = (T, c, t)
    rtol = 1e-10 if prec == 0 else 1e-7
    a = _solve(rve, True, prec, (8, 8, 4), 2, 1, states, rtol)
    b = _solve(rve, True, prec, (8, 8, 4), 2, 1, states, rtol)
    for x, y in zip(a, b):
        assert np.array_equal(x, y)
    atomic = _solve(rve, False, prec, (8, 8, 4), 2, 1, states, rtol)
    tol = 1e-8 if prec == 0 else 1e-6
    for x, y in zip(a, atomic):
        for g in range(len(T)):
            assert rel(x[g], y[g]) < tol


def test_deterministic_matches_oracle(rve):
    grid, p, bc = (6, 6, 4), 2, 1
    xyz, tets, phase, tangent = ri.weave_rve(*grid)
    T, c, t = np.array([60.0, 80.0]), np.array([0.5, 1.2]), np.array([100.0, 1500.0])
    Cg, Kg, Dg = _solve(rve, True, 0, grid, p, bc, (T, c, t), 1e-11)
    for g in range(2):
        w = mt.one_minus_omega(T[g], c[g], t[g])
        m = ri.MatrixProps(E=ri.NOMINAL_MATRIX.E * w, nu=ri.NOMINAL_MATRIX.nu, k=ri.NOMINAL_MATRIX.k,
                           d=ri.NOMINAL_MATRIX.d)
        D, K, Dd = mt.element_tensors(phase, tangent, m, ri.NOMINAL_YARN)
        Co, Ko, Do = fem.homogenise(xyz, tets, grid, p, bc, D, K, Dd)
        assert rel(Cg[g], Co) < 1e-9
        assert rel(Kg[g], Ko) < 1e-9
        assert rel(Dg[g], Do) < 1e-9


def test_deterministic_operator_is_reproducible(rve):
    """FP64 operator, p = 3, periodic: coloured launches twice (identical bits)
    and the one-launch operator (equal to rounding)."""
    xyz, tets, phase, tangent = ri.weave_rve(8, 8, 4)
    out = []
    for det in (True, True, False):
        with rve.Context(deterministic=det) as ctx:
            m = ctx.mesh_load(xyz, tets, 3, phase, tangent)
            m.set_materials(ri.NOMINAL_MATRIX, ri.NOMINAL_YARN)
            m.set_bc(1)
            n = m.info()["n_scalar_dofs"]
            x = np.random.default_rng(5).normal(size=(3 * n, 12))
            out.append(m.apply_operator(0, x))
            m.free()
    assert np.array_equal(out[0], out[1])
    assert rel(out[0], out[2]) < 1e-13
