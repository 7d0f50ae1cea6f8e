"""GPU path vs the FP64 CPU oracle, element by element, through the C ABI.

Tolerances (relative Frobenius per tensor): 1e-9 for the FP64 path, 1e-6 for
mixed precision; degradation factors and constituent tensors 1e-12.
"""
import numpy as np
import pytest

import rve_inputs as ri
from oracle import fem
from oracle import materials as mt

pytestmark = pytest.mark.gpu

TOL_FP64 = 1e-9
TOL_MIXED = 1e-6


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(b))


@pytest.fixture(scope="module")
def rve():
    import paper_1610_03484_gb300 as pkg
    from paper_1610_03484_gb300 import _build
    _build.build()
    pkg.load_library()
    return pkg


@pytest.fixture(scope="module")
def ctx64(rve):
    with rve.Context(precision=rve.PREC_FP64, rtol=1e-11) as c:
        yield c


def oracle_tensors(xyz, tets, grid, p, bc, phase, tangent, w=1.0, mat=ri.NOMINAL_MATRIX, yarn=ri.NOMINAL_YARN):
    m = ri.MatrixProps(E=mat.E * w, nu=mat.nu, k=mat.k, d=mat.d)
    D, K, Dd = mt.element_tensors(phase, tangent, m, yarn)
    return fem.homogenise(xyz, tets, grid, p, bc, D, K, Dd)


def test_degradation_factor(ctx64):
    T, c, t, _, _ = ri.gauss_point_states(1000, seed=7)
    got = ctx64.degradation_factor(T, c, t)
    want = mt.one_minus_omega(T, c, t)
    np.testing.assert_allclose(got, want, rtol=1e-13, atol=0)
    # edge cases: dry, zero time, saturated beyond c_sat
    got = ctx64.degradation_factor([60.0, 60.0, 80.0], [0.0, 1.5, 3.0], [1e4, 0.0, 2688.0])
    np.testing.assert_allclose(got, [1.0, 1.0, mt.one_minus_omega(80.0, 1.5, 2688.0)], rtol=1e-14)


def test_constituent_tensors(ctx64):
    xyz, tets, phase, tangent = ri.weave_rve(6, 6, 4)
    mesh = ctx64.mesh_load(xyz, tets, 1, phase, tangent)
    mesh.set_materials(ri.NOMINAL_MATRIX, ri.NOMINAL_YARN)
    D, K, Dd = mesh.tensors()
    Do, Ko, Ddo = mt.element_tensors(phase, tangent, ri.NOMINAL_MATRIX, ri.NOMINAL_YARN)
    assert np.abs(D - Do).max() / np.abs(Do).max() < 1e-12
    assert np.abs(K - Ko).max() / np.abs(Ko).max() < 1e-12
    assert np.abs(Dd - Ddo).max() / np.abs(Ddo).max() < 1e-12
    mesh.free()


def test_dof_counts(ctx64):
    for grid in ((12, 12, 6), (5, 3, 2)):
        xyz, tets = ri.kuhn_grid(*grid)
        V, E, F, T = ri.mesh_counts(*grid)
        for p in (1, 2, 3):
            mesh = ctx64.mesh_load(xyz, tets, p)
            info = mesh.info()
            assert (info["n_vertices"], info["n_edges"], info["n_faces"], info["n_tets"]) == (V, E, F, T)
            assert info["n_scalar_dofs"] == V + (p - 1) * E + (p - 1) * (p - 2) // 2 * F
            mesh.free()


@pytest.mark.parametrize("p", [1, 2, 3])
@pytest.mark.parametrize("bc", [0, 1, 2])
def test_tensors_fp64_vs_oracle(ctx64, p, bc):
    grid = (6, 6, 4) if p < 3 else (4, 4, 3)
    xyz, tets, phase, tangent = ri.weave_rve(*grid)
    mesh = ctx64.mesh_load(xyz, tets, p, phase, tangent)
    mesh.set_materials(ri.NOMINAL_MATRIX, ri.NOMINAL_YARN, T_C=50.0, c_wt=1.2, t_h=3000.0)
    mesh.set_bc(bc)
    res = mesh.homogenise()
    w = float(mt.one_minus_omega(50.0, 1.2, 3000.0))
    Co, Ko, Do = oracle_tensors(xyz, tets, grid, p, bc, phase, tangent, w)
    assert rel(res.C, Co) < TOL_FP64
    assert rel(res.K, Ko) < TOL_FP64
    assert rel(res.D, Do) < TOL_FP64
    assert res.stats["hill_mandel_mech"] < 1e-8
    mesh.free()


def test_config1_periodic_fp64(ctx64):
    # 12x12x6 plain weave, p = 2, periodic, PCG to 1e-10 (the config-1 case)
    grid, p = (12, 12, 6), 2
    xyz, tets, phase, tangent = ri.weave_rve(*grid)
    mesh = ctx64.mesh_load(xyz, tets, p, phase, tangent)
    mesh.set_materials(ri.NOMINAL_MATRIX, ri.NOMINAL_YARN)
    mesh.set_bc(1)
    res = mesh.homogenise()
    Co, Ko, Do = oracle_tensors(xyz, tets, grid, p, 1, phase, tangent)
    assert rel(res.C, Co) < TOL_FP64
    assert rel(res.K, Ko) < TOL_FP64
    assert rel(res.D, Do) < TOL_FP64
    mesh.free()


@pytest.mark.parametrize("bc", [0, 1, 2])
def test_tensors_mixed_vs_oracle(rve, bc):
    grid, p = (8, 8, 4), 2
    xyz, tets, phase, tangent = ri.weave_rve(*grid)
    with rve.Context(precision=rve.PREC_MIXED, rtol=1e-9, inner_rtol=1e-5) as ctx:
        mesh = ctx.mesh_load(xyz, tets, p, phase, tangent)
        mesh.set_materials(ri.NOMINAL_MATRIX, ri.NOMINAL_YARN)
        mesh.set_bc(bc)
        res = mesh.homogenise()
        mesh.free()
    Co, Ko, Do = oracle_tensors(xyz, tets, grid, p, bc, phase, tangent)
    assert rel(res.C, Co) < TOL_MIXED
    assert rel(res.K, Ko) < TOL_MIXED
    assert rel(res.D, Do) < TOL_MIXED


def test_batched_matches_single_and_oracle(rve):
    grid, p = (6, 6, 4), 2
    xyz, tets, phase, tangent = ri.weave_rve(*grid)
    T, c, t, _, _ = ri.gauss_point_states(10, seed=3)
    with rve.Context(precision=rve.PREC_FP64, rtol=1e-11, batch=4) as ctx:
        mesh = ctx.mesh_load(xyz, tets, p, phase, tangent)
        mesh.set_materials(ri.NOMINAL_MATRIX, ri.NOMINAL_YARN)
        mesh.set_bc(1)
        Cb, Kb, Db, st, stats, rc = ctx.macro_update([mesh], T, c, t, np.zeros(10, np.int32))
        assert (st == 0).all()
        for g in (0, 5, 9):
            w = float(mt.one_minus_omega(T[g], c[g], t[g]))
            Co, Ko, Do = oracle_tensors(xyz, tets, grid, p, 1, phase, tangent, w)
            assert rel(Cb[g], Co) < TOL_FP64
            assert rel(Kb[g], Ko) < TOL_FP64
            assert rel(Db[g], Do) < TOL_FP64
        mesh.free()


def test_homogeneous_and_voigt_edge_cases(ctx64):
    # single phase: C equals the material tensor for every BC
    xyz, tets = ri.kuhn_grid(3, 3, 2)
    nt = len(tets)
    mesh = ctx64.mesh_load(xyz, tets, 2, np.ones(nt, np.uint8), np.tile([0.3, 0.8, -0.2], (nt, 1)))
    mesh.set_materials(ri.NOMINAL_MATRIX, ri.NOMINAL_YARN)
    D0 = mt.ti_stiffness(45e9, 12e9, 5e9, 0.28, 0.4, [0.3, 0.8, -0.2])
    for bc in (0, 1, 2):
        mesh.set_bc(bc)
        res = mesh.homogenise()
        assert rel(res.C, D0) < 1e-10
    mesh.free()
    # one-cell mesh, Dirichlet, p = 1: every DOF constrained, C = Voigt average
    xyz, tets = ri.kuhn_grid(1, 1, 1)
    ph = np.array([0, 1, 0, 1, 0, 1], np.uint8)
    tg = np.tile([1.0, 0, 0], (6, 1))
    mesh = ctx64.mesh_load(xyz, tets, 1, ph, tg)
    mesh.set_materials(ri.NOMINAL_MATRIX, ri.NOMINAL_YARN)
    mesh.set_bc(0)
    res = mesh.homogenise()
    D, _, _ = mt.element_tensors(ph, tg, ri.NOMINAL_MATRIX, ri.NOMINAL_YARN)
    assert rel(res.C, D.mean(axis=0)) < 1e-12
    mesh.free()


def test_error_codes(rve, ctx64):
    xyz, tets = ri.kuhn_grid(2, 2, 2)
    bad = tets.copy()
    bad[0, 0] = 10_000
    with pytest.raises(rve.RveError) as e:
        ctx64.mesh_load(xyz, bad, 1)
    assert e.value.code == -2
    flat = xyz.copy()
    flat[:, 2] = 0.0
    with pytest.raises(rve.RveError) as e:
        ctx64.mesh_load(flat, tets, 1)
    assert e.value.code == -2
    mesh = ctx64.mesh_load(xyz, tets, 1)
    with pytest.raises(rve.RveError) as e:
        mesh.homogenise()
    assert e.value.code == -9
    with pytest.raises(rve.RveError) as e:
        mesh.set_materials(ri.MatrixProps(E=-1.0), ri.NOMINAL_YARN)
    assert e.value.code == -3
    with pytest.raises(rve.RveError) as e:
        mesh.set_materials(ri.NOMINAL_MATRIX, ri.NOMINAL_YARN, T_C=130.0)
    assert e.value.code == -1
    mesh.free()
    # periodic fold on a one-cell-thick mesh identifies vertices of one tet
    xyz, tets = ri.kuhn_grid(1, 2, 2)
    mesh = ctx64.mesh_load(xyz, tets, 1)
    with pytest.raises(rve.RveError) as e:
        mesh.set_bc(1)
    assert e.value.code == -2
    mesh.free()


def test_warm_started_batches_match_cold_and_oracle(rve):
    """Batches ordered by degradation factor and started from the previous
    batch's solutions (nearest, line, parabola in the factor, and the
    energy-optimal combination of up to four of them) give the same tensors as
    cold starts (and the oracle)."""
    grid, p = (6, 6, 4), 2
    xyz, tets, phase, tangent = ri.weave_rve(*grid)
    T, c, t, _, _ = ri.gauss_point_states(24, seed=9)
    out = {}
    for warm in (0, 1, 2, 3, 4):
        with rve.Context(precision=rve.PREC_MIXED, rtol=1e-7, inner_rtol=1e-6, batch=4, warm_start=warm) as ctx:
            mesh = ctx.mesh_load(xyz, tets, p, phase, tangent)
            mesh.set_materials(ri.NOMINAL_MATRIX, ri.NOMINAL_YARN)
            mesh.set_bc(1)
            Cb, Kb, Db, st, stats, rc = ctx.macro_update([mesh], T, c, t, np.zeros(24, np.int32))
            assert (st == 0).all()
            out[warm] = (Cb, Kb, Db, stats)
            mesh.free()
    for warm in (1, 2, 3, 4):
        for a, b in zip(out[warm][:3], out[0][:3]):
            for g in range(24):
                assert rel(a[g], b[g]) < 1e-6
    for g in (0, 11, 23):
        w = float(mt.one_minus_omega(T[g], c[g], t[g]))
        Co, Ko, Do = oracle_tensors(xyz, tets, grid, p, 1, phase, tangent, w)
        for warm in (1, 3, 4):
            assert rel(out[warm][0][g], Co) < TOL_MIXED
            assert rel(out[warm][1][g], Ko) < TOL_MIXED
            assert rel(out[warm][2][g], Do) < TOL_MIXED


@pytest.mark.parametrize("prec", [0, 1])
def test_energy_optimal_warm_start(rve, prec):
    """warm_start = 4 on a 12x12x6 p = 2 weave, 48 points in batches of 8: the
    tensors equal the cold-started ones to the solver tolerance, and the
    Galerkin start needs fewer operator launches than the line in w."""
    grid, p = (12, 12, 6), 2
    xyz, tets, phase, tangent = ri.weave_rve(*grid)
    T, c, t, _, _ = ri.gauss_point_states(48, seed=21)
    out = {}
    rtol = 1e-10 if prec == 0 else 1e-6
    for warm in (0, 2, 4):
        with rve.Context(precision=prec, rtol=rtol, inner_rtol=5e-7, batch=8, warm_start=warm) as ctx:
            mesh = ctx.mesh_load(xyz, tets, p, phase, tangent)
            mesh.set_materials(ri.NOMINAL_MATRIX, ri.NOMINAL_YARN)
            mesh.set_bc(1)
            Cb, Kb, Db, st, stats, rc = ctx.macro_update([mesh], T, c, t, np.zeros(48, np.int32))
            assert (st == 0).all()
            out[warm] = (Cb, Kb, Db, stats)
            mesh.free()
    tol = 1e-8 if prec == 0 else 1e-5
    for warm in (2, 4):
        for a, b in zip(out[warm][:3], out[0][:3]):
            for g in range(48):
                assert rel(a[g], b[g]) < tol
    assert out[4][3]["kernel_launches"] < out[2][3]["kernel_launches"], (out[4][3], out[2][3])
