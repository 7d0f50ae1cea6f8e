"""Batch scheduling: the batch-size autotuner (scheduling of the batched cell
solves; no counterpart in the paper).  Through the C ABI on the GPU."""
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


def test_autotune_batch_picks_a_candidate_and_is_used(rve):
    grid, p = (6, 6, 4), 2
    xyz, tets, phase, tangent = ri.weave_rve(*grid)
    Ts, cs, ts, _, _ = ri.gauss_point_states(24, seed=21)     # tuning sample
    T, c, t, _, _ = ri.gauss_point_states(20, seed=22)        # the call that uses it
    with rve.Context(precision=rve.PREC_MIXED, rtol=1e-8, inner_rtol=1e-6) as ctx:
        mesh = ctx.mesh_load(xyz, tets, p, phase, tangent)
        with pytest.raises(rve.RveError) as e:
            mesh.autotune_batch(Ts, cs, ts, [4, 8])
        assert e.value.code == -9                              # materials not set
        mesh.set_materials(ri.NOMINAL_MATRIX, ri.NOMINAL_YARN)
        mesh.set_bc(1)
        with pytest.raises(rve.RveError) as e:
            mesh.autotune_batch(Ts, cs, ts, [4, 0])
        assert e.value.code == -1
        best, rates = mesh.autotune_batch(Ts, cs, ts, [4, 8])
        assert best in (4, 8)
        assert all(r > 0 for r in rates.values())
        # the smallest candidate within 6 % of the fastest
        assert rates[best] >= 0.94 * max(rates.values())
        assert all(b >= best for b, r in rates.items() if r >= 0.94 * max(rates.values()))
        Ct, Kt, Dt, st, stats, rc = ctx.macro_update([mesh], T, c, t, np.zeros(20, np.int32))
        assert (st == 0).all()
        mesh.free()
    # the same points with the chosen batch size set explicitly
    with rve.Context(precision=rve.PREC_MIXED, rtol=1e-8, inner_rtol=1e-6, batch=best) as ctx:
        mesh = ctx.mesh_load(xyz, tets, p, phase, tangent)
        mesh.set_materials(ri.NOMINAL_MATRIX, ri.NOMINAL_YARN)
        mesh.set_bc(1)
        Ce, Ke, De, st, stats, rc = ctx.macro_update([mesh], T, c, t, np.zeros(20, np.int32))
        mesh.free()
    for g in range(20):
        assert rel(Ct[g], Ce[g]) < 1e-8
        assert rel(Kt[g], Ke[g]) < 1e-8
    # and against the oracle on two points
    for g in (0, 19):
        w = float(mt.one_minus_omega(T[g], c[g], t[g]))
        m = ri.MatrixProps(E=ri.NOMINAL_MATRIX.E * w, nu=ri.NOMINAL_MATRIX.nu, k=ri.NOMINAL_MATRIX.k,
                           d=ri.NOMINAL_MATRIX.d)
        D, K, Dd = mt.element_tensors(phase, tangent, m, ri.NOMINAL_YARN)
        Co, Ko, Do = fem.homogenise(xyz, tets, grid, p, 1, D, K, Dd)
        assert rel(Ct[g], Co) < 1e-6
        assert rel(Kt[g], Ko) < 1e-6
        assert rel(Dt[g], Do) < 1e-6


def test_transport_once_matches_per_point_solves(rve):
    """Thermal and moisture cell problems do not depend on the degradation
    state (transport is not degraded): solving them once per mesh gives the
    same K and D, and the same C, as solving all twelve load cases per point."""
    grid, p = (6, 6, 4), 2
    xyz, tets, phase, tangent = ri.weave_rve(*grid)
    T, c, t, _, _ = ri.gauss_point_states(20, seed=23)
    out = {}
    for once in (False, True):
        with rve.Context(precision=rve.PREC_MIXED, rtol=1e-8, inner_rtol=1e-6, batch=4,
                         transport_once=once) as ctx:
            mesh = ctx.mesh_load(xyz, tets, p, phase, tangent)
            mesh.set_materials(ri.NOMINAL_MATRIX, ri.NOMINAL_YARN)
            mesh.set_bc(1)
            Cb, Kb, Db, st, stats, rc = ctx.macro_update([mesh], T, c, t, np.zeros(20, np.int32))
            assert (st == 0).all()
            out[once] = (Cb, Kb, Db)
            mesh.free()
    for a, b in zip(out[True], out[False]):
        for g in range(20):
            assert rel(a[g], b[g]) < 1e-6
    # every point of the mesh carries the same transport tensors
    assert np.abs(out[True][1] - out[True][1][0]).max() <= 1e-12 * np.abs(out[True][1][0]).max()


def test_meshes_solved_concurrently_match_separate_calls(rve):
    """Points on several meshes in one call (one host thread and stream per mesh)
    give what each mesh gives on its own, and the oracle."""
    specs = [((6, 6, 4), 1), ((6, 6, 4), 2), ((4, 4, 3), 2)]
    T, c, t, _, _ = ri.gauss_point_states(30, seed=31)
    mid = np.arange(30, dtype=np.int32) % len(specs)
    with rve.Context(precision=rve.PREC_MIXED, rtol=1e-8, inner_rtol=1e-6, batch=4) as ctx:
        meshes = []
        for grid, p in specs:
            xyz, tets, phase, tangent = ri.weave_rve(*grid)
            m = ctx.mesh_load(xyz, tets, p, phase, tangent)
            m.set_materials(ri.NOMINAL_MATRIX, ri.NOMINAL_YARN)
            m.set_bc(1)
            meshes.append(m)
        Ca, Ka, Da, st, stats, rc = ctx.macro_update(meshes, T, c, t, mid)
        assert (st == 0).all()
        for k, m in enumerate(meshes):
            sel = np.nonzero(mid == k)[0]
            Cs, Ks, Ds, st2, _, _ = ctx.macro_update([m], T[sel], c[sel], t[sel], np.zeros(len(sel), np.int32))
            assert (st2 == 0).all()
            for i, g in enumerate(sel):
                assert rel(Ca[g], Cs[i]) < 1e-8
                assert rel(Ka[g], Ks[i]) < 1e-8
        for m in meshes:
            m.free()
    # one point of each mesh against the oracle
    for k, (grid, p) in enumerate(specs):
        g = int(np.nonzero(mid == k)[0][0])
        xyz, tets, phase, tangent = ri.weave_rve(*grid)
        w = float(mt.one_minus_omega(T[g], c[g], t[g]))
        mat = ri.MatrixProps(E=ri.NOMINAL_MATRIX.E * w, nu=ri.NOMINAL_MATRIX.nu, k=ri.NOMINAL_MATRIX.k,
                             d=ri.NOMINAL_MATRIX.d)
        D, K, Dd = mt.element_tensors(phase, tangent, mat, ri.NOMINAL_YARN)
        Co, Ko, Do = fem.homogenise(xyz, tets, grid, p, 1, D, K, Dd)
        assert rel(Ca[g], Co) < 1e-6
        assert rel(Ka[g], Ko) < 1e-6


@pytest.mark.parametrize("p", [2, 3])
def test_every_schedule_matches_oracle_and_the_tuned_one_is_used(rve, p):
    """Each (operator kernel, batch size) schedule the tuner can choose gives the
    oracle's tensors at the mixed-precision bound (1e-6); the tuner's choice is
    kept for the mesh and used by the next batched call."""
    grid = (6, 6, 4)
    xyz, tets, phase, tangent = ri.weave_rve(*grid)
    Ts, cs, ts, _, _ = ri.gauss_point_states(24, seed=31)
    T, c, t, _, _ = ri.gauss_point_states(16, seed=32)
    w = [float(mt.one_minus_omega(T[g], c[g], t[g])) for g in (0, 15)]
    oracle = {}
    for g, wg in zip((0, 15), w):
        m = ri.MatrixProps(E=ri.NOMINAL_MATRIX.E * wg, nu=ri.NOMINAL_MATRIX.nu, k=ri.NOMINAL_MATRIX.k,
                           d=ri.NOMINAL_MATRIX.d)
        D, K, Dd = mt.element_tensors(phase, tangent, m, ri.NOMINAL_YARN)
        oracle[g] = fem.homogenise(xyz, tets, grid, p, 1, D, K, Dd)
    results = {}
    for kern in (rve.KERNEL_CUDA_CORE, rve.KERNEL_TENSOR):
        for batch in (4, 8):
            with rve.Context(precision=rve.PREC_MIXED, rtol=1e-8, inner_rtol=1e-6, batch=batch,
                             operator_kernel=kern) as ctx:
                mesh = ctx.mesh_load(xyz, tets, p, phase, tangent)
                mesh.set_materials(ri.NOMINAL_MATRIX, ri.NOMINAL_YARN)
                mesh.set_bc(1)
                Cg, Kg, Dg, st, _, _ = ctx.macro_update([mesh], T, c, t, np.zeros(16, np.int32))
                mesh.free()
            assert (st == 0).all()
            results[(kern, batch)] = Cg
            for g in (0, 15):
                Co, Ko, Do = oracle[g]
                assert rel(Cg[g], Co) < 1e-6, (kern, batch, g)
                assert rel(Kg[g], Ko) < 1e-6
                assert rel(Dg[g], Do) < 1e-6
    with rve.Context(precision=rve.PREC_MIXED, rtol=1e-8, inner_rtol=1e-6) as ctx:
        mesh = ctx.mesh_load(xyz, tets, p, phase, tangent)
        mesh.set_materials(ri.NOMINAL_MATRIX, ri.NOMINAL_YARN)
        mesh.set_bc(1)
        bb, bk, rates = mesh.autotune_schedule(Ts, cs, ts, [4, 8])
        assert bb in (4, 8) and bk in (rve.KERNEL_CUDA_CORE, rve.KERNEL_TENSOR)
        top = max(rates.values())
        assert rates[(bk, bb)] >= 0.94 * top
        assert all(b >= bb for (k, b), r in rates.items() if r >= 0.94 * top)
        Ct, _, _, st, _, _ = ctx.macro_update([mesh], T, c, t, np.zeros(16, np.int32))
        mesh.free()
    assert (st == 0).all()
    for g in range(16):
        assert rel(Ct[g], results[(bk, bb)][g]) < 1e-8
