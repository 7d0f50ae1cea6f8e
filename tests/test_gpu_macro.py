"""Coupled macro step on the GPU (Secs. 3-5) against the FP64 oracle: nodal
temperature and moisture after implicit steps, Gauss-point degradation and
equivalent exposure times, and the RVE refresh of a few Gauss points through
macro_update_gauss_points against the oracle's cell solve at the same 1 - omega."""
import numpy as np
import pytest

import rve_inputs as ri
from oracle import fem
from oracle import macro as mo
from oracle import materials as mt

pytestmark = pytest.mark.gpu

KT = np.array([[0.40, 0.01, 0.0], [0.01, 0.35, 0.0], [0.0, 0.0, 0.30]])
DC = np.diag([1.2e-12, 1.0e-12, 8.0e-13])


@pytest.fixture(scope="module")
def rve():
    import paper_1610_03484_gb300 as pkg
    from paper_1610_03484_gb300 import _build
    _build.build()
    pkg.load_library()
    return pkg


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(b))


def test_macro_steps_match_oracle(rve):
    xyz, tets, face = ri.plate(8, 3, 5)
    ex = ri.PlateExposure()
    n_steps, dt_h = 4, 150.0
    ref = mo.march(xyz, tets, face, KT, ex.rho_cp, DC, ex.T0_C, ex.c0_wt, ex.T_face_C, ex.c_face_wt,
                   dt_h, n_steps)
    with rve.Context(precision=rve.PREC_FP64) as ctx:
        m = ctx.macro_load(xyz, tets)
        m.set_transport(KT, ex.rho_cp, DC)
        m.set_face(face, ex.T_face_C, ex.c_face_wt)
        m.reset(ex.T0_C, ex.c0_wt)
        for k in range(n_steps):
            st = m.step(dt_h, rtol=1e-13)
            g = m.get()
            o = ref[k]
            assert st["converged"] == 1
            # points ahead of the moisture front where the transport undershoots to
            # c <= 0 after some wetting: the same set and the same miss as the oracle
            miss = mo.handover_error(o["W"], o["Tg"], o["cg"])
            assert st["gauss_points_unencodable"] == int((miss > 0).sum())
            assert st["handover_max_err"] == pytest.approx(miss.max(), rel=1e-6, abs=1e-15)
            assert st["handover_max_err"] < 1e-3
            assert rel(g["T"], o["T"]) < 1e-10
            assert np.abs(g["c"] - o["c"]).max() < 1e-9 * ex.c_face_wt
            assert np.abs(g["Tg"] - o["Tg"]).max() < 1e-9 * ex.T_face_C
            assert np.abs(g["cg"] - o["cg"]).max() < 1e-9 * ex.c_face_wt
            assert np.abs(g["W"] - o["W"]).max() < 1e-11
            # t_eq = -24 ln W / lambda is what the RVE path receives: the closed form
            # at (T, c, t_eq) must give back W up to the hand-over miss; t_eq itself
            # is compared where it is well conditioned (W visibly below 1; for W
            # within rounding of 1 the moisture is ~0 and any t_eq reproduces W)
            back = mt.one_minus_omega(g["Tg"], g["cg"], g["t_eq"])
            assert np.abs(back - g["W"]).max() < 1e-12 + st["handover_max_err"]
            well = (miss == 0) & (o["W"] < 1 - 1e-8)
            assert well.sum() > 0
            assert np.allclose(g["t_eq"][well], o["t_eq"][well], rtol=1e-7)
        m.free()


def test_macro_refresh_through_rve_path(rve):
    """Gauss points handed to the RVE path as (T, c, t_eq) get the tensors of
    an RVE whose matrix is degraded by exactly their 1 - omega."""
    xyz, tets, face = ri.plate(6, 2, 6)
    ex = ri.PlateExposure()
    grid, p = (6, 6, 4), 1
    rxyz, rtets, phase, tangent = ri.weave_rve(*grid)
    with rve.Context(precision=rve.PREC_FP64, rtol=1e-11) as ctx:
        m = ctx.macro_load(xyz, tets)
        m.set_transport(KT, ex.rho_cp, DC)
        m.set_face(face, ex.T_face_C, ex.c_face_wt)
        m.reset(ex.T0_C, ex.c0_wt)
        for _ in range(3):
            m.step(1000.0, rtol=1e-13)
        g = m.get()
        W = g["W"].reshape(-1)
        order = np.argsort(W)
        pick = order[[0, len(W) // 2, len(W) - 1]]          # most, median and least degraded
        mesh = ctx.mesh_load(rxyz, rtets, p, phase, tangent)
        mesh.set_materials(ri.NOMINAL_MATRIX, ri.NOMINAL_YARN)
        mesh.set_bc(rve.BC_PERIODIC)
        T = g["Tg"].reshape(-1)[pick]
        c = g["cg"].reshape(-1)[pick]
        t = g["t_eq"].reshape(-1)[pick]
        assert np.allclose(mt.one_minus_omega(T, c, t), W[pick], rtol=1e-12)
        Cg, Kg, Dg, st, stats, rc = ctx.macro_update([mesh], T, c, t, np.zeros(3, np.int32))
        assert (st == 0).all()
        for i, gp in enumerate(pick):
            mat = ri.MatrixProps(E=ri.NOMINAL_MATRIX.E * W[gp], nu=ri.NOMINAL_MATRIX.nu, k=ri.NOMINAL_MATRIX.k,
                                 d=ri.NOMINAL_MATRIX.d)
            D, K, Dd = mt.element_tensors(phase, tangent, mat, ri.NOMINAL_YARN)
            Co, Ko, Do = fem.homogenise(rxyz, rtets, grid, p, 1, D, K, Dd)
            assert rel(Cg[i], Co) < 1e-9
            assert rel(Kg[i], Ko) < 1e-9
        assert W[pick[0]] < W[pick[2]]
        mesh.free()
        m.free()


def test_macro_errors(rve):
    xyz, tets, face = ri.plate(2, 2, 2)
    with rve.Context() as ctx:
        bad = tets.copy()
        bad[0, 0] = len(xyz) + 5
        with pytest.raises(rve.RveError) as e:
            ctx.macro_load(xyz, bad)
        assert e.value.code == -2
        flipped = tets.copy()
        flipped[:, [1, 2]] = flipped[:, [2, 1]]
        with pytest.raises(rve.RveError) as e:
            ctx.macro_load(xyz, flipped)
        assert e.value.code == -2
        m = ctx.macro_load(xyz, tets)
        with pytest.raises(rve.RveError) as e:
            m.step(10.0)
        assert e.value.code == -9
        with pytest.raises(rve.RveError) as e:
            m.set_transport(-np.eye(3), 1e6, np.eye(3))
        assert e.value.code == -3
        m.free()


def test_macro_checkpoint_resume(rve):
    """A state saved with get() and restored with set_state() on a fresh macro
    object continues as the run that saved it: same Gauss-point states at the
    restore, same fields after further steps (up to the summation order of the
    atomics), and the oracle's march agrees with the resumed run."""
    xyz, tets, face = ri.plate(6, 2, 4)
    ex = ri.PlateExposure()
    dt_h = 300.0
    ref = mo.march(xyz, tets, face, KT, ex.rho_cp, DC, ex.T0_C, ex.c0_wt, ex.T_face_C, ex.c_face_wt, dt_h, 5)
    with rve.Context(precision=rve.PREC_FP64) as ctx:
        a = ctx.macro_load(xyz, tets)
        a.set_transport(KT, ex.rho_cp, DC)
        a.set_face(face, ex.T_face_C, ex.c_face_wt)
        a.reset(ex.T0_C, ex.c0_wt)
        for _ in range(3):
            a.step(dt_h, rtol=1e-13)
        saved = a.get()
        b = ctx.macro_load(xyz, tets)
        b.set_transport(KT, ex.rho_cp, DC)
        b.set_face(face, ex.T_face_C, ex.c_face_wt)
        b.set_state(saved["T"], saved["c"], saved["W"])
        gb = b.get()
        assert (gb["W"] == saved["W"]).all()
        for k in ("T", "c", "Tg", "cg", "t_eq"):
            assert np.array_equal(gb[k], saved[k]), k
        for _ in range(2):
            a.step(dt_h, rtol=1e-13)
            b.step(dt_h, rtol=1e-13)
        ga, gb = a.get(), b.get()
        assert rel(gb["T"], ga["T"]) < 1e-12
        assert np.abs(gb["c"] - ga["c"]).max() < 1e-12 * ex.c_face_wt
        assert np.abs(gb["W"] - ga["W"]).max() < 1e-13
        assert np.abs(gb["W"] - ref[4]["W"]).max() < 1e-11
        assert rel(gb["T"], ref[4]["T"]) < 1e-10
        with pytest.raises(rve.RveError) as e:
            b.set_state(saved["T"], saved["c"], np.zeros_like(saved["W"]))
        assert e.value.code == -1
        a.free()
        b.free()
