"""Macro mechanics of the nested FE^2 step on the GPU (Sec. 5) against the FP64
oracle: displacements, Gauss-point stresses and nodal loads for per-Gauss-point
anisotropic stiffness, prescribed displacements, warm starts, and the whole
chain transport -> degradation -> RVE C_bar -> macro displacement."""
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


def spd6(rng, n, scale):
    A = rng.standard_normal((n, 6, 6))
    return scale * (np.einsum("nij,nkj->nik", A, A) + 6.0 * np.eye(6)[None])


def rollers(xyz):
    fixed = np.zeros((len(xyz), 3), bool)
    for i in range(3):
        fixed[:, i] = xyz[:, i] <= 1e-12 * np.abs(xyz).max()
    return fixed


def test_mech_matches_oracle(rve):
    rng = np.random.default_rng(11)
    xyz, tets, _ = ri.plate(9, 3, 4)
    Lx, Ly, Lz = ri.PLATE_LENGTHS
    C = spd6(rng, len(tets) * 4, 1e9).reshape(len(tets), 4, 6, 6)
    C += 1e-9 * np.abs(C).max() * rng.standard_normal(C.shape)   # a rounding-level asymmetric part
    fixed = rollers(xyz)
    top = xyz[:, 2] >= Lz * (1 - 1e-12)
    end = xyz[:, 0] >= Lx * (1 - 1e-12)
    t1, t2 = np.array([0.0, 0.0, -1.0e6]), np.array([2.0e6, 3.0e5, 0.0])
    f = mo.traction_load(xyz, tets, top, t1) + mo.traction_load(xyz, tets, end, t2)
    K = mo.elastic_assemble(xyz, tets, C)
    u_ref = mo.elastic_solve(K, f, fixed.reshape(-1))
    sig_ref = mo.gauss_stress(xyz, tets, u_ref, C)
    with rve.Context(precision=rve.PREC_FP64) as ctx:
        m = ctx.macro_load(xyz, tets)
        m.mech_set_bc(fixed)
        m.mech_set_traction(top, t1)
        m.mech_set_traction(end, t2, add=True)
        st = m.mech_solve(C, rtol=1e-13)
        g = m.mech_get()
        assert st["converged"] == 1 and st["iterations"] > 10
        assert np.abs(g["load"].reshape(-1) - f).max() < 1e-12 * np.abs(f).max()
        assert rel(g["u"].reshape(-1), u_ref) < 1e-10
        assert np.abs(g["stress"] - sig_ref).max() < 1e-9 * np.abs(sig_ref).max()
        assert (g["u"][fixed] == 0).all()
        # warm start: the same problem again needs (almost) no iteration; the
        # stiffness halved doubles the displacement (zero prescribed values)
        st2 = m.mech_solve(C, rtol=1e-13)
        assert st2["iterations"] <= 8
        m.mech_solve(0.5 * C, rtol=1e-13)
        g2 = m.mech_get()
        assert rel(g2["u"], 2.0 * g["u"]) < 1e-10
        assert np.abs(g2["stress"] - g["stress"]).max() < 1e-9 * np.abs(g["stress"]).max()
        m.free()


def test_mech_prescribed_displacement_patch(rve):
    """Boundary held at u = A y, no load, one anisotropic C everywhere: the
    interior reproduces A y (linear tetrahedra are exact for it)."""
    rng = np.random.default_rng(4)
    xyz, tets = ri.kuhn_grid(4, 3, 3, lengths=(0.4, 0.3, 0.3))
    Cm = spd6(rng, 1, 5e9)[0]
    C = np.broadcast_to(Cm, (len(tets), 4, 6, 6))
    A = 1e-3 * rng.standard_normal((3, 3))
    ulin = xyz @ A.T
    lo, hi = xyz.min(axis=0), xyz.max(axis=0)
    bnd = ((xyz <= lo + 1e-12) | (xyz >= hi - 1e-12)).any(axis=1)
    with rve.Context(precision=rve.PREC_FP64) as ctx:
        m = ctx.macro_load(xyz, tets)
        m.mech_set_bc(np.repeat(bnd[:, None], 3, axis=1), ulin)
        m.mech_set_traction(np.zeros(len(xyz), bool), [0.0, 0.0, 0.0])
        st = m.mech_solve(C, rtol=1e-14)
        g = m.mech_get()
        assert st["converged"] == 1
        assert np.abs(g["u"] - ulin).max() < 1e-12 * np.abs(ulin).max() + 1e-18
        eps = np.array([A[0, 0], A[1, 1], A[2, 2], A[0, 1] + A[1, 0], A[1, 2] + A[2, 1], A[2, 0] + A[0, 2]])
        assert np.abs(g["stress"] - Cm @ eps).max() < 1e-9 * np.abs(Cm @ eps).max()
        m.free()


def test_fe2_chain_transport_degradation_rve_mechanics(rve):
    """The nested FE^2 step end to end: implicit transport steps and the
    Gauss-point degradation on the macro plate, C_bar of every macro Gauss
    point from the RVE path at its (T, c, t_eq), the macro elastic solve with
    those C_bar (device pointer) against the oracle's solve with the same
    C_bar.  The RVE tensors are checked against the oracle's cell solve at a
    few points.  More degradation, more compliance f.u under the same load:
    C_bar falls in the Loewner order as the matrix modulus falls."""
    import torch
    xyz, tets, face = ri.plate(4, 1, 2)
    Lx, Ly, Lz = ri.PLATE_LENGTHS
    ex = ri.PlateExposure()
    grid, p = (6, 6, 4), 1
    rxyz, rtets, phase, tangent = ri.weave_rve(*grid)
    top = xyz[:, 2] >= Lz * (1 - 1e-12)
    fixed = rollers(xyz)
    t = np.array([0.0, 0.0, -5.0e6])
    with rve.Context(precision=rve.PREC_FP64, rtol=1e-11) as ctx:
        mesh = ctx.mesh_load(rxyz, rtets, p, phase, tangent)
        mesh.set_materials(ri.NOMINAL_MATRIX, ri.NOMINAL_YARN)
        mesh.set_bc(rve.BC_PERIODIC)
        m = ctx.macro_load(xyz, tets)
        m.set_transport(KT, ex.rho_cp, DC)
        m.set_face(face, ex.T_face_C, ex.c_face_wt)
        m.reset(ex.T0_C, ex.c0_wt)
        m.mech_set_bc(fixed)
        m.mech_set_traction(top, t)
        G = len(tets) * 4
        work = []
        for step in range(3):
            m.step(2000.0, rtol=1e-13)
            g = m.get()
            Cg, Kg, Dg, st, stats, rc = ctx.macro_update([mesh], g["Tg"].reshape(-1), g["cg"].reshape(-1),
                                                         g["t_eq"].reshape(-1), np.zeros(G, np.int32))
            assert (st == 0).all()
            Cd = torch.from_numpy(np.ascontiguousarray(Cg)).cuda()
            torch.cuda.synchronize()
            ms = m.mech_solve(Cd.data_ptr(), rtol=1e-13)
            assert ms["converged"] == 1
            u = m.mech_get()["u"]
            K = mo.elastic_assemble(xyz, tets, Cg.reshape(len(tets), 4, 6, 6))
            f = mo.traction_load(xyz, tets, top, t)
            u_ref = mo.elastic_solve(K, f, fixed.reshape(-1))
            assert rel(u.reshape(-1), u_ref) < 1e-9
            work.append(float(f @ u.reshape(-1)))
            if step == 2:
                # the RVE path receives (T, c, t_eq): its 1 - omega is the closed form there
                W = mt.one_minus_omega(g["Tg"].reshape(-1), g["cg"].reshape(-1), g["t_eq"].reshape(-1))
                assert W.min() < 0.97
                for i in (int(np.argmin(W)), int(np.argmax(W))):
                    mat = ri.MatrixProps(E=ri.NOMINAL_MATRIX.E * W[i], nu=ri.NOMINAL_MATRIX.nu,
                                         k=ri.NOMINAL_MATRIX.k, d=ri.NOMINAL_MATRIX.d)
                    D, Kt, Dd = mt.element_tensors(phase, tangent, mat, ri.NOMINAL_YARN)
                    Co, _, _ = fem.homogenise(rxyz, rtets, grid, p, fem.BC_PERIODIC, D, Kt, Dd)
                    assert rel(Cg[i], Co) < 1e-9
        assert work[0] < work[1] < work[2]
        del Cd
        m.free()
        mesh.free()


def test_mech_errors(rve):
    xyz, tets, _ = ri.plate(2, 2, 2)
    with rve.Context() as ctx:
        m = ctx.macro_load(xyz, tets)
        C = np.broadcast_to(mt.iso_stiffness(1e9, 0.3), (len(tets), 4, 6, 6))
        with pytest.raises(rve.RveError) as e:
            m.mech_solve(C)
        assert e.value.code == -9
        with pytest.raises(rve.RveError) as e:
            m.mech_get()
        assert e.value.code == -9
        with pytest.raises(rve.RveError) as e:
            m.mech_set_traction(np.ones(len(xyz), bool), [np.nan, 0.0, 0.0])
        assert e.value.code == -1
        with pytest.raises(ValueError):
            m.mech_solve(C[:-1])
        m.mech_set_bc(rollers(xyz))
        m.mech_set_traction(xyz[:, 0] >= xyz[:, 0].max() - 1e-12, [1e6, 0, 0])
        with pytest.raises(rve.RveError) as e:
            m.mech_solve(C, rtol=1e-14, max_iter=1)
        assert e.value.code == -4
        m.free()
