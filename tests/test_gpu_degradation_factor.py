"""The degradation factor handed straight to the RVE path (Sec. 5: the macro
level integrates 1 - omega at each Gauss point and the RVE's matrix modulus is
scaled by it).  A point that degraded and then lost its moisture (c = 0,
W < 1) cannot be written as an exposure time of the closed-form law at its own
(T, c); given W directly it must match the oracle's cell solve at that W."""
import numpy as np
import pytest

import rve_inputs as ri
from oracle import fem
from oracle import materials as mt

pytestmark = pytest.mark.gpu


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.fixture(scope="module")
def rve():
    import paper_1610_03484_gb300 as rve
    from paper_1610_03484_gb300 import _build
    _build.build()
    rve.load_library()
    return rve


def test_dry_degraded_point_matches_oracle(rve):
    grid, p = (4, 4, 2), 2
    xyz, tets, phase, tangent = ri.weave_rve(*grid)
    W = np.array([0.43, 1.0, 0.71])
    with rve.Context(precision=rve.PREC_FP64, rtol=1e-11) as ctx:
        mesh = ctx.mesh_load(xyz, tets, p, phase, tangent)
        mesh.set_materials(ri.NOMINAL_MATRIX, ri.NOMINAL_YARN)
        mesh.set_bc(rve.BC_PERIODIC)
        Cg, Kg, Dg, st, _, _ = ctx.macro_update_w([mesh], W, np.zeros(len(W), np.int32))
        mesh.free()
    assert (st == 0).all()
    m0 = ri.NOMINAL_MATRIX
    for k, w in enumerate(W):
        D, K, Dd = mt.element_tensors(phase, tangent, ri.MatrixProps(E=m0.E * w, nu=m0.nu, k=m0.k, d=m0.d),
                                      ri.NOMINAL_YARN)
        Co, Ko, Do = fem.homogenise(xyz, tets, grid, p, fem.BC_PERIODIC, D, K, Dd)
        assert rel(Cg[k], Co) < 1e-9
        assert rel(Kg[k], Ko) < 1e-9
        assert rel(Dg[k], Do) < 1e-9


def test_factor_route_equals_state_route(rve):
    """W from the degradation law at (T, c, t) gives the (T, c, t) route's tensors."""
    grid, p = (4, 4, 2), 1
    xyz, tets, phase, tangent = ri.weave_rve(*grid)
    T, c, t, _, _ = ri.gauss_point_states(24, 9)
    W = np.array([float(mt.one_minus_omega(a, b, d)) for a, b, d in zip(T, c, t)])
    with rve.Context(precision=rve.PREC_FP64, rtol=1e-11, batch=8) as ctx:
        mesh = ctx.mesh_load(xyz, tets, p, phase, tangent)
        mesh.set_materials(ri.NOMINAL_MATRIX, ri.NOMINAL_YARN)
        mesh.set_bc(rve.BC_PERIODIC)
        mid = np.zeros(len(W), np.int32)
        C1, K1, D1, s1, _, _ = ctx.macro_update([mesh], T, c, t, mid)
        C2, K2, D2, s2, _, _ = ctx.macro_update_w([mesh], W, mid)
        with pytest.raises(rve.RveError):
            ctx.macro_update_w([mesh], np.array([0.5, 0.0]), np.zeros(2, np.int32))
        with pytest.raises(rve.RveError):
            ctx.macro_update_w([mesh], np.array([1.5]), np.zeros(1, np.int32))
        mesh.free()
    assert (s1 == 0).all() and (s2 == 0).all()
    for a, b in ((C1, C2), (K1, K2), (D1, D2)):
        assert max(rel(a[i], b[i]) for i in range(len(W))) < 1e-10
