"""The single large RVE at full size: 48x48x16 Kuhn grid (221 184 tets), p = 3
(3 090 675 mechanical DOFs), constituents jittered by +-10 % (seed 1), all
three boundary conditions, FP64 path against the mixed FP32/FP64 path.

The oracle cannot solve this size, so the checks are the properties that hold
at any size: mixed == FP64 to 1e-6, symmetric positive definite tensors,
Voigt >= Dirichlet >= periodic >= Neumann >= Reuss, Hill-Mandel.
"""
import numpy as np
import pytest

import rve_inputs as ri

pytestmark = pytest.mark.gpu

GRID, P = (48, 48, 16), 3


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def loewner_ge(A, B, tol=1e-7):
    return np.linalg.eigvalsh(0.5 * ((A - B) + (A - B).T)).min() >= -tol * np.linalg.norm(B)


@pytest.fixture(scope="module")
def results():
    import paper_1610_03484_gb300 as rve
    from paper_1610_03484_gb300 import _build
    _build.build()
    rve.load_library()
    mat, yarn = ri.jitter_props(seed=1)
    xyz, tets, phase, tangent = ri.weave_rve(*GRID)
    out = {}
    for prec, rtol in ((rve.PREC_FP64, 1e-10), (rve.PREC_MIXED, 1e-8)):
        with rve.Context(precision=prec, rtol=rtol, inner_rtol=1e-5) as ctx:
            mesh = ctx.mesh_load(xyz, tets, P, phase, tangent)
            assert mesh.info()["n_scalar_dofs"] * 3 == 3_090_675
            mesh.set_materials(mat, yarn, T_C=40.0, c_wt=1.0, t_h=1000.0)
            for bc in (0, 1, 2):
                mesh.set_bc(bc)
                out[(prec, bc)] = mesh.homogenise()
            # constituent tensors as solved: the matrix modulus scaled by 1 - omega
            D, K, Dd = mesh.tensors()
            w = float(ctx.degradation_factor([40.0], [1.0], [1000.0])[0])
            D = np.where((phase == 0)[:, None, None], D * w, D)
            out["voigt"] = D.mean(axis=0)          # equal tet volumes on the Kuhn grid
            out["reuss"] = np.linalg.inv(np.linalg.inv(D).mean(axis=0))
            mesh.free()
    return out


@pytest.mark.parametrize("bc", [0, 1, 2])
def test_mixed_matches_fp64(results, bc):
    a, b = results[(1, bc)], results[(0, bc)]
    assert a.stats["converged"] and b.stats["converged"]
    assert rel(a.C, b.C) < 1e-6
    assert rel(a.K, b.K) < 1e-6
    assert rel(a.D, b.D) < 1e-6


@pytest.mark.parametrize("bc", [0, 1, 2])
def test_spd_symmetric_hill_mandel(results, bc):
    r = results[(0, bc)]
    for T in (r.C, r.K, r.D):
        assert np.abs(T - T.T).max() <= 1e-12 * np.abs(T).max()
        assert np.linalg.eigvalsh(T).min() > 0
    assert r.stats["hill_mandel_mech"] < 1e-7


def test_bounds_and_bc_ordering(results):
    d, p, n = (results[(0, bc)].C for bc in (0, 1, 2))
    assert loewner_ge(results["voigt"], d)
    assert loewner_ge(d, p)
    assert loewner_ge(p, n)
    assert loewner_ge(n, results["reuss"])
