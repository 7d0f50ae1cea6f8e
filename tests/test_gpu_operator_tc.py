"""The tensor-core operator of the mixed-precision inner solve (mechanics,
p = 2 and 3) against the oracle's element matrices, and against the
matrix-free CUDA-core kernel it replaces.

Both FP32 kernels apply y = sum_e s(col, phase_e) K_e x_e (Eq. RVE_Eq_var_final,
degradation as a per-column factor on the matrix phase).  The tensor-core kernel
multiplies FP32 operands split into two TF32 parts (three MMAs, FP32
accumulation), so it must agree with FP32 arithmetic: 2e-6 relative per column
against the oracle's element matrices (FP64), with a column count above one
128-column tile plus a ragged tail, inactive columns, per-column phase scales
and both DOF numberings (periodic fold, unfolded)."""
import numpy as np
import pytest

import rve_inputs as ri
from oracle import fem
from oracle import materials as mt

from test_gpu_operator import oracle_apply

pytestmark = pytest.mark.gpu
TOL_F32 = 2e-6


@pytest.fixture(scope="module")
def rve():
    import paper_1610_03484_gb300 as pkg
    from paper_1610_03484_gb300 import _build
    _build.build()
    pkg.load_library()
    return pkg


def colrel(a, b):
    return np.linalg.norm(a - b, axis=0) / np.linalg.norm(b, axis=0)


@pytest.mark.parametrize("p", [2, 3])
@pytest.mark.parametrize("bc", [1, 0])      # periodic (folded DOFs), Dirichlet numbering (no fold)
def test_tc_operator_matches_oracle_and_cuda_cores(rve, p, bc):
    grid = (3, 3, 2)
    xyz, tets, phase, tangent = ri.weave_rve(*grid)
    D, _, _ = mt.element_tensors(phase, tangent, ri.NOMINAL_MATRIX, ri.NOMINAL_YARN)
    nm = fem.build_nodal_mesh(xyz, tets, grid, p, periodic=False)
    KeM = fem.element_stiffness_mech(nm, D)
    rng = np.random.default_rng(7 * p + bc)
    ncols = 138                               # two 128-column tiles, the second ragged
    with rve.Context(precision=rve.PREC_MIXED) as ctx:
        mesh = ctx.mesh_load(xyz, tets, p, phase, tangent)
        mesh.set_materials(ri.NOMINAL_MATRIX, ri.NOMINAL_YARN)
        mesh.set_bc(bc)
        edofs, lverts = mesh.dofmap()
        N = mesh.info()["n_scalar_dofs"]
        x = rng.standard_normal((N * 3, ncols))
        x32 = x.astype(np.float32).astype(np.float64)       # what the kernels see
        scale = rng.uniform(0.2, 1.0, size=(ncols, 2))
        active = (rng.uniform(size=ncols) > 0.15).astype(np.int32)
        y_tc, e_tc = mesh.apply_operator_mixed(x, 0, scale, active)
        y_cc, e_cc = mesh.apply_operator_mixed(x, 1, scale, active)
        # the oracle, phase by phase: y = s0 K_matrix x + s1 K_yarn x
        want = np.zeros_like(x)
        for ph in (0, 1):
            Kp = KeM * (phase == ph)[:, None, None, None, None]
            yp = oracle_apply(xyz, tets, grid, p, Kp, 3, edofs.astype(np.int64), lverts.astype(np.int64), x32)
            want += yp * scale[:, ph][None, :]
        want[:, active == 0] = 0.0
        on = active == 1
        assert np.all(y_tc[:, ~on] == 0.0) and np.all(e_tc[~on] == 0.0)
        assert colrel(y_tc[:, on], want[:, on]).max() < TOL_F32
        assert colrel(y_cc[:, on], want[:, on]).max() < TOL_F32
        assert colrel(y_tc[:, on], y_cc[:, on]).max() < TOL_F32
        # energy x . K x per column, element by element
        e_want = np.einsum("rc,rc->c", x32, want)
        assert np.abs(e_tc[on] - e_want[on]).max() <= 2e-6 * np.abs(e_want[on]).max()
        assert np.abs(e_cc[on] - e_want[on]).max() <= 2e-6 * np.abs(e_want[on]).max()
        mesh.free()


def test_tc_operator_on_the_bench_mesh(rve):
    """32x32x10, p = 2 (the benchmark's largest class): a batch of 8 RVEs (48
    columns, one partial tile) against the CUDA-core kernel and the FP64
    operator (itself pinned to the oracle's element matrices)."""
    xyz, tets, phase, tangent = ri.weave_rve(32, 32, 10)
    rng = np.random.default_rng(3)
    with rve.Context(precision=rve.PREC_MIXED) as ctx:
        mesh = ctx.mesh_load(xyz, tets, 2, phase, tangent)
        mesh.set_materials(ri.NOMINAL_MATRIX, ri.NOMINAL_YARN)
        mesh.set_bc(1)
        N = mesh.info()["n_scalar_dofs"]
        x = rng.standard_normal((N * 3, 48))
        y_tc, e_tc = mesh.apply_operator_mixed(x, 0)
        y_cc, e_cc = mesh.apply_operator_mixed(x, 1)
        y64 = mesh.apply_operator(0, x.astype(np.float32).astype(np.float64))
        mesh.free()
    assert colrel(y_tc, y64).max() < TOL_F32
    assert colrel(y_cc, y64).max() < TOL_F32
    assert colrel(e_tc[None, :], e_cc[None, :]).max() < TOL_F32
