"""Parity at the benchmark's own settings: the batched mixed-precision path
with the tolerances bench.py times, on Gauss points sampled from the
benchmark's seeded draw, against the FP64 oracle (<= 1e-6 per tensor)."""
import numpy as np
import pytest

import rve_inputs as ri
from oracle import fem
from oracle import materials as mt

pytestmark = pytest.mark.gpu
TOL_MIXED = 1e-6


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("size_idx,p", [(0, 1), (0, 2), (1, 1), (2, 1)])
def test_bench_settings_match_oracle(size_idx, p):
    import bench
    import paper_1610_03484_gb300 as rve
    from paper_1610_03484_gb300 import _build
    _build.build()
    rve.load_library()
    G = 256
    T, c, t, size, pp = ri.gauss_point_states(G, bench.SEED)
    pick = np.nonzero((size == size_idx) & (pp == p))[0][:2]
    assert len(pick) == 2
    grid = ri.SIZE_CLASSES[size_idx]
    xyz, tets, phase, tangent = ri.weave_rve(*grid)
    with rve.Context(precision=rve.PREC_MIXED, rtol=bench.RTOL, inner_rtol=bench.INNER_RTOL,
                     max_refine=4) as ctx:
        mesh = ctx.mesh_load(xyz, tets, p, phase, tangent)
        mesh.set_materials(ri.NOMINAL_MATRIX, ri.NOMINAL_YARN)
        mesh.set_bc(rve.BC_PERIODIC)
        Cg, Kg, Dg, st, stats, rc = ctx.macro_update([mesh], T[pick], c[pick], t[pick],
                                                    np.zeros(len(pick), np.int32))
        mesh.free()
    assert (st == 0).all()
    for k, g in enumerate(pick):
        w = float(mt.one_minus_omega(T[g], c[g], t[g]))
        m0 = ri.NOMINAL_MATRIX
        D, K, Dd = mt.element_tensors(phase, tangent, ri.MatrixProps(E=m0.E * w, nu=m0.nu, k=m0.k, d=m0.d),
                                      ri.NOMINAL_YARN)
        Co, Ko, Do = fem.homogenise(xyz, tets, grid, p, fem.BC_PERIODIC, D, K, Dd)
        assert rel(Cg[k], Co) < TOL_MIXED
        assert rel(Kg[k], Ko) < TOL_MIXED
        assert rel(Dg[k], Do) < TOL_MIXED
