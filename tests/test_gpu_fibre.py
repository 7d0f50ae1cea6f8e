"""Yarn directions from potential flow (Sec. 6) on the GPU against the FP64
oracle, and an RVE homogenised with them against the oracle's cell solve."""
import numpy as np
import pytest

import rve_inputs as ri
from oracle import fem
from oracle import fibre as fo
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


@pytest.mark.parametrize("grid", [(16, 16, 6), (12, 12, 6)])
def test_directions_match_oracle(rve, grid):
    xyz, tets = ri.kuhn_grid(*grid)
    yid, axes = ri.plain_weave_yarns(xyz, tets)
    phase, tangent = ri.plain_weave(xyz, tets)
    want = fo.yarn_directions(xyz, tets, yid, axes, tangent)
    with rve.Context() as ctx:
        got = ctx.fibre_directions(xyz, tets, yid, axes, tangent, rtol=1e-13)
    assert np.abs(got - want).max() < 1e-9
    assert np.array_equal(got[yid < 0], tangent[yid < 0])


def test_straight_prism_gives_the_axis(rve):
    xyz, tets = ri.kuhn_grid(10, 6, 4, lengths=(2.0, 1.0, 1.0))
    c = ri.centroids(xyz, tets)
    yid = np.where((np.abs(c[:, 1] - 0.5) < 0.3) & (np.abs(c[:, 2] - 0.5) < 0.3), 0, -1).astype(np.int32)
    with rve.Context() as ctx:
        d = ctx.fibre_directions(xyz, tets, yid, [0], np.zeros((len(tets), 3)), rtol=1e-13)
    assert np.abs(d[yid == 0] - [1.0, 0.0, 0.0]).max() < 1e-10


def test_homogenisation_with_potential_flow_directions(rve):
    grid, p = (6, 6, 4), 2
    xyz, tets = ri.kuhn_grid(*grid)
    yid, axes = ri.plain_weave_yarns(xyz, tets)
    phase, tangent = ri.plain_weave(xyz, tets)
    with rve.Context(precision=rve.PREC_FP64, rtol=1e-11) as ctx:
        d = ctx.fibre_directions(xyz, tets, yid, axes, tangent, rtol=1e-13)
        mesh = ctx.mesh_load(xyz, tets, p, phase, d)
        mesh.set_materials(ri.NOMINAL_MATRIX, ri.NOMINAL_YARN)
        mesh.set_bc(rve.BC_PERIODIC)
        res = mesh.homogenise()
        mesh.free()
    D, K, Dd = mt.element_tensors(phase, d, ri.NOMINAL_MATRIX, ri.NOMINAL_YARN)
    Co, Ko, Do = fem.homogenise(xyz, tets, grid, p, fem.BC_PERIODIC, D, K, Dd)
    assert rel(res.C, Co) < 1e-9
    assert rel(res.K, Ko) < 1e-9
    assert rel(res.D, Do) < 1e-9
