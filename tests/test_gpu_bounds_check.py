"""Checking build (librve_check.so, -DRVE_BOUNDS_CHECK=1).

1. On valid meshes it reports no violation and gives the release library's
   tensors (the checks only skip work when an index is out of range).
2. With the test hook that lowers the DOF bound the kernels compare against,
   the elements touching the DOFs above it are counted and skipped, the call
   returns RVE_ERR_BOUNDS, and the first reported element does touch such a
   DOF.  Every access that runs stays inside the mesh's arrays: the lowered bound
   is below the true DOF count, so no out-of-range address is ever formed.

The checking library runs in a child process (RVE_LIBRARY selects it), since a
process loads one librve.
"""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

import rve_inputs as ri

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import json, sys
import numpy as np
sys.path.insert(0, ROOT)
import rve_inputs as ri
import paper_1610_03484_gb300 as rve
out = {}
xyz, tets, phase, tangent = ri.weave_rve(6, 6, 4)
for prec in (0, 1):
    with rve.Context(precision=prec, rtol=1e-10 if prec == 0 else 1e-7) as ctx:
        m = ctx.mesh_load(xyz, tets, 2, phase, tangent)
        m.set_materials(ri.NOMINAL_MATRIX, ri.NOMINAL_YARN, T_C=70.0, c_wt=0.8, t_h=400.0)
        m.set_bc(1)
        r = m.homogenise()
        out["C%d" % prec] = r.C.tolist()
        out["bounds%d" % prec] = ctx.debug_bounds(reset=True)
        m.free()
with rve.Context(max_iter=40) as ctx:
    m = ctx.mesh_load(xyz, tets, 2, phase, tangent)
    m.set_materials(ri.NOMINAL_MATRIX, ri.NOMINAL_YARN)
    m.set_bc(1)
    n = m.info()["n_scalar_dofs"]
    bound = n - n // 10
    m.debug_set_node_bound(bound)
    try:
        m.homogenise(allow_not_converged=True)
        out["planted_error"] = None
    except rve.RveError as e:
        out["planted_error"] = e.code
    out["planted_bound"] = bound
    out["planted"] = ctx.debug_bounds(reset=True)
    ed, _ = m.dofmap()
    fe = out["planted"]["first_element"]
    out["first_element_max_dof"] = int(ed[fe].max()) if fe >= 0 else -1
    out["n_elements_over"] = int((ed.max(axis=1) >= bound).sum())
    m.debug_set_node_bound(0)
    r = m.homogenise(allow_not_converged=True)
    out["after_reset"] = ctx.debug_bounds(reset=True)
    m.free()
print("RESULT " + json.dumps(out))
"""


@pytest.fixture(scope="module")
def libs():
    from paper_1610_03484_gb300 import _build
    return _build.build(), _build.build(check=True)


def test_checking_build_clean_and_planted(libs):
    release, check = libs
    env = dict(os.environ, RVE_LIBRARY=check)
    res = subprocess.run([sys.executable, "-c", "ROOT = %r\n" % ROOT + CHILD], env=env, capture_output=True,
                         text=True, timeout=600)
    assert res.returncode == 0, res.stderr[-3000:]
    line = [ln for ln in res.stdout.splitlines() if ln.startswith("RESULT ")][-1]
    out = json.loads(line[7:])
    for prec in (0, 1):
        b = out["bounds%d" % prec]
        assert b["checking_build"] == 1
        assert b["violations"] == 0 and b["first_element"] == -1
    # the planted bound: every element visit that touches a DOF >= bound is reported
    p = out["planted"]
    assert out["planted_error"] == -11
    assert p["violations"] > 0 and out["n_elements_over"] > 0
    assert out["first_element_max_dof"] >= out["planted_bound"]
    assert out["after_reset"]["violations"] == 0

    # the checking build's clean results equal the release library's
    import paper_1610_03484_gb300 as rve
    rve.load_library()
    xyz, tets, phase, tangent = ri.weave_rve(6, 6, 4)
    for prec in (0, 1):
        with rve.Context(precision=prec, rtol=1e-10 if prec == 0 else 1e-7) as ctx:
            m = ctx.mesh_load(xyz, tets, 2, phase, tangent)
            m.set_materials(ri.NOMINAL_MATRIX, ri.NOMINAL_YARN, T_C=70.0, c_wt=0.8, t_h=400.0)
            m.set_bc(1)
            r = m.homogenise()
            assert ctx.debug_bounds()["checking_build"] == 0
            m.free()
        C = np.array(out["C%d" % prec])
        assert np.linalg.norm(C - r.C) / np.linalg.norm(r.C) < (1e-9 if prec == 0 else 1e-6)
