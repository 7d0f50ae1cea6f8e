"""The paper's multiplier route on the GPU (Sec. 2): sigma_bar = -D^T lambda / V
(Eq. eq_homo_stress) with the constraint rows C and D = C X of each boundary
condition written out (Eqs. eq_RVE_disc_Eqs, eq_mat_C_and_D) and lambda from
the equilibrium of the total field, against the oracle's bordered total-field
system [[K, C^T], [C, 0]] solved densely (oracle.fem.paper_route) on 2x2x2
meshes, p = 1..3, all three boundary conditions, mechanics and both transport
fields, at 1e-9; and against the energy form of the same solve."""
import numpy as np
import pytest

import rve_inputs as ri
from oracle import fem
from oracle import materials as mt

pytestmark = pytest.mark.gpu
STATE = (45.0, 1.2, 3000.0)     # T [C], moisture [wt%], exposure [h]


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.fixture(scope="module")
def rve():
    import paper_1610_03484_gb300 as pkg
    from paper_1610_03484_gb300 import _build
    _build.build()
    pkg.load_library()
    return pkg


@pytest.mark.parametrize("p", [1, 2, 3])
@pytest.mark.parametrize("bc", [0, 1, 2])
def test_multiplier_route_matches_oracle(rve, p, bc):
    grid = (2, 2, 2)
    xyz, tets = ri.kuhn_grid(*grid)
    ph = (np.arange(len(tets)) % 3 == 0).astype(np.uint8)
    tg = ri.random_unit_vectors(len(tets), 11)
    w = float(mt.one_minus_omega(*STATE))
    m0 = ri.NOMINAL_MATRIX
    D, Kt, Dd = mt.element_tensors(ph, tg, ri.MatrixProps(E=m0.E * w, nu=m0.nu, k=m0.k, d=m0.d), ri.NOMINAL_YARN)
    with rve.Context(precision=rve.PREC_FP64, rtol=1e-13) as ctx:
        mesh = ctx.mesh_load(xyz, tets, p, ph, tg)
        mesh.set_materials(ri.NOMINAL_MATRIX, ri.NOMINAL_YARN, *STATE)
        mesh.set_bc(bc)
        Cw, Kw, Dw, Ce, Ke, De = mesh.homogenise_weak()
        mesh.free()
    for got, energy, mat, nc in ((Cw, Ce, D, 3), (Kw, Ke, Kt, 1), (Dw, De, Dd, 1)):
        want = fem.paper_route(xyz, tets, grid, p, bc, mat, nc)
        assert rel(got, want) < 1e-9, (p, bc, nc, rel(got, want))
        assert rel(got, energy) < 1e-9
