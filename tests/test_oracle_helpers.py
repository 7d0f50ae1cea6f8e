"""Direct pins for oracle helpers that the other pins reach only through
compositions: the volume-averaged flux of Eq. macro_stress, the box-surface node
set, the rate form of the degradation law (Eq. Eq_Model_RateForm) against its
closed form (Sec. 4), and the surrogate network's forward pass and activations."""
import numpy as np
import pytest

import rve_inputs as ri
from oracle import fem
from oracle import macro as mc
from oracle import materials as mt
from oracle import surrogate as sg


@pytest.mark.parametrize("p", [1, 2])
def test_volume_average_flux_of_a_linear_field_is_D_times_the_macro_gradient(p):
    """A homogeneous RVE under the unit macro fields with no fluctuation: the
    averaged stress (flux) is D e_J (k e_J) exactly, for every load case."""
    grid = (3, 2, 2)
    xyz, tets, _, _ = ri.weave_rve(*grid)
    m = fem.build_nodal_mesh(xyz, tets, grid, p)
    nt = len(tets)
    D = mt.iso_stiffness(3.5e9, 0.35) + 1e8 * np.eye(6)          # a full, non-isotropic stiffness
    k = np.array([[0.6, 0.1, 0.0], [0.1, 0.35, 0.05], [0.0, 0.05, 0.2]])
    for nc, mat in ((3, np.broadcast_to(D, (nt, 6, 6))), (1, np.broadcast_to(k, (nt, 3, 3)))):
        ue = [fem.linear_field_nodal(m, M, nc) for M in fem.unit_macro_fields(nc)]
        sig = fem.volume_average_flux(m, fem._KeFn(np.ascontiguousarray(mat), nc), ue, nc)
        ref = D if nc == 3 else k
        # load case J gives column J of the (symmetric) constitutive matrix
        np.testing.assert_allclose(sig, ref.T, rtol=1e-12, atol=1e-12 * np.abs(ref).max())


@pytest.mark.parametrize("grid", [(2, 2, 2), (4, 3, 2), (5, 1, 3)])
def test_boundary_nodes_p1_count(grid):
    """p = 1: the vertex lattice minus its strict interior."""
    xyz, tets, _, _ = ri.weave_rve(*grid)
    m = fem.build_nodal_mesh(xyz, tets, grid, 1)
    nx, ny, nz = grid
    n_all = (nx + 1) * (ny + 1) * (nz + 1)
    n_inner = max(nx - 1, 0) * max(ny - 1, 0) * max(nz - 1, 0)
    assert fem.n_nodes(m) == n_all
    assert len(fem.boundary_nodes(m)) == n_all - n_inner


@pytest.mark.parametrize("T_C,c_wt", [(20.0, 0.0), (40.0, 0.75), (60.0, 1.5), (70.0, 2.0)])
def test_rate_form_matches_the_closed_form(T_C, c_wt):
    """d(1 - omega)/dt = -lambda (1 - omega) with lambda in 1/day: the closed form
    at t hours equals exp(-lambda t / 24), and lambda >= 0."""
    lam = mc.degradation_rate(T_C, c_wt)
    assert lam >= 0.0
    for t_h in (1.0, 240.0, 1e4):
        assert mt.one_minus_omega(T_C, c_wt, t_h) == pytest.approx(np.exp(-lam * t_h / 24.0), rel=1e-13)
    # over-saturation clips to the saturated rate; dry points do not degrade
    assert mc.degradation_rate(T_C, 3.0) == pytest.approx(mc.degradation_rate(T_C, 1.5), rel=1e-15)
    assert mc.degradation_rate(T_C, 0.0) == 0.0
    # backward Euler over many small steps approaches the closed form
    W, n = 1.0, 4000
    for _ in range(n):
        W = mc.degradation_step(W, T_C, c_wt, 1e4 / n)
    assert W == pytest.approx(mt.one_minus_omega(T_C, c_wt, 1e4), rel=2e-3, abs=1e-12)


def test_activations_special_values():
    a = np.array([-50.0, -1.0, 0.0, 1.0, 50.0])
    np.testing.assert_allclose(sg.silu(a), a / (1.0 + np.exp(-a)), rtol=1e-15)
    assert sg.silu(np.array([0.0]))[0] == 0.0
    assert sg.silu(np.array([50.0]))[0] == pytest.approx(50.0, rel=1e-15)
    assert abs(sg.silu(np.array([-50.0]))[0]) < 1e-19
    # silu'(0) = 1/2, silu' -> 1 and 0 at the ends; softplus(0) = ln 2, stable tails
    assert sg.dsilu(np.array([0.0]))[0] == 0.5
    assert sg.dsilu(np.array([40.0]))[0] == pytest.approx(1.0, rel=1e-12)
    assert abs(sg.dsilu(np.array([-40.0]))[0]) < 1e-15
    assert sg.softplus(np.array([0.0]))[0] == pytest.approx(np.log(2.0), rel=1e-15)
    assert sg.softplus(np.array([800.0]))[0] == 800.0
    assert sg.softplus(np.array([-800.0]))[0] == 0.0
    assert sg.softplus(np.array([-30.0]))[0] == pytest.approx(np.exp(-30.0), rel=1e-12)


def test_forward_by_hand():
    """A 2 -> 2 -> 1 network with chosen weights, evaluated by hand: the hidden
    layer applies SiLU, the output layer is linear."""
    W1 = np.array([[1.0, -2.0], [0.5, 0.0]])
    b1 = np.array([0.0, 1.0])
    W2 = np.array([[2.0], [-1.0]])
    b2 = np.array([0.25])
    x = np.array([[1.0, 2.0], [0.0, 0.0]])
    z, cache = sg.forward([(W1, b1), (W2, b2)], x)

    def silu1(v):
        return v / (1.0 + np.exp(-v))
    # row 0: pre-activations (1 + 1, -2 + 1) = (2, -1); row 1: (0, 1)
    h0 = np.array([silu1(2.0), silu1(-1.0)])
    h1 = np.array([0.0, silu1(1.0)])
    expect = np.array([[2 * h0[0] - h0[1] + 0.25], [2 * h1[0] - h1[1] + 0.25]])
    np.testing.assert_allclose(z, expect, rtol=1e-15)
    np.testing.assert_allclose(cache[0][1], [[2.0, -1.0], [0.0, 1.0]], rtol=1e-15)
