"""Pins of the macro time-step oracle (Secs. 3-5): closed forms and invariants
that a mistake in the transport discretisation, the implicit step, the Gauss
rule or the degradation update would break."""
import numpy as np
import pytest

import rve_inputs as ri
from oracle import macro as mo
from oracle import materials as mt


def slab_series(z, t, L, D, n_terms=200):
    """1-D diffusion on [0, L], value 1 held at z = 0, zero flux at z = L, zero
    initially: 1 - sum 4/((2n+1) pi) sin(k_n z) exp(-k_n^2 D t), k_n = (2n+1) pi / (2L)."""
    n = np.arange(n_terms)[:, None]
    k = (2 * n + 1) * np.pi / (2 * L)
    return 1.0 - (4.0 / ((2 * n + 1) * np.pi) * np.sin(k * z[None]) * np.exp(-k ** 2 * D * t)).sum(axis=0)


def test_transient_slab_matches_series():
    xyz, tets = ri.kuhn_grid(2, 2, 40, lengths=(0.05, 0.05, 1.0))
    face = xyz[:, 2] <= 1e-12
    K, C = mo.assemble(xyz, tets, np.eye(3), 1.0)
    psi = np.zeros(len(xyz))
    dt, n = 0.002, 50
    for _ in range(n):
        psi = mo.backward_euler_step(K, C, psi, dt, face, 1.0)
    exact = slab_series(xyz[:, 2], dt * n, 1.0, 1.0)
    assert np.abs(psi - exact).max() < 1e-2


def test_steady_state_and_conservation():
    xyz, tets, face = ri.plate(6, 3, 2)
    KT = np.diag([0.4, 0.3, 0.25])
    K, C = mo.assemble(xyz, tets, KT, 2.0e6)
    # long implicit steps reach the held face value everywhere (zero flux elsewhere)
    psi = np.full(len(xyz), 20.0)
    for _ in range(3):
        psi = mo.backward_euler_step(K, C, psi, 1e9, face, 60.0)
    assert np.abs(psi - 60.0).max() < 1e-8
    # without a held face the capacity-weighted content is conserved exactly
    rng = np.random.default_rng(0)
    psi = rng.uniform(0, 1, len(xyz))
    content = C @ psi
    new = mo.backward_euler_step(K, C, psi, 10.0, np.zeros(len(xyz), bool), 0.0)
    assert abs((C @ new).sum() - content.sum()) <= 1e-12 * abs(content.sum())


def test_capacity_and_gauss_rule_exact():
    xyz, tets, face = ri.plate(3, 2, 2)
    vol, g = mo.p1_geometry(xyz, tets)
    assert np.isclose(vol.sum(), np.prod(ri.PLATE_LENGTHS), rtol=1e-12)
    # barycentric gradients sum to zero and reproduce x: sum_a x_a grad lambda_a = I
    assert np.abs(g.sum(axis=1)).max() < 1e-9 * np.abs(g).max()
    Ix = np.einsum("tai,taj->tij", xyz[tets], g)
    assert np.abs(Ix - np.eye(3)).max() < 1e-10
    # capacity matrix: total = capacity x volume, each element's row sums |T|/4
    K, C = mo.assemble(xyz, tets, np.eye(3), 3.0)
    assert np.isclose(C.sum(), 3.0 * vol.sum(), rtol=1e-12)
    # stiffness annihilates constants
    assert np.abs(K @ np.ones(len(xyz))).max() < 1e-9 * abs(K).max()
    # the 4-point rule integrates lambda_a lambda_b exactly: |T| (1 + delta_ab) / 20
    w = np.full(4, 0.25)
    M = np.einsum("g,ga,gb->ab", w, mo.GAUSS_BARY, mo.GAUSS_BARY)
    assert np.allclose(M, (np.ones((4, 4)) + np.eye(4)) / 20.0, atol=1e-15)
    # and a quadratic in space exactly: int x^2 over a tetrahedron
    X = xyz[tets[0]]
    pts = mo.GAUSS_BARY @ X
    quad = vol[0] * 0.25 * (pts[:, 0] ** 2).sum()
    exact = vol[0] / 20.0 * ((X[:, 0].sum()) ** 2 + (X[:, 0] ** 2).sum())
    assert np.isclose(quad, exact, rtol=1e-12)


@pytest.mark.parametrize("T_C,c_wt", [(60.0, 1.5), (40.0, 0.75), (25.0, 0.1)])
def test_degradation_backward_euler(T_C, c_wt):
    lam = mt.moisture_fraction(c_wt) * mt.alpha_of_T(T_C)
    assert lam > 0
    W = np.ones(1)
    dt_h, n = 100.0, 37
    for _ in range(n):
        W = mo.degradation_step(W, T_C, c_wt, dt_h)
    assert np.isclose(W[0], (1.0 + dt_h / 24.0 * lam) ** (-n), rtol=1e-13)
    # small steps approach the closed form of Eq. Eq_Model_final1 at first order
    t_h = 1.0e4
    Wf = np.ones(1)
    for _ in range(20000):
        Wf = mo.degradation_step(Wf, T_C, c_wt, t_h / 20000)
    closed = mt.one_minus_omega(T_C, c_wt, t_h)
    assert abs(Wf[0] - closed) < 5e-4 * closed
    # the equivalent exposure time reproduces W through the closed form
    t_eq = mo.equivalent_time(W, T_C, c_wt)
    assert np.isclose(mt.one_minus_omega(T_C, c_wt, t_eq)[0], W[0], rtol=1e-13)


def test_dry_points_do_not_degrade_and_equivalent_time_edge_cases():
    W = mo.degradation_step(np.ones(3), np.array([60.0, 60.0, 20.0]), np.array([0.0, 1.5, 0.0]), 500.0)
    assert W[0] == 1.0 and W[2] == 1.0 and W[1] < 1.0
    # no moisture now: handed over as undegraded, the miss is 1 - W
    T, c, Wd = np.array([60.0, 60.0]), np.array([0.0, -1e-4]), np.array([1.0, 0.9])
    t = mo.equivalent_time(Wd, T, c)
    assert (t == 0.0).all()
    assert np.allclose(mo.handover_error(Wd, T, c), [0.0, 0.1])
    assert np.allclose(mt.one_minus_omega(T, c, t), 1.0)


def test_march_moisture_front_and_thermal_equilibrium():
    xyz, tets, face = ri.plate(4, 2, 8)
    ex = ri.PlateExposure()
    out = mo.march(xyz, tets, face, np.diag([0.4, 0.4, 0.3]), ex.rho_cp, np.diag([1.2e-12, 1.2e-12, 8e-13]),
                   ex.T0_C, ex.c0_wt, ex.T_face_C, ex.c_face_wt, dt_h=100.0, n_steps=4)
    last = out[-1]
    # heat diffuses through 10 mm within one 100 h step; moisture is still a front
    assert np.abs(last["T"] - 60.0).max() < 1e-6
    z = xyz[:, 2]
    assert last["c"][z <= 0].min() == pytest.approx(1.5)
    assert last["c"][z >= z.max()].max() < 0.5
    # deeper points are wetter later and degrade less
    assert np.all(np.diff([o["W"].mean() for o in out]) < 0)
    assert ((last["W"] > 0) & (last["W"] <= 1)).all()
