"""Pins for oracle.materials: printed constants of the degradation model (Sec. 4)
and closed-form properties of the constituent tensors."""
import json
import os

import numpy as np
import pytest

from oracle import materials as mt


@pytest.fixture(scope="module")
def deg(golden_dir):
    with open(os.path.join(golden_dir, "degradation.json")) as f:
        return json.load(f)


def test_beta_refit_kelvin_matches_printed(deg):
    # Eq. alphaT_LSF with T in kelvin reproduces the printed beta to ~1 %.
    T = [float(k) for k in deg["alpha_per_day"]]
    a = [deg["alpha_per_day"][k] for k in deg["alpha_per_day"]]
    beta_K = mt.fit_beta(T, a, deg["Tg_C"], kelvin=True)
    assert beta_K == pytest.approx(-0.001701, abs=2e-6)
    assert abs(beta_K / deg["beta_per_day"] - 1.0) < 0.015
    # the Celsius reading is off by more than a factor two: kelvin is the reading
    beta_C = mt.fit_beta(T, a, deg["Tg_C"], kelvin=False)
    assert abs(beta_C / deg["beta_per_day"] - 1.0) > 1.0


def test_alpha_model_close_to_fitted_rates(deg):
    for T, a_fit in deg["alpha_per_day"].items():
        a_model = mt.alpha_of_T(float(T), deg["beta_per_day"], deg["Tg_C"])
        assert a_model > 0
        assert abs(a_model - a_fit) / a_fit < 0.15
    # rate increases with temperature and vanishes at 0 K
    assert mt.alpha_of_T(-273.15) == pytest.approx(0.0, abs=1e-15)
    assert mt.alpha_of_T(25.0) < mt.alpha_of_T(60.0) < mt.alpha_of_T(80.0)


def test_degradation_closed_form_values(deg):
    # 1 - omega after 112 days fully saturated (c = 1.5 wt% -> gamma = 1)
    t_h = deg["verification_exposure_days"] * 24.0
    vals = mt.one_minus_omega([25.0, 60.0, 80.0], 1.5, t_h)
    np.testing.assert_allclose(vals, [0.77192, 0.71246, 0.66562], atol=5e-5)
    # dry sample does not degrade; t = 0 does not degrade
    assert mt.one_minus_omega(60.0, 0.0, 1e4) == 1.0
    assert mt.one_minus_omega(60.0, 1.5, 0.0) == 1.0
    # moisture enters linearly in the exponent
    w_half = mt.one_minus_omega(60.0, 0.75, t_h)
    assert w_half == pytest.approx(np.sqrt(mt.one_minus_omega(60.0, 1.5, t_h)), rel=1e-12)


def test_backward_euler_converges_first_order():
    # Eq. Model_RateForm discretised by backward Euler tends to Eq. Model_final1
    exact = mt.one_minus_omega(80.0, 1.5, 112 * 24.0)
    errs = [abs(mt.one_minus_omega_backward_euler(80.0, 1.0, 112.0, n) - exact) for n in (10, 20, 40, 80)]
    ratios = [errs[i] / errs[i + 1] for i in range(3)]
    for r in ratios:
        assert 1.9 < r < 2.1
    assert mt.one_minus_omega_backward_euler(80.0, 1.0, 112.0, 20000) == pytest.approx(exact, rel=1e-5)


def test_iso_stiffness_engineering_constants():
    E, nu = 3.5e9, 0.35
    S = np.linalg.inv(mt.iso_stiffness(E, nu))
    assert 1 / S[0, 0] == pytest.approx(E)
    assert -S[0, 1] / S[0, 0] == pytest.approx(nu)
    assert 1 / S[3, 3] == pytest.approx(E / (2 * (1 + nu)))   # engineering shear


def test_ti_reduces_to_isotropic():
    E, nu = 10e9, 0.3
    G = E / (2 * (1 + nu))
    for axis in ([1, 0, 0], [0.3, -0.5, 0.8]):
        D = mt.ti_stiffness(E, E, G, nu, nu, axis)
        np.testing.assert_allclose(D, mt.iso_stiffness(E, nu), rtol=1e-12, atol=1e-3)


def test_ti_engineering_constants_along_fibre():
    E1, E2, G12, n12, n23 = 45e9, 12e9, 5e9, 0.28, 0.4
    # axis along global y: E_yy = E1, transverse E = E2, G_xy = G12, G_zx = E2/(2(1+nu23))
    D = mt.ti_stiffness(E1, E2, G12, n12, n23, [0, 1, 0])
    S = np.linalg.inv(D)
    assert 1 / S[1, 1] == pytest.approx(E1, rel=1e-12)
    assert 1 / S[0, 0] == pytest.approx(E2, rel=1e-12)
    assert 1 / S[2, 2] == pytest.approx(E2, rel=1e-12)
    assert -S[0, 1] / S[1, 1] == pytest.approx(n12, rel=1e-12)   # nu_yx with y the fibre
    assert -S[2, 0] / S[0, 0] == pytest.approx(n23, rel=1e-12)
    assert 1 / S[3, 3] == pytest.approx(G12, rel=1e-12)          # xy contains the fibre
    assert 1 / S[4, 4] == pytest.approx(G12, rel=1e-12)          # yz contains the fibre
    assert 1 / S[5, 5] == pytest.approx(E2 / (2 * (1 + n23)), rel=1e-12)
    assert np.all(np.linalg.eigvalsh(D) > 0)


def test_ti_frame_invariance():
    t = np.array([0.2, 0.9, -0.4])
    D1 = mt.ti_stiffness(45e9, 12e9, 5e9, 0.28, 0.4, t, helper=np.array([0, 0, 1.0]))
    D2 = mt.ti_stiffness(45e9, 12e9, 5e9, 0.28, 0.4, t, helper=np.array([1.0, 0.3, 0]))
    np.testing.assert_allclose(D1, D2, rtol=1e-12, atol=1e-3)


def test_rotation_is_tensorial():
    # rotating a stiffness then rotating back is the identity; energies invariant
    rng = np.random.default_rng(3)
    A = rng.normal(size=(6, 6))
    D = A @ A.T + 6 * np.eye(6)
    R = mt.frame_from_axis(rng.normal(size=3))
    D2 = mt.rotate_stiffness(mt.rotate_stiffness(D, R), R.T)
    np.testing.assert_allclose(D2, D, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(np.sort(np.linalg.eigvalsh(mt.rotate_stiffness(mt.iso_stiffness(1, .2), R))),
                               np.sort(np.linalg.eigvalsh(mt.iso_stiffness(1, .2))), rtol=1e-12)


def test_transport_tensor():
    t = np.array([1.0, 2.0, 2.0]) / 3
    k = mt.transport_tensor(0.6, 0.35, t)
    assert t @ k @ t == pytest.approx(0.6)
    n = np.cross(t, [0, 0, 1.0])
    n /= np.linalg.norm(n)
    assert n @ k @ n == pytest.approx(0.35)
