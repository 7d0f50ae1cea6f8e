"""Pins for oracle.surrogate: analytic gradients against central finite
differences, SPD reconstruction, factor round trip, Adam on a quadratic."""
import numpy as np

from oracle import surrogate as sg


def small_params(seed=0):
    return sg.init_params(seed, width=16, depth=2, n_in=8, n_out=33)


def test_gradients_match_finite_differences():
    rng = np.random.default_rng(1)
    params = small_params()
    x = rng.normal(size=(5, 8))
    target = rng.normal(size=(5, 33)) * 0.3 + 1.0
    sigma = np.full(33, 0.7)
    _, grads = sg.loss_and_grads(params, x, target, sigma)
    h = 1e-6
    for l, (W, b) in enumerate(params):
        for (i, j) in [(0, 0), (W.shape[0] - 1, W.shape[1] - 1), (2, 3)]:
            Wp = [(w.copy(), bb.copy()) for w, bb in params]
            Wm = [(w.copy(), bb.copy()) for w, bb in params]
            Wp[l][0][i, j] += h
            Wm[l][0][i, j] -= h
            fd = (sg.loss_and_grads(Wp, x, target, sigma)[0] - sg.loss_and_grads(Wm, x, target, sigma)[0]) / (2 * h)
            assert abs(fd - grads[l][0][i, j]) <= 1e-6 * max(1.0, abs(fd))
        k = b.shape[0] - 1
        Bp = [(w.copy(), bb.copy()) for w, bb in params]
        Bm = [(w.copy(), bb.copy()) for w, bb in params]
        Bp[l][1][k] += h
        Bm[l][1][k] -= h
        fd = (sg.loss_and_grads(Bp, x, target, sigma)[0] - sg.loss_and_grads(Bm, x, target, sigma)[0]) / (2 * h)
        assert abs(fd - grads[l][1][k]) <= 1e-6 * max(1.0, abs(fd))


def test_reconstruction_is_spd_for_any_output():
    z = np.random.default_rng(2).normal(size=(50, 33)) * 3
    C, K, D = sg.tensors_from_factors(sg.factor_entries(z))
    for T in (C, K, D):
        np.testing.assert_allclose(T, np.swapaxes(T, 1, 2))
        assert np.linalg.eigvalsh(T).min() > 0


def test_factor_round_trip():
    rng = np.random.default_rng(3)
    A = rng.normal(size=(4, 6, 6))
    C = A @ np.swapaxes(A, 1, 2) + 6 * np.eye(6)
    B3 = rng.normal(size=(4, 3, 3))
    K = B3 @ np.swapaxes(B3, 1, 2) + np.eye(3)
    Lv = sg.factors_from_tensors(C, K, K)
    C2, K2, D2 = sg.tensors_from_factors(Lv)
    np.testing.assert_allclose(C2, C, rtol=1e-12)
    np.testing.assert_allclose(K2, K, rtol=1e-12)
    assert (Lv[:, sg.DIAG] > 0).all()


def test_adam_minimises_a_quadratic():
    params = [(np.array([[3.0]]), np.array([-2.0]))]
    state = [(np.zeros((1, 1)), np.zeros((1, 1)), np.zeros(1), np.zeros(1))]
    for t in range(1, 3001):
        W, b = params[0]
        params = sg.adam_step(params, [(2 * W, 2 * b)], state, 0.01, t)
    assert abs(params[0][0][0, 0]) < 1e-3 and abs(params[0][1][0]) < 1e-3
