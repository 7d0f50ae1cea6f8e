"""Pins for oracle.surrogate: analytic gradients against central finite
differences, SPD reconstruction, factor round trip, Adam on a quadratic and
against the published update (Kingma & Ba 2015, Algorithm 1) evaluated by hand
for two steps, with planted mistakes (no bias correction, swapped betas)."""
import numpy as np
import pytest

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


# Adam (Kingma & Ba 2015, Algorithm 1): m_t = b1 m + (1 - b1) g,
# v_t = b2 v + (1 - b2) g^2, theta -= lr * m_t / (1 - b1^t) / (sqrt(v_t / (1 - b2^t)) + eps).
# Hand evaluation for two steps from m = v = 0, b1 = 0.9, b2 = 0.999:
#   step 1: m_hat = g1, v_hat = g1^2, so the step is -lr * g1 / (|g1| + eps);
#   step 2: m_hat = (0.09 g1 + 0.1 g2) / 0.19,
#           v_hat = (0.000999 g1^2 + 0.001 g2^2) / 0.001999.
# With g1 = 2, g2 = -1: m_hat = 8/19 and v_hat = 4996/1999.
# With g1 = -0.003, g2 = 0.005: m_hat = 0.00023/0.19 and
#   v_hat = (0.000999 * 9e-6 + 0.001 * 25e-6) / 0.001999 = 3.3991e-8 / 0.001999.
def _adam_two_steps(theta0, g1, g2, lr=0.01):
    params = [(np.array([[theta0[0]]]), np.array([theta0[1]]))]
    state = [(np.zeros((1, 1)), np.zeros((1, 1)), np.zeros(1), np.zeros(1))]
    p1 = sg.adam_step(params, [(np.array([[g1[0]]]), np.array([g1[1]]))], state, lr, 1)
    p2 = sg.adam_step(p1, [(np.array([[g2[0]]]), np.array([g2[1]]))], state, lr, 2)
    return (p1[0][0][0, 0], p1[0][1][0]), (p2[0][0][0, 0], p2[0][1][0])


def test_adam_matches_published_update_by_hand():
    lr, eps = 0.01, 1e-8
    (w1, b1), (w2, b2) = _adam_two_steps((1.5, -0.25), (2.0, -0.003), (-1.0, 0.005), lr)
    # first step: -lr * sign(g) up to eps / |g|
    assert w1 == pytest.approx(1.5 - lr * 2.0 / (2.0 + eps), rel=1e-15)
    assert b1 == pytest.approx(-0.25 + lr * 0.003 / (0.003 + eps), rel=1e-15)
    assert abs((w1 - 1.5) + lr) < 1e-10 and abs((b1 + 0.25) - lr) < 1e-7
    # second step
    assert w2 == pytest.approx(w1 - lr * (8.0 / 19.0) / (np.sqrt(4996.0 / 1999.0) + eps), rel=1e-14)
    assert b2 == pytest.approx(b1 - lr * (0.00023 / 0.19) / (np.sqrt(3.3991e-8 / 0.001999) + eps), rel=1e-12)


def test_planted_adam_mistakes_are_caught(monkeypatch):
    import oracle.surrogate as osg
    good = _adam_two_steps((1.5, -0.25), (2.0, -0.003), (-1.0, 0.005))
    orig = osg.adam_step

    def no_bias_correction(params, grads, state, lr, t, b1=0.9, b2=0.999, eps=1e-8):
        # c1 = c2 = 1: the same update without the bias correction
        out = []
        for l, ((W, b), (gW, gb)) in enumerate(zip(params, grads)):
            mW, vW, mb, vb = state[l]
            mW = b1 * mW + (1 - b1) * gW
            vW = b2 * vW + (1 - b2) * gW * gW
            mb = b1 * mb + (1 - b1) * gb
            vb = b2 * vb + (1 - b2) * gb * gb
            state[l] = (mW, vW, mb, vb)
            out.append((W - lr * mW / (np.sqrt(vW) + eps), b - lr * mb / (np.sqrt(vb) + eps)))
        return out

    for bad in (no_bias_correction,
                lambda p, g, s, lr, t: orig(p, g, s, lr, t, b1=0.999, b2=0.9)):
        monkeypatch.setattr(osg, "adam_step", bad)
        got = _adam_two_steps((1.5, -0.25), (2.0, -0.003), (-1.0, 0.005))
        assert abs(got[1][0] - good[1][0]) > 1e-4 or abs(got[0][0] - good[0][0]) > 1e-4
        monkeypatch.undo()
