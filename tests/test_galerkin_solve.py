"""The energy-optimal warm start's small solve, c = G^+ g with eigenvalues at or
below rel times the largest dropped (rve_debug_galerkin_solve, host code of the
library; no GPU needed).  Checked against the textbook solutions: a direct solve
for a well-conditioned G, the truncated eigen-expansion (numpy.linalg.eigh) for a
nearly singular one, the rank-one closed form, and the argument and error
contract."""
import numpy as np
import pytest


@pytest.fixture(scope="module")
def rve():
    from paper_1610_03484_gb300 import _build
    _build.build()
    import paper_1610_03484_gb300 as pkg
    pkg.load_library()
    return pkg


def spd(n, seed, cond=10.0):
    rng = np.random.default_rng(seed)
    Q, _ = np.linalg.qr(rng.normal(size=(n, n)))
    lam = np.geomspace(1.0, 1.0 / cond, n)
    return (Q * lam) @ Q.T, Q, lam


@pytest.mark.parametrize("n", [1, 2, 3, 4, 8])
def test_well_conditioned_equals_direct_solve(rve, n):
    G, _, _ = spd(n, n)
    g = np.random.default_rng(100 + n).normal(size=n)
    np.testing.assert_allclose(rve.galerkin_solve(G, g), np.linalg.solve(G, g), rtol=1e-12, atol=1e-12)


def test_only_the_symmetric_part_counts(rve):
    G, _, _ = spd(4, 7)
    S = np.random.default_rng(8).normal(size=(4, 4))
    g = np.arange(1.0, 5.0)
    np.testing.assert_allclose(rve.galerkin_solve(G + (S - S.T), g), np.linalg.solve(G, g), rtol=1e-12)


@pytest.mark.parametrize("rel", [1e-12, 1e-8, 1e-3])
def test_nearly_singular_is_the_truncated_expansion(rve, rel):
    """Eigenvalues 1, 1e-5, 1e-10, 1e-15: the ones above rel * 1 are kept."""
    rng = np.random.default_rng(3)
    Q, _ = np.linalg.qr(rng.normal(size=(4, 4)))
    lam = np.array([1.0, 1e-5, 1e-10, 1e-15])
    G = (Q * lam) @ Q.T
    g = rng.normal(size=4)
    keep = lam > rel
    ref = Q[:, keep] @ ((Q[:, keep].T @ g) / lam[keep])
    c = rve.galerkin_solve(G, g, rel)
    np.testing.assert_allclose(c, ref, rtol=1e-6 if rel < 1e-9 else 1e-9)
    # the kept part solves the system on its eigen-space: G c = projection of g
    np.testing.assert_allclose(G @ c, Q[:, keep] @ (Q[:, keep].T @ g), atol=1e-6 * np.abs(g).max())


def test_rank_one_closed_form(rve):
    """G = s s^T: c = (s . g) s / |s|^4, the minimum-norm solution."""
    s = np.array([1.0, -2.0, 0.5])
    g = np.array([0.3, 1.0, -0.7])
    c = rve.galerkin_solve(np.outer(s, s), g)
    np.testing.assert_allclose(c, (s @ g) * s / (s @ s) ** 2, rtol=1e-12)


def test_errors(rve):
    with pytest.raises(rve.RveError) as e:
        rve.galerkin_solve(np.zeros((3, 3)), np.ones(3))            # no positive eigenvalue
    assert e.value.code == -5
    G = np.eye(2)
    G[0, 1] = np.nan
    with pytest.raises(rve.RveError) as e:
        rve.galerkin_solve(G, np.ones(2))
    assert e.value.code == -5
    with pytest.raises(rve.RveError) as e:
        rve.galerkin_solve(np.eye(9), np.ones(9))                    # n above 8
    assert e.value.code == -1
    with pytest.raises(rve.RveError) as e:
        rve.galerkin_solve(np.eye(2), np.ones(2), rel=-1.0)
    assert e.value.code == -1
