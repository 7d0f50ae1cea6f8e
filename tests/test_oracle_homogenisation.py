"""Pins for oracle.fem: what the physics and the mathematics fix about the RVE
cell problems of Sec. 2, independent of the oracle's own arithmetic.

* single phase: the homogenised tensor is the material tensor, every BC, every p;
* laminate aligned with grid planes, periodic BC: exact textbook laminate
  averages (derived below from continuity of normal stress / flux and of
  in-plane strain / gradient);
* Voigt >= Dirichlet >= periodic >= Neumann >= Reuss in the Loewner order, and
  monotone decrease in p (nested minimisation sets, Sec. 2 and Sec. 7);
* symmetry, positive definiteness, Hill-Mandel (Eq. Hill_prin): the energy
  form equals eps_i . sigma_bar_j with sigma_bar the volume average;
* brute force: the paper's own bordered total-field system with
  sigma_bar = D^T lambda / V (Eqs. eq_RVE_disc_Eqs, eq_homo_stress) agrees with
  the elimination route on tiny meshes, for all three BCs and p = 1..3;
* planted mistakes in the oracle (dropped factor, wrong sign, transposed
  operand) each break at least one of these pins.
"""
import numpy as np
import pytest

import rve_inputs as ri
from oracle import fem
from oracle import materials as mt

BCS = (fem.BC_DIRICHLET, fem.BC_PERIODIC, fem.BC_NEUMANN)


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def loewner_ge(A, B, tol):
    """A >= B up to tol * ||B||."""
    return np.linalg.eigvalsh(0.5 * ((A - B) + (A - B).T)).min() >= -tol * np.linalg.norm(B)


def weave_tensors(grid, scale_mech=1e9, scale_k=1.0, scale_d=1e-12):
    xyz, tets, ph, tg = ri.weave_rve(*grid)
    D, K, Dd = mt.element_tensors(ph, tg, ri.NOMINAL_MATRIX, ri.NOMINAL_YARN)
    return xyz, tets, D / scale_mech, K / scale_k, Dd / scale_d


@pytest.mark.parametrize("p", [1, 2, 3])
@pytest.mark.parametrize("bc", BCS)
def test_single_phase_exact(p, bc):
    grid = (2, 2, 2)
    xyz, tets = ri.kuhn_grid(*grid)
    D = mt.ti_stiffness(45, 12, 5, 0.28, 0.4, [0.3, 0.8, -0.2])
    k = mt.transport_tensor(0.6, 0.35, [0.3, 0.8, -0.2])
    sm = fem.homogenise_field(xyz, tets, grid, p, bc, np.repeat(D[None], len(tets), 0), 3)
    ss = fem.homogenise_field(xyz, tets, grid, p, bc, np.repeat(k[None], len(tets), 0), 1)
    assert rel(sm.tensor, D) < 1e-12
    assert rel(ss.tensor, k) < 1e-12
    assert rel(sm.sigma_bar.T, D) < 1e-12
    assert np.abs(sm.u_tilde).max() < 1e-10


def laminate_average(Ds, fr, n_idx, t_idx):
    """Textbook laminate: normal stress / flux and in-plane strain / gradient
    continuous across layers; fr = volume fractions."""
    Ds = [np.asarray(D) for D in Ds]
    nn = np.ix_(n_idx, n_idx)
    nt = np.ix_(n_idx, t_idx)
    tn = np.ix_(t_idx, n_idx)
    tt = np.ix_(t_idx, t_idx)
    avg = lambda f: sum(w * f(D) for w, D in zip(fr, Ds))
    inv_nn = lambda D: np.linalg.inv(D[nn])
    Cnn = np.linalg.inv(avg(inv_nn))
    Cnt = Cnn @ avg(lambda D: inv_nn(D) @ D[nt])
    Ctn = avg(lambda D: D[tn] @ inv_nn(D)) @ Cnn
    Ctt = avg(lambda D: D[tt] - D[tn] @ inv_nn(D) @ D[nt]) + \
        avg(lambda D: D[tn] @ inv_nn(D)) @ Cnn @ avg(lambda D: inv_nn(D) @ D[nt])
    n = len(n_idx) + len(t_idx)
    C = np.zeros((n, n))
    C[nn], C[nt], C[tn], C[tt] = Cnn, Cnt, Ctn, Ctt
    return C


@pytest.mark.parametrize("p", [1, 2])
def test_laminate_periodic_exact(p):
    grid = (2, 2, 4)
    xyz, tets = ri.kuhn_grid(*grid)
    phase = ri.layered(xyz, tets, [0, 1, 1, 0], nz=4)
    D0 = mt.iso_stiffness(3.5, 0.35)
    D1 = mt.ti_stiffness(45, 12, 5, 0.28, 0.4, [1.0, 0.4, 0.0])
    k0 = 0.2 * np.eye(3)
    k1 = mt.transport_tensor(0.6, 0.35, [1.0, 0.4, 0.0])
    Dm = np.where(phase[:, None, None] == 0, D0, D1)
    km = np.where(phase[:, None, None] == 0, k0, k1)
    sm = fem.homogenise_field(xyz, tets, grid, p, fem.BC_PERIODIC, Dm, 3)
    ss = fem.homogenise_field(xyz, tets, grid, p, fem.BC_PERIODIC, km, 1)
    # Voigt indices: normal set {33, 23, 31}, in-plane set {11, 22, 12}
    C_lam = laminate_average([D0, D1], [0.5, 0.5], [2, 4, 5], [0, 1, 3])
    K_lam = laminate_average([k0, k1], [0.5, 0.5], [2], [0, 1])
    assert rel(sm.tensor, C_lam) < 1e-11
    assert rel(ss.tensor, K_lam) < 1e-11
    # and not the Voigt or Reuss average
    assert rel(0.5 * (D0 + D1), C_lam) > 1e-2


@pytest.fixture(scope="module")
def weave_results():
    grid = (4, 4, 2)
    xyz, tets, D, K, Dd = weave_tensors(grid)
    out = {}
    for p in (1, 2):
        for bc in BCS:
            out[(p, bc, "C")] = fem.homogenise_field(xyz, tets, grid, p, bc, D, 3)
            out[(p, bc, "K")] = fem.homogenise_field(xyz, tets, grid, p, bc, K, 1)
    m = fem.build_nodal_mesh(xyz, tets, grid, 1)
    w = m.vol / m.vol.sum()
    out["voigt_C"] = np.einsum("t,tij->ij", w, D)
    out["reuss_C"] = np.linalg.inv(np.einsum("t,tij->ij", w, np.linalg.inv(D)))
    out["voigt_K"] = np.einsum("t,tij->ij", w, K)
    out["reuss_K"] = np.linalg.inv(np.einsum("t,tij->ij", w, np.linalg.inv(K)))
    return out


@pytest.mark.parametrize("f", ["C", "K"])
@pytest.mark.parametrize("p", [1, 2])
def test_bounds_and_bc_ordering(weave_results, f, p):
    r = weave_results
    dirich, per, neu = (r[(p, bc, f)].tensor for bc in BCS)
    tol = 1e-10
    assert loewner_ge(r["voigt_" + f], dirich, tol)
    assert loewner_ge(dirich, per, tol)
    assert loewner_ge(per, neu, tol)
    assert loewner_ge(neu, r["reuss_" + f], tol)
    # strict: the three BCs give different answers on a heterogeneous RVE
    assert rel(dirich, per) > 1e-4 and rel(per, neu) > 1e-4


@pytest.mark.parametrize("f", ["C", "K"])
@pytest.mark.parametrize("bc", BCS)
def test_p_monotone(weave_results, f, bc):
    a = weave_results[(1, bc, f)].tensor
    b = weave_results[(2, bc, f)].tensor
    assert loewner_ge(a, b, 1e-10)
    assert rel(a, b) > 1e-4


@pytest.mark.parametrize("f", ["C", "K"])
@pytest.mark.parametrize("bc", BCS)
def test_spd_symmetric_hill_mandel(weave_results, f, bc):
    s = weave_results[(2, bc, f)]
    T = s.tensor
    assert np.abs(T - T.T).max() < 1e-12 * np.abs(T).max()
    assert np.linalg.eigvalsh(T).min() > 0
    # Hill-Mandel: eps_i . sigma_bar_j (volume average) equals the energy form
    assert rel(s.sigma_bar.T, T) < 1e-9


@pytest.mark.parametrize("p", [1, 2, 3])
@pytest.mark.parametrize("bc", BCS)
def test_paper_bordered_route_matches(p, bc):
    grid = (2, 2, 2)
    xyz, tets = ri.kuhn_grid(*grid)
    ph = (np.arange(len(tets)) % 3 == 0).astype(np.uint8)
    tg = ri.random_unit_vectors(len(tets), 11)
    D, K, _ = mt.element_tensors(ph, tg, ri.NOMINAL_MATRIX, ri.NOMINAL_YARN)
    D = D / 1e9
    em = fem.homogenise_field(xyz, tets, grid, p, bc, D, 3).tensor
    pr = fem.paper_route(xyz, tets, grid, p, bc, D, 3)
    assert rel(em, pr) < 1e-11
    ek = fem.homogenise_field(xyz, tets, grid, p, bc, K, 1).tensor
    pk = fem.paper_route(xyz, tets, grid, p, bc, K, 1)
    assert rel(ek, pk) < 1e-11


def test_ti_frame_choice_does_not_change_tensor():
    grid = (2, 2, 2)
    xyz, tets = ri.kuhn_grid(*grid)
    tg = ri.random_unit_vectors(len(tets), 5)
    D1 = np.stack([mt.ti_stiffness(45, 12, 5, .28, .4, t, helper=np.array([0, 0, 1.0])) for t in tg])
    D2 = np.stack([mt.ti_stiffness(45, 12, 5, .28, .4, t, helper=np.array([0.6, -0.7, 0.1])) for t in tg])
    a = fem.homogenise_field(xyz, tets, grid, 2, fem.BC_PERIODIC, D1, 3).tensor
    b = fem.homogenise_field(xyz, tets, grid, 2, fem.BC_PERIODIC, D2, 3).tensor
    assert rel(a, b) < 1e-12


# ------------------------------------------------------------ planted mistakes
def _laminate_error_with(monkeypatch, target, attr, bad):
    monkeypatch.setattr(target, attr, bad)
    grid = (2, 2, 4)
    xyz, tets = ri.kuhn_grid(*grid)
    phase = ri.layered(xyz, tets, [0, 1, 1, 0], nz=4)
    D0 = mt.iso_stiffness(3.5, 0.35)
    D1 = mt.ti_stiffness(45, 12, 5, 0.28, 0.4, [1.0, 0.4, 0.0])
    Dm = np.where(phase[:, None, None] == 0, D0, D1)
    sm = fem.homogenise_field(xyz, tets, grid, 1, fem.BC_PERIODIC, Dm, 3)
    return rel(sm.tensor, laminate_average([D0, D1], [0.5, 0.5], [2, 4, 5], [0, 1, 3]))


def test_planted_mistakes_are_caught(monkeypatch):
    # 1. engineering-shear factor dropped from the unit macro strains
    orig = fem.unit_macro_fields

    def bad_macros(nc):
        out = orig(nc)
        if nc == 3:
            out = [2 * E if J >= 3 else E for J, E in enumerate(out)]
        return out
    assert _laminate_error_with(monkeypatch, fem, "unit_macro_fields", bad_macros) > 1e-2
    monkeypatch.undo()

    # 2. sign error in the right-hand side (b = +a(eps y, phi))
    orig_load = fem.element_macro_load
    assert _laminate_error_with(monkeypatch, fem, "element_macro_load",
                                lambda K, u: -orig_load(K, u)) > 1e-2
    monkeypatch.undo()

    # 3. transposed Jacobian inverse in the barycentric gradients
    orig_build = fem.build_nodal_mesh

    def bad_build(*a, **k):
        m = orig_build(*a, **k)
        m.grad_lam = m.grad_lam.copy()
        m.grad_lam[:, 1:, :] = m.grad_lam[:, 1:, :].transpose(0, 2, 1)
        m.grad_lam[:, 0, :] = -m.grad_lam[:, 1:, :].sum(axis=1)
        return m
    assert _laminate_error_with(monkeypatch, fem, "build_nodal_mesh", bad_build) > 1e-2
    monkeypatch.undo()

    # 4. Voigt-to-tensor map without the minor symmetries
    from oracle import materials

    def bad_v2t(D):
        C = np.zeros((3, 3, 3, 3))
        for I, (i, j) in enumerate(materials.VOIGT):
            for J, (k, l) in enumerate(materials.VOIGT):
                C[i, j, k, l] = D[I, J]
        return C
    assert _laminate_error_with(monkeypatch, materials, "voigt_to_tensor", bad_v2t) > 1e-2
