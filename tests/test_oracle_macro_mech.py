"""Pins of the macro mechanics oracle (the linear elastic macro step of the
fully nested FE^2 scheme, Sec. 5): exact solutions that linear tetrahedra
reproduce, rigid-body modes, the traction resultant and a layered bar whose
end displacement has a closed form.  A transposed B, a wrong shear factor, a
Gauss point taken from the wrong tetrahedron or a lost face area fails one."""
import numpy as np
import pytest

import rve_inputs as ri
from oracle import macro as mo
from oracle import materials as mt


def spd6(rng, n):
    A = rng.standard_normal((n, 6, 6))
    return np.einsum("nij,nkj->nik", A, A) + 6.0 * np.eye(6)[None]


def rollers(xyz):
    """u_x = 0 on x = 0, u_y = 0 on y = 0, u_z = 0 on z = 0 (symmetry planes)."""
    fixed = np.zeros((len(xyz), 3), bool)
    for i in range(3):
        fixed[:, i] = xyz[:, i] <= 1e-12
    return fixed.reshape(-1)


def test_uniaxial_patch_test_is_exact():
    """Uniform isotropic C, traction t e_x on x = L, rollers on the three
    symmetry planes: u = (t/E x, -nu t/E y, -nu t/E z), sigma = t e_xx."""
    E, nu, t = 7.0e9, 0.3, 2.5e6
    xyz, tets = ri.kuhn_grid(4, 3, 2, lengths=(0.4, 0.2, 0.1))
    C = np.broadcast_to(mt.iso_stiffness(E, nu), (len(tets), 4, 6, 6))
    K = mo.elastic_assemble(xyz, tets, C)
    f = mo.traction_load(xyz, tets, xyz[:, 0] >= 0.4 - 1e-12, [t, 0, 0])
    u = mo.elastic_solve(K, f, rollers(xyz)).reshape(-1, 3)
    exact = np.stack([t / E * xyz[:, 0], -nu * t / E * xyz[:, 1], -nu * t / E * xyz[:, 2]], axis=1)
    assert np.abs(u - exact).max() < 1e-10 * np.abs(exact).max()
    sig = mo.gauss_stress(xyz, tets, u.reshape(-1), C)
    assert np.allclose(sig[..., 0], t, rtol=1e-9)
    assert np.abs(sig[..., 1:]).max() < 1e-9 * t


def test_linear_displacement_patch_test_anisotropic():
    """Every boundary node held at u = A y (A a full 3x3 gradient), no load,
    one anisotropic C for all Gauss points: the interior reproduces A y and
    the stress is C times the Voigt strain of sym(A) everywhere."""
    rng = np.random.default_rng(3)
    xyz, tets = ri.kuhn_grid(3, 3, 3)
    Cm = spd6(rng, 1)[0]
    C = np.broadcast_to(Cm, (len(tets), 4, 6, 6))
    A = rng.standard_normal((3, 3))
    ulin = xyz @ A.T
    bnd = ((xyz <= 1e-12) | (xyz >= 1 - 1e-12)).any(axis=1)
    fixed = np.repeat(bnd, 3)
    K = mo.elastic_assemble(xyz, tets, C)
    u = mo.elastic_solve(K, np.zeros(len(xyz) * 3), fixed, ulin.reshape(-1))
    assert np.abs(u - ulin.reshape(-1)).max() < 1e-12
    eps = np.array([A[0, 0], A[1, 1], A[2, 2], A[0, 1] + A[1, 0], A[1, 2] + A[2, 1], A[2, 0] + A[0, 2]])
    sig = mo.gauss_stress(xyz, tets, u, C)
    assert np.abs(sig - Cm @ eps).max() < 1e-11 * np.abs(Cm @ eps).max()


def test_rigid_modes_and_symmetry():
    rng = np.random.default_rng(5)
    xyz, tets = ri.kuhn_grid(2, 3, 2, lengths=(0.3, 0.5, 0.2))
    C = spd6(rng, len(tets) * 4).reshape(len(tets), 4, 6, 6)
    K = mo.elastic_assemble(xyz, tets, C)
    assert abs(K - K.T).max() < 1e-12 * abs(K).max()
    modes = []
    for i in range(3):
        m = np.zeros((len(xyz), 3))
        m[:, i] = 1.0
        modes.append(m)
        w = np.zeros(3)
        w[i] = 1.0
        modes.append(np.cross(w, xyz))       # infinitesimal rotation
    for m in modes:
        assert np.abs(K @ m.reshape(-1)).max() < 1e-10 * abs(K).max()
    # and K is positive on anything else: a random field with the rigid part removed
    Q, _ = np.linalg.qr(np.stack([m.reshape(-1) for m in modes], axis=1))
    v = rng.standard_normal(len(xyz) * 3)
    v -= Q @ (Q.T @ v)
    assert v @ (K @ v) > 0


def test_traction_resultant_and_moment():
    xyz, tets, _ = ri.plate(5, 3, 2)
    Lx, Ly, Lz = ri.PLATE_LENGTHS
    top = xyz[:, 2] >= Lz - 1e-12
    t = np.array([1.0e5, -2.0e5, -3.0e6])
    f = mo.traction_load(xyz, tets, top, t).reshape(-1, 3)
    assert np.allclose(f.sum(axis=0), t * Lx * Ly, rtol=1e-12)
    # the uniform load's resultant acts at the face centroid
    mx = (f[:, 2] * xyz[:, 0]).sum() / f[:, 2].sum()
    my = (f[:, 2] * xyz[:, 1]).sum() / f[:, 2].sum()
    assert mx == pytest.approx(Lx / 2, rel=1e-12) and my == pytest.approx(Ly / 2, rel=1e-12)
    assert (f[~top] == 0).all()


def test_layered_bar_closed_form():
    """Layers across x with their own Young's modulus (nu = 0), loaded by t e_x on
    x = L: uniaxial stress, u_x(L) = t sum h_i / E_i.  The Gauss points of a
    tetrahedron carry different C whose mean is the layer's, so a rule that
    ignored or misplaced per-point values would miss the closed form."""
    rng = np.random.default_rng(9)
    nx, L, t = 6, 0.6, 1.0e6
    xyz, tets = ri.kuhn_grid(nx, 2, 2, lengths=(L, 0.1, 0.1))
    E_layer = rng.uniform(2e9, 9e9, nx)
    layer = np.floor(xyz[tets].mean(axis=1)[:, 0] / (L / nx)).astype(int)
    C = np.zeros((len(tets), 4, 6, 6))
    spread = np.array([0.7, 1.1, 1.3, 0.9])                 # mean 1
    for q in range(4):
        C[:, q] = spread[q] * np.stack([mt.iso_stiffness(E, 0.0) for E in E_layer[layer]])
    K = mo.elastic_assemble(xyz, tets, C)
    f = mo.traction_load(xyz, tets, xyz[:, 0] >= L - 1e-12, [t, 0, 0])
    u = mo.elastic_solve(K, f, rollers(xyz)).reshape(-1, 3)
    end = xyz[:, 0] >= L - 1e-12
    assert np.allclose(u[end, 0], t * (L / nx) * (1.0 / E_layer).sum(), rtol=1e-10)
    assert np.abs(u[:, 1:]).max() < 1e-10 * u[end, 0].max()
    sig = mo.gauss_stress(xyz, tets, u.reshape(-1), C)
    # the stress at each Gauss point scales with its own C: spread[q] t
    assert np.allclose(sig[..., 0], spread[None, :] * t, rtol=1e-9)
