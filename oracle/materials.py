"""Constituent materials and the degradation law, FP64.

Test infrastructure (see ``oracle/__init__``).

Voigt order is the paper's (Sec. 2, macro-strain definition):
strain  [e11, e22, e33, 2e12, 2e23, 2e31], stress [s11, s22, s33, s12, s23, s31].

* isotropic matrix, transversely isotropic yarns rotated from the fibre frame
  to global axes (Sec. 1, Sec. 6, Sec. 7 with the material table);
* transport tensors k2 I + (k1 - k2) t t^T (isotropic when k1 = k2);
* degradation (Sec. 4): alpha(T) = beta ln(1 - T/Tg) with T in kelvin,
  1 - omega = exp(-c alpha(T) t) (Eq. Model_final1 applied to the matrix
  modulus), its rate form (Eq. Model_RateForm) integrated by backward Euler,
  and the least-squares beta of Eq. alphaT_LSF.

Pinned by: printed alpha/beta/Tg (tests/golden/degradation.json), closed form
vs backward Euler, TI engineering constants recovered from the compliance,
isotropic limit of the TI formula, rotation (frame) invariance.
"""
from __future__ import annotations

import numpy as np

VOIGT = ((0, 0), (1, 1), (2, 2), (0, 1), (1, 2), (2, 0))
KELVIN = 273.15


def iso_stiffness(E: float, nu: float) -> np.ndarray:
    lam = E * nu / ((1 + nu) * (1 - 2 * nu))
    mu = E / (2 * (1 + nu))
    D = np.zeros((6, 6))
    D[:3, :3] = lam
    D[[0, 1, 2], [0, 1, 2]] += 2 * mu
    D[[3, 4, 5], [3, 4, 5]] = mu
    return D


def ti_compliance_local(E1, E2, G12, nu12, nu23) -> np.ndarray:
    """Compliance in the fibre frame (axis 1 = fibre), engineering shear."""
    S = np.zeros((6, 6))
    S[0, 0] = 1 / E1
    S[1, 1] = S[2, 2] = 1 / E2
    S[0, 1] = S[1, 0] = S[0, 2] = S[2, 0] = -nu12 / E1
    S[1, 2] = S[2, 1] = -nu23 / E2
    S[3, 3] = 1 / G12                  # 12
    S[5, 5] = 1 / G12                  # 31
    S[4, 4] = 2 * (1 + nu23) / E2      # 23 (transverse isotropy)
    return S


def voigt_to_tensor(D: np.ndarray) -> np.ndarray:
    C = np.zeros((3, 3, 3, 3))
    for I, (i, j) in enumerate(VOIGT):
        for J, (k, l) in enumerate(VOIGT):
            for (a, b) in {(i, j), (j, i)}:
                for (c, d) in {(k, l), (l, k)}:
                    C[a, b, c, d] = D[I, J]
    return C


def tensor_to_voigt(C: np.ndarray) -> np.ndarray:
    D = np.zeros((6, 6))
    for I, (i, j) in enumerate(VOIGT):
        for J, (k, l) in enumerate(VOIGT):
            D[I, J] = C[i, j, k, l]
    return D


def frame_from_axis(t: np.ndarray, helper=None) -> np.ndarray:
    """Orthonormal columns (t, a, b); any a, b orthogonal to t."""
    t = np.asarray(t, float) / np.linalg.norm(t)
    if helper is None:
        helper = np.array([0.0, 0.0, 1.0]) if abs(t[2]) < 0.9 else np.array([1.0, 0.0, 0.0])
    a = helper - t * (helper @ t)
    a /= np.linalg.norm(a)
    b = np.cross(t, a)
    return np.stack([t, a, b], axis=1)


def rotate_stiffness(D_local: np.ndarray, R: np.ndarray) -> np.ndarray:
    """C_ijkl = R_ia R_jb R_kc R_ld C'_abcd with R columns = local axes in global."""
    C = voigt_to_tensor(D_local)
    Cg = np.einsum("ia,jb,kc,ld,abcd->ijkl", R, R, R, R, C)
    return tensor_to_voigt(Cg)


def ti_stiffness(E1, E2, G12, nu12, nu23, axis, helper=None) -> np.ndarray:
    D_local = np.linalg.inv(ti_compliance_local(E1, E2, G12, nu12, nu23))
    return rotate_stiffness(D_local, frame_from_axis(axis, helper))


def transport_tensor(k_axial, k_trans, axis) -> np.ndarray:
    t = np.asarray(axis, float) / np.linalg.norm(axis)
    return k_trans * np.eye(3) + (k_axial - k_trans) * np.outer(t, t)


# ------------------------------------------------------------- degradation
def alpha_of_T(T_C, beta=-0.001682, Tg_C=126.0):
    """Degradation rate [1/day] at exposure temperature T (Eq. alphaT, kelvin)."""
    return beta * np.log(1.0 - (np.asarray(T_C) + KELVIN) / (Tg_C + KELVIN))


def moisture_fraction(c_wt, c_sat_wt=1.5):
    """gamma(c) = c (Sec. 4) with c the saturation fraction, clipped to [0,1]."""
    return np.clip(np.asarray(c_wt, float) / c_sat_wt, 0.0, 1.0)


def one_minus_omega(T_C, c_wt, t_h, beta=-0.001682, Tg_C=126.0, c_sat_wt=1.5):
    """Closed form 1 - omega = exp(-c alpha(T) t), t in days = hours / 24."""
    c = moisture_fraction(c_wt, c_sat_wt)
    return np.exp(-c * alpha_of_T(T_C, beta, Tg_C) * (np.asarray(t_h, float) / 24.0))


def one_minus_omega_backward_euler(T_C, c, t_days, n_steps, beta=-0.001682, Tg_C=126.0):
    """Rate form d(1-w)/dt = -c beta ln(1 - T/Tg) (1-w), backward Euler with
    n_steps equal steps and constant T, c (c already a saturation fraction)."""
    dt = t_days / n_steps
    rate = c * alpha_of_T(T_C, beta, Tg_C)
    w = 1.0
    for _ in range(n_steps):
        w = w / (1.0 + dt * rate)
    return w


def fit_beta(T_C_list, alpha_list, Tg_C=126.0, kelvin=True):
    """argmin_beta sum_i (alpha_i - beta ln(1 - T_i/Tg))^2 (Eq. alphaT_LSF)."""
    T = np.asarray(T_C_list, float)
    Tg = Tg_C
    if kelvin:
        T = T + KELVIN
        Tg = Tg_C + KELVIN
    L = np.log(1.0 - T / Tg)
    a = np.asarray(alpha_list, float)
    return float((a @ L) / (L @ L))


# ------------------------------------------------------- per-element tensors
def element_tensors(phase, tangent, mat, yarn, w_matrix=1.0, w_yarn=1.0):
    """Per-tet 6x6 stiffness, 3x3 conductivity and 3x3 diffusivity.

    phase 0 = isotropic matrix (E scaled by w_matrix = 1 - omega), phase 1 =
    transversely isotropic yarn with fibre axis `tangent` (moduli scaled by
    w_yarn).  Transport properties are not degraded.
    """
    nt = len(phase)
    D = np.zeros((nt, 6, 6))
    K = np.zeros((nt, 3, 3))
    Dd = np.zeros((nt, 3, 3))
    Dm = iso_stiffness(mat.E * w_matrix, mat.nu)
    for e in range(nt):
        if phase[e] == 0:
            D[e] = Dm
            K[e] = mat.k * np.eye(3)
            Dd[e] = mat.d * np.eye(3)
        else:
            D[e] = ti_stiffness(yarn.E1 * w_yarn, yarn.E2 * w_yarn, yarn.G12 * w_yarn,
                                yarn.nu12, yarn.nu23, tangent[e])
            K[e] = transport_tensor(yarn.k1, yarn.k2, tangent[e])
            Dd[e] = transport_tensor(yarn.d1, yarn.d2, tangent[e])
    return D, K, Dd
