"""FP64 oracle for the coupled macro time step (Secs. 3, 4 and 5).

Test infrastructure (see ``oracle/__init__``).

What it computes, in the paper's terms:

* the macro heat and moisture transport problems (Eq. Eq_field), discretised
  with linear tetrahedra (Eq. Eq_T_disc) into C dpsi/dt + K psi = f
  (Eq. Eq_field_disc) with the consistent capacity matrix
  C = int rho c_p N^T N and K = int B^T K_bar B, K_bar the homogenised
  conductivity (heat) or diffusivity (moisture, capacity 1);
* one implicit (backward Euler) step in time,
  (C / dt + K) psi^{n+1} = C / dt psi^n, with the exposed face held at its
  prescribed value (Dirichlet rows) and zero flux elsewhere (f = 0);
* the degradation field 1 - omega at the macro Gauss points (4-point rule per
  tetrahedron), integrated with backward Euler from the rate form
  (Eq. Eq_Model_RateForm) at the new temperature and moisture:
  W^{n+1} = W^n / (1 + dt_days lambda), lambda = c beta ln(1 - T_K / T_g,K);
* the equivalent exposure time t_eq = -24 ln(W) / lambda [h], for which the
  closed form (Eq. Eq_Model_final1) at the point's current T and c gives W, so
  that a macro Gauss point can be handed to the RVE path as (T, c, t_eq); where
  there is no moisture now the closed form cannot reach W < 1, and t_eq = 0
  hands the point over undegraded (its error, 1 - W, is reported);
* the macro mechanical problem of the fully nested FE^2 step (Sec. 5): linear
  elasticity on the same linear tetrahedra with the homogenised stiffness
  C_bar given per macro Gauss point, K = sum_T sum_g |T| / 4 B^T C_g B (the
  4-point rule; C_g taken by its symmetric part, since the homogenised
  stiffness is symmetric and only rounding makes it otherwise), the load a
  uniform traction on a set of boundary faces (consistent nodal forces
  t |F| / 3 on each face node), displacements prescribed per degree of freedom
  (symmetry rollers), and the Gauss-point stresses sigma_g = C_g B u.

The linear systems are solved with a sparse direct factorisation.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import materials as mt

# 4-point rule on a tetrahedron, exact for quadratics: barycentric (a, b, b, b)
# and its permutations, equal weights |T| / 4.
_A = 0.5854101966249685
_B = 0.1381966011250105
GAUSS_BARY = np.array([[_A, _B, _B, _B], [_B, _A, _B, _B], [_B, _B, _A, _B], [_B, _B, _B, _A]])


def p1_geometry(xyz, tets):
    """Volumes |T| [nt] and barycentric gradients grad lambda_a [nt, 4, 3]."""
    X = xyz[tets]                                   # [nt, 4, 3]
    J = np.stack([X[:, 1] - X[:, 0], X[:, 2] - X[:, 0], X[:, 3] - X[:, 0]], axis=1)   # rows = edges
    det = np.linalg.det(J)
    if (det <= 0).any():
        raise ValueError("non-positive tetrahedron volume")
    Jinv = np.linalg.inv(J)                         # columns: gradients of lambda_1..3
    g = np.zeros((len(tets), 4, 3))
    g[:, 1:, :] = np.transpose(Jinv, (0, 2, 1))
    g[:, 0, :] = -g[:, 1:, :].sum(axis=1)
    return det / 6.0, g


def assemble(xyz, tets, Kbar, cap):
    """Stiffness K = sum |T| G^T K_bar G and consistent capacity
    C = sum cap |T| / 20 (1 + delta_ab) over linear tetrahedra."""
    vol, g = p1_geometry(xyz, tets)
    Ke = np.einsum("t,tai,ij,tbj->tab", vol, g, np.asarray(Kbar, float), g)
    Me = cap * vol[:, None, None] / 20.0 * (np.ones((4, 4)) + np.eye(4))[None]
    rows = np.repeat(tets, 4, axis=1).reshape(-1)
    cols = np.tile(tets, (1, 4)).reshape(-1)
    n = len(xyz)
    K = sp.csr_matrix((Ke.reshape(-1), (rows, cols)), shape=(n, n))
    C = sp.csr_matrix((Me.reshape(-1), (rows, cols)), shape=(n, n))
    return K, C


def backward_euler_step(K, C, psi, dt, face, value):
    """psi^{n+1} from (C/dt + K) psi^{n+1} = C/dt psi^n, psi = value on the face."""
    A = (C / dt + K).tocsr()
    b = C @ psi / dt
    new = psi.copy()
    new[face] = value
    free = np.nonzero(~face)[0]
    fixed = np.nonzero(face)[0]
    rhs = b[free] - A[free][:, fixed] @ new[fixed]
    new[free] = spla.splu(A[free][:, free].tocsc()).solve(rhs)
    return new


def gauss_values(tets, nodal):
    """Nodal field interpolated at the 4 Gauss points of every tetrahedron [nt, 4]."""
    return np.einsum("ga,ta->tg", GAUSS_BARY, nodal[tets])


def degradation_rate(T_C, c_wt, deg=None):
    """lambda = c beta ln(1 - T_K / T_g,K) [1/day] (Eq. Eq_Model_RateForm), >= 0."""
    d = deg or {}
    return mt.moisture_fraction(c_wt, d.get("c_sat_wt", 1.5)) * mt.alpha_of_T(
        T_C, d.get("beta", -0.001682), d.get("Tg_C", 126.0))


def degradation_step(W, T_C, c_wt, dt_h, deg=None):
    """Backward Euler of d(1-omega)/dt = -lambda (1-omega) over dt_h hours."""
    return W / (1.0 + (dt_h / 24.0) * degradation_rate(T_C, c_wt, deg))


def equivalent_time(W, T_C, c_wt, deg=None):
    """t_eq [h] with exp(-lambda t_eq / 24) = W where lambda > 0.  Where there is
    no moisture now (lambda = 0) no exposure time reproduces a W < 1: t_eq = 0
    hands the point over as undegraded, with the error of handover_error."""
    lam = degradation_rate(T_C, c_wt, deg)
    W = np.asarray(W, float)
    with np.errstate(divide="ignore", invalid="ignore"):
        t = np.where(lam > 0, -24.0 * np.log(W) / lam, 0.0)
    return t


def handover_error(W, T_C, c_wt, deg=None):
    """|closed form at (T, c, t_eq) - W|: 1 - W where lambda = 0, else 0."""
    lam = degradation_rate(T_C, c_wt, deg)
    return np.where(lam > 0, 0.0, 1.0 - np.asarray(W, float))


def march(xyz, tets, face, KT, rho_cp, Dc, T0, c0, T_face, c_face, dt_h, n_steps, deg=None):
    """n_steps coupled steps.  Returns the nodal T [C], c [wt%] and the Gauss-point
    T, c, W = 1 - omega and t_eq after each step (lists)."""
    dt_s = dt_h * 3600.0
    KTm, CT = assemble(xyz, tets, KT, rho_cp)
    KCm, CC = assemble(xyz, tets, Dc, 1.0)
    T = np.full(len(xyz), float(T0))
    c = np.full(len(xyz), float(c0))
    W = np.ones((len(tets), 4))
    out = []
    for _ in range(n_steps):
        T = backward_euler_step(KTm, CT, T, dt_s, face, T_face)
        c = backward_euler_step(KCm, CC, c, dt_s, face, c_face)
        Tg = gauss_values(tets, T)
        cg = gauss_values(tets, c)
        W = degradation_step(W, Tg, cg, dt_h, deg)
        out.append(dict(T=T.copy(), c=c.copy(), Tg=Tg, cg=cg, W=W.copy(),
                        t_eq=equivalent_time(W, Tg, cg, deg)))
    return out


# ------------------------------------------------ macro mechanics (Sec. 5)
def strain_operator(g):
    """B [nt, 6, 12]: the Voigt strain of a linear tetrahedron (order of
    materials.VOIGT, engineering shear) from its nodal displacements, DOF
    a * 3 + i for node a and component i; g are the barycentric gradients."""
    nt = len(g)
    B = np.zeros((nt, 6, 12))
    for a in range(4):
        for J, (i, j) in enumerate(mt.VOIGT):
            if i == j:
                B[:, J, a * 3 + i] = g[:, a, i]
            else:                       # 2 eps_ij = du_i/dx_j + du_j/dx_i
                B[:, J, a * 3 + i] += g[:, a, j]
                B[:, J, a * 3 + j] += g[:, a, i]
    return B


def _sym(C_gp):
    C = np.asarray(C_gp, float)
    return 0.5 * (C + np.swapaxes(C, -1, -2))


def elastic_assemble(xyz, tets, C_gp):
    """Macro stiffness from the Gauss-point stiffness C_gp [nt, 4, 6, 6]:
    K = sum over tetrahedra and their 4 Gauss points of |T| / 4 B^T C_g B,
    3 DOFs per node (node * 3 + component)."""
    vol, g = p1_geometry(xyz, tets)
    B = strain_operator(g)
    C = _sym(C_gp)
    Ke = np.zeros((len(tets), 12, 12))
    for q in range(4):
        Ke += np.einsum("t,tJa,tJK,tKb->tab", vol / 4.0, B, C[:, q], B)
    dof = (tets[:, :, None] * 3 + np.arange(3)[None, None, :]).reshape(len(tets), 12)
    rows = np.repeat(dof, 12, axis=1).reshape(-1)
    cols = np.tile(dof, (1, 12)).reshape(-1)
    n = len(xyz) * 3
    return sp.csr_matrix((Ke.reshape(-1), (rows, cols)), shape=(n, n))


# local vertex triples of the four faces of a tetrahedron
_FACES = ((1, 2, 3), (0, 2, 3), (0, 1, 3), (0, 1, 2))


def traction_load(xyz, tets, face_nodes, t):
    """Nodal forces [nv * 3] of a uniform traction t [3] (force per area) on
    every tetrahedron face whose three vertices are all in face_nodes: each
    of the three receives t |F| / 3, |F| the triangle's area."""
    f = np.zeros(len(xyz) * 3)
    t = np.asarray(t, float)
    for e in range(len(tets)):
        for tri in _FACES:
            v = tets[e, list(tri)]
            if face_nodes[v].all():
                X = xyz[v]
                area = 0.5 * np.linalg.norm(np.cross(X[1] - X[0], X[2] - X[0]))
                for k in v:
                    f[k * 3:k * 3 + 3] += t * area / 3.0
    return f


def elastic_solve(K, f, fixed, values=None):
    """u with K u = f on the free DOFs and u = values on the fixed ones."""
    u = np.zeros(K.shape[0]) if values is None else np.where(fixed, values, 0.0).astype(float)
    free = np.nonzero(~fixed)[0]
    fix = np.nonzero(fixed)[0]
    K = K.tocsr()
    rhs = f[free] - K[free][:, fix] @ u[fix]
    u[free] = spla.splu(K[free][:, free].tocsc()).solve(rhs)
    return u


def gauss_stress(xyz, tets, u, C_gp):
    """sigma_g = C_g B u_T at each Gauss point [nt, 4, 6] (B constant per tet)."""
    _, g = p1_geometry(xyz, tets)
    B = strain_operator(g)
    ue = u.reshape(-1, 3)[tets].reshape(len(tets), 12)
    eps = np.einsum("tJa,ta->tJ", B, ue)
    return np.einsum("tqJK,tK->tqJ", _sym(C_gp), eps)
