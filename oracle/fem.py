"""FP64 finite-element oracle for the RVE cell problems (Sec. 2).

Test infrastructure (see ``oracle/__init__``).

What it computes, in the paper's terms:

* micro displacement u = eps_bar y + u_tilde (Eq. micro_disp); the scalar
  fields use psi = grad_psi . y + psi_tilde (the X of Eq. eq_X_psi);
* the weak equilibrium int sigma : grad^s eta = 0 (Eq. RVE_Eq_var_final) on a
  Lagrange P_p space (``oracle.lagrange``), element matrices integrated
  exactly, assembled into scipy sparse matrices;
* the three boundary conditions of Sec. 2, written on the fluctuation:
    - linear Dirichlet: u_tilde = 0 on the boundary (nodes eliminated);
    - periodic: u_tilde(y+) = u_tilde(y-) (nodes identified on the lattice,
      one node pinned to remove translations);
    - uniform Neumann: int_Gamma sym(u_tilde (x) n) dA = 0, i.e. the constraint
      rows C = int H N^T N with H the six uniform traction modes sigma n
      (Eq. eq_mat_C_and_D), bordered with the rigid-body rows (rotation via
      the skew part of the same boundary integral, translation via the volume
      mean) that leave the strain field unchanged;
* homogenised tensors in energy form C_ij = (1/V) a(u_i, u_j) with u_i the total
  field of unit load case i (Eq. Hill_prin with Eq. Eq_C_stress), and the
  volume-averaged stress / flux (Eq. macro_stress) for the Hill-Mandel check;
* the paper's own bordered route on the total field,
  [[K, C^T], [C, 0]] [u; lambda] = [0; D eps_bar] (Eq. eq_RVE_disc_Eqs),
  D = int H N^T X (Eq. eq_mat_C_and_D, with X from Eq. eq_X_mech /
  eq_X_psi) and sigma_bar = -(1/V) D^T lambda (Eq. eq_homo_stress; the sign is
  fixed by the printed system, whose multiplier is minus the boundary
  reaction).  Used as a brute-force check on tiny meshes.

Meshes must be box meshes whose vertices lie on a regular lattice (the Kuhn
grids of ``rve_inputs``): nodes are identified by integer lattice keys, which
is how periodic images are matched.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import lagrange
from .materials import VOIGT

BC_DIRICHLET, BC_PERIODIC, BC_NEUMANN = 0, 1, 2
BC_NAMES = {BC_DIRICHLET: "dirichlet", BC_PERIODIC: "periodic", BC_NEUMANN: "neumann"}


# ----------------------------------------------------------------- mesh/nodes
@dataclass
class NodalMesh:
    xyz: np.ndarray          # [nv,3]
    tets: np.ndarray         # [nt,4]
    grid: tuple              # (nx, ny, nz)
    p: int
    lengths: np.ndarray = field(default=None)
    # derived
    elem_nodes: np.ndarray = field(default=None)   # [nt, n_local] global node ids
    node_key: np.ndarray = field(default=None)     # [nn, 3] lattice keys (units h/p)
    vol: np.ndarray = field(default=None)          # [nt]
    grad_lam: np.ndarray = field(default=None)     # [nt, 4, 3]
    node_xyz_e: np.ndarray = field(default=None)   # [nt, n_local, 3] actual coords


def build_nodal_mesh(xyz, tets, grid, p, periodic=False) -> NodalMesh:
    xyz = np.asarray(xyz, np.float64)
    tets = np.asarray(tets, np.int64)
    grid = tuple(int(g) for g in grid)
    lengths = xyz.max(axis=0) - xyz.min(axis=0)
    h = lengths / np.asarray(grid)
    iv = np.rint((xyz - xyz.min(axis=0)) / h).astype(np.int64)   # vertex lattice index
    ms = np.asarray(lagrange.node_multi_indices(p), np.int64)      # [n_local, 4]
    # element node keys in units of h/p: sum_a m_a * iv[v_a]
    keys = np.einsum("la,tak->tlk", ms, iv[tets])                  # [nt, nl, 3]
    if periodic:
        keys = keys % (p * np.asarray(grid))
    flat = keys.reshape(-1, 3)
    uniq, inv = np.unique(flat, axis=0, return_inverse=True)
    elem_nodes = inv.reshape(keys.shape[0], keys.shape[1])
    v = xyz[tets]                                                  # [nt,4,3]
    J = np.stack([v[:, 1] - v[:, 0], v[:, 2] - v[:, 0], v[:, 3] - v[:, 0]], axis=2)  # columns
    det = np.linalg.det(J)
    Jinv = np.linalg.inv(J)                                        # rows = grad xi_k
    g = np.zeros((len(tets), 4, 3))
    g[:, 1:, :] = Jinv
    g[:, 0, :] = -Jinv.sum(axis=1)
    node_xyz_e = np.einsum("la,tak->tlk", ms.astype(np.float64) / p, v)
    m = NodalMesh(xyz=xyz, tets=tets, grid=grid, p=p, lengths=lengths)
    m.elem_nodes = elem_nodes
    m.node_key = uniq
    m.vol = np.abs(det) / 6.0
    m.grad_lam = g
    m.node_xyz_e = node_xyz_e
    return m


def n_nodes(m: NodalMesh) -> int:
    return m.node_key.shape[0]


def boundary_nodes(m: NodalMesh) -> np.ndarray:
    """Nodes on the box surface (lattice coordinate 0 or p*n in some axis)."""
    top = m.p * np.asarray(m.grid)
    k = m.node_key
    return np.nonzero(((k == 0) | (k == top)).any(axis=1))[0]


def boundary_faces(m: NodalMesh):
    """(tet index, local face = opposite vertex, outward unit normal, area)."""
    h = m.lengths / np.asarray(m.grid)
    iv = np.rint((m.xyz - m.xyz.min(axis=0)) / h).astype(np.int64)
    out = []
    for f in range(4):
        others = [a for a in range(4) if a != f]
        vk = iv[m.tets[:, others]]                                 # [nt,3,3]
        for ax in range(3):
            for side, val in ((-1.0, 0), (1.0, m.grid[ax])):
                on = (vk[:, :, ax] == val).all(axis=1)
                for t in np.nonzero(on)[0]:
                    pts = m.xyz[m.tets[t, others]]
                    area = 0.5 * np.linalg.norm(np.cross(pts[1] - pts[0], pts[2] - pts[0]))
                    n = np.zeros(3)
                    n[ax] = side
                    out.append((t, f, n, area))
    return out


# ---------------------------------------------------------- element matrices
def element_stiffness_mech(m: NodalMesh, Dvoigt: np.ndarray) -> np.ndarray:
    """K_e[t, i, c, j, d] = |T| sum_ab S[a,b,i,j] g_a C_c.d. g_b (exact)."""
    from .materials import voigt_to_tensor
    S, _, _, _ = lagrange.reference_tables(m.p)
    C = np.stack([voigt_to_tensor(D) for D in Dvoigt])             # [nt,3,3,3,3]
    g = m.grad_lam
    GG = np.einsum("tak,tckdl,tbl->tacbd", g, C, g)                # [nt,4,3,4,3]
    return np.einsum("t,abij,tacbd->ticjd", m.vol, S, GG)


def element_stiffness_scalar(m: NodalMesh, kten: np.ndarray) -> np.ndarray:
    S, _, _, _ = lagrange.reference_tables(m.p)
    g = m.grad_lam
    GG = np.einsum("tak,tkl,tbl->tab", g, kten, g)
    return np.einsum("t,abij,tab->tij", m.vol, S, GG)


def assemble(m: NodalMesh, Ke: np.ndarray, nc: int) -> sp.csr_matrix:
    nt, nl = m.elem_nodes.shape
    dofs = (m.elem_nodes[:, :, None] * nc + np.arange(nc)[None, None, :]).reshape(nt, nl * nc)
    Kf = Ke.reshape(nt, nl * nc, nl * nc)
    rows = np.repeat(dofs, nl * nc, axis=1).reshape(-1)
    cols = np.tile(dofs, (1, nl * nc)).reshape(-1)
    N = n_nodes(m) * nc
    return sp.csr_matrix((Kf.reshape(-1), (rows, cols)), shape=(N, N))


def unit_macro_fields(nc: int):
    """Unit macro strains (Voigt, engineering shear) as 3x3 tensors, or unit
    gradients for the scalar fields."""
    if nc == 3:
        out = []
        for J in range(6):
            E = np.zeros((3, 3))
            i, j = VOIGT[J]
            if i == j:
                E[i, i] = 1.0
            else:
                E[i, j] = E[j, i] = 0.5
            out.append(E)
        return out
    return [np.eye(3)[k] for k in range(3)]


def linear_field_nodal(m: NodalMesh, macro, nc: int) -> np.ndarray:
    """Element nodal values of eps_bar y (mech) or grad_psi . y (scalar)."""
    y = m.node_xyz_e
    if nc == 3:
        return np.einsum("ck,tlk->tlc", macro, y)
    return np.einsum("k,tlk->tl", macro, y)[:, :, None]


# ------------------------------------------------------------------ solving
def _cg_beta(rz_new, rz):
    """Fletcher-Reeves coefficient of preconditioned CG, beta = (r'.z') / (r.z)."""
    return np.where(rz != 0, rz_new / np.where(rz != 0, rz, 1.0), 0.0)


def _true_residual_met(A, B, X, rtol, bnorm):
    """||b - A x|| <= rtol ||b|| for every column, recomputed from x."""
    return np.linalg.norm(B - A @ X, axis=0) <= rtol * bnorm


def pcg_columns(A: sp.spmatrix, B: np.ndarray, rtol=1e-13, maxiter=100_000, info=None):
    """Textbook Jacobi-preconditioned CG run independently on every column of
    B (each column has its own alpha, beta); returns once every column
    satisfies ||b - A x|| <= rtol ||b|| in the TRUE residual.  The recursive
    residual only proposes the stop: when it passes but the true residual
    b - A x misses rtol (the two drift apart in floating point), the recursion
    restarts from the true residual.  ``info`` (a dict), when given, receives
    the iteration count and the number of restarts."""
    A = A.tocsr()
    dinv = 1.0 / A.diagonal()
    X = np.zeros_like(B)
    Rr = B.copy()
    Z = dinv[:, None] * Rr
    P = Z.copy()
    rz = np.einsum("ij,ij->j", Rr, Z)
    bnorm = np.linalg.norm(B, axis=0)
    bnorm[bnorm == 0] = 1.0
    restarts = 0
    for it in range(maxiter + 1):
        if (np.linalg.norm(Rr, axis=0) <= rtol * bnorm).all():
            if _true_residual_met(A, B, X, rtol, bnorm).all():
                if info is not None:
                    info["iterations"] = it
                    info["restarts"] = restarts
                return X
            restarts += 1
            Rr = B - A @ X
            Z = dinv[:, None] * Rr
            P = Z.copy()
            rz = np.einsum("ij,ij->j", Rr, Z)
        if it == maxiter:
            break
        Q = A @ P
        pq = np.einsum("ij,ij->j", P, Q)
        alpha = np.where(pq != 0, rz / np.where(pq != 0, pq, 1.0), 0.0)
        X += alpha * P
        Rr -= alpha * Q
        Z = dinv[:, None] * Rr
        rz_new = np.einsum("ij,ij->j", Rr, Z)
        beta = _cg_beta(rz_new, rz)
        P = Z + beta * P
        rz = rz_new
    raise RuntimeError("oracle CG did not converge")


def _solve_spd(A: sp.spmatrix, B: np.ndarray, direct_max=4000, rtol=1e-13):
    if A.shape[0] <= direct_max:
        lu = spla.splu(A.tocsc(), permc_spec="MMD_AT_PLUS_A")
        return lu.solve(B)
    return pcg_columns(A, B, rtol=rtol)


def neumann_rows(m: NodalMesh, nc: int) -> sp.csr_matrix:
    """Bordering rows for the uniform-traction RVE, on the fluctuation.

    mech: 6 traction modes int_Gamma (E_k n) . u  (E_k unit symmetric, Voigt
          stress order), 3 rotation rows int_Gamma skew(u (x) n), 3 translation
          rows int_Omega u.
    scalar: 3 rows int_Gamma psi n_k and 1 row int_Omega psi.
    """
    _, _, M0, Fc = lagrange.reference_tables(m.p)
    nn = n_nodes(m)
    rows = []
    if nc == 3:
        modes = []
        for J in range(6):
            E = np.zeros((3, 3))
            i, j = VOIGT[J]
            E[i, j] = E[j, i] = 1.0
            modes.append(E)
        skews = []
        for (a, b) in ((1, 2), (2, 0), (0, 1)):
            W = np.zeros((3, 3))
            W[a, b], W[b, a] = 1.0, -1.0
            skews.append(W)
        R = np.zeros((12, nn * 3))
        for (t, f, n, area) in boundary_faces(m):
            nodes = m.elem_nodes[t]
            w = area * Fc[f]                                       # [nl]
            for k, E in enumerate(modes):
                tr = E @ n
                for c in range(3):
                    np.add.at(R[k], nodes * 3 + c, w * tr[c])
            for k, W in enumerate(skews):
                # skew part of int u (x) n : (u_a n_b - u_b n_a)
                v = W @ n
                for c in range(3):
                    np.add.at(R[6 + k], nodes * 3 + c, w * v[c])
        for t in range(len(m.tets)):
            nodes = m.elem_nodes[t]
            for c in range(3):
                np.add.at(R[9 + c], nodes * 3 + c, m.vol[t] * M0)
        rows = R
    else:
        R = np.zeros((4, nn))
        for (t, f, n, area) in boundary_faces(m):
            nodes = m.elem_nodes[t]
            w = area * Fc[f]
            for k in range(3):
                np.add.at(R[k], nodes, w * n[k])
        for t in range(len(m.tets)):
            np.add.at(R[3], m.elem_nodes[t], m.vol[t] * M0)
        rows = R
    return sp.csr_matrix(rows)


def element_macro_load(Kef: np.ndarray, ulin_e: np.ndarray) -> np.ndarray:
    """Element load -a_e(eps_bar y, phi_i) = -K_e u_lin (the linear part moved
    to the right-hand side of the fluctuation problem)."""
    return -np.einsum("tab,tb->ta", Kef, ulin_e)


@dataclass
class CellSolution:
    bc: int
    nc: int
    tensor: np.ndarray            # energy form, [6,6] or [3,3]
    sigma_bar: np.ndarray         # volume-averaged stress/flux per load case, [R, 6 or 3]
    u_tilde: np.ndarray           # [N_dof, R] fluctuation on the (possibly folded) node set
    volume: float


def solve_cell(xyz, tets, grid, p, bc, Ke_fn, nc, direct_max=4000) -> CellSolution:
    """Solve the R unit cell problems of one field for one boundary condition.

    Ke_fn(mesh) -> element matrices; nc = 3 (mechanics) or 1 (scalar field).
    """
    m = build_nodal_mesh(xyz, tets, grid, p, periodic=(bc == BC_PERIODIC))
    Ke = Ke_fn(m)                                                  # [nt, nl, nc, nl, nc] or [nt,nl,nl]
    nt, nl = m.elem_nodes.shape
    Kef = Ke.reshape(nt, nl * nc, nl * nc)
    K = assemble(m, Kef, nc)
    macros = unit_macro_fields(nc)
    R = len(macros)
    N = n_nodes(m) * nc
    # right-hand sides b_i = -a(eps_i y, phi)   (element-local linear fields)
    B = np.zeros((N, R))
    ulin = [linear_field_nodal(m, M, nc).reshape(nt, nl * nc) for M in macros]
    dofs = (m.elem_nodes[:, :, None] * nc + np.arange(nc)[None, None, :]).reshape(nt, nl * nc)
    for i in range(R):
        np.add.at(B[:, i], dofs.reshape(-1), element_macro_load(Kef, ulin[i]).reshape(-1))

    U = np.zeros((N, R))
    if bc in (BC_DIRICHLET, BC_PERIODIC):
        if bc == BC_DIRICHLET:
            fixed_nodes = boundary_nodes(m)
        else:
            fixed_nodes = np.nonzero((m.node_key == 0).all(axis=1))[0]
        fixed = (fixed_nodes[:, None] * nc + np.arange(nc)[None, :]).reshape(-1)
        free = np.setdiff1d(np.arange(N), fixed)
        Kff = K[free][:, free]
        U[free] = _solve_spd(Kff, B[free], direct_max=direct_max)
    elif bc == BC_NEUMANN:
        Cn = neumann_rows(m, nc)
        nr = Cn.shape[0]
        A = sp.bmat([[K, Cn.T], [Cn, None]], format="csc")
        rhs = np.vstack([B, np.zeros((nr, R))])
        sol = spla.splu(A, permc_spec="MMD_AT_PLUS_A").solve(rhs)
        U = sol[:N]
    else:
        raise ValueError(bc)

    V = float(m.vol.sum())
    # energy-form tensor
    tens = np.zeros((R, R))
    ue = [ulin[i] + U[dofs, i] for i in range(R)]
    Ku = [np.einsum("tab,tb->ta", Kef, ue[j]) for j in range(R)]
    for i in range(R):
        for j in range(R):
            tens[i, j] = np.einsum("ta,ta->", ue[i], Ku[j]) / V
    sig = volume_average_flux(m, Ke_fn, ue, nc)
    return CellSolution(bc=bc, nc=nc, tensor=tens, sigma_bar=sig, u_tilde=U, volume=V)


def volume_average_flux(m: NodalMesh, Ke_fn, ue, nc):
    """sigma_bar = (1/V) int sigma dV (Eq. macro_stress), per load case."""
    _, G, _, _ = lagrange.reference_tables(m.p)
    nt, nl = m.elem_nodes.shape
    mat = Ke_fn.material  # per-element D [nt,6,6] or k [nt,3,3]
    V = m.vol.sum()
    out = []
    for u in ue:
        u = u.reshape(nt, nl, nc)
        # mean gradient per element: sum_i sum_a G[a,i] u_i (x) g_a
        grad = np.einsum("ai,tic,tak->tck", G, u, m.grad_lam)     # [nt, nc, 3]
        if nc == 3:
            eps = 0.5 * (grad + grad.transpose(0, 2, 1))
            ev = np.stack([eps[:, i, j] * (1.0 if i == j else 2.0) for (i, j) in VOIGT], axis=1)
            s = np.einsum("tIJ,tJ->tI", mat, ev)
        else:
            s = np.einsum("tkl,tl->tk", mat, grad[:, 0, :])
        out.append(np.einsum("t,tI->I", m.vol, s) / V)
    return np.stack(out)


class _KeFn:
    """Callable producing element matrices; carries the per-element material."""

    def __init__(self, material, nc):
        self.material = material
        self.nc = nc

    def __call__(self, m):
        if self.nc == 3:
            return element_stiffness_mech(m, self.material)
        return element_stiffness_scalar(m, self.material)


def homogenise_field(xyz, tets, grid, p, bc, material, nc, direct_max=4000) -> CellSolution:
    """material: per-tet D [nt,6,6] (nc=3) or conductivity [nt,3,3] (nc=1)."""
    return solve_cell(xyz, tets, grid, p, bc, _KeFn(np.asarray(material, float), nc), nc,
                      direct_max=direct_max)


def homogenise(xyz, tets, grid, p, bc, Dmech, Kth, Dmo, direct_max=4000):
    """C_bar (6x6), K_bar (3x3), D_bar (3x3) of one RVE under one BC type."""
    c = homogenise_field(xyz, tets, grid, p, bc, Dmech, 3, direct_max)
    k = homogenise_field(xyz, tets, grid, p, bc, Kth, 1, direct_max)
    d = homogenise_field(xyz, tets, grid, p, bc, Dmo, 1, direct_max)
    return c.tensor, k.tensor, d.tensor


# ------------------------------------------------- paper's bordered route
def paper_route(xyz, tets, grid, p, bc, material, nc):
    """Total-field saddle system of Eq. eq_RVE_disc_Eqs with sigma_bar from
    Eq. eq_homo_stress.  Dense; tiny meshes only.

    H (admissible nodal traction distributions) per boundary condition:
      Dirichlet: a unit nodal force per boundary node and component, so
                 C u = D eps_bar pins every boundary node to eps_bar y;
      periodic:  equal and opposite unit forces on each image node and its
                 master (each image node mapped to exactly one master), plus
                 one pinned corner node;
      Neumann:   the six uniform traction modes sigma n, integrated over the
                 boundary, plus rotation and translation rows whose
                 multipliers vanish at equilibrium.
    D = int H N^T X is evaluated as C applied to the nodal interpolant of X,
    which is exact because X is linear in y (Eqs. eq_X_mech, eq_X_psi).
    """
    m = build_nodal_mesh(xyz, tets, grid, p, periodic=False)
    kefn = _KeFn(np.asarray(material, float), nc)
    Ke = kefn(m)
    nt, nl = m.elem_nodes.shape
    K = assemble(m, Ke.reshape(nt, nl * nc, nl * nc), nc).toarray()
    nn = n_nodes(m)
    N = nn * nc
    # node coordinates (unique nodes)
    h = m.lengths / (m.p * np.asarray(m.grid))
    ycoord = m.node_key * h + m.xyz.min(axis=0)
    macros = unit_macro_fields(nc)
    R = len(macros)
    Xn = np.zeros((N, R))     # nodal interpolant of the columns of X
    for J, M in enumerate(macros):
        if nc == 3:
            Xn[:, J] = (ycoord @ M.T).reshape(-1)
        else:
            Xn[:, J] = ycoord @ M
    rows = []
    top = m.p * np.asarray(m.grid)
    if bc == BC_DIRICHLET:
        for n in boundary_nodes(m):
            for c in range(nc):
                r = np.zeros(N)
                r[n * nc + c] = 1.0
                rows.append(r)
    elif bc == BC_PERIODIC:
        key_to_node = {tuple(k): i for i, k in enumerate(m.node_key)}
        for s, k in enumerate(m.node_key):
            if (k == top).any():
                mk = tuple(np.where(k == top, 0, k))
                mn = key_to_node[mk]
                for c in range(nc):
                    r = np.zeros(N)
                    r[s * nc + c] = 1.0
                    r[mn * nc + c] -= 1.0
                    rows.append(r)
        origin = key_to_node[(0, 0, 0)]
        for c in range(nc):
            r = np.zeros(N)
            r[origin * nc + c] = 1.0
            rows.append(r)
    elif bc == BC_NEUMANN:
        rows = list(neumann_rows(m, nc).toarray())
    C = np.asarray(rows)
    Dm = C @ Xn
    nr = C.shape[0]
    A = np.block([[K, C.T], [C, np.zeros((nr, nr))]])
    V = float(m.vol.sum())
    sig = np.zeros((R, R))
    for J in range(R):
        e = np.zeros(R)
        e[J] = 1.0
        rhs = np.concatenate([np.zeros(N), Dm @ e])
        sol = np.linalg.solve(A, rhs)
        lam = sol[N:]
        if bc == BC_NEUMANN:
            # only the traction-mode rows carry the macro stress / flux
            ntr = 6 if nc == 3 else 3
            sig[:, J] = -(Dm[:ntr].T @ lam[:ntr]) / V
        else:
            sig[:, J] = -(Dm.T @ lam) / V
    return sig
