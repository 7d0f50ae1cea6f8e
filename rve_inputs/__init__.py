"""Seeded synthetic inputs shared by the oracle and the CUDA path.

This module produces *inputs only*: meshes, phase labels, fibre tangents,
constituent properties and macro Gauss-point states.  It holds none of the
homogenisation arithmetic (no element matrices, no constraint handling, no
solver, no degradation law); both the CPU oracle and the GPU library consume
what it returns and must compute everything else on their own.

Geometry follows the synthetic plain-weave RVE used throughout this project
(the paper's own RVE, Sec. 7 "Numerical example", is only shown in a figure and
its geometry table is not self-consistent, so a synthetic weave stands in):

* unit box meshed as an nx x ny x nz structured hex grid, each hex split into
  six tetrahedra around its main diagonal (Kuhn split, identical orientation in
  every hex, hence a conforming and periodic-compatible mesh);
* four yarns of elliptical cross-section 0.4 x 0.1 (full axes) following
  sinusoidal centrelines z = 0.5 +/- 0.125 sin(2 pi s), two warp yarns along x
  (at y = 0.25, 0.75) and two weft yarns along y (at x = 0.25, 0.75), with
  alternating phase so that crossing yarns do not interpenetrate;
* a tetrahedron is yarn if its centroid lies inside a yarn cross-section; its
  fibre axis is the centreline tangent there.
"""
from __future__ import annotations

import itertools
from dataclasses import dataclass, asdict

import numpy as np

PHASE_MATRIX = 0
PHASE_YARN = 1


# --------------------------------------------------------------------------- mesh
def kuhn_grid(nx: int, ny: int, nz: int, lengths=(1.0, 1.0, 1.0)):
    """Structured box mesh: (nx+1)(ny+1)(nz+1) vertices, 6*nx*ny*nz tetrahedra.

    Vertex id v = i + (nx+1)*(j + (ny+1)*k).  Each hex with lowest corner
    (i,j,k) is split into the six tetrahedra (v000, v000+e_a, v000+e_a+e_b,
    v111) over the six orderings (a,b,c) of the axes.  Every tetrahedron has
    positive orientation after the per-permutation vertex swap below.

    Returns xyz float64 [nv,3], tets int32 [nt,4].
    """
    lx, ly, lz = lengths
    ii, jj, kk = np.meshgrid(np.arange(nx + 1), np.arange(ny + 1), np.arange(nz + 1), indexing="ij")
    # lexicographic with i fastest
    ii = ii.transpose(2, 1, 0).reshape(-1)
    jj = jj.transpose(2, 1, 0).reshape(-1)
    kk = kk.transpose(2, 1, 0).reshape(-1)
    xyz = np.stack([ii * (lx / nx), jj * (ly / ny), kk * (lz / nz)], axis=1).astype(np.float64)

    def vid(i, j, k):
        return i + (nx + 1) * (j + (ny + 1) * k)

    ci, cj, ck = np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="ij")
    ci = ci.transpose(2, 1, 0).reshape(-1)
    cj = cj.transpose(2, 1, 0).reshape(-1)
    ck = ck.transpose(2, 1, 0).reshape(-1)
    unit = np.eye(3, dtype=np.int64)
    tets = []
    for perm in itertools.permutations(range(3)):
        a, b, _ = perm
        o0 = np.zeros(3, dtype=np.int64)
        o1 = unit[a]
        o2 = unit[a] + unit[b]
        o3 = np.ones(3, dtype=np.int64)
        corners = [vid(ci + o[0], cj + o[1], ck + o[2]) for o in (o0, o1, o2, o3)]
        # orientation sign of the permutation decides the vertex order
        sign = np.linalg.det(np.stack([o1, o2, o3]).astype(float))
        if sign < 0:
            corners[1], corners[2] = corners[2], corners[1]
        tets.append(np.stack(corners, axis=1))
    # interleave so the 6 tets of one hex are adjacent in memory
    tets = np.stack(tets, axis=1).reshape(-1, 4).astype(np.int32)
    return xyz, tets


def mesh_counts(nx: int, ny: int, nz: int):
    """Closed-form entity counts (V, E, F, T) of the Kuhn grid (topology only)."""
    V = (nx + 1) * (ny + 1) * (nz + 1)
    T = 6 * nx * ny * nz
    # edges: axis edges + face diagonals (one per quad face) + one body diagonal per hex
    E_axis = nx * (ny + 1) * (nz + 1) + (nx + 1) * ny * (nz + 1) + (nx + 1) * (ny + 1) * nz
    E_face = nx * ny * (nz + 1) + nx * (ny + 1) * nz + (nx + 1) * ny * nz
    E = E_axis + E_face + nx * ny * nz
    F = 1 - V + E + T  # Euler characteristic of a ball: V - E + F - T = 1
    return V, E, F, T


def centroids(xyz, tets):
    return xyz[tets].mean(axis=1)


# ----------------------------------------------------------------- plain weave
@dataclass(frozen=True)
class WeaveGeometry:
    amplitude: float = 0.125      # centreline amplitude
    width: float = 0.4            # cross-section full axis, in-plane
    thickness: float = 0.1        # cross-section full axis, through-thickness
    z_mid: float = 0.5


def _yarns(g: WeaveGeometry):
    """(direction axis, transverse position, sign of the sine) for the four yarns."""
    # warp along x at y = 0.25 (+), y = 0.75 (-); weft along y at x = 0.25 (-), x = 0.75 (+)
    return [(0, 0.25, +1.0), (0, 0.75, -1.0), (1, 0.25, -1.0), (1, 0.75, +1.0)]


def plain_weave(xyz, tets, geom: WeaveGeometry = WeaveGeometry(), lengths=(1.0, 1.0, 1.0)):
    """Phase (uint8: 0 matrix, 1 yarn) and unit fibre axis (float64 [nt,3]) per tet.

    Coordinates are normalised by the box lengths so the weave always spans the
    box.  Matrix tets get fibre axis (1,0,0); it is ignored for isotropic phases.
    """
    c = centroids(xyz, tets) / np.asarray(lengths, dtype=np.float64)
    nt = c.shape[0]
    phase = np.zeros(nt, dtype=np.uint8)
    tangent = np.tile(np.array([1.0, 0.0, 0.0]), (nt, 1))
    a = geom.amplitude
    hw, ht = 0.5 * geom.width, 0.5 * geom.thickness
    for axis, pos, sgn in _yarns(geom):
        s = c[:, axis]                        # coordinate along the yarn
        q = c[:, 1 - axis]                    # in-plane transverse coordinate
        zc = geom.z_mid + sgn * a * np.sin(2 * np.pi * s)
        inside = ((q - pos) / hw) ** 2 + ((c[:, 2] - zc) / ht) ** 2 <= 1.0
        new = inside & (phase == PHASE_MATRIX)
        t = np.zeros((nt, 3))
        t[:, axis] = 1.0
        t[:, 2] = sgn * a * 2 * np.pi * np.cos(2 * np.pi * s)
        t /= np.linalg.norm(t, axis=1, keepdims=True)
        phase[new] = PHASE_YARN
        tangent[new] = t[new]
    return phase, tangent


def plain_weave_yarns(xyz, tets, geom: WeaveGeometry = WeaveGeometry(), lengths=(1.0, 1.0, 1.0)):
    """Which yarn each tet belongs to (int32, -1 for matrix; same centroid test and
    tie-break as plain_weave) and each yarn's axis (0 = x for warp, 1 = y for weft)."""
    c = centroids(xyz, tets) / np.asarray(lengths, dtype=np.float64)
    yid = np.full(c.shape[0], -1, dtype=np.int32)
    axes = []
    hw, ht = 0.5 * geom.width, 0.5 * geom.thickness
    for k, (axis, pos, sgn) in enumerate(_yarns(geom)):
        s = c[:, axis]
        q = c[:, 1 - axis]
        zc = geom.z_mid + sgn * geom.amplitude * np.sin(2 * np.pi * s)
        inside = ((q - pos) / hw) ** 2 + ((c[:, 2] - zc) / ht) ** 2 <= 1.0
        yid[inside & (yid < 0)] = k
        axes.append(axis)
    return yid, np.array(axes, dtype=np.int32)


def layered(xyz, tets, layer_phase, nz: int, lz: float = 1.0):
    """Laminate along z: tet in z-cell k gets phase layer_phase[k % len]."""
    zc = centroids(xyz, tets)[:, 2]
    k = np.clip(np.floor(zc / (lz / nz)).astype(int), 0, nz - 1)
    lp = np.asarray(layer_phase, dtype=np.uint8)
    return lp[k % len(lp)]


# --------------------------------------------------------------- constituents
@dataclass(frozen=True)
class MatrixProps:
    """Isotropic matrix: Young's modulus [Pa], Poisson ratio, conductivity
    [W/mK], moisture diffusivity [m^2/s]."""
    E: float = 3.5e9
    nu: float = 0.35
    k: float = 0.2
    d: float = 1e-12


@dataclass(frozen=True)
class YarnProps:
    """Transversely isotropic yarn, axis 1 along the fibre."""
    E1: float = 45e9
    E2: float = 12e9
    G12: float = 5e9
    nu12: float = 0.28
    nu23: float = 0.4
    k1: float = 0.6
    k2: float = 0.35
    d1: float = 2e-12
    d2: float = 5e-13


@dataclass(frozen=True)
class DegradationParams:
    """Constants of the degradation law (Sec. 4): beta [1/day], glass
    transition temperature [deg C], saturation moisture [wt%] that maps to
    c = 1, and whether yarn moduli degrade too (paper: matrix only)."""
    beta: float = -0.001682
    Tg_C: float = 126.0
    c_sat_wt: float = 1.5
    apply_to_yarn: bool = False


NOMINAL_MATRIX = MatrixProps()
NOMINAL_YARN = YarnProps()
NOMINAL_DEGRADATION = DegradationParams()


def jitter_props(seed: int, mat: MatrixProps = NOMINAL_MATRIX, yarn: YarnProps = NOMINAL_YARN, frac=0.10):
    """Every constituent scalar multiplied by an independent U(1-frac, 1+frac) draw."""
    rng = np.random.default_rng(seed)
    m = {k: v * rng.uniform(1 - frac, 1 + frac) for k, v in asdict(mat).items()}
    y = {k: v * rng.uniform(1 - frac, 1 + frac) for k, v in asdict(yarn).items()}
    return MatrixProps(**m), YarnProps(**y)


# --------------------------------------------------------- macro Gauss points
SIZE_CLASSES = ((16, 16, 6), (24, 24, 8), (32, 32, 10))
P_CLASSES = (1, 2)


def gauss_point_states(G: int, seed: int):
    """Per Gauss point: T [deg C] ~ U(20,60), moisture [wt%] ~ U(0,1.5),
    exposure time [h] = 10^U(0,4), size-class index in SIZE_CLASSES and order
    p in P_CLASSES, all uniform and seeded."""
    rng = np.random.default_rng(seed)
    T = rng.uniform(20.0, 60.0, G)
    c = rng.uniform(0.0, 1.5, G)
    t = 10.0 ** rng.uniform(0.0, 4.0, G)
    size = rng.integers(0, len(SIZE_CLASSES), G).astype(np.int32)
    p = np.asarray(P_CLASSES, dtype=np.int32)[rng.integers(0, len(P_CLASSES), G)]
    return T, c, t, size, p


def aged_states(G: int, seed: int):
    """Per Gauss point, the long-exposure part of the state space that a macro
    structure held hot reaches while moisture diffuses in: T [deg C] ~ U(40,60),
    moisture [wt%] ~ U(0,1.5), exposure time [h] = 10^U(2,4), seeded."""
    rng = np.random.default_rng(seed)
    T = rng.uniform(40.0, 60.0, G)
    c = rng.uniform(0.0, 1.5, G)
    t = 10.0 ** rng.uniform(2.0, 4.0, G)
    return T, c, t


def weave_rve(nx: int, ny: int, nz: int):
    """Convenience: Kuhn grid plus plain-weave phases and tangents."""
    xyz, tets = kuhn_grid(nx, ny, nz)
    phase, tangent = plain_weave(xyz, tets)
    return xyz, tets, phase, tangent


def random_unit_vectors(n: int, seed: int):
    rng = np.random.default_rng(seed)
    v = rng.normal(size=(n, 3))
    return v / np.linalg.norm(v, axis=1, keepdims=True)


__all__ = [
    "PHASE_MATRIX", "PHASE_YARN", "kuhn_grid", "mesh_counts", "centroids", "plain_weave",
    "layered", "WeaveGeometry", "MatrixProps", "YarnProps", "DegradationParams",
    "NOMINAL_MATRIX", "NOMINAL_YARN", "NOMINAL_DEGRADATION", "jitter_props", "SIZE_CLASSES",
    "P_CLASSES", "gauss_point_states", "aged_states", "weave_rve", "random_unit_vectors",
]



# ------------------------------------------------------------ macro plate
PLATE_LENGTHS = (0.5, 0.1, 0.01)      # m


@dataclass(frozen=True)
class PlateExposure:
    """Synthetic coupled macro problem: a composite plate with one hot, wet
    face (z = 0), the rest insulated and sealed; everything starts dry at
    room temperature.  rho_cp is a typical glass/polyester value."""
    T0_C: float = 20.0
    c0_wt: float = 0.0
    T_face_C: float = 60.0
    c_face_wt: float = 1.5
    rho_cp: float = 1.9e6             # J / (m^3 K)
    total_h: float = 1.0e4
    n_steps: int = 100


def plate(nx: int, ny: int, nz: int, lengths=PLATE_LENGTHS):
    """Kuhn-split hex grid of the plate; returns xyz [m], tets and the node mask
    of the exposed face z = 0."""
    xyz, tets = kuhn_grid(nx, ny, nz, lengths)
    face = xyz[:, 2] <= 1e-12 * lengths[2]
    return xyz, tets, face
