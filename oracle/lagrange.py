"""Lagrange P_p shape functions on a tetrahedron, exact integration.

Test infrastructure (see ``oracle/__init__``).

The paper discretises with hierarchic H1 functions of order p = 1..3 (Sec. 1,
Sec. 7, citing Ainsworth and Coyle).  Any conforming basis spanning the same
P_p space gives the same Galerkin solution, so the oracle uses the textbook
nodal (Lagrange) basis written in barycentric coordinates:

    phi_m(lam) = prod_a prod_{s < m_a} (p lam_a - s) / (s + 1),   |m| = p,

with node m at barycentric point m / p.  Polynomials are kept as exact
rational coefficients of barycentric monomials and integrated with

    int_T lam^alpha dV = alpha! 3! |T| / (|alpha| + 3)!,
    int_F lam^alpha dA = alpha! 2! |F| / (|alpha| + 2)!   (alpha_opposite = 0),

so no quadrature rule enters.  Pinned by: partition of unity and the
Kronecker property (tests), linear-field reproduction, and every downstream
homogenisation pin.
"""
from __future__ import annotations

import itertools
from fractions import Fraction
from functools import lru_cache
from math import factorial

import numpy as np

# A polynomial is a dict {(e0,e1,e2,e3): Fraction}


def _mul(a, b):
    out = {}
    for ea, ca in a.items():
        for eb, cb in b.items():
            e = tuple(x + y for x, y in zip(ea, eb))
            out[e] = out.get(e, 0) + ca * cb
    return {e: c for e, c in out.items() if c != 0}


def _diff(a, k):
    out = {}
    for e, c in a.items():
        if e[k] > 0:
            e2 = list(e)
            e2[k] -= 1
            out[tuple(e2)] = out.get(tuple(e2), 0) + c * e[k]
    return out


def _vol_integral(a):
    """(1/|T|) int_T poly dV."""
    tot = Fraction(0)
    for e, c in a.items():
        num = 1
        for x in e:
            num *= factorial(x)
        tot += c * Fraction(num * factorial(3), factorial(sum(e) + 3))
    return tot


def _face_integral(a, opposite):
    """(1/|F|) int_F poly dA over the face opposite to vertex `opposite`."""
    tot = Fraction(0)
    for e, c in a.items():
        if e[opposite] != 0:
            continue
        num = 1
        for x in e:
            num *= factorial(x)
        tot += c * Fraction(num * factorial(2), factorial(sum(e) + 2))
    return tot


@lru_cache(maxsize=None)
def node_multi_indices(p: int):
    """All m in N^4 with |m| = p; the four vertex nodes come first, vertex a at
    position a, then the remaining nodes in a fixed order."""
    ms = [m for m in itertools.product(range(p + 1), repeat=4) if sum(m) == p]
    ms.sort(key=lambda m: (-max(m), tuple(-x for x in m)))
    return tuple(ms)


@lru_cache(maxsize=None)
def basis_polys(p: int):
    out = []
    for m in node_multi_indices(p):
        poly = {(0, 0, 0, 0): Fraction(1)}
        for a in range(4):
            for s in range(m[a]):
                e = [0, 0, 0, 0]
                e[a] = 1
                factor = {tuple(e): Fraction(p, s + 1), (0, 0, 0, 0): Fraction(-s, s + 1)}
                poly = _mul(poly, factor)
        out.append(poly)
    return tuple(out)


def evaluate(p: int, lam):
    """Values of all basis functions at barycentric points lam [..., 4]."""
    lam = np.asarray(lam, dtype=np.float64)
    vals = []
    for poly in basis_polys(p):
        v = np.zeros(lam.shape[:-1])
        for e, c in poly.items():
            v = v + float(c) * np.prod(lam ** np.asarray(e), axis=-1)
        vals.append(v)
    return np.stack(vals, axis=-1)


@lru_cache(maxsize=None)
def reference_tables(p: int):
    """Exact reference integrals, normalised by the element measure.

    S[a,b,i,j] = (1/|T|) int dphi_i/dlam_a * dphi_j/dlam_b
    G[a,i]     = (1/|T|) int dphi_i/dlam_a
    M0[i]      = (1/|T|) int phi_i
    Fc[f,i]    = (1/|F_f|) int_{F_f} phi_i   (face f opposite vertex f)
    """
    polys = basis_polys(p)
    n = len(polys)
    d = [[_diff(polys[i], a) for i in range(n)] for a in range(4)]
    S = np.zeros((4, 4, n, n))
    G = np.zeros((4, n))
    M0 = np.zeros(n)
    Fc = np.zeros((4, n))
    for i in range(n):
        M0[i] = float(_vol_integral(polys[i]))
        for f in range(4):
            Fc[f, i] = float(_face_integral(polys[i], f))
        for a in range(4):
            G[a, i] = float(_vol_integral(d[a][i]))
            for b in range(4):
                for j in range(n):
                    S[a, b, i, j] = float(_vol_integral(_mul(d[a][i], d[b][j])))
    return S, G, M0, Fc


def n_local(p: int) -> int:
    return (p + 1) * (p + 2) * (p + 3) // 6
