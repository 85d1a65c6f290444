"""Exact rational reference for the mortar integrals on tiny meshes (Sec. 2.3).

TEST INFRASTRUCTURE ONLY.  Used to pin the FP64 oracle, with code that shares
nothing with it:

* every double input is an exact rational (``Fraction(float)``);
* E ∩ C is found by vertex enumeration: every d-subset of the 3d+1 bounding
  hyperplanes (2d cell faces, d+1 element faces) is intersected exactly and
  the points that satisfy all constraints are the vertices;
* the polytope is coned from its vertex centroid over its faces (3-D) or its
  edges (2-D), vertices ordered by exact orientation tests;
* every simplex is integrated with the Grundmann-Moeller rule of degree 2s+1
  (rational points and weights; s=1 in 2-D, s=2 in 3-D), exact for the
  integrand lambda_a * psi_b of degree d+1.
"""
from __future__ import annotations

import functools
import itertools
from fractions import Fraction as Fr
from math import factorial


def _solve(A, b):
    """Exact Gauss elimination; returns None if singular."""
    n = len(A)
    M = [list(A[i]) + [b[i]] for i in range(n)]
    for c in range(n):
        piv = next((r for r in range(c, n) if M[r][c] != 0), None)
        if piv is None:
            return None
        M[c], M[piv] = M[piv], M[c]
        for r in range(n):
            if r != c and M[r][c] != 0:
                f = M[r][c] / M[c][c]
                M[r] = [M[r][j] - f * M[c][j] for j in range(n + 1)]
    return [M[i][n] / M[i][i] for i in range(n)]


def _det(rows):
    n = len(rows)
    if n == 2:
        return rows[0][0] * rows[1][1] - rows[0][1] * rows[1][0]
    return (rows[0][0] * (rows[1][1] * rows[2][2] - rows[1][2] * rows[2][1])
            - rows[0][1] * (rows[1][0] * rows[2][2] - rows[1][2] * rows[2][0])
            + rows[0][2] * (rows[1][0] * rows[2][1] - rows[1][1] * rows[2][0]))


@functools.lru_cache(maxsize=None)
def gm_rule(n: int, s: int):
    """Grundmann-Moeller rule on the n-simplex: list of (weight, barycentric point).

    Weights are normalised so that they sum to 1 (i.e. they approximate the mean
    value over the simplex); exact for polynomials of degree 2s+1."""
    d = 2 * s + 1
    out = []
    for i in range(s + 1):
        w = Fr((-1) ** i * (d + n - 2 * i) ** d, 2 ** (2 * s) * factorial(i) * factorial(d + n - i))
        w *= factorial(n)  # the raw weights integrate over the unit simplex of volume 1/n!
        den = d + n - 2 * i
        for beta in _compositions(s - i, n + 1):
            out.append((w, tuple(Fr(2 * bj + 1, den) for bj in beta)))
    return out


def _compositions(total, parts):
    if parts == 1:
        yield (total,)
        return
    for first in range(total + 1):
        for rest in _compositions(total - first, parts - 1):
            yield (first,) + rest


def simplex_integral(verts, f, s):
    """Exact integral of polynomial f over the simplex with rational vertices."""
    n = len(verts) - 1
    rows = [[verts[i + 1][k] - verts[0][k] for k in range(n)] for i in range(n)]
    vol = abs(_det(rows)) / factorial(n)
    if vol == 0:
        return None, Fr(0)
    acc = None
    for w, mu in gm_rule(n, s):
        x = [sum(mu[j] * verts[j][k] for j in range(n + 1)) for k in range(n)]
        v = f(x)
        acc = [w * vi for vi in v] if acc is None else [a + w * vi for a, vi in zip(acc, v)]
    return [a * vol for a in acc], vol


def _order_ccw(points, centre, normal=None):
    """Sort coplanar points around their centre with exact orientation tests."""
    dim = len(centre)

    def rel(p):
        return [p[k] - centre[k] for k in range(dim)]

    if dim == 2:
        def cross(u, v):
            return u[0] * v[1] - u[1] * v[0]
        ref = rel(points[0])
        def key_half(p):
            u = rel(p)
            c = cross(ref, u)
            dot = ref[0] * u[0] + ref[1] * u[1]
            return 0 if (c > 0 or (c == 0 and dot > 0)) else 1
        def cmp(p, q):
            hp, hq = key_half(p), key_half(q)
            if hp != hq:
                return -1 if hp < hq else 1
            c = cross(rel(p), rel(q))
            return -1 if c > 0 else (1 if c < 0 else 0)
        return sorted(points, key=functools.cmp_to_key(cmp))

    def cross3(u, v):
        return [u[1] * v[2] - u[2] * v[1], u[2] * v[0] - u[0] * v[2], u[0] * v[1] - u[1] * v[0]]

    def orient(u, v):
        c = cross3(u, v)
        return c[0] * normal[0] + c[1] * normal[1] + c[2] * normal[2]

    ref = rel(points[0])
    def half(p):
        u = rel(p)
        o = orient(ref, u)
        dot = sum(ref[k] * u[k] for k in range(3))
        return 0 if (o > 0 or (o == 0 and dot > 0)) else 1
    def cmp(p, q):
        hp, hq = half(p), half(q)
        if hp != hq:
            return -1 if hp < hq else 1
        o = orient(rel(p), rel(q))
        return -1 if o > 0 else (1 if o < 0 else 0)
    return sorted(points, key=functools.cmp_to_key(cmp))


def pair_block_exact(dim, verts, cell_lo, h, dual=False, cell_hi=None):
    """Exact block int_{E cap C} lambda_a psi_b and vol(E cap C).

    ``verts``: element vertex coordinates (floats), ``cell_lo``: the cell's lower
    corner (floats), ``h``: cell widths (floats).  Returns (block, vol) with
    block[a][b] Fractions, b = corner bits (x bit 0).  With ``dual`` the weight
    lambda_a is replaced by the element dual function (dim+2) lambda_a - 1
    (Eq. (biorth)), integrated as it stands.  ``cell_hi`` (floats) gives the
    upper corner instead of ``h``: the widths are then the exact differences
    (a cell of a stretched grid)."""
    V = [[Fr(verts[i][k]) - Fr(cell_lo[k]) for k in range(dim)] for i in range(dim + 1)]
    H = ([Fr(h[k]) for k in range(dim)] if cell_hi is None
         else [Fr(cell_hi[k]) - Fr(cell_lo[k]) for k in range(dim)])
    # barycentric coordinates: lambda(x) = L @ (x, 1)
    A = [[V[j][r] for j in range(dim + 1)] for r in range(dim)] + [[Fr(1)] * (dim + 1)]
    L = []
    for a in range(dim + 1):
        # row a of A^{-1}: solve A^T y = e_a
        At = [[A[r][c] for r in range(dim + 1)] for c in range(dim + 1)]
        e = [Fr(int(i == a)) for i in range(dim + 1)]
        L.append(_solve(At, e))
    # constraints g(x) = n.x + c >= 0
    cons = []
    for k in range(dim):
        n = [Fr(0)] * dim; n[k] = Fr(1); cons.append((n, Fr(0)))
        n = [Fr(0)] * dim; n[k] = Fr(-1); cons.append((n, H[k]))
    for a in range(dim + 1):
        cons.append((L[a][:dim], L[a][dim]))

    def val(cn, x):
        return sum(cn[0][k] * x[k] for k in range(dim)) + cn[1]

    verts_p = set()
    for sub in itertools.combinations(range(len(cons)), dim):
        x = _solve([cons[i][0] for i in sub], [-cons[i][1] for i in sub])
        if x is None:
            continue
        if all(val(c, x) >= 0 for c in cons):
            verts_p.add(tuple(x))
    nb = 1 << dim
    zero = [[Fr(0)] * nb for _ in range(dim + 1)]
    if len(verts_p) < dim + 1:
        return zero, Fr(0)
    P = list(verts_p)
    cen = [sum(p[k] for p in P) / len(P) for k in range(dim)]

    def integrand(x):
        lam = [sum(L[a][k] * x[k] for k in range(dim)) + L[a][dim] for a in range(dim + 1)]
        if dual:
            lam = [(dim + 2) * la - 1 for la in lam]
        t = [x[k] / H[k] for k in range(dim)]
        out = []
        for a in range(dim + 1):
            for b in range(nb):
                psi = Fr(1)
                for k in range(dim):
                    psi *= t[k] if (b >> k) & 1 else 1 - t[k]
                out.append(lam[a] * psi)
        return out

    s = 1 if dim == 2 else 2
    acc = [Fr(0)] * ((dim + 1) * nb)
    vol = Fr(0)
    if dim == 2:
        ring = _order_ccw(P, cen)
        simplices = [[cen, ring[i], ring[(i + 1) % len(ring)]] for i in range(len(ring))]
    else:
        simplices = []
        for cn in cons:
            on = [p for p in P if val(cn, p) == 0]
            if len(on) < 3:
                continue
            fc = [sum(p[k] for p in on) / len(on) for k in range(3)]
            ring = _order_ccw(on, fc, normal=cn[0])
            for i in range(len(ring)):
                simplices.append([cen, fc, ring[i], ring[(i + 1) % len(ring)]])
    for S in simplices:
        r, v = simplex_integral(S, integrand, s)
        if r is None:
            continue
        acc = [x + y for x, y in zip(acc, r)]
        vol += v
    block = [[acc[a * nb + b] for b in range(nb)] for a in range(dim + 1)]
    return block, vol
