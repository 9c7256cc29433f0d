"""Fully symmetric volume rules of degree 2p on the reference triangle.

TEST INFRASTRUCTURE ONLY (part of the oracle): the tests, ``smoke()`` and the
benchmark's CPU-baseline leg are the only callers.

The paper evaluates its volume integrals with symmetric rules of degree 2p
(Section 4.3.2; 3 points at p = 1 and 16 at p = 4 in Section 6.1) and does not
print them.  This module derives rules of that kind from their defining
conditions.  A rule invariant under the six symmetries of the triangle
T = {(0,0), (1,0), (0,1)} is a union of orbits in barycentric coordinates
(l1, l2, l3), every point of an orbit carrying the same weight w:

  S3    the centroid (1/3, 1/3, 1/3)                     1 point,  parameters (w)
  S21   (a, a, 1-2a) and its permutations                3 points, parameters (w, a)
  S111  (a, b, 1-a-b) and its permutations               6 points, parameters (w, a, b)

With (r, s) = (l2, l3) the rule is exact for degree d when
  sum_k w_k r_k^i s_k^j = int_T r^i s^j = i! j! / (i+j+2)!     for all i + j <= d.
For each p the orbit structure below has as many parameters as there are
independent symmetric moment conditions of degree 2p, and the point counts are
the paper's (3, 6, 12, 16, 25 for p = 1..5).  The conditions are solved by
Gauss-Newton on all the monomial moments (an overdetermined, consistent system;
each linear step from the normal equations by Gaussian elimination) from the
start values below.  The monomial system is ill-conditioned (solved in float64
the p = 5 points come out wrong by about 2e-13), so every step runs in 50-digit
decimal arithmetic (Python's decimal module) and the result is rounded to
float64 once at the end.

The solution is not unique for every structure (at p = 3 there are at least
two rules with positive weights and interior points).  The rule used is the
one this iteration reaches from START; among the positive-interior solutions
that the seeded multi-start search of search_symmetric_rules.py finds, it is
the one whose points lie farthest from the edges (largest smallest barycentric
coordinate), and START is that rule to three significant digits.

Point order within the rule: the orbits in START's order; an S21 orbit as
(r, s) = (a, a), (a, 1-2a), (1-2a, a); an S111 orbit, with c = 1-a-b, as
(a, b), (b, a), (a, c), (c, a), (b, c), (c, b).
"""
from __future__ import annotations

from decimal import Decimal, localcontext
from math import factorial

import numpy as np

# orbit structure and start values, per p: a list of (kind, parameters) with
# kind 0 = S3 (w), 1 = S21 (w, a), 2 = S111 (w, a, b); w is the weight of one point
START = {
    1: [(1, (0.167, 0.167))],
    2: [(1, (0.0550, 0.0916)), (1, (0.112, 0.446))],
    3: [(1, (0.0254, 0.0631)), (1, (0.0584, 0.249)), (2, (0.0414, 0.0531, 0.310))],
    4: [(0, (0.0722,)), (1, (0.0162, 0.0505)), (1, (0.0516, 0.171)), (1, (0.0475, 0.459)),
        (2, (0.0136, 0.00839, 0.263))],
    5: [(0, (0.0416,)), (1, (0.00548, 0.0285)), (1, (0.0263, 0.163)), (2, (0.0177, 0.0293, 0.363)),
        (2, (0.0147, 0.0337, 0.153)), (2, (0.0281, 0.147, 0.337))],
}

DIGITS = 50


def _points(structure, x):
    """Points of the rule with parameter vector x: a list of (r, s, w, dr, ds, dw)
    with d* the derivatives of r, s and w with respect to x (dicts index -> value)."""
    one = Decimal(1)
    pts = []
    off = 0
    for kind, prm0 in structure:
        w = x[off]
        dw = {off: one}
        if kind == 0:
            third = one / 3
            pts.append((third, third, w, {}, {}, dw))
        elif kind == 1:
            a, ia = x[off + 1], off + 1
            c = one - 2 * a
            # (a, a), (a, c), (c, a); dc/da = -2
            pts.append((a, a, w, {ia: one}, {ia: one}, dw))
            pts.append((a, c, w, {ia: one}, {ia: -2 * one}, dw))
            pts.append((c, a, w, {ia: -2 * one}, {ia: one}, dw))
        else:
            a, b, ia, ib = x[off + 1], x[off + 2], off + 1, off + 2
            c = one - a - b
            da, db, dc = {ia: one}, {ib: one}, {ia: -one, ib: -one}
            for (u, du), (v, dv) in (((a, da), (b, db)), ((b, db), (a, da)), ((a, da), (c, dc)),
                                     ((c, dc), (a, da)), ((b, db), (c, dc)), ((c, dc), (b, db))):
                pts.append((u, v, w, du, dv, dw))
        off += len(prm0)
    return pts


def _moment_system(structure, x, degree):
    """Relative residuals of the monomial moment conditions and their Jacobian."""
    n = len(x)
    pts = _points(structure, x)
    res, jac = [], []
    for i in range(degree + 1):
        for j in range(degree + 1 - i):
            exact = Decimal(factorial(i) * factorial(j)) / Decimal(factorial(i + j + 2))
            f = Decimal(0)
            g = [Decimal(0)] * n
            for r, s, w, dr, ds, dw in pts:
                v = r ** i * s ** j
                f += w * v
                for k, d in dw.items():
                    g[k] += d * v
                if i:
                    vr = i * r ** (i - 1) * s ** j
                    for k, d in dr.items():
                        g[k] += w * vr * d
                if j:
                    vs = j * r ** i * s ** (j - 1)
                    for k, d in ds.items():
                        g[k] += w * vs * d
            res.append((f - exact) / exact)
            jac.append([gk / exact for gk in g])
    return res, jac


def _solve(A, b):
    """Gaussian elimination with partial pivoting (A square, lists of Decimal)."""
    n = len(b)
    A = [row[:] + [b[i]] for i, row in enumerate(A)]
    for col in range(n):
        piv = max(range(col, n), key=lambda r: abs(A[r][col]))
        A[col], A[piv] = A[piv], A[col]
        for r in range(col + 1, n):
            f = A[r][col] / A[col][col]
            for c in range(col, n + 1):
                A[r][c] -= f * A[col][c]
    x = [Decimal(0)] * n
    for r in range(n - 1, -1, -1):
        x[r] = (A[r][n] - sum(A[r][c] * x[c] for c in range(r + 1, n))) / A[r][r]
    return x


def symmetric_rule(p: int, max_iter: int = 60):
    """Points r, s and weights w (sum 1/2) of the symmetric degree-2p rule, float64."""
    if p not in START:
        raise ValueError("no symmetric rule for p=%d" % p)
    structure = START[p]
    with localcontext() as ctx:
        ctx.prec = DIGITS
        x = [Decimal(repr(v)) for _, prm in structure for v in prm]
        n = len(x)
        tol = Decimal(10) ** (-(DIGITS - 8))
        for _ in range(max_iter):
            res, jac = _moment_system(structure, x, 2 * p)
            # normal equations J^T J step = -J^T res
            JtJ = [[sum(row[a] * row[b] for row in jac) for b in range(n)] for a in range(n)]
            Jtr = [-sum(row[a] * rv for row, rv in zip(jac, res)) for a in range(n)]
            step = _solve(JtJ, Jtr)
            x = [xi + si for xi, si in zip(x, step)]
            if max(abs(si) for si in step) < tol:
                break
        res, _ = _moment_system(structure, x, 2 * p)
        if not max(abs(rv) for rv in res) < Decimal(10) ** (-(DIGITS - 10)):
            raise RuntimeError("symmetric rule p=%d did not converge" % p)
        pts = _points(structure, x)
        R = np.array([float(r) for r, _, _, _, _, _ in pts])
        S = np.array([float(s) for _, s, _, _, _, _ in pts])
        W = np.array([float(w) for _, _, w, _, _, _ in pts])
    return R, S, W


def orbit_structure(p: int):
    """(number of S3, S21, S111 orbits) of the rule for p."""
    kinds = [k for k, _ in START[p]]
    return tuple(kinds.count(k) for k in (0, 1, 2))
