"""Seeded multi-start search for the fully symmetric degree-2p rules of
oracle/symmetric_rules.py (reading of Sections 4.3.2 and 6.1).

TEST INFRASTRUCTURE ONLY (part of the oracle): it shows where the start values
of symmetric_rules.START come from, and tests/test_oracle_symmetric_rules.py runs
it.  ``python oracle/search_symmetric_rules.py`` prints, for p = 1..5, every
distinct rule with positive weights and interior points that the search finds,
and START.

For each p the orbit structure is fixed (symmetric_rules.START's kinds: S3, S21,
S111 orbits; the paper's point counts 3, 6, 12, 16, 25).  From seeded random
orbit parameters, a Levenberg-Marquardt iteration in float64 solves the moment
conditions of degree 2p on the reference triangle T = {(0,0), (1,0), (0,1)},
written against an orthogonal basis of the polynomials of degree <= 2p (the
products of Jacobi polynomials in the collapsed coordinates, of which only the
constant has a nonzero integral, 1/2): sum_k w_k psi(x_k) = int_T psi.  Against
monomials the same conditions are too ill-conditioned for float64 at p = 4-5.
A converged solution is kept if its weights are positive and its points lie
inside T; it is written in a canonical form (an S21 orbit by a, an S111 orbit by
its barycentric coordinates sorted, a < b < c, listed as (w, a, b); orbits of
one kind sorted by a), so that the same rule found twice is recognised.  The
rule chosen is the one whose points lie farthest from the edges (the largest
smallest barycentric coordinate over its points); START holds its parameters
to three significant digits, from which symmetric_rules.rule converges to it
in 50-digit arithmetic on the monomial conditions.  With the default 100 starts
per p the search finds 1, 1, 2, 1 and 4 such rules at p = 1..5.
"""
from __future__ import annotations

import numpy as np

try:
    from .symmetric_rules import START
except ImportError:                   # run as a script from oracle/
    from symmetric_rules import START


def structure(p):
    """The orbit kinds of the rule of degree 2p (0 = S3, 1 = S21, 2 = S111)."""
    return [kind for kind, _ in START[p]]


def _points(kinds, x):
    """Barycentric coordinates (l1, l2, l3) [n, 3] and weights [n] of the rule."""
    bary, w, off = [], [], 0
    for kind in kinds:
        if kind == 0:
            bary.append((1 / 3, 1 / 3, 1 / 3)); w.append(x[off]); off += 1
        elif kind == 1:
            a = x[off + 1]
            for t in ((a, a, 1 - 2 * a), (a, 1 - 2 * a, a), (1 - 2 * a, a, a)):
                bary.append(t); w.append(x[off])
            off += 2
        else:
            a, b = x[off + 1], x[off + 2]
            c = 1 - a - b
            for t in ((a, b, c), (b, a, c), (a, c, b), (c, a, b), (b, c, a), (c, b, a)):
                bary.append(t); w.append(x[off])
            off += 3
    return np.array(bary, dtype=float), np.array(w, dtype=float)


def _jacobi(n, al, x):
    """P_0..P_n^{(al, 0)}(x) (numpy arrays), by the three-term recurrence."""
    P = [np.ones_like(x)]
    if n >= 1:
        P.append(0.5 * ((al + 2) * x + al))
    for k in range(2, n + 1):
        a1 = 2 * k * (k + al) * (2 * k + al - 2)
        a2 = (2 * k + al - 1) * al * al
        a3 = (2 * k + al - 2) * (2 * k + al - 1) * (2 * k + al)
        a4 = 2 * (k + al - 1) * (k - 1) * (2 * k + al)
        P.append(((a2 + a3 * x) * P[k - 1] - a4 * P[k - 2]) / a1)
    return P


def _basis(d, r, s):
    """The orthogonal polynomials psi_ij = P_i(e1) ((1 - e2)/2)^i P_j^{(2i+1,0)}(e2),
    i + j <= d, on T (collapsed coordinates e1 = 2 r / (1 - s) - 1, e2 = 2 s - 1),
    at the points (r, s) [..., n]: an array [n_basis, ..., n].  Only psi_00 = 1
    has a nonzero integral over T (1/2), which makes the moment conditions well
    conditioned."""
    e2 = 2 * s - 1
    t = 1 - s
    e1 = np.where(t > 1e-300, 2 * r / np.where(t > 1e-300, t, 1.0) - 1, -1.0)
    Pi = _jacobi(d, 0, e1)
    out = []
    for i in range(d + 1):
        Pj = _jacobi(d - i, 2 * i + 1, e2)
        fac = (t) ** i                       # ((1 - e2)/2)^i = (1 - s)^i
        for j in range(d - i + 1):
            out.append(Pi[i] * fac * Pj[j])
    return np.array(out)


def _residual_many(kinds, X, d):
    """Residuals [m, n_basis] of the parameter sets X [m, n_par]."""
    bary, w = _points_many(kinds, X)
    B = _basis(d, bary[..., 1], bary[..., 2])         # [n_basis, m, n]
    res = np.einsum("bmn,mn->mb", B, w)
    res[:, 0] -= 0.5
    return res


def _points_many(kinds, X):
    """Barycentric coordinates [m, n, 3] and weights [m, n] of parameter sets X."""
    cols_b, cols_w, off = [], [], 0
    one = np.ones(X.shape[0])
    for kind in kinds:
        w = X[:, off]
        if kind == 0:
            cols_b.append(np.stack([one / 3, one / 3, one / 3], -1)); cols_w.append(w); off += 1
        elif kind == 1:
            a = X[:, off + 1]
            c = 1 - 2 * a
            for t in ((a, a, c), (a, c, a), (c, a, a)):
                cols_b.append(np.stack(t, -1)); cols_w.append(w)
            off += 2
        else:
            a, b = X[:, off + 1], X[:, off + 2]
            c = 1 - a - b
            for t in ((a, b, c), (b, a, c), (a, c, b), (c, a, b), (b, c, a), (c, b, a)):
                cols_b.append(np.stack(t, -1)); cols_w.append(w)
            off += 3
    return np.stack(cols_b, 1), np.stack(cols_w, 1)


def _random_start(kinds, rng, npts):
    x = []
    for kind in kinds:
        w = rng.uniform(0.2, 1.8) * 0.5 / npts          # the weights sum to the area 1/2
        if kind == 0:
            x += [w]
        elif kind == 1:
            x += [w, rng.uniform(0.0, 0.5)]
        else:
            l = rng.dirichlet((1.0, 1.0, 1.0))
            x += [w, l[0], l[1]]
    return np.array(x)


def _lm(kinds, x, d, iters=100, h=1e-6):
    """Levenberg-Marquardt on the moment residual (central-difference Jacobian,
    all perturbed parameter sets in one evaluation); returns (x, |residual|)."""
    n = x.size
    E = np.eye(n) * h
    mu = 1e-3
    f = _residual_many(kinds, x[None], d)[0]
    cost = f @ f
    for _ in range(iters):
        R = _residual_many(kinds, np.concatenate([x[None] + E, x[None] - E]), d)
        J = ((R[:n] - R[n:]) / (2 * h)).T
        A = J.T @ J
        g = J.T @ f
        try:
            step = np.linalg.solve(A + mu * np.diag(np.diag(A) + 1e-30), -g)
        except np.linalg.LinAlgError:
            break
        xn = x + step
        fn = _residual_many(kinds, xn[None], d)[0]
        cn = fn @ fn
        if np.isfinite(cn) and cn < cost:
            x, f, cost, mu = xn, fn, cn, max(mu / 3, 1e-12)
            if cost < 1e-30:
                break
        else:
            mu *= 4
            if mu > 1e10:
                break
    return x, np.sqrt(cost)


def canonical(kinds, x):
    """The orbits of a solution as sorted tuples: (kind, w, a[, b])."""
    out, off = [], 0
    for kind in kinds:
        if kind == 0:
            out.append((0, x[off])); off += 1
        elif kind == 1:
            out.append((1, x[off], x[off + 1])); off += 2
        else:
            a, b = x[off + 1], x[off + 2]
            l = sorted((a, b, 1 - a - b))
            out.append((2, x[off], l[0], l[1])); off += 3
    return sorted(out, key=lambda o: (o[0], o[2] if len(o) > 2 else 0.0))


def min_barycentric(kinds, x):
    bary, _ = _points(kinds, x)
    return float(bary.min())


def search(p, starts=100, seed=2016, tol=1e-13):
    """Distinct positive-interior rules of degree 2p found from `starts` seeded
    random starts: a list of (canonical orbits, smallest barycentric coordinate),
    the farthest from the edges first."""
    kinds = structure(p)
    bary0, _ = _points(kinds, np.zeros(sum(1 if k == 0 else k + 1 for k in kinds)))
    npts = len(bary0)
    rng = np.random.default_rng(seed + p)
    found = {}
    for _ in range(starts):
        x, res = _lm(kinds, _random_start(kinds, rng, npts), 2 * p)
        if not res <= tol:
            continue
        bary, w = _points(kinds, x)
        if (w <= 0).any() or bary.min() <= 1e-9:
            continue
        can = canonical(kinds, x)
        key = tuple(round(v, 7) for o in can for v in o)
        found.setdefault(key, (can, min_barycentric(kinds, x)))
    return sorted(found.values(), key=lambda t: -t[1])


def chosen(p, **kw):
    """The rule the oracle uses: the found rule farthest from the edges."""
    rules = search(p, **kw)
    return rules[0] if rules else None


def as_start(can):
    """A canonical rule in START's form, three significant digits."""
    sig = lambda v: float("%.3g" % v)
    return [(o[0], tuple(sig(v) for v in o[1:])) for o in can]


if __name__ == "__main__":
    for p in range(1, 6):
        rules = search(p)
        print("p = %d: %d positive-interior rule(s) of %d points" % (p, len(rules), len(_points(
            structure(p), np.zeros(sum(1 if k == 0 else k + 1 for k in structure(p))))[1])))
        for can, mb in rules:
            print("   smallest barycentric coordinate %.4f: %s" % (mb, as_start(can)))
        print("   START[%d] = %s" % (p, START[p]))
