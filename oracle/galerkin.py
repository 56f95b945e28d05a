"""Oracle: Galerkin single-layer entries for piecewise-constant elements.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

The Galerkin scheme of Section 2 (eq. (bie_semi_indirect)) needs, for the
single layer with piecewise-constant test and trial functions,

    V(s)[i, j] = int_{tau_i} int_{tau_j} exp(-s |x - y|) / (4 pi |x - y|) dy dx.

Readings (Section 2, paragraph after eq. (bie_semi_neum): Gauss rules for the
regular integrals, the Erichsen-Sauter rules for the weakly singular ones):

* Regular pairs (no common vertex): a 4-point rule on each triangle, 16
  kernel evaluations per entry.  The 4-point rule is the conical product of a
  2-point Gauss-Jacobi rule (weight 1 - u) in u and a 2-point Gauss-Legendre
  rule in v, mapped by l1 = u, l2 = v (1 - u); it is exact for polynomials of
  degree 3.
* Pairs with a common vertex, a common edge, or identical panels: the
  Sauter-Schwab transformations to [0, 1]^4 (Sauter and Schwab, Boundary
  Element Methods, Section 5.2), whose Jacobians cancel the 1/r singularity,
  with an n-point Gauss-Legendre rule per coordinate (n = 6 by default),
  float64.

Reference triangle T = {(x1, x2): 0 <= x2 <= x1 <= 1}; the panel with
vertices (P0, P1, P2) is chi(x1, x2) = P0 + x1 (P1 - P0) + x2 (P2 - P1), with
Jacobian 2 |tau|.  For a common edge both panels list the shared vertices
first in the same order (the edge is x2 = 0); for a common vertex both list
it first.

``potential_triangle`` is the closed-form integral of 1/|x - y| over a flat
triangle (Wilton et al. 1984); the tests use it, with an independent outer
quadrature, to pin the singular rules.
"""
from __future__ import annotations

import numpy as np

FOUR_PI = 4.0 * np.pi


# ---------------------------------------------------------------------------
# rules

def stroud4() -> tuple[np.ndarray, np.ndarray]:
    """Barycentric points (l0, l1, l2) [4, 3] and weights [4] (sum 1) of the
    4-point degree-3 conical product rule."""
    r6 = np.sqrt(6.0)
    u = np.array([(4.0 - r6) / 10.0, (4.0 + r6) / 10.0])
    wu = np.array([(9.0 + r6) / 36.0, (9.0 - r6) / 36.0])     # Gauss-Jacobi, weight (1 - u), sum 1/2
    v = np.array([0.5 - 0.5 / np.sqrt(3.0), 0.5 + 0.5 / np.sqrt(3.0)])
    pts, w = [], []
    for a in range(2):
        for b in range(2):
            l1 = u[a]
            l2 = v[b] * (1.0 - u[a])
            pts.append([1.0 - l1 - l2, l1, l2])
            w.append(2.0 * wu[a] * 0.5)                       # reference area 1/2 -> weights sum to 1
    return np.array(pts), np.array(w)


def gauss_legendre01(n: int) -> tuple[np.ndarray, np.ndarray]:
    x, w = np.polynomial.legendre.leggauss(n)
    return 0.5 * (x + 1.0), 0.5 * w


# ---------------------------------------------------------------------------
# Sauter-Schwab rules on [0, 1]^4

def _chi(P: np.ndarray, x1: np.ndarray, x2: np.ndarray) -> np.ndarray:
    return P[0] + x1[..., None] * (P[1] - P[0]) + x2[..., None] * (P[2] - P[1])


def _area(P: np.ndarray) -> float:
    return 0.5 * np.linalg.norm(np.cross(P[1] - P[0], P[2] - P[0]))


def _grid4(n: int):
    g, w = gauss_legendre01(n)
    X = np.meshgrid(g, g, g, g, indexing="ij")
    W = np.einsum("a,b,c,d->abcd", w, w, w, w)
    return [x.ravel() for x in X], W.ravel()


def _maps(case: str, xi, e1, e2, e3):
    """(weight factor, x-hat, y-hat) for every region of the case."""
    one = np.ones_like(xi)
    if case == "identical":
        f = xi ** 3 * e1 ** 2 * e2
        return [
            (f, (xi, xi * (1 - e1 + e1 * e2)), (xi * (1 - e1 * e2 * e3), xi * (1 - e1))),
            (f, (xi * (1 - e1 * e2 * e3), xi * (1 - e1)), (xi, xi * (1 - e1 + e1 * e2))),
            (f, (xi, xi * e1 * (1 - e2 + e2 * e3)), (xi * (1 - e1 * e2), xi * e1 * (1 - e2))),
            (f, (xi * (1 - e1 * e2), xi * e1 * (1 - e2)), (xi, xi * e1 * (1 - e2 + e2 * e3))),
            (f, (xi * (1 - e1 * e2 * e3), xi * e1 * (1 - e2 * e3)), (xi, xi * e1 * (1 - e2))),
            (f, (xi, xi * e1 * (1 - e2)), (xi * (1 - e1 * e2 * e3), xi * e1 * (1 - e2 * e3))),
        ]
    if case == "edge":
        f1 = xi ** 3 * e1 ** 2
        f = xi ** 3 * e1 ** 2 * e2
        return [
            (f1, (xi, xi * e1 * e3), (xi * (1 - e1 * e2), xi * e1 * (1 - e2))),
            (f, (xi, xi * e1), (xi * (1 - e1 * e2 * e3), xi * e1 * e2 * (1 - e3))),
            (f, (xi * (1 - e1 * e2), xi * e1 * (1 - e2)), (xi, xi * e1 * e2 * e3)),
            (f, (xi * (1 - e1 * e2 * e3), xi * e1 * e2 * (1 - e3)), (xi, xi * e1)),
            (f, (xi * (1 - e1 * e2 * e3), xi * e1 * (1 - e2 * e3)), (xi, xi * e1 * e2)),
        ]
    if case == "vertex":
        f = xi ** 3 * e2
        return [
            (f, (xi, xi * e1), (xi * e2, xi * e2 * e3)),
            (f, (xi * e2, xi * e2 * e3), (xi, xi * e1)),
        ]
    raise ValueError(case)


def sauter_schwab(case: str, Px: np.ndarray, Py: np.ndarray, kernel, n: int = 6) -> np.ndarray:
    """int_{tau_x} int_{tau_y} kernel(x - y) dy dx for the given case; kernel
    maps differences [..., 3] to values [..., m] (m outputs, e.g. frequencies).
    Px, Py: [3, 3] vertex arrays ordered as the module docstring says."""
    (xi, e1, e2, e3), W = _grid4(n)
    total = 0.0
    for f, (a1, a2), (b1, b2) in _maps(case, xi, e1, e2, e3):
        z = _chi(Px, a1, a2) - _chi(Py, b1, b2)
        total = total + np.einsum("q,qm->m", W * f, kernel(z))
    return total * (2.0 * _area(Px)) * (2.0 * _area(Py))


def helmholtz_kernel(s: np.ndarray):
    s = np.atleast_1d(np.asarray(s, dtype=np.complex128))

    def k(z):
        r = np.linalg.norm(z, axis=-1)[..., None]
        return np.exp(-s[None, :] * r) / (FOUR_PI * r)
    return k


# ---------------------------------------------------------------------------
# closed-form potential of a uniform triangle (static kernel, pins only)

def potential_triangle(P: np.ndarray, x: np.ndarray) -> np.ndarray:
    """int_T 1/|x - y| dy for points x [m, 3] (any position)."""
    P = np.asarray(P, dtype=np.float64)
    x = np.atleast_2d(np.asarray(x, dtype=np.float64))
    nrm = np.cross(P[1] - P[0], P[2] - P[0])
    nrm = nrm / np.linalg.norm(nrm)
    d = (x - P[0]) @ nrm                      # signed height
    rho = x - d[:, None] * nrm                # projection onto the plane
    out = np.zeros(x.shape[0])
    ad = np.abs(d)
    for e in range(3):
        a, b = P[e], P[(e + 1) % 3]
        lvec = (b - a) / np.linalg.norm(b - a)
        u = np.cross(lvec, nrm)               # in-plane edge normal, outward for counter-clockwise vertices
        lp = (b - rho) @ lvec
        lm = (a - rho) @ lvec
        p0 = (a - rho) @ u                    # signed distance of the projection to the edge line
        r0sq = p0 ** 2 + d ** 2
        rp = np.sqrt(lp ** 2 + r0sq)
        rm = np.sqrt(lm ** 2 + r0sq)
        with np.errstate(divide="ignore", invalid="ignore"):
            # r + l without cancellation when l < 0: (r^2 - l^2) / (r - l)
            sp = np.where(lp >= 0, rp + lp, r0sq / (rp - lp))
            sm = np.where(lm >= 0, rm + lm, r0sq / (rm - lm))
            logt = np.log(sp / sm)
            logt = np.where(np.abs(p0) > 0, logt, 0.0)
            at = np.arctan2(p0 * lp, r0sq + ad * rp) - np.arctan2(p0 * lm, r0sq + ad * rm)
        out += p0 * logt - ad * at
    return out


# ---------------------------------------------------------------------------
# entries

def classify(tris: np.ndarray, i: int, j: int):
    """('regular' | 'vertex' | 'edge' | 'identical', vertex order of tau_i,
    vertex order of tau_j) with the shared vertices first (same order)."""
    a, b = list(tris[i]), list(tris[j])
    common = [v for v in a if v in b]
    if len(common) == 0:
        return "regular", a, b
    if len(common) == 3:
        return "identical", a, a
    if len(common) == 1:
        v = common[0]
        return "vertex", [v] + [x for x in a if x != v], [v] + [x for x in b if x != v]
    # common edge: keep the edge direction of tau_i for both
    ia = [a.index(c) for c in common]
    if (ia[0] + 1) % 3 == ia[1]:
        e0, e1 = common[0], common[1]
    else:
        e0, e1 = common[1], common[0]
    return "edge", [e0, e1] + [x for x in a if x not in common], [e0, e1] + [x for x in b if x not in common]


def entries(verts, tris, I, J, s, n: int = 6) -> np.ndarray:
    """V(s)[I[t], J[t]] for the pairs t, all s: [n_pairs, len(s)] complex128."""
    verts = np.asarray(verts, dtype=np.float64)
    tris = np.asarray(tris)
    s = np.atleast_1d(np.asarray(s, dtype=np.complex128))
    k = helmholtz_kernel(s)
    L, W = stroud4()
    out = np.zeros((len(I), s.size), dtype=np.complex128)
    for t, (i, j) in enumerate(zip(I, J)):
        case, oa, ob = classify(tris, int(i), int(j))
        if case == "regular":
            Pi, Pj = verts[tris[i]], verts[tris[j]]
            xp = L @ Pi
            yq = L @ Pj
            z = xp[:, None, :] - yq[None, :, :]
            wt = np.outer(W * _area(Pi), W * _area(Pj))
            out[t] = np.einsum("pq,pqm->m", wt, k(z))
        else:
            out[t] = sauter_schwab(case, verts[oa], verts[ob], k, n)
    return out


def dense(verts, tris, s, rows=None, cols=None, n: int = 6) -> np.ndarray:
    """Dense V(s)[rows, cols, k] (original element indices)."""
    E = np.asarray(tris).shape[0]
    rows = np.arange(E) if rows is None else np.asarray(rows)
    cols = np.arange(E) if cols is None else np.asarray(cols)
    I = np.repeat(rows, cols.size)
    J = np.tile(cols, rows.size)
    return entries(verts, tris, I, J, s, n).reshape(rows.size, cols.size, -1)
