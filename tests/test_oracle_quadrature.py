"""Pins for the oracle's collocation entries: polynomial exactness of the
triangle rule, the unit-sphere closed forms for V and K, the static Gauss
identity on the cube, coplanar zeros, and two independent singular
quadratures."""
import math

import numpy as np
import pytest

from inputs import meshes
from oracle import quadrature as Q


def _monomial_exact(a: int, b: int) -> float:
    # int over {x, y >= 0, x + y <= 1} of x^a y^b = a! b! / (a + b + 2)!
    return math.factorial(a) * math.factorial(b) / math.factorial(a + b + 2)


def test_radon7_degree5_exact_not_degree6():
    bary, w = Q.radon7()
    assert abs(w.sum() - 1.0) < 1e-15
    x, y = bary[:, 1], bary[:, 2]      # reference triangle (0,0),(1,0),(0,1), area 1/2
    for deg in range(6):
        for a in range(deg + 1):
            b = deg - a
            quad = 0.5 * np.sum(w * x ** a * y ** b)
            assert abs(quad - _monomial_exact(a, b)) < 1e-15, (a, b)
    errs = [abs(0.5 * np.sum(w * x ** a * y ** (6 - a)) - _monomial_exact(a, 6 - a)) for a in range(7)]
    assert max(errs) > 1e-6


def _sphere_rowsums(level, s, rows=(0, 17, 101)):
    g = Q.Geometry(*meshes.icosphere(level))
    out_v, out_k = [], []
    for i in rows:
        I = np.full(g.E, i)
        J = np.arange(g.E)
        out_v.append(Q.entries(g, "slp", I, J, s).sum(0))
        out_k.append(Q.entries(g, "dlp", I, J, s).sum(0))
    return np.array(out_v), np.array(out_k)


def test_unit_sphere_identities_converge_second_order():
    """int_{S^2} exp(-s r)/(4 pi r) dS_y = (1 - e^{-2s})/(2s) and
    int_{S^2} dU/dn_y dS_y = -(1 - (1 + s) e^{-2s})/(2s) for |x| = 1
    (derived from (x - y).y = -r^2/2 on the unit sphere); the flat
    icosphere approximation converges with order 2 in h."""
    s = np.array([0.5, 2.0, 5.0 + 5.0j, 1e-8, 3.0 - 12.0j])
    exact_v = -np.expm1(-2 * s) / (2 * s)
    exact_k = -(1 - (1 + s) * np.exp(-2 * s)) / (2 * s)
    ev, ek = [], []
    for lvl in (2, 3, 4):
        v, k = _sphere_rowsums(lvl, s)
        ev.append(np.abs(v - exact_v).max())
        ek.append(np.abs(k - exact_k).max())
    for e in (ev, ek):
        orders = [math.log2(e[i] / e[i + 1]) for i in range(2)]
        assert min(orders) > 1.8, (e, orders)
        assert e[-1] < 2e-3


def test_cube_static_gauss_identity_dlp():
    """sum_j K[i, j](s -> 0) = -1/2 at points on the smooth part of a closed
    surface (Gauss' solid-angle integral; sign fixed by (x - y).n_y)."""
    g = Q.Geometry(*meshes.cube(8))
    # centroids away from cube edges: centroid more than 2 h from every edge
    c = g.centroid
    far_from_edges = np.sum((c > 0.25) & (c < 0.75), axis=1) == 2
    rows = np.nonzero(far_from_edges)[0][:6]
    assert rows.size == 6
    for i in rows:
        val = Q.entries(g, "dlp", np.full(g.E, i), np.arange(g.E), np.array([1e-9]))[:, 0].sum()
        assert abs(val - (-0.5)) < 2e-3, (i, val)


def test_coplanar_dlp_entries_exactly_zero():
    g = Q.Geometry(*meshes.lshape(4))
    s = np.array([1.0 + 2.0j, 7.0])
    n = g.normal
    for i in range(0, g.E, 7):
        J = np.nonzero((np.abs(n @ n[i]) == 1.0) &
                       (np.abs(np.einsum("jd,d->j", g.v0 - g.centroid[i], n[i])) == 0.0))[0]
        A = Q.entries(g, "dlp", np.full(J.size, i), J, s)
        assert np.all(A == 0.0)


def test_self_term_two_methods_agree():
    g = Q.Geometry(*meshes.icosphere(3))
    g2 = Q.Geometry(*meshes.lshape(32))
    s = np.array([1e-12, 0.5, 3.0 + 10.0j, 50.0 - 100.0j, 200.0, 3.6 - 12.0j])
    for geo, js in ((g, [0, 9, 500]), (g2, [0, 77, 12000])):
        for j in js:
            a = Q.slp_self(geo, j, s)
            b = Q.slp_self_duffy_full(geo, j, s)
            assert np.max(np.abs(a - b)) <= 1e-10 * np.max(np.abs(a))
            # s -> 0: the closed-form static integral
            assert abs(a[0] - Q.slp_static_self(geo, j)) < 1e-10 * abs(a[0])


def test_static_self_matches_duffy_at_s0():
    """Closed-form int 1/r over a triangle vs. the Duffy map of the three
    sub-triangles with apex x at s = 0, 120 x 120 Gauss-Legendre points."""
    v, t = meshes.icosphere(1)
    g = Q.Geometry(v, t)
    j = 3
    ref = Q.slp_static_self(g, j)
    alt = Q.slp_self_duffy_full(g, j, np.array([0.0]), n_gauss=120)[0].real
    assert abs(ref - alt) < 1e-12 * ref


def test_conjugate_symmetry_of_entries():
    g = Q.Geometry(*meshes.cube(4))
    s = np.array([0.7 + 3.0j, 12.0 - 40.0j])
    I = np.arange(0, g.E, 3)
    J = (I * 7 + 1) % g.E
    for ker in ("slp", "dlp"):
        a = Q.entries(g, ker, I, J, s)
        b = Q.entries(g, ker, I, J, np.conj(s))
        assert np.max(np.abs(a - np.conj(b))) <= 1e-15 * np.max(np.abs(a))


def test_regular_entry_converges_to_subdivided_integral():
    """The 7-point rule on a well-separated pair agrees with a fine
    subdivision of the trial triangle to the rule's O(h^6) error (about 5e-6
    relative for h = 1/4, |s| = 5.4, r = 0.95)."""
    g = Q.Geometry(*meshes.cube(4))
    i, j = 0, 150
    s = np.array([2.0 + 5.0j])
    base = Q.entries(g, "slp", [i], [j], s)[0, 0]
    # subdivide tau_j into 4^3 triangles, 7 points each
    bary, w = Q.radon7()
    tri = [np.array([g.v0[j], g.v1[j], g.v2[j]])]
    for _ in range(3):
        nxt = []
        for a, b, c in tri:
            ab, bc, ca = (a + b) / 2, (b + c) / 2, (c + a) / 2
            nxt += [np.array(x) for x in ([a, ab, ca], [b, bc, ab], [c, ca, bc], [ab, bc, ca])]
        tri = nxt
    x = g.centroid[i]
    tot = 0.0
    for a, b, c in tri:
        area = 0.5 * np.linalg.norm(np.cross(b - a, c - a))
        y = bary @ np.array([a, b, c])
        r = np.linalg.norm(x - y, axis=1)
        tot += area * np.sum(w * np.exp(-s[0] * r) / (4 * np.pi * r))
    assert abs(base - tot) < 5e-5 * abs(tot)
