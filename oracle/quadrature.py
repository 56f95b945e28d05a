"""Oracle: collocation entries of the Laplace-domain single and double layer.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Definitions followed (paper, Section "Boundary element method:
Discretisation", eq. (bie_semi_diri), and the Laplace-domain kernel given
after eq. (conv)):

* Laplace-domain fundamental solution with c = 1:
      U(r, s) = exp(-s r) / (4 pi r),  r = |x - y|.
* Single layer (V), piecewise-constant trial functions, collocation at the
  element centroids x_i (the workloads collocate at centroids):
      V[i, j](s) = int_{tau_j} U(|x_i - y|, s) dS_y.
* Double layer (K), normal derivative at y (eq. (dlp) with the trace
  gamma_{1,y}):  dU/dn_y = exp(-s r) (1 + s r) ((x - y) . n_y) / (4 pi r^3),
      K[i, j](s) = int_{tau_j} dU/dn_y dS_y.
  For y in the plane of tau_j, (x - y) . n_j = (x - v0_j) . n_j, so the plane
  distance is evaluated once per pair; coplanar pairs give exactly 0.
* Regular entries (i != j): the 7-point degree-5 triangle rule (Radon's
  rule; the constants are computed from their closed forms below).  The
  paper's distance-dependent point count is unspecified, so one fixed rule
  is used for every regular pair; no quasi-singular treatment is applied,
  as in the paper.
* Self entries (i == j): V[i, i] is weakly singular.  The oracle splits it
  into the static part, integrated in closed form,
      (1/4pi) int 1/r dS = (1/4pi) sum_edges d_e [asinh(t2/d_e) - asinh(t1/d_e)],
  plus the bounded remainder (exp(-s r) - 1)/(4 pi r), integrated by a Duffy
  map of the three sub-triangles with apex x_i and 48 x 48 Gauss-Legendre
  (converged to about 1e-15 relative on the workloads' triangles).
  K[i, i] = 0 because x_i lies in the plane of tau_i.

Everything is complex128 / float64.
"""
from __future__ import annotations

import math

import numpy as np

FOUR_PI = 4.0 * math.pi


def radon7() -> tuple[np.ndarray, np.ndarray]:
    """Barycentric points (7 x 3) and weights (7, summing to 1) of the
    7-point degree-5 rule on a triangle."""
    r15 = math.sqrt(15.0)
    a1 = (6.0 - r15) / 21.0
    b1 = (9.0 + 2.0 * r15) / 21.0
    a2 = (6.0 + r15) / 21.0
    b2 = (9.0 - 2.0 * r15) / 21.0
    w1 = (155.0 - r15) / 1200.0
    w2 = (155.0 + r15) / 1200.0
    third = 1.0 / 3.0
    pts = np.array([
        [third, third, third],
        [a1, a1, b1], [a1, b1, a1], [b1, a1, a1],
        [a2, a2, b2], [a2, b2, a2], [b2, a2, a2],
    ])
    w = np.array([9.0 / 40.0, w1, w1, w1, w2, w2, w2])
    return pts, w


class Geometry:
    """Per-triangle data in the ORIGINAL element order (float64)."""

    def __init__(self, verts: np.ndarray, tris: np.ndarray):
        self.verts = np.asarray(verts, dtype=np.float64)
        self.tris = np.asarray(tris, dtype=np.int64)
        self.v0 = self.verts[self.tris[:, 0]]
        self.v1 = self.verts[self.tris[:, 1]]
        self.v2 = self.verts[self.tris[:, 2]]
        self.centroid = ((self.v0 + self.v1) + self.v2) / 3.0
        cr = np.cross(self.v1 - self.v0, self.v2 - self.v0)
        nrm = np.linalg.norm(cr, axis=1)
        self.area = 0.5 * nrm
        self.normal = cr / nrm[:, None]
        bary, w = radon7()
        # quadrature points y_q = l0 v0 + l1 v1 + l2 v2 and weights * area
        self.qpts = (bary[None, :, 0, None] * self.v0[:, None, :]
                     + bary[None, :, 1, None] * self.v1[:, None, :]
                     + bary[None, :, 2, None] * self.v2[:, None, :])
        self.qw = w[None, :] * self.area[:, None]

    @property
    def E(self) -> int:
        return self.tris.shape[0]


def _regular(geom: Geometry, kernel: str, I: np.ndarray, J: np.ndarray, s: np.ndarray) -> np.ndarray:
    """Regular-rule entries for pairs (I[n], J[n]) at frequencies s -> [n, nk]."""
    x = geom.centroid[I]                       # [n,3]
    y = geom.qpts[J]                           # [n,7,3]
    diff = x[:, None, :] - y                   # [n,7,3]
    r = np.sqrt(np.einsum("nqd,nqd->nq", diff, diff))   # [n,7]
    sr = s[None, None, :] * r[:, :, None]      # [n,7,nk]
    e = np.exp(-sr)
    w = geom.qw[J]                             # [n,7]
    if kernel == "slp":
        val = e / (FOUR_PI * r[:, :, None])
    elif kernel == "dlp":
        dist = np.einsum("nd,nd->n", x - geom.v0[J], geom.normal[J])   # (x - v0).n
        val = e * (1.0 + sr) * dist[:, None, None] / (FOUR_PI * r[:, :, None] ** 3)
    else:
        raise ValueError(kernel)
    return np.einsum("nq,nqk->nk", w, val)


def gauss_legendre01(n: int) -> tuple[np.ndarray, np.ndarray]:
    x, w = np.polynomial.legendre.leggauss(n)
    return 0.5 * (x + 1.0), 0.5 * w


def slp_static_self(geom: Geometry, j: int) -> float:
    """(1/4pi) int_{tau_j} 1/|x_j - y| dS_y in closed form (x_j = centroid)."""
    x = geom.centroid[j]
    vs = [geom.v0[j], geom.v1[j], geom.v2[j]]
    total = 0.0
    for e in range(3):
        a, b = vs[e], vs[(e + 1) % 3]
        t = b - a
        L = np.linalg.norm(t)
        t = t / L
        t1 = float(np.dot(a - x, t))
        t2 = float(np.dot(b - x, t))
        foot = a - t1 * t
        d = float(np.linalg.norm(foot - x))
        total += d * (math.asinh(t2 / d) - math.asinh(t1 / d))
    return total / FOUR_PI


def slp_self(geom: Geometry, j: int, s: np.ndarray, n_gauss: int = 48) -> np.ndarray:
    """V[j, j](s): closed-form static part + Duffy/Gauss remainder."""
    s = np.atleast_1d(np.asarray(s, dtype=np.complex128))
    x = geom.centroid[j]
    vs = [geom.v0[j], geom.v1[j], geom.v2[j]]
    gx, gw = gauss_legendre01(n_gauss)
    rem = np.zeros(s.shape, dtype=np.complex128)
    for e in range(3):
        a, b = vs[e], vs[(e + 1) % 3]
        two_area = np.linalg.norm(np.cross(a - x, b - x))
        # y(u, v) = x + u ((a - x) + v (b - a)),  dS = two_area * u du dv
        dirs = (a - x)[None, :] + gx[:, None] * (b - a)[None, :]    # [nv,3]
        rho = np.linalg.norm(dirs, axis=1)                           # [nv]
        # integrand (exp(-s u rho) - 1)/(4 pi u rho) * two_area * u
        u = gx[:, None, None]
        rr = rho[None, :, None]
        val = np.expm1(-s[None, None, :] * u * rr) / (FOUR_PI * rr) * two_area
        rem += np.einsum("u,v,uvk->k", gw, gw, val)
    return slp_static_self(geom, j) + rem


def slp_self_duffy_full(geom: Geometry, j: int, s: np.ndarray, n_gauss: int = 60) -> np.ndarray:
    """V[j, j](s) by a Duffy map of the whole integrand (a second method,
    used only to cross-check `slp_self`)."""
    s = np.atleast_1d(np.asarray(s, dtype=np.complex128))
    x = geom.centroid[j]
    vs = [geom.v0[j], geom.v1[j], geom.v2[j]]
    gx, gw = gauss_legendre01(n_gauss)
    out = np.zeros(s.shape, dtype=np.complex128)
    for e in range(3):
        a, b = vs[e], vs[(e + 1) % 3]
        two_area = np.linalg.norm(np.cross(a - x, b - x))
        dirs = (a - x)[None, :] + gx[:, None] * (b - a)[None, :]
        rho = np.linalg.norm(dirs, axis=1)
        u = gx[:, None, None]
        rr = rho[None, :, None]
        val = np.exp(-s[None, None, :] * u * rr) / (FOUR_PI * rr) * two_area
        out += np.einsum("u,v,uvk->k", gw, gw, val)
    return out


def entries(geom: Geometry, kernel: str, I, J, s, chunk: int = 4096) -> np.ndarray:
    """ENTRY(I[n], J[n], s_k) for all pairs and frequencies -> [n, nk] complex128.

    I, J are ORIGINAL element indices (same length); s is a 1-D array.
    """
    I = np.atleast_1d(np.asarray(I, dtype=np.int64))
    J = np.atleast_1d(np.asarray(J, dtype=np.int64))
    s = np.atleast_1d(np.asarray(s, dtype=np.complex128))
    out = np.empty((I.size, s.size), dtype=np.complex128)
    for a in range(0, I.size, chunk):
        Ii = I[a:a + chunk]
        Jj = J[a:a + chunk]
        reg = Ii != Jj
        blk = np.zeros((Ii.size, s.size), dtype=np.complex128)
        if reg.any():
            blk[reg] = _regular(geom, kernel, Ii[reg], Jj[reg], s)
        for n in np.nonzero(~reg)[0]:
            if kernel == "slp":
                blk[n] = slp_self(geom, int(Jj[n]), s)
            else:
                blk[n] = 0.0
        out[a:a + chunk] = blk
    return out


def dense(geom: Geometry, kernel: str, s, rows=None, cols=None) -> np.ndarray:
    """Dense array A[i, j, k] = ENTRY(rows[i], cols[j], s_k) (complex128)."""
    rows = np.arange(geom.E) if rows is None else np.asarray(rows)
    cols = np.arange(geom.E) if cols is None else np.asarray(cols)
    s = np.atleast_1d(np.asarray(s, dtype=np.complex128))
    I = np.repeat(rows, cols.size)
    J = np.tile(cols, rows.size)
    return entries(geom, kernel, I, J, s).reshape(rows.size, cols.size, s.size)
