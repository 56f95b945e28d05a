"""Oracle: Galerkin hypersingular operator D and adjoint double layer K' with
linear continuous elements (the Neumann problem, eq. (bie_semi_neum)).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

The Neumann problem of Section 2 is discretised with the nodal (piecewise
linear, continuous) shape functions phi_i and the Galerkin scheme:

    D(s)[i, j]  = <phi_i, gamma_1,x W phi_j>     (hypersingular operator)
    K'(s)[i, j] = int phi_i(x) int d/dn_x U(x - y, s) phi_j(y) dy dx

with U(r, s) = exp(-s r) / (4 pi r), the Laplace-domain fundamental solution
of the section on the wave equation.

Readings (the paper states the operators, not how their integrals are done):

* D by integration by parts (the Maue form for the operator s^2 - Delta):
      D[i, j] = int int U(x - y, s) [ curl phi_i(x) . curl phi_j(y)
                                      + s^2 (n_x . n_y) phi_i(x) phi_j(y) ] dy dx,
  curl phi = n x grad_Gamma phi, constant on a flat triangle.  This is the
  symmetric form whose value on the unit sphere is the positive eigenvalue
  -s^3 i_n'(s) k_n'(s) (pinned); the paper's sign convention for gamma_1
  enters the right side of eq. (bie_semi_neum), not the operator's
  compression or application.
* d/dn_x U(x - y, s) = -exp(-s r) (1 + s r) ((x - y) . n_x) / (4 pi r^3),
  the derivative of U in the outward normal at the test point; for x and y on
  one flat triangle it is exactly zero.
* The integrals are assembled element pair by element pair in local 3 x 3
  blocks (test element tau, local vertex a; trial element sigma, local
  vertex b), D[i, j] = sum over tau containing i and sigma containing j of the
  local entries.  Regular pairs (no common vertex) use the 4-point degree-3
  rule on each triangle (16 kernel evaluations per pair), the pairs with a
  common vertex, a common edge or identical panels the Sauter-Schwab
  transformations to [0, 1]^4 with n Gauss-Legendre points per coordinate,
  as the piecewise-constant single layer (Section 2: Erichsen-Sauter rules
  for the weakly singular integrals, Gauss rules for the regular ones).

The local functions are the barycentric coordinates: on the panel
chi(x1, x2) = P0 + x1 (P1 - P0) + x2 (P2 - P1) of the reference triangle
0 <= x2 <= x1 <= 1, lambda = (1 - x1, x1 - x2, x2) for (P0, P1, P2).
"""
from __future__ import annotations

import numpy as np

from . import galerkin as G

FOUR_PI = 4.0 * np.pi


def panel(verts: np.ndarray, tri) -> tuple[np.ndarray, np.ndarray, float]:
    """(vertices [3, 3], unit normal [3], area) of a triangle (counter-clockwise
    vertices seen from outside give the outward normal)."""
    P = verts[np.asarray(tri)]
    c = np.cross(P[1] - P[0], P[2] - P[0])
    a2 = np.linalg.norm(c)
    return P, c / a2, 0.5 * a2


def surface_curls(P: np.ndarray, n: np.ndarray, area: float) -> np.ndarray:
    """curl_Gamma lambda_a = n x grad_Gamma lambda_a [3 (local a), 3] for the
    barycentric coordinates of the flat triangle P (vertices in any order) and
    its outward unit normal n: grad_Gamma lambda_a = m x (P_{a+2} - P_{a+1}) /
    (2 area) with m the unit normal of the vertex order of P."""
    c = np.cross(P[1] - P[0], P[2] - P[0])
    m = c / np.linalg.norm(c)
    g = np.array([np.cross(m, P[(a + 2) % 3] - P[(a + 1) % 3]) / (2.0 * area) for a in range(3)])
    return np.cross(n[None, :], g)


def _bary(x1, x2) -> np.ndarray:
    return np.stack([1.0 - x1, x1 - x2, x2], axis=-1)


def _kernels(s: np.ndarray):
    """U and d/dn_x U as functions of (z = x - y [..., 3], n_x [3]) -> [..., m]."""
    s = np.atleast_1d(np.asarray(s, dtype=np.complex128))

    def U(z):
        r = np.linalg.norm(z, axis=-1)[..., None]
        return np.exp(-s[None, :] * r) / (FOUR_PI * r)

    def dUdnx(z, nx):
        r = np.linalg.norm(z, axis=-1)[..., None]
        zn = (z @ nx)[..., None]
        return -np.exp(-s[None, :] * r) * (1.0 + s[None, :] * r) * zn / (FOUR_PI * r ** 3)

    return U, dUdnx


def _local_regular(Px, nx, ax, Py, ny, ay, s, op):
    """Local 3 x 3 block [a, b, m] of a regular pair (4-point rule on each panel)."""
    U, dUdnx = _kernels(s)
    L, W = G.stroud4()                      # barycentric points [4, 3], weights sum 1
    xp = L @ Px
    yq = L @ Py
    z = xp[:, None, :] - yq[None, :, :]     # [4, 4, 3]
    wt = np.outer(W * ax, W * ay)           # [4, 4]
    phix, phiy = L, L                       # lambda_a at the points [4, 3]
    if op == "kp":
        k = dUdnx(z, nx)                    # [4, 4, m]
        return np.einsum("pq,pa,qb,pqm->abm", wt, phix, phiy, k)
    k = U(z)
    i0 = np.einsum("pq,pqm->m", wt, k)
    iab = np.einsum("pq,pa,qb,pqm->abm", wt, phix, phiy, k)
    cx, cy = surface_curls(Px, nx, ax), surface_curls(Py, ny, ay)
    s = np.atleast_1d(np.asarray(s, dtype=np.complex128))
    return (cx @ cy.T)[:, :, None] * i0[None, None, :] + (s ** 2)[None, None, :] * float(nx @ ny) * iab


def _local_singular(case, Px, nx, ax, Py, ny, ay, s, op, n):
    """Local 3 x 3 block of a pair with a common vertex / edge / panel, in the
    vertex order of Px and Py (shared vertices first), by the Sauter-Schwab
    maps of oracle.galerkin."""
    U, dUdnx = _kernels(s)
    (xi, e1, e2, e3), W = G._grid4(n)
    s = np.atleast_1d(np.asarray(s, dtype=np.complex128))
    m = s.size
    i0 = np.zeros(m, complex)
    iab = np.zeros((3, 3, m), complex)
    for f, (a1, a2), (b1, b2) in G._maps(case, xi, e1, e2, e3):
        x = G._chi(Px, a1, a2)
        y = G._chi(Py, b1, b2)
        z = x - y
        w = W * f
        lx, ly = _bary(a1, a2), _bary(b1, b2)          # [q, 3]
        k = dUdnx(z, nx) if op == "kp" else U(z)       # [q, m]
        iab += np.einsum("q,qa,qb,qm->abm", w, lx, ly, k)
        if op == "d":
            i0 += np.einsum("q,qm->m", w, k)
    jac = (2.0 * ax) * (2.0 * ay)
    iab *= jac
    i0 *= jac
    if op == "kp":
        return iab
    cx, cy = surface_curls(Px, nx, ax), surface_curls(Py, ny, ay)
    return (cx @ cy.T)[:, :, None] * i0[None, None, :] + (s ** 2)[None, None, :] * float(nx @ ny) * iab


def local_block(verts, tris, t: int, u: int, s, op: str, n: int = 6) -> np.ndarray:
    """Local block [3, 3, m] of the element pair (test tau_t, trial sigma_u) in
    the original vertex order of both triangles; op = "d" (hypersingular, Maue
    form) or "kp" (adjoint double layer)."""
    verts = np.asarray(verts, dtype=np.float64)
    tris = np.asarray(tris)
    case, oa, ob = G.classify(tris, int(t), int(u))
    Px, nx, ax = panel(verts, tris[t])
    Py, ny, ay = panel(verts, tris[u])
    if case == "regular":
        return _local_regular(Px, nx, ax, Py, ny, ay, s, op)
    if case == "identical" and op == "kp":
        return np.zeros((3, 3, np.atleast_1d(s).size), complex)   # (x - y) . n_x = 0 on a flat panel
    Pa, Pb = verts[oa], verts[ob]
    blk = _local_singular(case, Pa, nx, ax, Pb, ny, ay, s, op, n)
    # back to the original local numbering of both triangles
    ia = [list(tris[t]).index(v) for v in oa]
    ib = [list(tris[u]).index(v) for v in ob]
    out = np.zeros_like(blk)
    for p in range(3):
        for q in range(3):
            out[ia[p], ib[q]] = blk[p, q]
    return out


def dense_nodal(verts, tris, s, op: str, n: int = 6) -> np.ndarray:
    """Dense nodal Galerkin matrix [nv, nv, m] of D ("d") or K' ("kp"),
    assembled from all element pairs (small meshes only): the regular pairs
    with the 4-point rule on each panel in one array pass, the others one by
    one through local_block."""
    verts = np.asarray(verts, dtype=np.float64)
    tris = np.asarray(tris)
    s = np.atleast_1d(np.asarray(s, dtype=np.complex128))
    nv, E = verts.shape[0], tris.shape[0]
    out = np.zeros((nv, nv, s.size), complex)
    # geometry of all panels
    P = verts[tris]                                               # [E, 3, 3]
    c = np.cross(P[:, 1] - P[:, 0], P[:, 2] - P[:, 0])
    area = 0.5 * np.linalg.norm(c, axis=1)
    nrm = c / (2.0 * area[:, None])
    curls = np.array([surface_curls(P[e], nrm[e], area[e]) for e in range(E)])   # [E, 3, 3]
    L, W = G.stroud4()
    X = np.einsum("qa,eac->eqc", L, P)                           # [E, 4, 3] quadrature points
    Wa = W[None, :] * area[:, None]                               # [E, 4]
    shared = np.zeros((E, E), dtype=bool)
    for v in range(nv):
        els = np.flatnonzero((tris == v).any(axis=1))
        shared[np.ix_(els, els)] = True
    for t in range(E):
        us = np.flatnonzero(~shared[t])
        z = X[t][None, :, None, :] - X[us][:, None, :, :]         # [u, 4, 4, 3]
        r = np.linalg.norm(z, axis=-1)[..., None]                 # [u, 4, 4, 1]
        e = np.exp(-s[None, None, None, :] * r)
        wt = Wa[t][None, :, None] * Wa[us][:, None, :]            # [u, 4, 4]
        if op == "kp":
            zn = (z @ nrm[t])[..., None]
            k = -e * (1.0 + s[None, None, None, :] * r) * zn / (FOUR_PI * r ** 3)
            blk = np.einsum("upq,pa,qb,upqm->uabm", wt, L, L, k)
        else:
            k = e / (FOUR_PI * r)
            i0 = np.einsum("upq,upqm->um", wt, k)
            iab = np.einsum("upq,pa,qb,upqm->uabm", wt, L, L, k)
            cc = np.einsum("ac,ubc->uab", curls[t], curls[us])
            nn = nrm[us] @ nrm[t]
            blk = cc[..., None] * i0[:, None, None, :] + (s ** 2)[None, None, None, :] * nn[:, None, None, None] * iab
        for a in range(3):
            for b in range(3):
                np.add.at(out, (tris[t][a], tris[us, b]), blk[:, a, b])
        for u in np.flatnonzero(shared[t]):
            out[np.ix_(tris[t], tris[u])] += local_block(verts, tris, t, int(u), s, op, n)
    return out


def nodal_rows(verts, tris, rows, s, op: str, n: int = 6) -> np.ndarray:
    """Rows [len(rows), nv, m] of the nodal Galerkin matrix of D ("d") or K'
    ("kp"): for each row vertex, the sum over the elements that contain it of
    their local blocks with every element."""
    verts = np.asarray(verts, dtype=np.float64)
    tris = np.asarray(tris)
    s = np.atleast_1d(np.asarray(s, dtype=np.complex128))
    nv, E = verts.shape[0], tris.shape[0]
    out = np.zeros((len(rows), nv, s.size), complex)
    for r, i in enumerate(rows):
        for t in np.flatnonzero((tris == i).any(axis=1)):
            a = list(tris[t]).index(i)
            for u in range(E):
                blk = local_block(verts, tris, int(t), u, s, op, n)
                for b in range(3):
                    out[r, tris[u][b]] += blk[a, b]
    return out


def mass_p1(verts, tris) -> np.ndarray:
    """Nodal mass matrix int phi_i phi_j (exact: area / 12 (1 + delta_ab))."""
    verts = np.asarray(verts, dtype=np.float64)
    tris = np.asarray(tris)
    nv = verts.shape[0]
    Mm = np.zeros((nv, nv))
    loc = (np.ones((3, 3)) + np.eye(3)) / 12.0
    for tri in tris:
        _, _, a = panel(verts, tri)
        Mm[np.ix_(tri, tri)] += a * loc
    return Mm
