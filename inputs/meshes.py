"""Seeded synthetic surface meshes (flat triangles, outward counter-clockwise).

This module only builds geometry: vertex coordinates and triangle index
triples.  It holds none of the boundary element arithmetic, so both the
CPU oracle and the CUDA path consume its output.

The geometries stand in for the paper's test bodies (Section "Numerical
examples"): the unit cube, the cube with a re-entrant corner ("L-shape")
and the unit ball.  The paper's own meshes are not available, so uniform
structured meshes of the same bodies are generated here.

Every mesh is closed (each edge is shared by exactly two triangles) and
oriented so that the right-hand normal of (v0, v1, v2) points out of the
body.
"""
from __future__ import annotations

import numpy as np


def _orient_outward(verts: np.ndarray, tris: np.ndarray, outward: np.ndarray) -> np.ndarray:
    """Swap v1/v2 of every triangle whose right-hand normal opposes `outward`."""
    a = verts[tris[:, 0]]
    b = verts[tris[:, 1]]
    c = verts[tris[:, 2]]
    n = np.cross(b - a, c - a)
    flip = np.einsum("ij,ij->i", n, outward) < 0
    out = tris.copy()
    out[flip, 1], out[flip, 2] = tris[flip, 2], tris[flip, 1]
    return out


class _LatticeMesh:
    """Collects axis-aligned unit squares on an integer lattice and splits them.

    Vertices are identified by integer lattice coordinates, so shared edges
    are shared exactly; coordinates are scaled by `h` at the end (h is a
    power of two for every workload here, so the scaling is exact).
    """

    def __init__(self) -> None:
        self.vid: dict[tuple[int, int, int], int] = {}
        self.tris: list[tuple[int, int, int]] = []
        self.normals: list[tuple[int, int, int]] = []

    def _v(self, p: tuple[int, int, int]) -> int:
        if p not in self.vid:
            self.vid[p] = len(self.vid)
        return self.vid[p]

    def square(self, axis: int, level: int, u0: int, v0: int, sign: int) -> None:
        """Add the unit square {axis = level, u in [u0,u0+1], v in [v0,v0+1]}.

        (u, v) are the two other axes in increasing order.  The square is
        split along the diagonal through its lowest (u, v) corner.
        """
        ua, va = [d for d in range(3) if d != axis]

        def P(u: int, v: int) -> tuple[int, int, int]:
            p = [0, 0, 0]
            p[axis] = level
            p[ua] = u
            p[va] = v
            return tuple(p)  # type: ignore[return-value]

        p00 = self._v(P(u0, v0))
        p10 = self._v(P(u0 + 1, v0))
        p11 = self._v(P(u0 + 1, v0 + 1))
        p01 = self._v(P(u0, v0 + 1))
        nrm = [0, 0, 0]
        nrm[axis] = sign
        self.tris.append((p00, p10, p11))
        self.tris.append((p00, p11, p01))
        self.normals.append(tuple(nrm))
        self.normals.append(tuple(nrm))

    def finish(self, h: float) -> tuple[np.ndarray, np.ndarray]:
        pts = np.zeros((len(self.vid), 3), dtype=np.float64)
        for p, i in self.vid.items():
            pts[i] = p
        verts = pts * h
        tris = np.asarray(self.tris, dtype=np.int32)
        outward = np.asarray(self.normals, dtype=np.float64)
        return verts, _orient_outward(verts, tris, outward)


def cube(n: int, origin: float = 0.0) -> tuple[np.ndarray, np.ndarray]:
    """Surface of the cube [origin, origin+1]^3 with n x n squares per face.

    Returns (verts [nv,3] float64, tris [12 n^2, 3] int32).  n must be a
    power of two for exact coordinates; other n are allowed (coordinates are
    then rounded once from k/n).
    """
    m = _LatticeMesh()
    for axis in range(3):
        for level, sign in ((0, -1), (n, +1)):
            for u in range(n):
                for v in range(n):
                    m.square(axis, level, u, v, sign)
    if n & (n - 1) == 0:
        verts, tris = m.finish(1.0 / n)
    else:
        vi, tris = m.finish(1.0)
        verts = vi / n
    return verts + origin, tris


def lshape(n: int) -> tuple[np.ndarray, np.ndarray]:
    """Unit cube [0,1]^3 minus the octant [1/2,1]^3, uniform squares of side 1/n.

    n must be even.  The surface has nine planar faces (three full unit
    squares, three L-shaped faces of area 3/4, three inner faces of area
    1/4), total area 6, hence 12 n^2 triangles (n = 32 gives 12,288).
    """
    assert n % 2 == 0
    half = n // 2
    m = _LatticeMesh()

    def removed(c: tuple[float, float, float]) -> bool:
        return all(x > half for x in c)

    # A lattice square lies on the surface iff exactly one of the two unit
    # cells on either side of it belongs to the solid.
    def solid(cell: tuple[int, int, int]) -> bool:
        if any(x < 0 or x >= n for x in cell):
            return False
        centre = tuple(x + 0.5 for x in cell)
        return not removed(centre)  # type: ignore[arg-type]

    for axis in range(3):
        ua, va = [d for d in range(3) if d != axis]
        for level in range(n + 1):
            for u in range(n):
                for v in range(n):
                    lo = [0, 0, 0]
                    lo[axis] = level - 1
                    lo[ua] = u
                    lo[va] = v
                    hi = list(lo)
                    hi[axis] = level
                    s_lo = solid(tuple(lo))  # type: ignore[arg-type]
                    s_hi = solid(tuple(hi))  # type: ignore[arg-type]
                    if s_lo != s_hi:
                        m.square(axis, level, u, v, +1 if s_lo else -1)
    return m.finish(1.0 / n)


def _icosahedron() -> tuple[np.ndarray, np.ndarray]:
    t = (1.0 + 5.0 ** 0.5) / 2.0
    v = np.array(
        [[-1, t, 0], [1, t, 0], [-1, -t, 0], [1, -t, 0],
         [0, -1, t], [0, 1, t], [0, -1, -t], [0, 1, -t],
         [t, 0, -1], [t, 0, 1], [-t, 0, -1], [-t, 0, 1]], dtype=np.float64)
    f = np.array(
        [[0, 11, 5], [0, 5, 1], [0, 1, 7], [0, 7, 10], [0, 10, 11],
         [1, 5, 9], [5, 11, 4], [11, 10, 2], [10, 7, 6], [7, 1, 8],
         [3, 9, 4], [3, 4, 2], [3, 2, 6], [3, 6, 8], [3, 8, 9],
         [4, 9, 5], [2, 4, 11], [6, 2, 10], [8, 6, 7], [9, 8, 1]], dtype=np.int32)
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    return v, f


def icosphere(level: int) -> tuple[np.ndarray, np.ndarray]:
    """Unit sphere: icosahedron refined `level` times by edge midpoints.

    Every new vertex is projected onto the unit sphere.  20 * 4^level
    triangles (level 5 gives 20,480; level 6 gives 81,920).
    """
    verts, tris = _icosahedron()
    vl = [tuple(p) for p in verts]
    for _ in range(level):
        cache: dict[tuple[int, int], int] = {}

        def mid(a: int, b: int) -> int:
            key = (a, b) if a < b else (b, a)
            if key not in cache:
                p = np.asarray(vl[a]) + np.asarray(vl[b])
                p = p / np.linalg.norm(p)
                cache[key] = len(vl)
                vl.append(tuple(p))
            return cache[key]

        new = []
        for a, b, c in tris:
            ab, bc, ca = mid(a, b), mid(b, c), mid(c, a)
            new += [(a, ab, ca), (b, bc, ab), (c, ca, bc), (ab, bc, ca)]
        tris = np.asarray(new, dtype=np.int32)
    verts = np.asarray(vl, dtype=np.float64)
    cen = verts[tris].mean(axis=1)
    return verts, _orient_outward(verts, tris, cen)


def random_rotation(rng: np.random.Generator) -> np.ndarray:
    """Uniform random rotation (QR of a Gaussian matrix, sign-fixed, det +1)."""
    a = rng.standard_normal((3, 3))
    q, r = np.linalg.qr(a)
    q = q * np.sign(np.diag(r))
    if np.linalg.det(q) < 0:
        q[:, 0] = -q[:, 0]
    return q


def transformed(verts: np.ndarray, rot: np.ndarray, scale: float, shift: np.ndarray) -> np.ndarray:
    """Rigid rotation, uniform scaling and translation (orientation is kept)."""
    return (verts @ rot.T) * scale + shift


def check_closed(tris: np.ndarray) -> bool:
    """True iff every undirected edge is used by exactly two triangles, once in each direction."""
    directed: dict[tuple[int, int], int] = {}
    for a, b, c in tris:
        for e in ((a, b), (b, c), (c, a)):
            directed[(int(e[0]), int(e[1]))] = directed.get((int(e[0]), int(e[1])), 0) + 1
    for (a, b), cnt in directed.items():
        if cnt != 1 or directed.get((b, a), 0) != 1:
            return False
    return True


def signed_volume(verts: np.ndarray, tris: np.ndarray) -> float:
    """Volume enclosed by the surface (positive for outward orientation)."""
    a = verts[tris[:, 0]]
    b = verts[tris[:, 1]]
    c = verts[tris[:, 2]]
    return float(np.einsum("ij,ij->i", a, np.cross(b, c)).sum() / 6.0)
