"""Oracle: balanced binary cluster tree and geometric block partition.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

The paper builds its H-matrix on balanced cluster trees with a purely
geometric admissibility condition, one block structure for all frequencies
(Section "Three-dimensional adaptive cross approximation", the paragraph on
eq. (outerProd) and the first implementation remark).  It gives no further
detail, so this reading is used, and the CUDA library must reproduce it
bit for bit:

* A cluster is a set of elements; its box is the axis-aligned bounding box
  of all vertices of its elements.
* A cluster with n > leaf elements is split: axis = the box's longest side
  (lowest axis index on ties); the elements are sorted stably by
  (centroid[axis], element index) ascending, centroid = ((v0 + v1) + v2) / 3;
  the first floor(n/2) go left, the rest right.  Node ids are preorder.
* Admissibility of (tau, sigma):  min(diam2(tau), diam2(sigma))
  <= eta^2 dist2(tau, sigma)  and  dist2 > 0, with
  diam2 = dx*dx + dy*dy + dz*dz of the box sides and
  dist2 = sum over x, y, z of max(0, lo_s - hi_t, lo_t - hi_s)^2, all in
  float64, left to right, without fused multiply-adds.
* Block recursion from (root, root): admissible -> far block; both leaves
  -> near block; both inner -> the four child pairs (LL, LR, RL, RR);
  otherwise only the inner cluster is split (left child first).
  Blocks are listed in this depth-first order.
* Optional cap max_block > 0 (not in the paper; it bounds the work of one
  block): an admissible pair whose larger cluster has more than max_block
  elements is split like an inadmissible pair, unless both are leaves.

Output blocks are given as cluster-order index ranges
(row_begin, row_end, col_begin, col_end, admissible).
"""
from __future__ import annotations

import sys

import numpy as np


class Tree:
    def __init__(self, perm, begin, end, left, right, lo, hi, blocks):
        self.perm = perm            # cluster position -> original element
        self.begin = begin          # node -> first cluster position
        self.end = end
        self.left = left            # -1 for leaves
        self.right = right
        self.lo = lo                # node -> box corner [3]
        self.hi = hi
        self.blocks = blocks        # [nb, 5] int64

    @property
    def far(self):
        return self.blocks[self.blocks[:, 4] == 1]

    @property
    def near(self):
        return self.blocks[self.blocks[:, 4] == 0]


def _diam2(lo, hi) -> float:
    dx = hi[0] - lo[0]
    dy = hi[1] - lo[1]
    dz = hi[2] - lo[2]
    return dx * dx + dy * dy + dz * dz


def _dist2(lo_t, hi_t, lo_s, hi_s) -> float:
    acc = 0.0
    for d in range(3):
        g = max(0.0, lo_s[d] - hi_t[d], lo_t[d] - hi_s[d])
        acc = acc + g * g
    return acc


def admissible(lo_t, hi_t, lo_s, hi_s, eta: float) -> bool:
    d2 = _dist2(lo_t, hi_t, lo_s, hi_s)
    return min(_diam2(lo_t, hi_t), _diam2(lo_s, hi_s)) <= eta * eta * d2 and d2 > 0.0


def build(verts: np.ndarray, tris: np.ndarray, leaf: int = 32, eta: float = 1.0, max_block: int = 0) -> Tree:
    verts = np.asarray(verts, dtype=np.float64)
    tris = np.asarray(tris, dtype=np.int64)
    v0, v1, v2 = verts[tris[:, 0]], verts[tris[:, 1]], verts[tris[:, 2]]
    cen = ((v0 + v1) + v2) / 3.0
    tmin = np.minimum(np.minimum(v0, v1), v2)
    tmax = np.maximum(np.maximum(v0, v1), v2)

    begin, end, left, right, lo, hi = [], [], [], [], [], []
    order_out: list[np.ndarray] = []

    def node(idx: np.ndarray, start: int) -> int:
        nid = len(begin)
        begin.append(start)
        end.append(start + idx.size)
        left.append(-1)
        right.append(-1)
        blo = tmin[idx].min(axis=0)
        bhi = tmax[idx].max(axis=0)
        lo.append([float(x) for x in blo])
        hi.append([float(x) for x in bhi])
        if idx.size > leaf:
            ext = [bhi[d] - blo[d] for d in range(3)]
            axis = 0
            for d in (1, 2):
                if ext[d] > ext[axis]:
                    axis = d
            srt = idx[np.lexsort((idx, cen[idx, axis]))]
            h = idx.size // 2
            l = node(srt[:h], start)
            r = node(srt[h:], start + h)
            left[nid] = l
            right[nid] = r
        else:
            order_out.append(idx)
        return nid

    old = sys.getrecursionlimit()
    sys.setrecursionlimit(max(old, 10000))
    node(np.arange(tris.shape[0], dtype=np.int64), 0)
    perm = np.concatenate(order_out)

    blocks: list[tuple[int, int, int, int, int]] = []

    def part(t: int, s: int) -> None:
        tl, sl = left[t] < 0, left[s] < 0
        if admissible(lo[t], hi[t], lo[s], hi[s], eta):
            big = max(end[t] - begin[t], end[s] - begin[s])
            if max_block <= 0 or big <= max_block or (tl and sl):
                blocks.append((begin[t], end[t], begin[s], end[s], 1))
                return
        elif tl and sl:
            blocks.append((begin[t], end[t], begin[s], end[s], 0))
            return
        if not tl and not sl:
            part(left[t], left[s])
            part(left[t], right[s])
            part(right[t], left[s])
            part(right[t], right[s])
        elif tl:
            part(t, left[s])
            part(t, right[s])
        else:
            part(left[t], s)
            part(right[t], s)

    part(0, 0)
    sys.setrecursionlimit(old)
    return Tree(perm, np.asarray(begin), np.asarray(end), np.asarray(left), np.asarray(right),
                np.asarray(lo), np.asarray(hi), np.asarray(blocks, dtype=np.int64))
