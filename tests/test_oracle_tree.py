"""Pins for the oracle's cluster tree and block partition: exact cover,
admissibility re-checked independently, leaf and balance structure."""
import numpy as np
import pytest

from inputs import meshes, workloads
from oracle import tree


def _check(verts, tris, leaf, eta, max_block=0):
    T = tree.build(verts, tris, leaf, eta, max_block)
    E = tris.shape[0]
    assert np.array_equal(np.sort(T.perm), np.arange(E))
    # every (i, j) covered exactly once
    cover = np.zeros((E, E), dtype=np.int32)
    for rb, re, cb, ce, adm in T.blocks:
        cover[rb:re, cb:ce] += 1
    assert np.all(cover == 1)
    # balance: children sizes differ by at most one; leaves <= leaf
    for n in range(T.begin.size):
        size = T.end[n] - T.begin[n]
        if T.left[n] < 0:
            assert size <= leaf
        else:
            l, r = T.left[n], T.right[n]
            assert T.end[l] == T.begin[r] and T.begin[l] == T.begin[n] and T.end[r] == T.end[n]
            assert (T.end[r] - T.begin[r]) - (T.end[l] - T.begin[l]) in (0, 1)
            assert size > leaf
    # admissibility recomputed from element boxes (numpy, vectorised)
    tv = verts[tris[T.perm]]                 # [E,3,3] cluster order
    tmin, tmax = tv.min(axis=1), tv.max(axis=1)
    leaf_ranges = {(T.begin[n], T.end[n]) for n in range(T.begin.size) if T.left[n] < 0}
    for rb, re, cb, ce, adm in T.blocks:
        lo_t, hi_t = tmin[rb:re].min(0), tmax[rb:re].max(0)
        lo_s, hi_s = tmin[cb:ce].min(0), tmax[cb:ce].max(0)
        gap = np.maximum(0, np.maximum(lo_s - hi_t, lo_t - hi_s))
        dist = np.sqrt(np.sum(gap ** 2))
        diam = min(np.linalg.norm(hi_t - lo_t), np.linalg.norm(hi_s - lo_s))
        if adm:
            assert dist > 0 and diam <= eta * dist * (1 + 1e-12)
        else:
            assert (rb, re) in leaf_ranges and (cb, ce) in leaf_ranges
    return T


@pytest.mark.parametrize("name", ["cube48", "cube192", "cube768", "lshape768", "sphere1280"])
def test_partition_invariants(name):
    w = workloads.get(name)
    _check(w.verts, w.tris, w.leaf, w.eta)


def test_small_leaf_and_eta():
    v, t = meshes.icosphere(2)
    _check(v, t, 8, 0.5)
    _check(v, t, 5, 2.0)


def test_cube768_structure():
    w = workloads.get("cube768")
    T = tree.build(w.verts, w.tris, 32, 1.0)
    sizes = T.end - T.begin
    # 768 -> 384 -> 192 -> 96 -> 48 -> 24 : 63 nodes, 32 leaves of 24
    assert T.begin.size == 63
    assert sorted(set(sizes[T.left < 0])) == [24]
    assert T.far.shape[0] > 0 and T.near.shape[0] > 0


def test_tree_is_deterministic_and_preorder():
    w = workloads.get("lshape768")
    a = tree.build(w.verts, w.tris, 32, 1.0)
    b = tree.build(w.verts.copy(), w.tris.copy(), 32, 1.0)
    assert np.array_equal(a.perm, b.perm) and np.array_equal(a.blocks, b.blocks)
    # preorder: a node's left child is the next id
    for n in range(a.begin.size):
        if a.left[n] >= 0:
            assert a.left[n] == n + 1


@pytest.mark.parametrize("cap", [48, 96, 192])
def test_far_block_cap(cap):
    """With a cap, the partition is still an exact cover with admissible far
    blocks; no far block's larger side exceeds the cap; the near blocks are
    unchanged; and every capped far block lies inside one far block of the
    uncapped partition."""
    w = workloads.get("lshape3072")
    plain = tree.build(w.verts, w.tris, w.leaf, w.eta)
    T = _check(w.verts, w.tris, w.leaf, w.eta, cap)
    far = T.blocks[T.blocks[:, 4] == 1]
    assert np.max(np.maximum(far[:, 1] - far[:, 0], far[:, 3] - far[:, 2])) <= cap
    assert np.array_equal(plain.blocks[plain.blocks[:, 4] == 0], T.blocks[T.blocks[:, 4] == 0])
    pf = plain.blocks[plain.blocks[:, 4] == 1]
    for rb, re, cb, ce, _ in far:
        inside = (pf[:, 0] <= rb) & (re <= pf[:, 1]) & (pf[:, 2] <= cb) & (ce <= pf[:, 3])
        assert inside.sum() == 1
    # a cap below the largest block adds blocks; one at or above it changes nothing
    big = int(np.max(np.maximum(pf[:, 1] - pf[:, 0], pf[:, 3] - pf[:, 2])))
    if cap < big:
        assert far.shape[0] > pf.shape[0]
    else:
        assert np.array_equal(T.blocks, plain.blocks)
