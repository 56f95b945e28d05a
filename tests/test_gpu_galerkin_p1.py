"""GPU parity of the Galerkin operators of the Neumann problem with linear
continuous elements (eq. (bie_semi_neum)): the hypersingular operator D (Maue
form) and the adjoint double layer K', on element-local shape functions
(build_p1_tree), against oracle.galerkin_p1, through the C ABI.

* Entries of regular element pairs (g3_entries): float64 1e-10, float32 3e-5.
* Near-field blocks with identical, edge- and vertex-adjacent pairs
  (Sauter-Schwab) and regular pairs, every local entry: float64 1e-9,
  float32 3e-5 (relative to the block).
* The three-way ACA of Algorithm 1 on the 3 M x 3 N blocks: each checked
  block within 10 eps3 of the oracle's dense block, with the entries formed
  on each of the kernel's three paths (dense residual working faces, residual
  rows and columns, exact dense faces).
* apply_gcq on nodal densities (gather at the vertices, near + compressed far
  field, sum into the vertices) against the oracle's nodal rows on sampled
  vertices: <= 1e-4 relative.
"""
import numpy as np
import pytest

from inputs import workloads
from oracle import freqs as O_freqs, galerkin as O_gal, galerkin_p1 as P1

pytestmark = pytest.mark.gpu

OPS = {"hyp": "d", "adj": "kp"}


@pytest.fixture(scope="module")
def ctx(g3):
    return g3.Context(0)


@pytest.fixture(scope="module")
def setup(g3, ctx):
    w = workloads.get("sphere1280g")
    T = g3.build_cluster_tree(ctx, w.verts, w.tris, w.leaf, w.eta)
    T1 = g3.build_p1_tree(ctx, T)
    F = g3.freqs_from_spec(ctx, w.freq)
    fs = O_freqs.frequency_set(w.freq)
    return w, T, T1, F, fs


def _dof(perm3, d):
    return perm3[d] // 3, perm3[d] % 3


def test_p1_tree_triples_the_partition(setup):
    w, T, T1, F, fs = setup
    g, g1 = T.get(), T1.get()
    E = w.tris.shape[0]
    assert g1["perm"].size == 3 * E
    assert np.array_equal(g1["perm"].reshape(E, 3), 3 * g["perm"][:, None] + np.arange(3)[None, :])
    assert np.array_equal(g1["blocks"][:, :4], 3 * g["blocks"][:, :4])
    assert np.array_equal(g1["blocks"][:, 4], g["blocks"][:, 4])


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-10), ("mixed", 3e-5)])
@pytest.mark.parametrize("kernel", ["hyp", "adj"])
def test_p1_regular_entries(g3, ctx, setup, kernel, prec, tol):
    w, T, T1, F, fs = setup
    E = w.tris.shape[0]
    rng = np.random.default_rng(7)
    rows, cols = [], []
    while len(rows) < 40:
        e, f = rng.integers(0, E, 2)
        if O_gal.classify(w.tris, int(e), int(f))[0] != "regular":
            continue
        a, b = rng.integers(0, 3, 2)
        rows.append(3 * e + a)
        cols.append(3 * f + b)
    kidx = np.array([0, 3, 17, 40, 63])
    got = g3.g3_entries(ctx, T1, F, kernel, np.array(rows), np.array(cols), kidx, prec=prec, scheme="galerkin4x4")
    ref = np.array([P1.local_block(w.verts, w.tris, r // 3, c // 3, fs["s"][kidx], OPS[kernel])[r % 3, c % 3]
                    for r, c in zip(rows, cols)])
    assert np.max(np.abs(got - ref)) <= tol * np.max(np.abs(ref))


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-9), ("mixed", 3e-5)])
@pytest.mark.parametrize("kernel", ["hyp", "adj"])
def test_p1_near_blocks(g3, ctx, setup, kernel, prec, tol):
    w, T, T1, F, fs = setup
    nf = g3.assemble_near(ctx, T1, F, kernel, scheme="galerkin4x4", prec=prec)
    g1 = T1.get()
    perm3, blocks = g1["perm"], g1["blocks"]
    su = fs["s"][fs["uniq"]]
    near = [b for b in range(blocks.shape[0]) if blocks[b, 4] == 0]
    diag = [b for b in near if blocks[b, 0] == blocks[b, 2]]
    off = [b for b in near if blocks[b, 0] != blocks[b, 2]]
    cases = set()
    for b in diag[:1] + off[:1]:
        rb, re, cb, ce, _ = blocks[b]
        M, N = re - rb, ce - cb
        got = nf.block(b, M, N, su.size)            # [Ku, M, N]
        ref = np.zeros((su.size, M, N), complex)
        for ie in range(rb // 3, re // 3):
            for je in range(cb // 3, ce // 3):
                e, f = perm3[3 * ie] // 3, perm3[3 * je] // 3
                cases.add(O_gal.classify(w.tris, int(e), int(f))[0])
                blk = P1.local_block(w.verts, w.tris, int(e), int(f), su, OPS[kernel])
                ref[:, 3 * ie - rb:3 * ie - rb + 3, 3 * je - cb:3 * je - cb + 3] = blk.transpose(2, 0, 1)
        assert np.max(np.abs(got - ref)) <= tol * np.max(np.abs(ref)), b
    assert {"identical", "edge", "vertex", "regular"} <= cases


def _check_block(w, g1, far, i, fa, fs, kernel, eps3, strict=True):
    """Far block i of the compression within 10 eps3 of the oracle's dense
    block (strict: asserted here); returns the relative error."""
    perm3, blocks = g1["perm"], g1["blocks"]
    su = fs["s"][fs["uniq"]]
    rb, re, cb, ce, _ = blocks[far[i]]
    M, N = re - rb, ce - cb
    blk = fa.block(i, M, N, su.size)
    A = np.zeros((M, N, su.size), complex)
    for U, V, f in zip(blk["U"], blk["V"], blk["f"]):
        A += (U @ V.conj().T)[:, :, None] * f[None, None, :]
    D = np.zeros((M, N, su.size), complex)
    for ie in range(rb // 3, re // 3):
        for je in range(cb // 3, ce // 3):
            e, f = perm3[3 * ie] // 3, perm3[3 * je] // 3
            D[3 * ie - rb:3 * ie - rb + 3, 3 * je - cb:3 * je - cb + 3] = \
                P1.local_block(w.verts, w.tris, int(e), int(f), su, OPS[kernel])
    err = np.linalg.norm(A - D) / np.linalg.norm(D)
    if strict:
        assert err <= 10 * eps3, (i, M, N, err)
    return err


@pytest.mark.parametrize("kernel", ["hyp", "adj"])
def test_p1_compression_and_nodal_apply(g3, ctx, setup, kernel):
    import torch
    w, T, T1, F, fs = setup
    eps3 = 1e-4
    nf = g3.assemble_near(ctx, T1, F, kernel, scheme="galerkin4x4", prec="mixed")
    fa = g3.aca3_compress(ctx, T1, F, kernel, scheme="galerkin4x4", prec="mixed", eps3=eps3)
    st = fa.stats()
    assert st["status_bits"] & 1 == 0 and st["crosses"] > 0
    g1 = T1.get()
    far = [b for b in range(g1["blocks"].shape[0]) if g1["blocks"][b, 4] == 1]
    rng = np.random.default_rng(2)
    for i in rng.choice(len(far), 2, replace=False):
        _check_block(w, g1, far, int(i), fa, fs, kernel, eps3)
    nv = w.verts.shape[0]
    W = workloads.densities(nv, w.freq.K, w.density_seed)
    y = g3.apply_gcq(ctx, T1, nf, fa, torch.from_numpy(W).to("cuda", torch.complex64)).cpu().numpy()
    assert y.shape == (nv,)
    rows = np.random.default_rng(5).choice(nv, 4, replace=False)
    R = P1.nodal_rows(w.verts, w.tris, rows, fs["s"], OPS[kernel])   # [rows, nv, K]
    yref = np.einsum("rjk,jk->r", R, W)
    assert np.linalg.norm(y[rows] - yref) <= 1e-4 * np.linalg.norm(yref)


# The hypersingular operator's later faces on the 40-element blocks need face
# ranks 68-87 (the oracle's Algorithm 1 on the same blocks): the oracle capped
# at 48 gives 8.3-8.8 eps3, at 64 1.4 eps3, uncapped 0.44 eps3, so the kernel
# caps the face ranks of the linear-element operators at 64 (48 elsewhere).
@pytest.mark.parametrize("kernel,path", [
    ("hyp", "dense_residual"), ("hyp", "lines"), ("hyp", "dense_faces"),
    ("adj", "dense_residual"), ("adj", "lines"), ("adj", "dense_faces")])
def test_p1_compression_entry_paths(g3, ctx, setup, kernel, path):
    """Each way the compression forms entries of linear elements: dense
    residual working faces (the default), the residual rows and columns of
    the partial-pivot ACA (dense residual working faces off), and the exact
    faces of dense-face blocks (every far block of this mesh made one).  Two
    blocks of each shape (20 and 40 elements a side) against the oracle's
    dense blocks, 10 eps3."""
    w, T, T1, F, fs = setup
    eps3 = 1e-4
    opts = {"dense_residual": {}, "lines": {"residual_face_max": -1},
            "dense_faces": {"dense_face_max": 120 * 120}}[path]
    fa = g3.aca3_compress(ctx, T1, F, kernel, scheme="galerkin4x4", prec="mixed", eps3=eps3, **opts)
    st = fa.stats()
    assert st["status_bits"] & 1 == 0 and st["crosses"] > 0
    assert (st["entries_face_dense"] > 0) == (path == "dense_residual")
    assert st["dense_crosses"] == (st["crosses"] if path == "dense_faces" else 0)
    g1 = T1.get()
    far = [b for b in range(g1["blocks"].shape[0]) if g1["blocks"][b, 4] == 1]
    size = np.array([g1["blocks"][b, 1] - g1["blocks"][b, 0] for b in far])
    assert set(size.tolist()) == {60, 120}
    errs = []
    for M0 in (60, 120):
        for i in np.flatnonzero(size == M0)[:2]:
            errs.append(_check_block(w, g1, far, int(i), fa, fs, kernel, eps3, strict=False))
    assert max(errs) <= 10 * eps3, errs
