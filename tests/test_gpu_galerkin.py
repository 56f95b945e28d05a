"""GPU parity of the Galerkin single layer (4 x 4-point rule for regular pairs,
Sauter-Schwab rules for pairs with a common vertex) against the oracle, and
the three-way ACA and apply built on it."""
import numpy as np
import pytest

from inputs import workloads
from oracle import aca3 as O_aca, freqs as O_freqs, galerkin as O_gal, tree as O_tree

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx(g3):
    return g3.Context(0)


def _maxrel(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


def _adjacent_pairs(tris, n, seed):
    """(rows, cols): identical pairs, pairs with a common edge or vertex, and
    random (mostly regular) pairs."""
    rng = np.random.default_rng(seed)
    E = tris.shape[0]
    by_vertex = {}
    for e, t in enumerate(tris):
        for v in t:
            by_vertex.setdefault(int(v), []).append(e)
    rows, cols = [], []
    for i in rng.choice(E, n, replace=False):
        nb = sorted({f for v in tris[i] for f in by_vertex[int(v)]})
        for j in nb:
            rows.append(i)
            cols.append(j)
        rows.append(i)
        cols.append(int(rng.integers(0, E)))
    return np.array(rows), np.array(cols)


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-11), ("mixed", 2e-5)])
def test_galerkin_entries_parity(g3, ctx, prec, tol):
    w = workloads.get("sphere320g")
    T = g3.build_cluster_tree(ctx, w.verts, w.tris, w.leaf, w.eta)
    F = g3.freqs_from_spec(ctx, w.freq)
    fs = O_freqs.frequency_set(w.freq)
    r, c = _adjacent_pairs(w.tris, 10, 4)
    cases = {O_gal.classify(w.tris, i, j)[0] for i, j in zip(r, c)}
    assert cases == {"regular", "vertex", "edge", "identical"}
    kidx = np.array([0, 1, 7, 31, 32, 63])
    ref = O_gal.entries(w.verts, w.tris, r, c, fs["s"][kidx])
    got = g3.g3_entries(ctx, T, F, "slp", r, c, kidx, prec=prec, scheme="galerkin4x4")
    if prec == "fp64":
        # per entry, relative to the entry; entries of strongly damped
        # frequencies between distant panels underflow to 0 on both sides
        live = np.abs(ref) > 1e-250
        assert np.all(np.abs(got[~live]) <= 1e-250)
        rel = np.abs(got - ref)[live] / np.abs(ref)[live]
    else:
        # relative to the largest entry of the same frequency (float32 range)
        rel = np.abs(got - ref) / np.max(np.abs(ref), axis=0, keepdims=True)
    assert rel.max() <= tol, rel.max()


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-11), ("mixed", 2e-5)])
def test_galerkin_near_field_blocks(g3, ctx, prec, tol):
    w = workloads.get("sphere320g")
    T = g3.build_cluster_tree(ctx, w.verts, w.tris, w.leaf, w.eta)
    F = g3.freqs_from_spec(ctx, w.freq)
    nf = g3.assemble_near(ctx, T, F, "slp", scheme="galerkin4x4", prec=prec)
    fs = O_freqs.frequency_set(w.freq)
    su = fs["s"][fs["uniq"]]
    tr = T.get()
    near = [b for b in range(tr["blocks"].shape[0]) if tr["blocks"][b, 4] == 0]
    rng = np.random.default_rng(5)
    diag = [b for b in near if tr["blocks"][b, 0] == tr["blocks"][b, 2]]
    for b in list(rng.choice(near, 3, replace=False)) + diag[:1]:
        rb, re, cb, ce, _ = tr["blocks"][b]
        M, N = re - rb, ce - cb
        got = nf.block(int(b), M, N, su.size)                                    # [k, i, j]
        ref = O_gal.dense(w.verts, w.tris, su, rows=tr["perm"][rb:re], cols=tr["perm"][cb:ce])
        ref = np.moveaxis(ref, 2, 0)
        assert _maxrel(got, ref) <= tol, b


def test_galerkin_compression_and_apply(g3, ctx):
    import torch
    w = workloads.get("sphere1280g")
    T = g3.build_cluster_tree(ctx, w.verts, w.tris, w.leaf, w.eta)
    F = g3.freqs_from_spec(ctx, w.freq)
    fs = O_freqs.frequency_set(w.freq)
    su = fs["s"][fs["uniq"]]
    OT = O_tree.build(w.verts, w.tris, w.leaf, w.eta)
    far = [b for b in range(OT.blocks.shape[0]) if OT.blocks[b, 4] == 1]
    for prec in ("fp64", "mixed"):
        fa = g3.aca3_compress(ctx, T, F, "slp", scheme="galerkin4x4", prec=prec, eps3=w.eps3)
        st = fa.stats()
        assert st["n_far"] == len(far) and st["crosses"] > 0 and st["status_bits"] & 1 == 0
        # blocks against the oracle's dense Galerkin blocks
        rng = np.random.default_rng(1)
        for i in rng.choice(len(far), 4, replace=False):
            rb, re, cb, ce, _ = OT.blocks[far[i]]
            M, N = re - rb, ce - cb
            D = O_gal.dense(w.verts, w.tris, su, rows=OT.perm[rb:re], cols=OT.perm[cb:ce])
            blk = fa.block(int(i), M, N, su.size)
            A = np.zeros_like(D)
            for U, V, f in zip(blk["U"], blk["V"], blk["f"]):
                A += (U @ V.conj().T)[:, :, None] * f[None, None, :]
            assert np.linalg.norm(A - D) <= 10 * w.eps3 * np.linalg.norm(D), (prec, i)
        # apply: sampled rows of the dense Galerkin apply
        nf = g3.assemble_near(ctx, T, F, "slp", scheme="galerkin4x4", prec=prec)
        Wn = workloads.densities(w.E, w.freq.K, w.density_seed)
        dt = torch.complex64 if prec == "mixed" else torch.complex128
        y = g3.apply_gcq(ctx, T, nf, fa, torch.from_numpy(Wn).to("cuda", dt)).cpu().numpy()
        rows = workloads.frobenius_sample_rows(w.E, 12, 3)
        A = O_gal.dense(w.verts, w.tris, fs["s"], rows=rows)                      # all K frequencies
        yref = np.einsum("ijk,jk->i", A, Wn)
        assert np.linalg.norm(y[rows] - yref) / np.linalg.norm(yref) <= 1e-4, prec


def test_autotune_picks_and_caches_a_launch_shape(g3, ctx):
    w = workloads.get("lshape768")
    T = g3.build_cluster_tree(ctx, w.verts, w.tris, w.leaf, w.eta)
    F = g3.freqs_from_spec(ctx, w.freq)
    first = g3.autotune(ctx, T, F, "slp", prec="mixed", eps3=w.eps3)
    assert first["threads"] in (128, 256, 512) and first["dense_face_max"] in (24 * 24, 48 * 48, 64 * 64)
    assert first["ms"] > 0
    again = g3.autotune(ctx, T, F, "slp", prec="mixed", eps3=w.eps3)
    assert again == {**first, "ms": 0.0}            # served from the context's cache
    fa = g3.aca3_compress(ctx, T, F, "slp", prec="mixed", eps3=w.eps3, threads=first["threads"],
                          dense_face_max=first["dense_face_max"])
    assert fa.stats()["status_bits"] & 1 == 0 and fa.stats()["crosses"] > 0
    # float64: 256 threads only
    assert g3.autotune(ctx, T, F, "slp", prec="fp64", eps3=w.eps3)["threads"] == 256
