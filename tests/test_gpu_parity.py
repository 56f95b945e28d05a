"""GPU parity: every step of the CUDA path against the CPU oracle.

All calls go through the C ABI (ctypes binding).  Tolerances:
  * cluster tree / block partition: bit-exact;
  * frequencies (float64): 1e-12 relative (multistep CQ), 1e-10 (gCQ, elliptic
    functions by a different method than the oracle's);
  * float64 entries: 1e-6 relative to the largest entry of the sample
    (the stated bar; observed ~1e-13);
  * float32 entries (mixed): 2e-5 relative to the largest entry (float32
    rounding of geometry and phase, |Im s| r up to ~100);
  * compression: per-block reconstruction error <= 10 eps3 against the dense
    oracle block (eps3 = 1e-4);
  * apply: relative error <= 1e-4 against the dense oracle apply (every
    entry at all K frequencies); the near field alone against the oracle's
    near-field apply (1e-10 float64, 1e-5 mixed).
"""
import numpy as np
import pytest

from inputs import workloads
from oracle import aca3 as O_aca, apply as O_apply, freqs as O_freqs, quadrature as O_q, tree as O_tree

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx(g3):
    return g3.Context(0)


def _maxrel(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


# ---------------------------------------------------------------- frequencies

@pytest.mark.parametrize("K,dt", [(32, 0.1), (128, 0.02), (256, 0.01)])
def test_bdf2_frequencies(g3, ctx, K, dt):
    spec = workloads.bdf2_spec(K, dt)
    f = g3.g3_freqs_bdf2(ctx, K, spec.lam, dt)
    got = f.get()
    ref = O_freqs.bdf2(K, dt, spec.lam)
    uniq, partner = O_freqs.bdf2_unique(K)
    assert np.array_equal(got["uniq"], uniq) and np.array_equal(got["partner"], partner)
    assert _maxrel(got["s"], ref) < 1e-12


def test_gcq_frequencies_and_weights(g3, ctx):
    st = workloads.graded_steps(64)
    f = g3.g3_freqs_gcq(ctx, 256, float(st.min()), float(st.max()))
    got = f.get()
    s, w = O_freqs.gcq(256, float(st.min()), float(st.max()))
    assert _maxrel(got["s"], s) < 1e-10
    assert _maxrel(got["omega"], w) < 1e-10
    # the contour property holds for the device set too
    for dt in st[::8]:
        assert abs(np.sum(got["omega"] / (got["s"] - 1.0 / dt)) - 1.0) < 1e-9


def test_gcq_constant_steps_rejected(g3, ctx):
    with pytest.raises(g3.G3Error) as e:
        g3.g3_freqs_gcq(ctx, 64, 0.01, 0.01)
    assert "EINVAL" in str(e.value)


# ---------------------------------------------------------------- tree

@pytest.mark.parametrize("name", ["cube48", "cube768", "lshape768", "lshape12288", "sphere1280", "sphere20480"])
def test_tree_bit_exact(g3, ctx, name):
    w = workloads.get(name)
    T = g3.build_cluster_tree(ctx, w.verts, w.tris, w.leaf, w.eta)
    got = T.get()
    ref = O_tree.build(w.verts, w.tris, w.leaf, w.eta)
    assert np.array_equal(got["perm"], ref.perm)
    assert np.array_equal(got["blocks"], ref.blocks)
    assert np.array_equal(got["nodes"][:, 0], ref.begin) and np.array_equal(got["nodes"][:, 2], ref.left)
    assert np.array_equal(got["boxes"][:, :3], ref.lo) and np.array_equal(got["boxes"][:, 3:], ref.hi)


@pytest.mark.parametrize("name,cap", [("cube768", 96), ("lshape12288", 384), ("lshape12288", 192)])
def test_tree_capped_bit_exact(g3, ctx, name, cap):
    w = workloads.get(name)
    T = g3.build_cluster_tree(ctx, w.verts, w.tris, w.leaf, w.eta, max_block=cap)
    got = T.get()
    ref = O_tree.build(w.verts, w.tris, w.leaf, w.eta, cap)
    assert np.array_equal(got["perm"], ref.perm)
    assert np.array_equal(got["blocks"], ref.blocks)


def test_tree_batch_geometries_bit_exact(g3, ctx):
    for w in workloads.batch64(n_geom=6):
        T = g3.build_cluster_tree(ctx, w.verts, w.tris, w.leaf, w.eta)
        ref = O_tree.build(w.verts, w.tris, w.leaf, w.eta)
        got = T.get()
        assert np.array_equal(got["perm"], ref.perm) and np.array_equal(got["blocks"], ref.blocks)


def test_tree_rejects_bad_input(g3, ctx):
    w = workloads.get("cube48")
    bad = w.tris.copy()
    bad[3] = [0, 0, 1]
    with pytest.raises(g3.G3Error):
        g3.build_cluster_tree(ctx, w.verts, bad, 32, 1.0)
    bad = w.tris.copy()
    bad[0, 0] = 10 ** 6
    with pytest.raises(g3.G3Error):
        g3.build_cluster_tree(ctx, w.verts, bad, 32, 1.0)
    with pytest.raises(g3.G3Error):
        g3.build_cluster_tree(ctx, w.verts, w.tris, 0, 1.0)


# ---------------------------------------------------------------- entries

def _pairs(E, n, seed, with_self=True):
    rng = np.random.default_rng(seed)
    r = rng.integers(0, E, n)
    c = rng.integers(0, E, n)
    if with_self:
        c[: n // 8] = r[: n // 8]
        # neighbours: consecutive element ids are usually adjacent on the structured meshes
        c[n // 8: n // 4] = np.minimum(r[n // 8: n // 4] + 1, E - 1)
    return r, c


@pytest.mark.parametrize("name", ["cube768", "lshape12288", "sphere1280"])
@pytest.mark.parametrize("kernel", ["slp", "dlp"])
def test_entries_parity(g3, ctx, name, kernel):
    w = workloads.get(name)
    T = g3.build_cluster_tree(ctx, w.verts, w.tris, w.leaf, w.eta)
    F = g3.freqs_from_spec(ctx, w.freq)
    fs = O_freqs.frequency_set(w.freq)
    geo = O_q.Geometry(w.verts, w.tris)
    r, c = _pairs(w.E, 512, 7)
    K = w.freq.K
    kidx = np.unique(np.r_[0, 1, K // 2, K - 1, np.arange(0, K, max(1, K // 8))])
    ref = O_q.entries(geo, kernel, r, c, fs["s"][kidx])
    d64 = g3.g3_entries(ctx, T, F, kernel, r, c, kidx, prec="fp64")
    assert _maxrel(d64, ref) < 1e-6
    d32 = g3.g3_entries(ctx, T, F, kernel, r, c, kidx, prec="mixed")
    assert _maxrel(d32, ref) < 2e-5
    # per-entry relative error of the float64 path (regular and singular entries)
    big = np.abs(ref) > 1e-3 * np.abs(ref).max()
    assert np.max(np.abs(d64 - ref)[big] / np.abs(ref)[big]) < 1e-9


def test_self_entries_fp64(g3, ctx):
    w = workloads.get("lshape12288")
    T = g3.build_cluster_tree(ctx, w.verts, w.tris, w.leaf, w.eta)
    F = g3.freqs_from_spec(ctx, w.freq)
    fs = O_freqs.frequency_set(w.freq)
    geo = O_q.Geometry(w.verts, w.tris)
    idx = np.arange(0, w.E, 997)
    kidx = np.arange(0, 128, 9)
    ref = O_q.entries(geo, "slp", idx, idx, fs["s"][kidx])
    got = g3.g3_entries(ctx, T, F, "slp", idx, idx, kidx, prec="fp64")
    assert np.max(np.abs(got - ref) / np.abs(ref)) < 1e-10


# ---------------------------------------------------------------- near field

@pytest.mark.parametrize("prec,tol", [("fp64", 1e-9), ("mixed", 2e-5)])
@pytest.mark.parametrize("kernel", ["slp", "dlp"])
def test_near_field_blocks(g3, ctx, prec, tol, kernel):
    w = workloads.get("lshape768")
    T = g3.build_cluster_tree(ctx, w.verts, w.tris, w.leaf, w.eta)
    F = g3.freqs_from_spec(ctx, w.freq)
    nf = g3.assemble_near(ctx, T, F, kernel, prec=prec)
    fs = O_freqs.frequency_set(w.freq)
    su = fs["s"][fs["uniq"]]
    geo = O_q.Geometry(w.verts, w.tris)
    tr = T.get()
    near = [b for b in range(tr["blocks"].shape[0]) if tr["blocks"][b, 4] == 0]
    rng = np.random.default_rng(3)
    for b in rng.choice(near, 6, replace=False):
        rb, re, cb, ce, _ = tr["blocks"][b]
        M, N = re - rb, ce - cb
        got = nf.block(int(b), M, N, su.size)                    # [k, i, j]
        ref = O_q.dense(geo, kernel, su, rows=tr["perm"][rb:re], cols=tr["perm"][cb:ce])  # [i, j, k]
        ref = np.moveaxis(ref, 2, 0)
        assert _maxrel(got, ref) < tol, b
    assert nf.info()["entries"] == sum(
        (tr["blocks"][b, 1] - tr["blocks"][b, 0]) * (tr["blocks"][b, 3] - tr["blocks"][b, 2]) for b in near) * su.size


# ---------------------------------------------------------------- compression

def _rand(rng, *shape):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


@pytest.mark.parametrize("dense", [0, -1])
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_separable_rank1_exact(g3, ctx, prec, dense):
    rng = np.random.default_rng(2)
    a, b, c = _rand(rng, 1, 40), _rand(rng, 1, 33), _rand(rng, 1, 17)
    fa = g3.aca3_compress_separable(ctx, a, b, c, prec=prec, eps3=1e-4, dense_face_max=dense)
    st = fa.stats()
    assert fa.ranks()[0] == 1
    blk = fa.block(0, 40, 33, 17)
    D = np.einsum("ti,tj,tk->ijk", a, b, c)
    A = sum((U @ V.conj().T)[:, :, None] * f[None, None, :] for U, V, f in zip(blk["U"], blk["V"], blk["f"]))
    tol = 1e-12 if prec == "fp64" else 1e-5
    assert np.linalg.norm(A - D) <= tol * np.linalg.norm(D)
    assert st["status_bits"] & 1 == 0


@pytest.mark.parametrize("dense", [0, -1])
@pytest.mark.parametrize("R", [2, 4])
def test_separable_rank_r_recovered(g3, ctx, R, dense):
    rng = np.random.default_rng(10 + R)
    c = _rand(rng, R, 12) * (0.3 ** np.arange(R))[:, None]
    a, b = _rand(rng, R, 22), _rand(rng, R, 19)
    fa = g3.aca3_compress_separable(ctx, a, b, c, prec="fp64", eps3=1e-10, dense_face_max=dense)
    r3 = fa.ranks()[0]
    assert r3 <= R
    blk = fa.block(0, 22, 19, 12)
    D = np.einsum("ti,tj,tk->ijk", a, b, c)
    A = sum((U @ V.conj().T)[:, :, None] * f[None, None, :] for U, V, f in zip(blk["U"], blk["V"], blk["f"]))
    assert np.linalg.norm(A - D) <= 1e-9 * np.linalg.norm(D)
    # same ranks as the oracle on the same tensor
    ref = O_aca.aca3(O_aca.SeparableBlock(a, b, c), 1e-10, dense_max=O_aca.DENSE_MAX if dense == 0 else -1)
    assert ref.rank == r3


def _oracle_blocks(w, kernel, eps3):
    geo = O_q.Geometry(w.verts, w.tris)
    T = O_tree.build(w.verts, w.tris, w.leaf, w.eta)
    fs = O_freqs.frequency_set(w.freq)
    su = fs["s"][fs["uniq"]]
    ef = lambda I, J, s: O_q.entries(geo, kernel, I, J, s)
    return geo, T, fs, su, ef


@pytest.mark.parametrize("dense", [0, -1])
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_compression_cube768_blockwise(g3, ctx, prec, dense):
    w = workloads.get("cube768")
    eps3 = 1e-4
    geo, OT, fs, su, ef = _oracle_blocks(w, "slp", eps3)
    T = g3.build_cluster_tree(ctx, w.verts, w.tris, w.leaf, w.eta)
    F = g3.freqs_from_spec(ctx, w.freq)
    fa = g3.aca3_compress(ctx, T, F, "slp", prec=prec, eps3=eps3, dense_face_max=dense)
    st = fa.stats()
    assert st["status_bits"] & 1 == 0
    assert (st["dense_crosses"] == st["crosses"]) if dense == 0 else (st["dense_crosses"] == 0)
    r3 = fa.ranks()
    far = [b for b in range(OT.blocks.shape[0]) if OT.blocks[b, 4] == 1]
    assert r3.size == len(far)
    oranks = []
    rng = np.random.default_rng(5)
    check = set(rng.choice(len(far), 24, replace=False).tolist()) | {int(np.argmax(
        [(OT.blocks[b, 1] - OT.blocks[b, 0]) * (OT.blocks[b, 3] - OT.blocks[b, 2]) for b in far]))}
    for i in sorted(check):
        rb, re, cb, ce, _ = OT.blocks[far[i]]
        M, N = re - rb, ce - cb
        D = O_q.dense(geo, "slp", su, rows=OT.perm[rb:re], cols=OT.perm[cb:ce])
        blk = fa.block(i, M, N, su.size)
        A = np.zeros_like(D)
        for U, V, f in zip(blk["U"], blk["V"], blk["f"]):
            A += (U @ V.conj().T)[:, :, None] * f[None, None, :]
        err = np.linalg.norm(A - D) / np.linalg.norm(D)
        assert err <= 10 * eps3, (i, err)
        ref = O_aca.aca3(O_aca.BemBlock(ef, OT.perm[rb:re], OT.perm[cb:ce], su), eps3, s_abs=np.abs(su),
                         dense_max=O_aca.DENSE_MAX if dense == 0 else -1)
        oranks.append((ref.rank, r3[i]))
        assert abs(ref.rank - r3[i]) <= 2
        # the first frequency is always the first one used
        assert blk["piv"][0, 2] == 0
    o, g = np.array(oranks).T
    assert abs(o.mean() - g.mean()) <= 0.1 * o.mean() + 0.5


@pytest.mark.parametrize("threads", [128, 256, 512])
def test_compression_launch_shapes(g3, ctx, threads):
    """Every CTA size of the low-rank launch computes Algorithm 1: blocks
    within 10 eps3 of the oracle's dense blocks, and every cross's pivot the
    largest entry of its face approximant H_l (the pivot step of Algorithm 1),
    checked on blocks that span several 64-row tiles of the pivot search."""
    w = workloads.get("lshape3072")
    eps3 = 1e-4
    geo, OT, fs, su, ef = _oracle_blocks(w, "slp", eps3)
    T = g3.build_cluster_tree(ctx, w.verts, w.tris, w.leaf, w.eta)
    F = g3.freqs_from_spec(ctx, w.freq)
    fa = g3.aca3_compress(ctx, T, F, "slp", prec="mixed", eps3=eps3, dense_face_max=-1, threads=threads)
    st = fa.stats()
    assert st["status_bits"] & 1 == 0 and st["dense_crosses"] == 0
    far = [b for b in range(OT.blocks.shape[0]) if OT.blocks[b, 4] == 1]
    rows = np.array([OT.blocks[b, 1] - OT.blocks[b, 0] for b in far])
    cols = np.array([OT.blocks[b, 3] - OT.blocks[b, 2] for b in far])
    big = np.flatnonzero((rows > 64) & (rows * cols <= 256 * 256))
    assert big.size > 0
    rng = np.random.default_rng(11)
    order = np.argsort(-(rows * cols)[big], kind="stable")
    check = sorted(set(big[order[:3]].tolist()) | set(rng.choice(big, min(3, big.size), replace=False).tolist()))
    n_piv = 0
    for i in check:
        rb, re, cb, ce, _ = OT.blocks[far[i]]
        M, N = re - rb, ce - cb
        blk = fa.block(i, M, N, su.size)
        for U, V, piv in zip(blk["U"], blk["V"], blk["piv"]):
            H = np.abs(U @ V.conj().T)
            assert H[piv[0], piv[1]] >= (1 - 1e-3) * H.max(), (i, piv, H.max())
            n_piv += 1
        D = O_q.dense(geo, "slp", su, rows=OT.perm[rb:re], cols=OT.perm[cb:ce])
        A = np.zeros_like(D)
        for U, V, f in zip(blk["U"], blk["V"], blk["f"]):
            A += (U @ V.conj().T)[:, :, None] * f[None, None, :]
        assert np.linalg.norm(A - D) <= 10 * eps3 * np.linalg.norm(D), i
    assert n_piv > 0


@pytest.mark.parametrize("kernel", ["slp", "dlp"])
@pytest.mark.parametrize("threads", [256, 512])
def test_dense_residual_faces(g3, ctx, kernel, threads):
    """Low-rank faces evaluated through the dense residual working face
    (opts residual_face_max; the default up to 192 x 192 entries, the sum over
    the earlier crosses on the tensor cores at 256 threads, on the CUDA cores
    at 512) compute Algorithm 1 as the on-demand rows and columns do: blocks within 10 eps3 of the oracle's dense blocks, block ranks
    within 2 of the on-demand run, and every stored pivot the largest entry of
    its face approximant H_l."""
    w = workloads.get("lshape3072")
    eps3 = 1e-4
    geo, OT, fs, su, ef = _oracle_blocks(w, kernel, eps3)
    T = g3.build_cluster_tree(ctx, w.verts, w.tris, w.leaf, w.eta)
    F = g3.freqs_from_spec(ctx, w.freq)
    ref = g3.aca3_compress(ctx, T, F, kernel, prec="mixed", eps3=eps3, dense_face_max=-1, threads=threads,
                           residual_face_max=-1)
    fa = g3.aca3_compress(ctx, T, F, kernel, prec="mixed", eps3=eps3, dense_face_max=-1, threads=threads,
                          residual_face_max=256 * 256)
    st, st0 = fa.stats(), ref.stats()
    assert st["status_bits"] & 1 == 0 and st["dense_crosses"] == 0
    assert st["entries_face_dense"] > 0 and st0["entries_face_dense"] == 0
    far = [b for b in range(OT.blocks.shape[0]) if OT.blocks[b, 4] == 1]
    rows = np.array([OT.blocks[b, 1] - OT.blocks[b, 0] for b in far])
    cols = np.array([OT.blocks[b, 3] - OT.blocks[b, 2] for b in far])
    r3, r30 = fa.ranks(), ref.ranks()
    assert np.abs(r3 - r30).max() <= 2
    assert abs(r3.mean() - r30.mean()) <= 0.1 * r30.mean()
    inside = np.flatnonzero(rows * cols <= 256 * 256)
    assert inside.size > 0
    rng = np.random.default_rng(21)
    order = np.argsort(-(rows * cols)[inside], kind="stable")
    check = sorted(set(inside[order[:2]].tolist()) | set(rng.choice(inside, min(3, inside.size), replace=False).tolist()))
    for i in check:
        rb, re, cb, ce, _ = OT.blocks[far[i]]
        M, N = re - rb, ce - cb
        blk = fa.block(i, M, N, su.size)
        for U, V, piv in zip(blk["U"], blk["V"], blk["piv"]):
            H = np.abs(U @ V.conj().T)
            assert H[piv[0], piv[1]] >= (1 - 1e-3) * H.max(), (i, piv, H.max())
        D = O_q.dense(geo, kernel, su, rows=OT.perm[rb:re], cols=OT.perm[cb:ce])
        A = np.zeros_like(D)
        for U, V, f in zip(blk["U"], blk["V"], blk["f"]):
            A += (U @ V.conj().T)[:, :, None] * f[None, None, :]
        assert np.linalg.norm(A - D) <= 10 * eps3 * np.linalg.norm(D), i


@pytest.mark.parametrize("dense", [0, -1])
def test_apply_cube768_against_oracle(g3, ctx, dense):
    import torch
    w = workloads.get("cube768")
    eps3 = 1e-4
    geo, OT, fs, su, ef = _oracle_blocks(w, "slp", eps3)
    W = workloads.densities(w.E, w.freq.K, w.density_seed)
    yd = O_apply.dense_apply(ef, w.E, fs["s"], W)
    T = g3.build_cluster_tree(ctx, w.verts, w.tris, w.leaf, w.eta)
    F = g3.freqs_from_spec(ctx, w.freq)
    for prec in ("fp64", "mixed"):
        nf = g3.assemble_near(ctx, T, F, "slp", prec=prec)
        fa = g3.aca3_compress(ctx, T, F, "slp", prec=prec, eps3=eps3, dense_face_max=dense)
        Wd = torch.from_numpy(W).to("cuda")
        y = g3.apply_gcq(ctx, T, nf, fa, Wd).cpu().numpy()
        err = np.linalg.norm(y - yd) / np.linalg.norm(yd)
        assert err <= 1e-4, (prec, err)
        # host-buffer path gives the same result
        yh = g3.apply_gcq(ctx, T, nf, fa, W)
        assert np.linalg.norm(yh - y) <= 1e-6 * np.linalg.norm(y)
        # near field alone equals the oracle's near-field apply
        yn = g3.apply_gcq(ctx, T, nf, None, Wd).cpu().numpy()
        ynr = O_apply.compressed_apply(OT, {b: O_aca.Result([], 0, [], False) for b in range(OT.blocks.shape[0])
                                            if OT.blocks[b, 4] == 1}, ef, fs["s"], fs["uniq"], fs["partner"], W)
        assert np.linalg.norm(yn - ynr) <= (1e-10 if prec == "fp64" else 1e-5) * np.linalg.norm(ynr)
