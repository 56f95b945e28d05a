"""Edge cases of the path on the GPU, through the C ABI.

* A mesh with no admissible block (the 192-triangle cube at leaf 32, eta = 1:
  all 64 blocks are near blocks): the compression has nothing to do and the
  apply is the near field alone, equal to the dense oracle apply in both
  modes (SUM and PERFREQ) and through the allocation-free entry point.
* One triangle: one 1 x 1 block, the self term (Section 3, singular
  integration).  Single layer: y = sum_l V_00(s_l) w_l against the oracle's
  self term; double layer: exactly 0 (the collocation point lies in the
  element's plane, so (x - y) . n_y = 0 on the whole element).
* Zero densities give an exactly zero y on a mesh with far blocks (every
  kernel of the apply, float64 and float32 with the tensor-core x formation).
* Ragged block sizes: the 2,352-triangle L-shape has far blocks of 18, 19,
  36, 37, 73 and 74 rows, so every tile of the compression (the dense
  residual working faces' 64-row tiles, the tensor cores' 16 x 32 sub-tiles)
  and of the apply ends on a partial tile.  Blocks against the dense oracle
  (<= 10 eps3, ranks within 2 of the oracle's), the apply against the dense
  oracle apply on sampled rows (<= 1e-4).
* An empty mesh is rejected before any launch.
"""
import numpy as np
import pytest

from inputs import meshes, workloads
from oracle import aca3 as O_aca, apply as O_apply, freqs as O_freqs, quadrature as O_q, tree as O_tree

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx(g3):
    return g3.Context(0)


@pytest.fixture(scope="module")
def cube192():
    w = workloads.get("cube192")
    geo = O_q.Geometry(w.verts, w.tris)
    fs = O_freqs.frequency_set(w.freq)
    W = workloads.densities(w.E, w.freq.K, w.density_seed)
    Y = O_apply.dense_apply_perfreq(lambda I, J, s: O_q.entries(geo, "slp", I, J, s), w.E, fs["s"], W)
    return w, W, Y


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_mesh_without_admissible_blocks(g3, ctx, cube192, prec):
    import torch
    w, W, Yref = cube192
    T = g3.build_cluster_tree(ctx, w.verts, w.tris, w.leaf, w.eta)
    blocks = T.get()["blocks"]
    assert blocks.shape[0] == 64 and not (blocks[:, 4] == 1).any()
    F = g3.freqs_from_spec(ctx, w.freq)
    nf = g3.assemble_near(ctx, T, F, "slp", prec=prec)
    fa = g3.aca3_compress(ctx, T, F, "slp", prec=prec, eps3=w.eps3)
    st = fa.stats()
    assert st["n_far"] == 0 and st["crosses"] == 0 and fa.ranks().size == 0
    tol = 1e-9 if prec == "fp64" else 1e-5
    Wd = torch.from_numpy(W).to("cuda")
    yref = Yref.sum(axis=1)
    y = g3.apply_gcq(ctx, T, nf, fa, Wd).cpu().numpy()
    assert np.linalg.norm(y - yref) <= tol * np.linalg.norm(yref)
    Y = g3.apply_gcq(ctx, T, nf, fa, Wd, mode="perfreq").cpu().numpy()
    err = np.linalg.norm(Y - Yref, axis=0) / np.linalg.norm(Yref, axis=0)
    assert err.max() <= tol, err
    # the empty factors alone contribute nothing
    assert torch.count_nonzero(g3.apply_gcq(ctx, T, None, fa, Wd)) == 0
    if prec == "mixed":
        Wt = Wd.to(torch.complex64).t().contiguous()
        Yn = torch.empty(w.E, dtype=torch.complex64, device="cuda")
        g3.apply_gcq_noalloc(ctx, T, nf, fa, Wt.t(), Yn)
        yn = Yn.cpu().numpy()
        assert np.linalg.norm(yn - yref) <= tol * np.linalg.norm(yref)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_single_triangle(g3, ctx, prec):
    import torch
    v = np.array([[0.0, 0.0, 0.0], [0.9, 0.1, 0.0], [0.2, 0.7, 0.3]])
    t = np.array([[0, 1, 2]], dtype=np.int32)
    spec = workloads.bdf2_spec(8, 0.1)
    s = O_freqs.frequency_set(spec)["s"]
    T = g3.build_cluster_tree(ctx, v, t, 32, 1.0)
    info = T.get()
    assert np.array_equal(info["perm"], [0]) and np.array_equal(info["blocks"], [[0, 1, 0, 1, 0]])
    F = g3.freqs_from_spec(ctx, spec)
    rng = np.random.default_rng(21)
    W = (rng.standard_normal((1, s.size)) + 1j * rng.standard_normal((1, s.size)))
    Wd = torch.from_numpy(W).to("cuda")
    geo = O_q.Geometry(v, t)
    v00 = O_q.entries(geo, "slp", [0], [0], s)[0]
    tol = 1e-9 if prec == "fp64" else 1e-5
    for ker in ("slp", "dlp"):
        nf = g3.assemble_near(ctx, T, F, ker, prec=prec)
        fa = g3.aca3_compress(ctx, T, F, ker, prec=prec, eps3=1e-4)
        assert fa.stats()["n_far"] == 0
        y = g3.apply_gcq(ctx, T, nf, fa, Wd).cpu().numpy()
        Y = g3.apply_gcq(ctx, T, nf, fa, Wd, mode="perfreq").cpu().numpy()
        if ker == "slp":
            ref = v00 * W[0]
            assert abs(y[0] - ref.sum()) <= tol * abs(ref.sum())
            assert np.abs(Y[0] - ref).max() <= tol * np.abs(ref).max()
        else:
            assert y[0] == 0 and not Y.any()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_zero_densities_give_exact_zero(g3, ctx, prec):
    import torch
    w = workloads.get("cube768")
    T = g3.build_cluster_tree(ctx, w.verts, w.tris, w.leaf, w.eta)
    F = g3.freqs_from_spec(ctx, w.freq)
    nf = g3.assemble_near(ctx, T, F, "slp", prec=prec)
    fa = g3.aca3_compress(ctx, T, F, "slp", prec=prec, eps3=w.eps3)
    assert fa.stats()["n_far"] > 0
    Wd = torch.zeros((w.E, w.freq.K), dtype=torch.complex128, device="cuda")
    assert torch.count_nonzero(g3.apply_gcq(ctx, T, nf, fa, Wd)) == 0
    assert torch.count_nonzero(g3.apply_gcq(ctx, T, nf, fa, Wd, mode="perfreq")) == 0


@pytest.fixture(scope="module")
def lshape2352():
    v, t = meshes.lshape(14)
    w = workloads.Workload("lshape2352", v, t, workloads.bdf2_spec(32, 0.05), kernels=("slp", "dlp"),
                           density_seed=23)
    OT = O_tree.build(w.verts, w.tris, w.leaf, w.eta)
    return w, O_q.Geometry(w.verts, w.tris), OT, O_freqs.frequency_set(w.freq)


@pytest.mark.parametrize("mode", ["fp64", "mixed", "mixed_no_dense_residual"])
@pytest.mark.parametrize("kernel", ["slp", "dlp"])
def test_ragged_block_sizes(g3, ctx, lshape2352, kernel, mode):
    import torch
    w, geo, OT, fs = lshape2352
    su = fs["s"][fs["uniq"]]
    ef = lambda I, J, s: O_q.entries(geo, kernel, I, J, s)
    far = np.flatnonzero(OT.blocks[:, 4] == 1)
    sizes = OT.blocks[far, 1] - OT.blocks[far, 0]
    assert set(sizes.tolist()) == {18, 19, 36, 37, 73, 74}
    prec = "fp64" if mode == "fp64" else "mixed"
    kw = {"residual_face_max": -1} if mode == "mixed_no_dense_residual" else {}
    T = g3.build_cluster_tree(ctx, w.verts, w.tris, w.leaf, w.eta)
    F = g3.freqs_from_spec(ctx, w.freq)
    fa = g3.aca3_compress(ctx, T, F, kernel, prec=prec, eps3=w.eps3, **kw)
    st = fa.stats()
    assert st["status_bits"] & 1 == 0 and st["n_far"] == far.size
    assert (st["entries_face_dense"] > 0) == (mode == "mixed")
    r3 = fa.ranks()
    rng = np.random.default_rng(31)
    check = set(rng.choice(far.size, 10, replace=False).tolist())
    check |= {int(np.flatnonzero(sizes == sz)[0]) for sz in (19, 37, 73, 74)}
    for i in sorted(check):
        rb, re, cb, ce, _ = OT.blocks[far[i]]
        M, N = re - rb, ce - cb
        D = O_q.dense(geo, kernel, su, rows=OT.perm[rb:re], cols=OT.perm[cb:ce])
        if not D.any():
            assert r3[i] == 0
            continue
        blk = fa.block(i, M, N, su.size)
        A = np.zeros_like(D)
        for U, V, f in zip(blk["U"], blk["V"], blk["f"]):
            A += (U @ V.conj().T)[:, :, None] * f[None, None, :]
        err = np.linalg.norm(A - D) / np.linalg.norm(D)
        assert err <= 10 * w.eps3, (i, M, N, err)
        ref = O_aca.aca3(O_aca.BemBlock(ef, OT.perm[rb:re], OT.perm[cb:ce], su), w.eps3, s_abs=np.abs(su))
        assert abs(ref.rank - r3[i]) <= 2, (i, ref.rank, r3[i])
    nf = g3.assemble_near(ctx, T, F, kernel, prec=prec)
    W = workloads.densities(w.E, w.freq.K, w.density_seed)
    rows = workloads.frobenius_sample_rows(w.E, 24, 3)
    yref = O_apply.dense_apply(ef, w.E, fs["s"], W, rows=rows)
    y = g3.apply_gcq(ctx, T, nf, fa, torch.from_numpy(W).to("cuda")).cpu().numpy()
    assert np.linalg.norm(y[rows] - yref) <= 1e-4 * np.linalg.norm(yref)


def test_empty_mesh_rejected(g3, ctx):
    w = workloads.get("cube48")
    for v, t in ((w.verts, np.zeros((0, 3), dtype=np.int32)), (np.zeros((0, 3)), w.tris[:0])):
        with pytest.raises(g3.G3Error) as e:
            g3.build_cluster_tree(ctx, v, t, w.leaf, w.eta)
        assert "EINVAL" in str(e.value)
