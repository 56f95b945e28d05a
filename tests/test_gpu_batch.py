"""GPU tests of the batched compression: the admissible blocks of several
meshes (different sizes and frequency counts) in one persistent launch.

Each block's computation depends only on its own mesh, frequencies and the
tolerances, so the batch must reproduce, mesh by mesh, the ranks and the
applied result of compressing that mesh alone (which the parity tests check
against the oracle), and the cube member is checked against the oracle's
dense apply directly.
"""
import numpy as np
import pytest

from inputs import workloads
from oracle import apply as O_apply, freqs as O_freqs, quadrature as O_q

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx(g3):
    return g3.Context(0)


def _members():
    ws = workloads.batch64(n_geom=5)
    ws.append(workloads.get("cube768"))
    return ws


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_batch_matches_single_compressions(g3, ctx, prec):
    import torch
    ws = _members()
    trees = [g3.build_cluster_tree(ctx, w.verts, w.tris, w.leaf, w.eta) for w in ws]
    freqs = [g3.freqs_from_spec(ctx, w.freq) for w in ws]
    assert len({F.info()[1] for F in freqs}) > 1          # several frequency counts in the batch
    batch = g3.aca3_compress_batch(ctx, trees, freqs, "slp", prec=prec, eps3=1e-4)
    assert len(batch) == len(ws)
    dt = torch.complex64 if prec == "mixed" else torch.complex128
    for w, T, F, fb in zip(ws, trees, freqs, batch):
        single = g3.aca3_compress(ctx, T, F, "slp", prec=prec, eps3=1e-4)
        sb, ss = fb.stats(), single.stats()
        assert sb["n_far"] == ss["n_far"] == T.info()["n_far"]
        assert np.array_equal(fb.ranks(), single.ranks())
        assert sb["factor_bytes"] == ss["factor_bytes"] and sb["crosses"] == ss["crosses"]
        W = torch.from_numpy(workloads.densities(w.E, w.freq.K, w.density_seed)).to("cuda", dt)
        yb = g3.apply_gcq(ctx, T, None, fb, W)
        ys = g3.apply_gcq(ctx, T, None, single, W)
        torch.cuda.synchronize()
        scale = float(ys.abs().max())
        if scale > 0:
            assert float((yb - ys).abs().max()) <= (1e-5 if prec == "mixed" else 1e-12) * scale


def test_batch_member_against_dense_oracle(g3, ctx):
    import torch
    ws = _members()
    trees = [g3.build_cluster_tree(ctx, w.verts, w.tris, w.leaf, w.eta) for w in ws]
    freqs = [g3.freqs_from_spec(ctx, w.freq) for w in ws]
    batch = g3.aca3_compress_batch(ctx, trees, freqs, "slp", prec="mixed", eps3=1e-4)
    w, T, F, fa = ws[-1], trees[-1], freqs[-1], batch[-1]
    # release the other members first: the shared pool stays alive with fa
    del batch[:-1]
    geo = O_q.Geometry(w.verts, w.tris)
    fs = O_freqs.frequency_set(w.freq)
    ef = lambda I, J, s: O_q.entries(geo, "slp", I, J, s)
    Wn = workloads.densities(w.E, w.freq.K, w.density_seed)
    yd = O_apply.dense_apply(ef, w.E, fs["s"], Wn)
    nf = g3.assemble_near(ctx, T, F, "slp", prec="mixed")
    y = g3.apply_gcq(ctx, T, nf, fa, torch.from_numpy(Wn).to("cuda", torch.complex64)).cpu().numpy()
    assert np.linalg.norm(y - yd) / np.linalg.norm(yd) <= 1e-4


def test_batch_with_predictor_and_spills(g3, ctx):
    ws = _members()
    trees = [g3.build_cluster_tree(ctx, w.verts, w.tris, w.leaf, w.eta) for w in ws]
    freqs = [g3.freqs_from_spec(ctx, w.freq) for w in ws]
    plain = g3.aca3_compress_batch(ctx, trees, freqs, "slp", prec="mixed", eps3=1e-4)
    # pool far too small: blocks spill and rerun; same ranks
    sp = g3.aca3_compress_batch(ctx, trees, freqs, "slp", prec="mixed", eps3=1e-4, pool_factor=0.02)
    assert sp[0].stats()["spilled_blocks"] > 0
    for a, b in zip(plain, sp):
        assert np.array_equal(a.ranks(), b.ranks())
    # predictor trained on the batch's own labels, queue order + pool size only
    X = np.concatenate([g3.block_features(ctx, T, F, "slp", 1e-4) for T, F in zip(trees, freqs)])
    Y = np.concatenate([fa.labels() for fa in plain])
    net = g3.mlp_train(ctx, X, Y, epochs=60, batch=256, seed=3)
    lm = g3.aca3_compress_batch(ctx, trees, freqs, "slp", prec="mixed", eps3=1e-4, mlp=net, mlp_use=3)
    assert lm[0].stats()["mlp_used"] == 3
    for a, b in zip(plain, lm):
        assert np.array_equal(a.ranks(), b.ranks())


def test_batch_rejects_bad_input(g3, ctx):
    w = workloads.get("cube768")
    T = g3.build_cluster_tree(ctx, w.verts, w.tris, w.leaf, w.eta)
    F = g3.freqs_from_spec(ctx, w.freq)
    with pytest.raises(g3.G3Error):
        g3.aca3_compress_batch(ctx, [T, T], [F, F], "slp", k1=np.zeros(10, dtype=np.int32))
    with pytest.raises(g3.G3Error):
        g3.aca3_compress_batch(ctx, [T], [F], "slp", unbatched=1)


def test_compression_as_captured_graph_matches_plain_launches(g3):
    """opts.graph: the queue resets and both persistent launches captured into
    one CUDA graph give the same compression, block for block, as the plain
    launches (and the same apply)."""
    import torch
    ctx = g3.Context(0)
    w = workloads.get("lshape3072")
    T = g3.build_cluster_tree(ctx, w.verts, w.tris, w.leaf, w.eta)
    F = g3.freqs_from_spec(ctx, w.freq)
    Wd = torch.from_numpy(workloads.densities(w.E, w.freq.K, 3)).to("cuda")
    for ker in ("slp", "dlp"):
        fa = g3.aca3_compress(ctx, T, F, ker, prec="mixed", eps3=w.eps3)
        fg = g3.aca3_compress(ctx, T, F, ker, prec="mixed", eps3=w.eps3, graph=1)
        assert np.array_equal(fa.ranks(), fg.ranks())
        sa, sg = fa.stats(), fg.stats()
        assert sa["entries"] == sg["entries"] and sa["factor_bytes"] == sg["factor_bytes"]
        assert ctx.kernel_launches().get("graph_launch", 0) >= 1
        ya = g3.apply_gcq(ctx, T, None, fa, Wd)
        yg = g3.apply_gcq(ctx, T, None, fg, Wd)
        assert torch.linalg.norm(ya - yg) <= 1e-6 * torch.linalg.norm(ya)
