"""GPU parity of the three-way ACA of the H-matrix as a whole (Section 4,
first implementation remark; ``whole_matrix=1``) through the C ABI:

* against the oracle's `aca3_whole` on the 768-triangle cube: the same
  number of crosses (within 2) and, in float64, the same first frequencies;
* every block keeps the same number of crosses, at least the largest rank
  the block-wise compression needs (the literal stopping test in both);
* the apply of the whole-matrix factors against the dense oracle apply on
  sampled rows (<= 1e-4), both precisions.
"""
import numpy as np
import pytest

from inputs import workloads
from oracle import aca3 as O_aca, apply as O_apply, freqs as O_freqs, quadrature as O_q, tree as O_tree

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx(g3):
    return g3.Context(0)


def test_whole_matrix_matches_oracle_cube768(g3, ctx):
    w = workloads.get("cube768")
    geo = O_q.Geometry(w.verts, w.tris)
    OT = O_tree.build(w.verts, w.tris, w.leaf, w.eta)
    fs = O_freqs.frequency_set(w.freq)
    su = fs["s"][fs["uniq"]]
    ef = lambda I, J, s: O_q.entries(geo, "slp", I, J, s)
    far = [b for b in range(OT.blocks.shape[0]) if OT.blocks[b, 4] == 1]
    assert len(far) > 100
    ops = [O_aca.BemBlock(ef, OT.perm[OT.blocks[b, 0]:OT.blocks[b, 1]], OT.perm[OT.blocks[b, 2]:OT.blocks[b, 3]], su)
           for b in far]
    ref = O_aca.aca3_whole(ops, w.eps3, s_abs=np.abs(su))
    T = g3.build_cluster_tree(ctx, w.verts, w.tris, w.leaf, w.eta)
    F = g3.freqs_from_spec(ctx, w.freq)
    fa = g3.aca3_compress(ctx, T, F, "slp", prec="fp64", eps3=w.eps3, whole_matrix=1)
    r3 = fa.ranks()
    assert np.all(r3 == r3[0])
    assert abs(int(r3[0]) - ref.rank) <= 2, (r3[0], ref.rank)
    b0 = fa.block(0, OT.blocks[far[0], 1] - OT.blocks[far[0], 0], OT.blocks[far[0], 3] - OT.blocks[far[0], 2],
                  su.size)
    n = min(3, ref.rank, int(r3[0]))
    assert b0["piv"][:n, 2].tolist() == [p[3] for p in ref.pivots[:n]]
    # the shared fibers: every block holds the same fiber of each cross
    b1 = fa.block(len(far) - 1, OT.blocks[far[-1], 1] - OT.blocks[far[-1], 0],
                  OT.blocks[far[-1], 3] - OT.blocks[far[-1], 2], su.size)
    assert np.allclose(b0["f"], b1["f"], rtol=0, atol=1e-12 * np.abs(b0["f"]).max())


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_whole_matrix_apply_and_rank(g3, ctx, prec):
    import torch
    w = workloads.get("cube768")
    geo = O_q.Geometry(w.verts, w.tris)
    fs = O_freqs.frequency_set(w.freq)
    T = g3.build_cluster_tree(ctx, w.verts, w.tris, w.leaf, w.eta)
    F = g3.freqs_from_spec(ctx, w.freq)
    fa = g3.aca3_compress(ctx, T, F, "slp", prec=prec, eps3=w.eps3, whole_matrix=1)
    st = fa.stats()
    assert st["status_bits"] & 1 == 0
    r3 = fa.ranks()
    assert np.all(r3 == r3[0]) and r3[0] >= 1
    blockwise = g3.aca3_compress(ctx, T, F, "slp", prec=prec, eps3=w.eps3, dense_face_max=-1, literal_stop=1)
    assert r3[0] >= blockwise.ranks().max() - 2
    nf = g3.assemble_near(ctx, T, F, "slp", prec=prec)
    W = workloads.densities(w.E, w.freq.K, w.density_seed)
    y = g3.apply_gcq(ctx, T, nf, fa, torch.from_numpy(W).to("cuda")).cpu().numpy()
    rows = np.arange(0, w.E, 23)
    yd = O_apply.dense_apply(lambda I, J, s: O_q.entries(geo, "slp", I, J, s), w.E, fs["s"], W, rows=rows)
    assert np.linalg.norm(y[rows] - yd) <= 1e-4 * np.linalg.norm(yd)
