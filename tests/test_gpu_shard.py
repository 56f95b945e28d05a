"""GPU test of the row-cluster sharding through the C ABI: the shards of a
partition (g3_shard_rows + g3_tree_subset), each assembled, compressed and
applied on its own as a rank would, reproduce the unsharded result: the same
rank for every block, disjoint output rows, and partial applies that add up
to the whole apply (up to the order of float32 sums)."""
import numpy as np
import pytest

from inputs import workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx(g3):
    return g3.Context(0)


@pytest.mark.parametrize("n_ranks", [2, 3])
def test_shards_reassemble_the_whole(g3, ctx, n_ranks):
    import torch
    w = workloads.get("lshape3072")
    T = g3.build_cluster_tree(ctx, w.verts, w.tris, w.leaf, w.eta, max_block=96)
    F = g3.freqs_from_spec(ctx, w.freq)
    tg = T.get()
    sh = g3.shard_rows(tg["nodes"], tg["blocks"], n_ranks)
    assert sh["n_units"] >= n_ranks
    Wd = torch.from_numpy(workloads.densities(w.E, w.freq.K, 31)).to("cuda")
    for ker in ("slp", "dlp"):
        nf = g3.assemble_near(ctx, T, F, ker, prec="mixed")
        fa = g3.aca3_compress(ctx, T, F, ker, prec="mixed", eps3=w.eps3)
        y = g3.apply_gcq(ctx, T, nf, fa, Wd).cpu().numpy()
        r_full = fa.ranks()
        far_full = tg["far_index"]
        ysum = np.zeros_like(y)
        entries = 0
        seen = np.zeros(w.E, int)
        for rank in range(n_ranks):
            S = g3.tree_subset(ctx, T, sh["owner"], rank)
            sg = S.get()
            nfs = g3.assemble_near(ctx, S, F, ker, prec="mixed")
            fas = g3.aca3_compress(ctx, S, F, ker, prec="mixed", eps3=w.eps3)
            ys = g3.apply_gcq(ctx, S, nfs, fas, Wd).cpu().numpy()
            # the rank's blocks, in the whole tree's order, with the same ranks
            mine = np.flatnonzero(sh["owner"] == rank)
            assert np.array_equal(sg["blocks"], tg["blocks"][mine])
            full_pos = {int(b): i for i, b in enumerate(far_full)}
            own_far = [full_pos[int(b)] for b in mine if tg["blocks"][b, 4] == 1]
            assert np.array_equal(fas.ranks(), r_full[own_far])
            rows = np.zeros(w.E, bool)
            for rb, re, _, _, _ in sg["blocks"]:
                rows[sg["perm"][rb:re]] = True
            assert np.all(ys[~rows] == 0)
            seen += rows
            ysum += ys
            entries += fas.stats()["entries"] + nfs.info()["entries"]
        assert np.all(seen == 1)
        assert np.linalg.norm(ysum - y) <= 1e-5 * np.linalg.norm(y)
        assert entries == fa.stats()["entries"] + nf.info()["entries"]
