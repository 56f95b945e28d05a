"""GPU parity at the benchmark's full size: the 12,288-triangle L-shape,
K = 128 multistep-CQ frequencies, single and double layer, in the launch
configuration bench.py times (mixed precision, persistent batched launch).

The oracle cannot form the whole problem, so it checks sampled outputs it can
compute one by one:
  * rows of y = sum_l A(s_l) w_l from its dense definition (relative error
    <= 1e-4 on the sampled rows, the accuracy target);
  * admissible blocks of every size class reconstructed from the returned
    factors against the oracle's dense block (<= 10 eps3);
  * near-field blocks entry by entry (float32 rounding, 2e-5).
"""
import numpy as np
import pytest

from inputs import workloads
from oracle import apply as O_apply, freqs as O_freqs, quadrature as O_q, tree as O_tree

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def setup(g3):
    import torch
    ctx = g3.Context(0)
    w = workloads.get("lshape12288")
    T = g3.build_cluster_tree(ctx, w.verts, w.tris, w.leaf, w.eta, max_block=w.max_block)
    F = g3.freqs_from_spec(ctx, w.freq)
    geo = O_q.Geometry(w.verts, w.tris)
    OT = O_tree.build(w.verts, w.tris, w.leaf, w.eta, w.max_block)
    fs = O_freqs.frequency_set(w.freq)
    W = workloads.densities(w.E, w.freq.K, w.density_seed)
    out = {}
    for ker in w.kernels:
        nf = g3.assemble_near(ctx, T, F, ker, prec="mixed")
        fa = g3.aca3_compress(ctx, T, F, ker, prec="mixed", eps3=w.eps3)
        y = g3.apply_gcq(ctx, T, nf, fa, torch.from_numpy(W).to("cuda")).cpu().numpy()
        out[ker] = (nf, fa, y)
    return dict(ctx=ctx, w=w, T=T, F=F, geo=geo, OT=OT, fs=fs, W=W, out=out)


@pytest.mark.parametrize("kernel", ["slp", "dlp"])
def test_fullsize_apply_sampled_rows(setup, kernel):
    d = setup
    w, geo, fs, W = d["w"], d["geo"], d["fs"], d["W"]
    rows = workloads.frobenius_sample_rows(w.E, 8, seed=3 + (kernel == "dlp"))
    ef = lambda I, J, s: O_q.entries(geo, kernel, I, J, s)
    yref = O_apply.dense_apply(ef, w.E, fs["s"], W, rows=rows)
    y = d["out"][kernel][2]
    err = np.linalg.norm(y[rows] - yref) / np.linalg.norm(yref)
    assert err <= 1e-4, err


@pytest.mark.parametrize("kernel", ["slp", "dlp"])
def test_fullsize_blocks_every_size(setup, kernel):
    d = setup
    w, geo, OT, fs = d["w"], d["geo"], d["OT"], d["fs"]
    fa = d["out"][kernel][1]
    su = fs["s"][fs["uniq"]]
    far = np.nonzero(OT.blocks[:, 4] == 1)[0]
    size = np.maximum(OT.blocks[far, 1] - OT.blocks[far, 0], OT.blocks[far, 3] - OT.blocks[far, 2])
    rng = np.random.default_rng(17)
    st = fa.stats()
    assert st["status_bits"] & 1 == 0 and st["n_far"] == far.size
    for sz in sorted(set(size.tolist()))[:5]:
        i = int(rng.choice(np.nonzero(size == sz)[0]))
        rb, re, cb, ce, _ = OT.blocks[far[i]]
        M, N = re - rb, ce - cb
        D = O_q.dense(geo, kernel, su, rows=OT.perm[rb:re], cols=OT.perm[cb:ce])
        blk = fa.block(i, M, N, su.size)
        A = np.zeros_like(D)
        for U, V, f in zip(blk["U"], blk["V"], blk["f"]):
            A += (U @ V.conj().T)[:, :, None] * f[None, None, :]
        nD = np.linalg.norm(D)
        if nD == 0:
            assert np.linalg.norm(A) == 0
            continue
        assert np.linalg.norm(A - D) <= 10 * w.eps3 * nD, (sz, np.linalg.norm(A - D) / nD)


def test_fullsize_near_blocks(setup):
    d = setup
    w, geo, OT, fs = d["w"], d["geo"], d["OT"], d["fs"]
    su = fs["s"][fs["uniq"]]
    near = np.nonzero(OT.blocks[:, 4] == 0)[0]
    rng = np.random.default_rng(5)
    for kernel in w.kernels:
        nf = d["out"][kernel][0]
        for b in rng.choice(near, 3, replace=False):
            rb, re, cb, ce, _ = OT.blocks[b]
            got = nf.block(int(b), re - rb, ce - cb, su.size)
            ref = np.moveaxis(O_q.dense(geo, kernel, su, rows=OT.perm[rb:re], cols=OT.perm[cb:ce]), 2, 0)
            assert np.max(np.abs(got - ref)) <= 2e-5 * np.max(np.abs(ref))
