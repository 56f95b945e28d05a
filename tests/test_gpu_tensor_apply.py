"""GPU parity of the far-field apply whose x_p = sum_k f_p[k] w_k formation
runs on the tensor cores (eq. (product); mma.sync m16n8k8 TF32 in the
three-term split, float32 accumulation), through the C ABI.

* Against the same apply on the CUDA cores (float32 fused multiply-adds):
  the two orders of float32 sums agree to 2e-6 relative, far field alone and
  near + far, single and double layer, both launch widths of the low-rank
  kernel (blocks of at most 128 and of more than 128 columns).
* Against the oracle's dense apply of the float64 entries on sampled rows:
  <= 1e-4 relative (the far field is compressed to eps3 = 1e-4).
* The allocation-free apply takes the same path and gives the same y.
"""
import numpy as np
import pytest

from inputs import workloads
from oracle import apply as O_apply, freqs as O_freqs, quadrature as O_q

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx(g3):
    return g3.Context(0)


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("kernel", ["slp", "dlp"])
def test_tensor_core_far_apply_matches_cuda_cores_and_oracle(g3, ctx, kernel):
    import torch
    w = workloads.get("lshape3072")
    T = g3.build_cluster_tree(ctx, w.verts, w.tris, w.leaf, w.eta)
    F = g3.freqs_from_spec(ctx, w.freq)
    nf = g3.assemble_near(ctx, T, F, kernel, prec="mixed")
    fa = g3.aca3_compress(ctx, T, F, kernel, prec="mixed", eps3=w.eps3, dense_face_max=-1)
    st = fa.stats()
    assert st["dense_crosses"] == 0 and st["crosses"] > 0
    # both launch widths of the low-rank kernel occur
    tg = T.get()
    far = tg["blocks"][tg["blocks"][:, 4] == 1]
    ncols = far[:, 3] - far[:, 2]
    assert (ncols <= 128).any() and (ncols > 128).any()
    W = workloads.densities(w.E, w.freq.K, w.density_seed)
    Wd = torch.from_numpy(W).to("cuda", torch.complex64)
    out = {}
    for tc in (True, False):
        ctx.set_apply_tensor_cores(tc)
        n0 = ctx.kernel_launches().get("k_far_lr_tc", 0)
        yf = g3.apply_gcq(ctx, T, None, fa, Wd).cpu().numpy()
        y = g3.apply_gcq(ctx, T, nf, fa, Wd).cpu().numpy()
        used = ctx.kernel_launches().get("k_far_lr_tc", 0) - n0
        assert (used > 0) == tc
        out[tc] = (yf, y)
    ctx.set_apply_tensor_cores(True)
    assert _rel(out[True][0], out[False][0]) <= 2e-6
    assert _rel(out[True][1], out[False][1]) <= 2e-6
    # against the float64 dense oracle on sampled rows
    geo = O_q.Geometry(w.verts, w.tris)
    fs = O_freqs.frequency_set(w.freq)
    rows = np.random.default_rng(3).choice(w.E, 12, replace=False)
    yref = O_apply.dense_apply(lambda I, J, s: O_q.entries(geo, kernel, I, J, s), w.E, fs["s"], W, rows=rows)
    assert _rel(out[True][1][rows], yref) <= 1e-4
    # the allocation-free apply takes the tensor-core path too
    Wt = torch.from_numpy(np.ascontiguousarray(W.T)).to("cuda", torch.complex64)
    Y = torch.empty(w.E, dtype=torch.complex64, device="cuda")
    n0 = ctx.kernel_launches().get("k_far_lr_tc", 0)
    g3.apply_gcq_noalloc(ctx, T, nf, fa, Wt.t(), Y)
    assert ctx.kernel_launches().get("k_far_lr_tc", 0) > n0
    assert _rel(Y.cpu().numpy(), out[True][1]) <= 2e-6
