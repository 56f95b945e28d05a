"""GPU test of apply_gcq_noalloc, the allocation-free apply.

Callers that cannot allocate device memory during the step (memory-capped or
pre-reserved arenas, runtimes that forbid cudaMalloc and the synchronisation
it may cause on their hot path) use apply_gcq_noalloc instead of apply_gcq.
It must give the same y as apply_gcq on device buffers, on consecutive calls
that reuse its fixed scratch, and reject problems larger than that scratch.
The file is named to be collected last.
"""
import numpy as np
import pytest

from inputs import workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx(g3):
    return g3.Context(0)


@pytest.mark.parametrize("name,kernel,prec,tol", [
    ("cube768", "slp", "mixed", 1e-5),
    ("lshape768", "dlp", "mixed", 1e-5),
    ("cube768", "slp", "fp64", 1e-12),
])
def test_noalloc_matches_apply_on_two_calls(g3, ctx, name, kernel, prec, tol):
    import torch
    w = workloads.get(name)
    T = g3.build_cluster_tree(ctx, w.verts, w.tris, w.leaf, w.eta)
    F = g3.freqs_from_spec(ctx, w.freq)
    nf = g3.assemble_near(ctx, T, F, kernel, prec=prec)
    fa = g3.aca3_compress(ctx, T, F, kernel, prec=prec, eps3=w.eps3)
    dt = torch.complex64 if prec == "mixed" else torch.complex128
    y = torch.empty(w.E, dtype=dt, device="cuda")
    for call, seed in enumerate((w.density_seed, w.density_seed + 1)):
        # W [M, K] with contiguous columns, as the allocation-free call wants it
        W = torch.from_numpy(workloads.densities(w.E, w.freq.K, seed).T.copy()).to("cuda", dt).t()
        y_ref = g3.apply_gcq(ctx, T, nf, fa, W)
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        allocs0 = torch.cuda.memory_stats().get("allocation.all.allocated", 0)
        g3.apply_gcq_noalloc(ctx, T, nf, fa, W, y)
        torch.cuda.synchronize()
        if call == 1:
            # the second call allocates nothing: neither the device nor torch's allocator moves
            assert torch.cuda.mem_get_info()[0] == free0
            assert torch.cuda.memory_stats().get("allocation.all.allocated", 0) == allocs0
        err = float((y - y_ref).abs().max() / y_ref.abs().max())
        assert err <= tol, (call, err)
    # near field alone and far field alone
    W = torch.from_numpy(workloads.densities(w.E, w.freq.K, 99).T.copy()).to("cuda", dt).t()
    for a, b in ((nf, None), (None, fa)):
        y_ref = g3.apply_gcq(ctx, T, a, b, W)
        g3.apply_gcq_noalloc(ctx, T, a, b, W, y)
        torch.cuda.synchronize()
        assert float((y - y_ref).abs().max() / y_ref.abs().max()) <= tol


def test_noalloc_rejects_problems_beyond_its_scratch(g3, ctx):
    import torch
    from inputs import meshes
    v, t = meshes.lshape(48)                   # 27,648 triangles
    spec = workloads.bdf2_spec(128, 0.02)      # 65 unique frequencies
    T = g3.build_cluster_tree(ctx, v, t, 32, 1.0)
    F = g3.freqs_from_spec(ctx, spec)
    fa = g3.aca3_compress(ctx, T, F, "slp", prec="fp64", eps3=1e-4, max_blocks=1)
    W = torch.zeros((128, t.shape[0]), dtype=torch.complex128, device="cuda").t()
    Y = torch.empty(t.shape[0], dtype=torch.complex128, device="cuda")
    with pytest.raises(g3.G3Error) as e:
        g3.apply_gcq_noalloc(ctx, T, None, fa, W, Y)
    assert "EINVAL" in str(e.value) and "scratch" in str(e.value)
