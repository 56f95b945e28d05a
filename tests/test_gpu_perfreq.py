"""GPU parity of the per-frequency apply (G3_APPLY_PERFREQ) and of frequency
sets given as arrays (g3_freqs_from_array), through the C ABI.

* g3_freqs_from_array pairs conjugates exactly as the oracle's
  pair_conjugates (bit-exact unique set and partners) and, fed the values of
  a closed-form set, reproduces its ranks exactly and its apply up to the
  order of float32 atomic sums.
* PERFREQ: Y[:, l] = A(s_l) w_l for every l against the oracle's dense
  per-frequency apply, per column <= 1e-4 relative (the far field is
  compressed to eps3 = 1e-4); the columns sum to the SUM-mode result.
"""
import numpy as np
import pytest

from inputs import workloads
from oracle import apply as O_apply, freqs as O_freqs, quadrature as O_q

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx(g3):
    return g3.Context(0)


def test_from_array_pairing_matches_oracle(g3, ctx):
    rng = np.random.default_rng(9)
    sets = [O_freqs.bdf2(32, 0.1, (1e-8) ** (1 / 64)), O_freqs.gcq(64, 0.005, 0.015)[0]]
    s = O_freqs.bdf2(16, 0.05, (1e-8) ** (1 / 32))
    sets.append(np.r_[s[rng.permutation(16)], 2.0 + 3.0j, 5.0])
    for s in sets:
        F = g3.g3_freqs_from_array(ctx, s)
        got = F.get()
        u, p = O_freqs.pair_conjugates(s)
        assert np.array_equal(got["uniq"], u) and np.array_equal(got["partner"], p)
        assert np.array_equal(got["s"], s)


def test_from_array_rejects_bad_sets(g3, ctx):
    for bad in (np.array([-1.0 + 1j, -1.0 - 1j]), np.array([1.0, np.nan]), np.zeros(0, complex),
                np.arange(1, 600) * (1 + 1j)):
        with pytest.raises(g3.G3Error) as e:
            g3.g3_freqs_from_array(ctx, bad)
        assert "EINVAL" in str(e.value)


def test_from_array_reproduces_closed_form_set(g3, ctx):
    import torch
    w = workloads.get("cube768")
    T = g3.build_cluster_tree(ctx, w.verts, w.tris, w.leaf, w.eta)
    F = g3.freqs_from_spec(ctx, w.freq)
    F2 = g3.g3_freqs_from_array(ctx, F.get()["s"])
    assert F2.info() == F.info()
    assert np.array_equal(F2.get()["uniq"], F.get()["uniq"])
    assert np.array_equal(F2.get()["partner"], F.get()["partner"])
    Wd = torch.from_numpy(workloads.densities(w.E, w.freq.K, w.density_seed)).to("cuda")
    ys = []
    for FF in (F, F2):
        nf = g3.assemble_near(ctx, T, FF, "slp", prec="mixed")
        fa = g3.aca3_compress(ctx, T, FF, "slp", prec="mixed", eps3=w.eps3)
        ys.append((fa.ranks(), g3.apply_gcq(ctx, T, nf, fa, Wd).cpu().numpy()))
    assert np.array_equal(ys[0][0], ys[1][0])
    # same factors; the apply's float32 atomic sums may add in another order
    assert np.linalg.norm(ys[0][1] - ys[1][1]) <= 1e-6 * np.linalg.norm(ys[0][1])


@pytest.mark.parametrize("dense", [0, -1])
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_perfreq_against_dense_oracle(g3, ctx, prec, dense):
    import torch
    w = workloads.get("cube768")
    geo = O_q.Geometry(w.verts, w.tris)
    fs = O_freqs.frequency_set(w.freq)
    W = workloads.densities(w.E, w.freq.K, w.density_seed)
    rows = np.arange(0, w.E, 5)
    Yref = O_apply.dense_apply_perfreq(lambda I, J, s: O_q.entries(geo, "slp", I, J, s), w.E, fs["s"], W, rows=rows)
    T = g3.build_cluster_tree(ctx, w.verts, w.tris, w.leaf, w.eta)
    F = g3.freqs_from_spec(ctx, w.freq)
    nf = g3.assemble_near(ctx, T, F, "slp", prec=prec)
    fa = g3.aca3_compress(ctx, T, F, "slp", prec=prec, eps3=w.eps3, dense_face_max=dense)
    Wd = torch.from_numpy(W).to("cuda")
    Y = g3.apply_gcq(ctx, T, nf, fa, Wd, mode="perfreq").cpu().numpy()     # [M, K]
    assert Y.shape == (w.E, w.freq.K)
    err = np.linalg.norm(Y[rows] - Yref, axis=0) / np.linalg.norm(Yref, axis=0)
    assert err.max() <= 1e-4, err
    # the columns sum to the SUM-mode apply
    y = g3.apply_gcq(ctx, T, nf, fa, Wd).cpu().numpy()
    assert np.linalg.norm(Y.sum(axis=1) - y) <= (1e-12 if prec == "fp64" else 1e-5) * np.linalg.norm(y)
    # host buffers give the same columns
    Yh = g3.apply_gcq(ctx, T, nf, fa, W, mode="perfreq")
    assert np.linalg.norm(Yh - Y) <= 1e-6 * np.linalg.norm(Y)
    la = ctx.last_apply()
    assert la["ms"] > 0 and la["bytes"] > 0


def test_perfreq_near_and_far_parts_separately(g3, ctx):
    """Near field only, far field only, and both: the per-frequency outputs add."""
    import torch
    w = workloads.get("lshape768")
    T = g3.build_cluster_tree(ctx, w.verts, w.tris, w.leaf, w.eta)
    F = g3.freqs_from_spec(ctx, w.freq)
    Wd = torch.from_numpy(workloads.densities(w.E, w.freq.K, 4)).to("cuda")
    for ker in ("slp", "dlp"):
        nf = g3.assemble_near(ctx, T, F, ker, prec="fp64")
        fa = g3.aca3_compress(ctx, T, F, ker, prec="fp64", eps3=1e-4)
        Yn = g3.apply_gcq(ctx, T, nf, None, Wd, mode="perfreq")
        Yf = g3.apply_gcq(ctx, T, None, fa, Wd, mode="perfreq")
        Y = g3.apply_gcq(ctx, T, nf, fa, Wd, mode="perfreq")
        assert torch.linalg.norm(Y - Yn - Yf) <= 1e-12 * torch.linalg.norm(Y)
        # far-field only SUM and PERFREQ agree
        yf = g3.apply_gcq(ctx, T, None, fa, Wd)
        assert torch.linalg.norm(Yf.sum(dim=1) - yf) <= 1e-12 * torch.linalg.norm(yf)
