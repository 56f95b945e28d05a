"""GPU parity of the gCQ time-stepping consumer (g3_gcq_history) through the
C ABI, against the oracle's compact algorithm (implicit-Euler reading):

* one history update and its weights on seeded data, float64 and float32;
* three time steps on the 1,280-triangle icosphere with the gCQ set of the
  graded steps: the history sum apply_gcq(W_n) against the oracle's dense
  apply of the oracle's W_n on sampled rows (<= 1e-4, the compression's
  tolerance), and the operator at the real frequency 1/dt_n (a one-frequency
  set from g3_freqs_from_array) against the dense oracle.
"""
import numpy as np
import pytest

from inputs import workloads
from oracle import apply as O_apply, freqs as O_freqs, gcq as O_gcq, quadrature as O_q

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx(g3):
    return g3.Context(0)


@pytest.mark.parametrize("dtype,tol", [("c128", 1e-13), ("c64", 2e-6)])
def test_history_step_matches_oracle(g3, ctx, dtype, tol):
    import torch
    tdt = torch.complex128 if dtype == "c128" else torch.complex64
    F = g3.g3_freqs_gcq(ctx, 64, 0.005, 0.015)
    fr = F.get()
    s, om = fr["s"], fr["omega"]
    rng = np.random.default_rng(2)
    M = 1000
    X0 = rng.standard_normal((M, 64)) + 1j * rng.standard_normal((M, 64))
    th = rng.standard_normal(M) + 1j * rng.standard_normal(M)
    X = torch.from_numpy(X0.T.copy()).to("cuda", tdt).t()
    W = g3.gcq_history(ctx, F, X, torch.from_numpy(th).to("cuda", tdt), 0.012, 0.007)
    Xr = O_gcq.history_step(X0, th, s, 0.012)
    Wr = O_gcq.history_weights(Xr, s, om, 0.007)
    Xg, Wg = X.cpu().numpy(), W.cpu().numpy()
    assert np.linalg.norm(Xg - Xr) <= tol * np.linalg.norm(Xr)
    assert np.linalg.norm(Wg - Wr) <= tol * np.linalg.norm(Wr)
    # no density: the update only divides
    W2 = g3.gcq_history(ctx, F, X, None, 0.009, 0.011)
    Xr2 = O_gcq.history_step(Xr, None, s, 0.009)
    assert np.linalg.norm(X.cpu().numpy() - Xr2) <= tol * np.linalg.norm(Xr2)
    assert np.linalg.norm(W2.cpu().numpy() - O_gcq.history_weights(Xr2, s, om, 0.011)) <= tol * np.linalg.norm(Xr2)


def test_history_rejects_sets_without_weights(g3, ctx):
    import torch
    F = g3.g3_freqs_bdf2(ctx, 8, 0.1, 0.1)
    X = torch.zeros((8, 10), dtype=torch.complex128, device="cuda").t()
    with pytest.raises(g3.G3Error) as e:
        g3.gcq_history(ctx, F, X, None, 0.1, 0.1)
    assert "EINVAL" in str(e.value)


def test_time_steps_history_sum_and_real_frequency_operator(g3, ctx):
    import torch
    w = workloads.get("sphere1280")
    dts = workloads.graded_steps(64)
    geo = O_q.Geometry(w.verts, w.tris)
    ef = lambda I, J, s: O_q.entries(geo, "slp", I, J, s)
    T = g3.build_cluster_tree(ctx, w.verts, w.tris, w.leaf, w.eta)
    F = g3.freqs_from_spec(ctx, w.freq)
    fr = F.get()
    s, om = fr["s"], fr["omega"]
    nf = g3.assemble_near(ctx, T, F, "slp", prec="fp64")
    fa = g3.aca3_compress(ctx, T, F, "slp", prec="fp64", eps3=w.eps3)
    rng = np.random.default_rng(7)
    E, K = w.E, s.size
    thetas = [rng.standard_normal(E) + 0j for _ in range(4)]
    X = torch.zeros((K, E), dtype=torch.complex128, device="cuda").t()
    Xr = np.zeros((E, K), complex)
    rows = np.sort(rng.choice(E, 12, replace=False))
    for n in range(1, 4):
        W = g3.gcq_history(ctx, F, X, torch.from_numpy(thetas[n - 1]).to("cuda"), float(dts[n - 1]), float(dts[n]))
        Xr = O_gcq.history_step(Xr, thetas[n - 1], s, float(dts[n - 1]))
        Wr = O_gcq.history_weights(Xr, s, om, float(dts[n]))
        assert np.linalg.norm(W.cpu().numpy() - Wr) <= 1e-12 * np.linalg.norm(Wr)
        hist = g3.apply_gcq(ctx, T, nf, fa, W).cpu().numpy()
        ref = O_apply.dense_apply(ef, E, s, Wr, rows=rows)
        assert np.linalg.norm(hist[rows] - ref) <= 1e-4 * np.linalg.norm(ref), n
        # V((dt_n A)^{-1}) theta_n: the operator at the real frequency 1/dt_n
        F1 = g3.g3_freqs_from_array(ctx, np.array([1.0 / dts[n] + 0j]))
        assert F1.info() == (1, 1)
        nf1 = g3.assemble_near(ctx, T, F1, "slp", prec="fp64")
        fa1 = g3.aca3_compress(ctx, T, F1, "slp", prec="fp64", eps3=w.eps3)
        th = torch.from_numpy(thetas[n].reshape(E, 1).copy()).to("cuda")
        v1 = g3.apply_gcq(ctx, T, nf1, fa1, th).cpu().numpy()
        ref1 = O_apply.dense_apply(ef, E, np.array([1.0 / dts[n] + 0j]), thetas[n].reshape(E, 1), rows=rows)
        assert np.linalg.norm(v1[rows] - ref1) <= 1e-4 * np.linalg.norm(ref1), n
