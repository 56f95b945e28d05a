"""Pins for the oracle's frequency sets (multistep CQ and the gCQ contour of
Appendix A).  None of these re-types the oracle's formulas: each checks a
property the frequencies must have."""
import numpy as np
import pytest
from scipy import special

from inputs import workloads
from oracle import freqs


def bdf2_impulse_response(a: float, dt: float, n: int) -> np.ndarray:
    """Textbook BDF2 for y' = -a y + g with g a discrete unit impulse (scaled
    by 1/dt): (3 y_m - 4 y_{m-1} + y_{m-2}) / (2 dt) = -a y_m + g_m.
    The resulting y_m are the CQ weights of F(s) = 1/(s + a)."""
    y = np.zeros(n)
    for m in range(n):
        g = 1.0 / dt if m == 0 else 0.0
        ym1 = y[m - 1] if m >= 1 else 0.0
        ym2 = y[m - 2] if m >= 2 else 0.0
        y[m] = (g + (4.0 * ym1 - ym2) / (2.0 * dt)) / (1.5 / dt + a)
    return y * dt


@pytest.mark.parametrize("K,dt", [(32, 0.1), (128, 0.02), (64, 0.05)])
def test_bdf2_frequencies_reproduce_bdf2_weights(K, dt):
    spec = workloads.bdf2_spec(K, dt)
    s = freqs.bdf2(K, dt, spec.lam)
    a = 1.7
    # trapezoidal inversion of the generating function on the circle |zeta| = lam
    n = np.arange(K // 2)
    Fs = 1.0 / (s + a)
    k = np.arange(K)
    w_cq = np.array([(spec.lam ** (-m) / K) * np.sum(Fs * np.exp(-2j * np.pi * m * k / K)) for m in n])
    w_ref = bdf2_impulse_response(a, dt, K // 2)
    assert np.max(np.abs(w_cq.imag)) < 1e-10
    assert np.max(np.abs(w_cq.real - w_ref)) < 1e-3 * np.max(np.abs(w_ref))


@pytest.mark.parametrize("K,dt", [(32, 0.1), (128, 0.02)])
def test_bdf2_conjugate_pairs_and_stability(K, dt):
    spec = workloads.bdf2_spec(K, dt)
    s = freqs.bdf2(K, dt, spec.lam)
    uniq, partner = freqs.bdf2_unique(K)
    assert uniq.size == K // 2 + 1
    assert np.all(s.real > 0)                  # A-stability of BDF2, |zeta| < 1
    assert np.max(np.abs(s[partner] - np.conj(s))) < 1e-12 * np.abs(s).max()
    # the unique set plus partners covers every index
    assert set(uniq) | set(partner[uniq]) == set(range(K))


def _gcq_sphere():
    st = workloads.graded_steps(64)
    return 256, float(st.min()), float(st.max())


def test_gcq_contour_residues():
    NQ, dmin, dmax = _gcq_sphere()
    s, w = freqs.gcq(NQ, dmin, dmax)
    # (1/2 pi i) contour integral of 1/(s - a) = 1 for a enclosed, 0 outside
    for dt in (dmin, 0.5 * (dmin + dmax), dmax, 0.0073, 0.0121):
        val = np.sum(w / (s - 1.0 / dt))
        assert abs(val - 1.0) < 1e-10, (dt, val)
    for a in (-50.0, 1500.0, 3000.0 + 10.0j):
        assert abs(np.sum(w / (s - a))) < 1e-6
    assert abs(np.sum(w)) < 1e-10
    # the contour encloses all poles 1/dt_n of the graded mesh
    for dt in workloads.graded_steps(64):
        assert abs(np.sum(w / (s - 1.0 / dt)) - 1.0) < 1e-10


def test_gcq_conjugate_symmetry_and_halfplane():
    NQ, dmin, dmax = _gcq_sphere()
    s, w = freqs.gcq(NQ, dmin, dmax)
    uniq, partner = freqs.gcq_unique(NQ)
    assert uniq.size == NQ // 2
    assert np.max(np.abs(s[partner] - np.conj(s))) < 1e-10 * np.abs(s).max()
    assert np.max(np.abs(w[partner] - np.conj(w))) < 1e-10 * np.abs(w).max()
    assert np.all(s.real > 0)


def test_jacobi_complex_identities():
    m = 0.0213
    u = np.array([0.3 + 0.7j, -1.1 + 1.9j, 2.0 + 0.1j, -0.4 - 2.2j])
    sn, cn, dn = freqs.jacobi_complex(u, m)
    assert np.max(np.abs(sn ** 2 + cn ** 2 - 1)) < 1e-12
    assert np.max(np.abs(dn ** 2 + m * sn ** 2 - 1)) < 1e-12
    # d sn / du = cn dn, checked by a central difference along the real axis
    h = 1e-5
    sp, _, _ = freqs.jacobi_complex(u + h, m)
    sm, _, _ = freqs.jacobi_complex(u - h, m)
    assert np.max(np.abs((sp - sm) / (2 * h) - cn * dn)) < 1e-8
    # and along the imaginary axis (analyticity): d/du = -i d/dy
    sp, _, _ = freqs.jacobi_complex(u + 1j * h, m)
    sm, _, _ = freqs.jacobi_complex(u - 1j * h, m)
    assert np.max(np.abs((sp - sm) / (2j * h) - cn * dn)) < 1e-8
    assert abs(special.ellipk(0.0) - np.pi / 2) < 1e-15


def test_gcq_constant_steps_rejected():
    with pytest.raises(ValueError):
        freqs.gcq(64, 0.01, 0.01)


# ---------------------------------------------------------------- conjugate pairing of a given set

def test_pair_conjugates_reproduces_the_closed_form_pairings():
    """The closed-form sets are conjugate-closed; pairing them by value gives
    the index rules of the multistep CQ (k <-> K - k) and the gCQ
    (l <-> N_Q + 1 - l)."""
    for K in (8, 32, 128):
        s = freqs.bdf2(K, 0.1, (1e-8) ** (1.0 / (2 * K)))
        u, p = freqs.pair_conjugates(s)
        u0, p0 = freqs.bdf2_unique(K)
        assert np.array_equal(u, u0) and np.array_equal(p, p0)
    s, _ = freqs.gcq(64, 0.005, 0.015)
    u, p = freqs.pair_conjugates(s)
    u0, p0 = freqs.gcq_unique(64)
    assert np.array_equal(u, u0) and np.array_equal(p, p0)


def test_pair_conjugates_arbitrary_order_and_unpaired():
    rng = np.random.default_rng(3)
    s = freqs.bdf2(16, 0.05, (1e-8) ** (1.0 / 32))
    order = rng.permutation(16)
    t = np.r_[s[order], 2.0 + 3.0j, 5.0]        # one complex frequency without partner, one real
    u, p = freqs.pair_conjugates(t)
    K = t.size
    assert np.array_equal(p[p], np.arange(K))                  # an involution
    paired = p != np.arange(K)
    assert np.allclose(t[p][paired], np.conj(t[paired]))       # partner = conjugate
    # self-partners: the real frequencies (BDF2 k = 0, K/2 and the extra 5) and the unpaired 2 + 3i
    assert np.sum(~paired) == 4 and np.all(np.abs(t[~paired].imag[:-2]) < 1e-12 * np.abs(t[~paired][:-2]))
    assert np.all(np.diff(u) > 0)                              # increasing
    covered = np.zeros(K, bool)
    covered[u] = True
    covered[p[u]] = True
    assert covered.all() and u.size == 9 + 2                   # 9 unique BDF2 (two real) + the two extras
    assert p[16] == 16 and p[17] == 17
    for l in u:                                                # the lower index of each pair is unique
        assert p[l] >= l


# ---------------------------------------------------------------- the gCQ time-stepping consumer

def test_gcq_history_reproduces_implicit_euler():
    """For the transfer function F(s) = 1/(s + a) the implicit-Euler gCQ is
    the implicit-Euler solution of y' = -a y + theta on the same (graded)
    steps: y_n = (y_{n-1} + dt_n theta_n) / (1 + a dt_n).  The compact
    algorithm with the contour of Appendix A must reproduce it to the
    quadrature's accuracy (the contour runs from near s = 0 around
    [1/dt_max, 1/dt_min], so the pole -a of F is kept well away from it:
    a >= 20); a wrong sign of the contour weights flips the history term, a
    wrong update index shifts it by a step."""
    from oracle import gcq
    from inputs import workloads
    dts = workloads.graded_steps(64)
    s, omega = freqs.gcq(256, float(dts.min()), float(dts.max()))
    rng = np.random.default_rng(5)
    theta = 1.0 + 0.5 * np.sin(np.arange(dts.size) / 5.0) + 0.1 * rng.standard_normal(dts.size)
    for a in (20.0, 50.0, 200.0):
        g = gcq.convolution(lambda z: 1.0 / (z + a), theta, dts, s, omega)
        y = np.zeros(dts.size)
        prev = 0.0
        for n in range(dts.size):
            prev = (prev + dts[n] * theta[n]) / (1.0 + a * dts[n])
            y[n] = prev
        assert np.max(np.abs(g - y)) <= 1e-10 * np.max(np.abs(y)), a
        # the opposite orientation of the weights fails by O(1)
        g_bad = gcq.convolution(lambda z: 1.0 / (z + a), theta, dts, s, -omega)
        assert np.max(np.abs(g_bad - y)) > 0.1 * np.max(np.abs(y))


def test_gcq_history_weights_sign_and_first_step():
    """x_0 = 0 gives W = 0 at the first step; one step of a unit density gives
    x_1(s) = dt / (1 - dt s), whose weighted sum with F = 1 is the quadrature
    of (1/2 pi i) times the clockwise contour integral of dt / ((1 - dt s)(1 - dt' s)):
    the residues at s = 1/dt and 1/dt' give dt / (1 - dt'/dt) * (-1/dt) * ... =
    0 for the sum of both (the integrand decays as s^-2), so the weights of
    the two enclosed poles cancel: sum_l W_l = 0."""
    from oracle import gcq
    s, omega = freqs.gcq(128, 0.005, 0.015)
    X = np.zeros((3, s.size), complex)
    assert np.all(gcq.history_weights(X, s, omega, 0.01) == 0)
    X = gcq.history_step(X, np.ones(3), s, 0.012)
    assert np.allclose(X[0], 0.012 / (1 - 0.012 * s))
    W = gcq.history_weights(X, s, omega, 0.008)
    assert abs(W[0].sum()) <= 1e-10 * np.abs(W[0]).sum()
