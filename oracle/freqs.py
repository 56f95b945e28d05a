"""Oracle: complex Laplace frequencies of the (g)CQ, in float64.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Two frequency sets:

* Multistep CQ with the BDF2 generating function (the constant-step special
  case the workloads use):  s_k = delta(zeta_k) / dt,
  delta(zeta) = (1 - zeta) + (1 - zeta)^2 / 2,  zeta_k = lam exp(2 pi i k / K),
  k = 0..K-1.  Conjugate partners: k <-> K - k.
* gCQ contour points and weights of Appendix A ("Parameters of the gCQ"):
  s_l = gamma(sigma_l),  omega_l = -4 K(k^2) gamma'(sigma_l) / (2 pi i N_Q),
  sigma_l = -K + (l - 1/2) 4K/N_Q + i K'/2,  l = 1..N_Q, with
  q = dt_max / dt_min (the implicit-Euler reading of q, factor 5 and the
  Runge-Kutta eigenvalues dropped), k = (q - sqrt(2q-1)) / (q + sqrt(2q-1)),
  K = K(k^2), K' = K(1 - k^2) (parameter convention m = k^2).
  Conjugate partners: l <-> N_Q + 1 - l.

The Jacobi elliptic functions at a complex argument are assembled from
real-argument values by the addition formula with Jacobi's imaginary
transformation (Abramowitz & Stegun 16.21.1-16.21.3); scipy supplies the
real-argument sn, cn, dn and K(m).

The unique set used by the compression is: BDF2, k = 0..K/2 (k = 0 and
K/2 are self-conjugate); gCQ, l = 1..N_Q/2 (no self-conjugate points for even
N_Q).  `partner[k]` is the index of conj(s_k) in the full set.

A set given as an array (any rule) is paired by `pair_conjugates`: a real
operator has A(conj s) = conj A(s) (Appendix A: half of a conjugate-closed
set suffices), so each frequency whose conjugate is also in the set needs
only one of the two.
"""
from __future__ import annotations

import numpy as np
from scipy import special


def bdf2(K: int, dt: float, lam: float) -> np.ndarray:
    """All K multistep-CQ frequencies s_k = delta(zeta_k)/dt (complex128)."""
    k = np.arange(K, dtype=np.float64)
    zeta = lam * np.exp(2j * np.pi * k / K)
    one_minus = 1.0 - zeta
    return (one_minus + 0.5 * one_minus * one_minus) / dt


def bdf2_unique(K: int) -> tuple[np.ndarray, np.ndarray]:
    """(unique indices 0..K/2, partner of each full index)."""
    uniq = np.arange(K // 2 + 1)
    partner = (K - np.arange(K)) % K
    return uniq, partner


def jacobi_complex(u: np.ndarray, m: float) -> tuple[np.ndarray, np.ndarray, np.ndarray]:
    """sn, cn, dn of complex u = x + i y with parameter m (A&S 16.21.1-3)."""
    x = np.real(u)
    y = np.imag(u)
    s, c, d, _ = special.ellipj(x, m)
    s1, c1, d1, _ = special.ellipj(y, 1.0 - m)
    den = c1 * c1 + m * (s * s) * (s1 * s1)
    sn = (s * d1 + 1j * c * d * s1 * c1) / den
    cn = (c * c1 - 1j * s * d * s1 * d1) / den
    dn = (d * c1 * d1 - 1j * m * s * c * s1) / den
    return sn, cn, dn


def gcq(NQ: int, dt_min: float, dt_max: float) -> tuple[np.ndarray, np.ndarray]:
    """gCQ contour points s_l and weights omega_l, l = 1..NQ (Appendix A).

    Raises ValueError when dt_max/dt_min <= 1: the paper notes that constant
    steps give q = 1, k = 0, where the construction breaks down.
    """
    q = dt_max / dt_min
    if not q > 1.0:
        raise ValueError("gCQ contour needs dt_max > dt_min (q = 1 gives k = 0)")
    r = np.sqrt(2.0 * q - 1.0)
    k = (q - r) / (q + r)
    m = k * k
    Kk = special.ellipk(m)
    Kp = special.ellipk(1.0 - m)
    ell = np.arange(1, NQ + 1, dtype=np.float64)
    sigma = -Kk + (ell - 0.5) * 4.0 * Kk / NQ + 0.5j * Kp
    sn, cn, dn = jacobi_complex(sigma, m)
    pref = 1.0 / (dt_min * (q - 1.0))
    s = pref * (r * (1.0 / k + sn) / (1.0 / k - sn) - 1.0)
    dgamma = pref * r * 2.0 * cn * dn / (k * (1.0 / k - sn) ** 2)
    omega = -4.0 * Kk * dgamma / (2j * np.pi * NQ)
    return s, omega


def gcq_unique(NQ: int) -> tuple[np.ndarray, np.ndarray]:
    """(unique indices 0..NQ/2-1, partner of each full index), 0-based."""
    uniq = np.arange(NQ // 2)
    partner = NQ - 1 - np.arange(NQ)
    return uniq, partner


def frequency_set(spec) -> dict:
    """All frequencies of a workload's FreqSpec plus the unique subset."""
    if spec.kind == "bdf2":
        s = bdf2(spec.K, spec.dt, spec.lam)
        uniq, partner = bdf2_unique(spec.K)
        w = None
    elif spec.kind == "gcq":
        s, w = gcq(spec.K, spec.dt_min, spec.dt_max)
        uniq, partner = gcq_unique(spec.K)
    else:
        raise ValueError(spec.kind)
    return {"s": s, "omega": w, "uniq": uniq, "partner": partner}


def pair_conjugates(s: np.ndarray, tol: float = 1e-12) -> tuple[np.ndarray, np.ndarray]:
    """Unique indices and conjugate partners of an arbitrary frequency array.

    Scanning l = 0, 1, ...: an l not yet paired is unique; if Im s_l is not
    zero (|Im s_l| > tol |s_l|) it is paired with the first not-yet-paired
    l' > l whose s_l' is conj(s_l) within tol |s_l|.  Real frequencies and
    complex ones without a conjugate in the set are their own partners.
    """
    s = np.asarray(s, dtype=np.complex128)
    K = s.size
    partner = np.full(K, -1, dtype=np.int64)
    uniq = []
    for l in range(K):
        if partner[l] >= 0:
            continue
        uniq.append(l)
        partner[l] = l
        if abs(s[l].imag) <= tol * abs(s[l]):
            continue
        for m in range(l + 1, K):
            if partner[m] < 0 and abs(s[m] - np.conj(s[l])) <= tol * abs(s[l]):
                partner[l], partner[m] = m, l
                break
    return np.asarray(uniq, dtype=np.int64), partner
