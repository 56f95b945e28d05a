"""Seeded synthetic workloads: geometry, frequency-set parameters, densities.

Only inputs live here: meshes, the parameters that select a frequency set
(the frequencies themselves are computed by the method, separately by the
oracle and by the CUDA path), and the seeded densities W.  No boundary
element arithmetic is done in this module.

Workloads (all synthetic; the paper's meshes and load data are not used):

* ``cube768``     unit cube surface, 8x8 squares per face (768 triangles),
                  collocation, single layer, K = 32 multistep-CQ frequencies.
* ``lshape12288`` unit cube minus the [1/2,1]^3 octant, h = 1/32
                  (12,288 triangles), collocation, single + double layer,
                  K = 128 multistep-CQ frequencies (``lshape12288_nocap``:
                  the same without the far-block cap).
* ``sphere20480`` icosphere level 5 (20,480 triangles), Galerkin, single
                  layer, N_Q = 256 gCQ frequencies for steps in [0.005, 0.015].
* ``batch64``     64 seeded cubes/icospheres (about 500-8,000 triangles each).
* ``sphere81920`` icosphere level 6 (81,920 triangles), collocation, single
                  layer, the gCQ set of ``sphere20480``.
* ``sphere5120n`` icosphere level 4 (5,120 triangles, 2,562 vertices),
                  Galerkin with linear continuous elements: hypersingular
                  operator and adjoint double layer (the Neumann problem),
                  N_Q = 64 gCQ frequencies, nodal densities.

Small variants (``cube48``, ``cube192``, ``lshape768``, ``sphere1280``...) serve
the tests.  The large workloads cap far blocks at 192 elements per side
(``max_block``; a scheduling choice that bounds the longest block of the
persistent launch, not part of the paper's partition).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

from . import meshes


@dataclass(frozen=True)
class FreqSpec:
    """Parameters of a frequency set.

    kind = "bdf2": s_k = delta(zeta_k)/dt, zeta_k = lam * exp(2 pi i k / K).
    kind = "gcq":  N_Q = K contour points for time steps in [dt_min, dt_max].
    """
    kind: str
    K: int
    dt: float = 0.0
    lam: float = 0.0
    dt_min: float = 0.0
    dt_max: float = 0.0


@dataclass
class Workload:
    name: str
    verts: np.ndarray
    tris: np.ndarray
    freq: FreqSpec
    kernels: tuple[str, ...] = ("slp",)
    scheme: str = "colloc7"
    leaf: int = 32
    eta: float = 1.0
    max_block: int = 0           # cap of the larger side of a far block (0 = the plain partition)
    eps3: float = 1e-4
    density_seed: int = 1
    extra: dict = field(default_factory=dict)

    @property
    def E(self) -> int:
        return int(self.tris.shape[0])


def bdf2_spec(K: int, dt: float) -> FreqSpec:
    """Multistep-CQ parameters with radius lam = (1e-8)^(1/(2K))."""
    return FreqSpec("bdf2", K, dt=dt, lam=(1e-8) ** (1.0 / (2 * K)))


def gcq_spec(NQ: int, dt_min: float, dt_max: float) -> FreqSpec:
    return FreqSpec("gcq", NQ, dt_min=dt_min, dt_max=dt_max)


def graded_steps(n_steps: int = 64) -> np.ndarray:
    """Time steps dt_n = 0.01 (1 + 0.5 sin(2 pi n / 64)), n = 1..n_steps."""
    n = np.arange(1, n_steps + 1, dtype=np.float64)
    return 0.01 * (1.0 + 0.5 * np.sin(2.0 * np.pi * n / 64.0))


def densities(M: int, K: int, seed: int) -> np.ndarray:
    """W in C^{M x K}: real and imaginary parts i.i.d. N(0,1) (numpy PCG64, `seed`)."""
    rng = np.random.default_rng(seed)
    re = rng.standard_normal((M, K))
    im = rng.standard_normal((M, K))
    return (re + 1j * im).astype(np.complex128)


def mean_edge(verts: np.ndarray, tris: np.ndarray) -> float:
    e = np.concatenate([verts[tris[:, 1]] - verts[tris[:, 0]],
                        verts[tris[:, 2]] - verts[tris[:, 1]],
                        verts[tris[:, 0]] - verts[tris[:, 2]]])
    return float(np.linalg.norm(e, axis=1).mean())


def _gcq_sphere_spec() -> FreqSpec:
    steps = graded_steps(64)
    return gcq_spec(256, float(steps.min()), float(steps.max()))


def get(name: str) -> Workload:
    if name == "cube768":
        v, t = meshes.cube(8)
        return Workload(name, v, t, bdf2_spec(32, 0.1), density_seed=1)
    if name == "lshape12288":
        v, t = meshes.lshape(32)
        return Workload(name, v, t, bdf2_spec(128, 0.02), kernels=("slp", "dlp"), density_seed=2, max_block=192)
    if name == "lshape12288_nocap":
        # the 12,288-triangle L-shape on the plain partition (no far-block cap)
        v, t = meshes.lshape(32)
        return Workload(name, v, t, bdf2_spec(128, 0.02), kernels=("slp", "dlp"), density_seed=2)
    if name == "sphere20480":
        v, t = meshes.icosphere(5)
        return Workload(name, v, t, _gcq_sphere_spec(), scheme="galerkin4x4", density_seed=3, max_block=192)
    if name == "sphere81920":
        v, t = meshes.icosphere(6)
        return Workload(name, v, t, _gcq_sphere_spec(), density_seed=5, max_block=192)
    # small variants for tests
    if name == "cube48":
        v, t = meshes.cube(2)
        return Workload(name, v, t, bdf2_spec(32, 0.3), density_seed=11)
    if name == "cube192":
        v, t = meshes.cube(4)
        return Workload(name, v, t, bdf2_spec(32, 0.15), density_seed=12)
    if name == "lshape768":
        v, t = meshes.lshape(8)
        return Workload(name, v, t, bdf2_spec(32, 0.08), kernels=("slp", "dlp"), density_seed=13)
    if name == "lshape3072":
        v, t = meshes.lshape(16)
        return Workload(name, v, t, bdf2_spec(64, 0.04), kernels=("slp", "dlp"), density_seed=14)
    if name == "sphere1280":
        v, t = meshes.icosphere(3)
        return Workload(name, v, t, _gcq_sphere_spec(), density_seed=15)
    if name == "sphere1280g":
        v, t = meshes.icosphere(3)
        return Workload(name, v, t, gcq_spec(64, 0.005, 0.015), scheme="galerkin4x4", density_seed=17)
    if name == "sphere5120n":
        # the Neumann problem (Galerkin, linear continuous elements): the
        # hypersingular operator and the adjoint double layer on nodal densities
        v, t = meshes.icosphere(4)
        return Workload(name, v, t, gcq_spec(64, 0.005, 0.015), kernels=("hyp", "adj"), scheme="galerkin4x4",
                        density_seed=19, extra={"p1": True})
    if name == "sphere320g":
        v, t = meshes.icosphere(2)
        return Workload(name, v, t, gcq_spec(64, 0.005, 0.015), scheme="galerkin4x4", density_seed=16)
    raise KeyError(name)


def batch64(seed: int = 4, n_geom: int = 64) -> list[Workload]:
    """64 seeded geometries: cubes (n in [7,25] per face) alternating with
    icospheres (levels 3-4), randomly rotated, scaled by [0.5, 2] and shifted;
    K drawn from {32, 64, 128, 256}; multistep CQ with dt = 0.7 h."""
    rng = np.random.default_rng(seed)
    out = []
    for g in range(n_geom):
        if g % 2 == 0:
            n = int(rng.integers(7, 26))
            v, t = meshes.cube(n, origin=-0.5)
        else:
            lvl = int(rng.integers(3, 5))
            v, t = meshes.icosphere(lvl)
        rot = meshes.random_rotation(rng)
        scale = float(rng.uniform(0.5, 2.0))
        shift = rng.uniform(-1.0, 1.0, size=3)
        v = meshes.transformed(v, rot, scale, shift)
        K = int(rng.choice([32, 64, 128, 256]))
        h = mean_edge(v, t)
        out.append(Workload(f"batch64[{g}]", v, t, bdf2_spec(K, 0.7 * h), density_seed=1000 + g, max_block=192))
    return out


def frobenius_sample_rows(M: int, n: int, seed: int) -> np.ndarray:
    """Seeded sorted sample of n distinct row indices out of M."""
    rng = np.random.default_rng(seed)
    return np.sort(rng.choice(M, size=min(n, M), replace=False)).astype(np.int64)


def describe(w: Workload) -> dict:
    f = w.freq
    d = {"workload": w.name, "triangles": w.E, "K": f.K, "freqs": f.kind,
         "kernels": list(w.kernels), "scheme": w.scheme, "leaf": w.leaf,
         "eta": w.eta, "max_block": w.max_block, "eps3": w.eps3}
    if f.kind == "bdf2":
        d.update(dt=f.dt, lam=f.lam)
    else:
        d.update(dt_min=f.dt_min, dt_max=f.dt_max)
    return d


__all__ = ["FreqSpec", "Workload", "get", "batch64", "densities", "graded_steps",
           "bdf2_spec", "gcq_spec", "describe", "frobenius_sample_rows", "mean_edge",
           "math"]
