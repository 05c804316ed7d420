"""Seeded synthetic inputs shared by the CUDA path, the oracle tests and the bench.

This module holds scene descriptions (media, sources, sensors, source-sensor
pairs, run settings) and seeded generators of path states.  It contains none
of the method's arithmetic: no density, no move, no estimator.  Both the
oracle (FP64 CPU) and the CUDA library consume these plain values, and
neither side imports the other.

Scene presets follow the paper's synthetic-detector setting (section
"Implementation": point source, spherical light-sensitive elements,
homogeneous or piecewise-constant scattering/absorption coefficients,
Henyey-Greenstein phase function) with the sizes of the five workloads the
library is measured on:

* ``plain``      - isotropic source at the origin, one sensor of radius 0.1 m at
                   1 m, scattering length 0.5 m, absorption length 5 m, g=0.9;
                   64 chains x 10,000 steps, vertex cap 64.
* ``detector``   - source-sensor distance 50 m, sensor radius 0.165 m,
                   scattering length 5 m, absorption length 100 m, g=0.94;
                   65,536 chains x 100,000 steps, vertex cap 256.
* ``batched``    - 4,096 pairs, distances U(5, 150) m, chains per pair
                   U{16..512}, caps 64..1,024 growing with distance.
* ``gradients``  - the ``plain`` geometry with MALA moves (step 0.02 m) over
                   65,536 chains, gradients w.r.t. (lambda_s, lambda_a, g).
* ``layered``    - 100 horizontal 10 m layers with log-normal lengths
                   (medians 5 m / 100 m, sigma_log 0.3), g=0.94, one source and
                   60 sensors of radius 0.165 m on a vertical string (17 m pitch),
                   8,192 chains per sensor, vertex cap 1,024.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Sequence

import numpy as np

HOMOGENEOUS = 0
LAYERED = 1

EMIT_ISOTROPIC = 0
EMIT_VMF = 1

RHO_ONE = 0
RHO_PAPER = 1

INIT_DIRECT = 0
INIT_STRAIGHT = 1
INIT_USER = 2

WITHIN_PERTURB = 0
WITHIN_MALA = 1
WITHIN_TREE = 2
WITHIN_HMC = 3

LAYOUT_AUTO = 0
LAYOUT_WARP = 1
LAYOUT_LANE = 2

BASE_SEED = 0x181104156


@dataclasses.dataclass
class Medium:
    kind: int = HOMOGENEOUS
    lambda_s: float = 0.5          # scattering length (m), homogeneous
    lambda_a: float = 5.0          # absorption length (m), homogeneous
    g: float = 0.9                 # mean cosine of the phase function
    f_sl: float = 0.0              # weight of the simplified-Liu component
    z0: float = 0.0                # bottom of layer 0 (m), layered
    dz: float = 10.0               # layer thickness (m), layered
    lambda_s_layers: Optional[np.ndarray] = None
    lambda_a_layers: Optional[np.ndarray] = None
    # wavelength dependence: coefficients b (l / lambda0)^(-k_s), a (l / lambda0)^(-k_a) (0: none)
    lambda0: float = 0.0           # reference wavelength (nm) of lambda_s, lambda_a
    k_s: float = 0.0
    k_a: float = 0.0

    @property
    def n_layers(self) -> int:
        return 0 if self.lambda_s_layers is None else int(len(self.lambda_s_layers))


@dataclasses.dataclass
class Source:
    pos: Sequence[float] = (0.0, 0.0, 0.0)
    emission: int = EMIT_ISOTROPIC
    kappa: float = 0.0
    direction: Sequence[float] = (0.0, 0.0, 1.0)


@dataclasses.dataclass
class Sensor:
    centre: Sequence[float] = (0.0, 0.0, 1.0)
    radius: float = 0.1
    rho: int = RHO_ONE
    rho_hat: Sequence[float] = (0.0, -1.0, 0.0)


@dataclasses.dataclass
class Pair:
    source: int
    sensor: int
    n_chains: int
    cap: int


@dataclasses.dataclass
class Run:
    seed: int = BASE_SEED
    n_steps: int = 10_000
    burn_in: int = 1_000
    p_within: float = 0.6
    p_birth: float = 0.2
    p_death: float = 0.2
    within: int = WITHIN_PERTURB
    sigma: float = 0.05            # Gaussian perturbation scale (m)
    mala_step: float = 0.02        # MALA step epsilon (m)
    kappa_end: float = 0.0         # vMF concentration of end moves; 0 -> (R/sigma)^2
    init: int = INIT_DIRECT
    init_k: int = 0                # interior vertices of a straight initial path
    init_jitter: float = 0.0       # N(0, jitter^2) per coordinate
    thin_bridge: int = 0           # 0 = no reference-density bridge terms
    gradients: bool = False
    hmc_steps: int = 10            # leapfrog steps of a full-path gradient (HMC) move, step mala_step
    layout: int = LAYOUT_AUTO      # LAYOUT_WARP: one warp per chain; LAYOUT_LANE: one lane per chain (lean runs)
    # wavelength as a sampled coordinate: spectrum table (nm, any positive scale); None = off
    spectrum_nm: Optional[Sequence[float]] = None
    spectrum: Optional[Sequence[float]] = None
    sigma_lambda: float = 10.0     # Gaussian step of a wavelength move (nm)


@dataclasses.dataclass
class Scene:
    name: str
    medium: Medium
    sources: List[Source]
    sensors: List[Sensor]
    pairs: List[Pair]
    run: Run

    @property
    def total_chains(self) -> int:
        return int(sum(p.n_chains for p in self.pairs))


def plain(n_chains: int = 64, n_steps: int = 10_000, cap: int = 64) -> Scene:
    """Plain RJMCMC workload: 64 chains x 10,000 steps, caps 2..64."""
    med = Medium(HOMOGENEOUS, lambda_s=0.5, lambda_a=5.0, g=0.9)
    run = Run(seed=BASE_SEED + 0, n_steps=n_steps, burn_in=n_steps // 10,
              init=INIT_DIRECT, sigma=0.05)
    return Scene("plain", med, [Source()], [Sensor((0.0, 0.0, 1.0), 0.1)],
                 [Pair(0, 0, n_chains, cap)], run)


def detector(n_chains: int = 65_536, n_steps: int = 100_000, cap: int = 256) -> Scene:
    """Detector-scale single pair: 50 m, R=0.165 m, lambda_s=5, lambda_a=100, g=0.94."""
    med = Medium(HOMOGENEOUS, lambda_s=5.0, lambda_a=100.0, g=0.94)
    run = Run(seed=BASE_SEED + 1, n_steps=n_steps, burn_in=n_steps // 10,
              init=INIT_STRAIGHT, init_k=4, init_jitter=0.5, sigma=0.05)
    return Scene("detector", med, [Source()], [Sensor((0.0, 0.0, 50.0), 0.165)],
                 [Pair(0, 0, n_chains, cap)], run)


def batched_cap(distance: float) -> int:
    """Vertex cap growing linearly from 64 at 5 m to 1,024 at 150 m, rounded up to 32."""
    raw = 64.0 + 960.0 * (distance - 5.0) / 145.0
    return int(32 * math.ceil(raw / 32.0))


def batched(n_pairs: int = 4096, n_steps: int = 10_000, chain_lo: int = 16,
            chain_hi: int = 512, d_lo: float = 5.0, d_hi: float = 150.0,
            radius: float = 0.1) -> Scene:
    """Uneven batch: pairs with random distances/directions, chain counts and caps."""
    rng = np.random.default_rng(BASE_SEED + 2)
    med = Medium(HOMOGENEOUS, lambda_s=0.5, lambda_a=5.0, g=0.9)
    sensors, pairs = [], []
    for i in range(n_pairs):
        d = float(rng.uniform(d_lo, d_hi))
        v = rng.normal(size=3)
        v /= np.linalg.norm(v)
        sensors.append(Sensor(tuple(float(x) for x in d * v), radius))
        pairs.append(Pair(0, i, int(rng.integers(chain_lo, chain_hi + 1)), batched_cap(d)))
    run = Run(seed=BASE_SEED + 2, n_steps=n_steps, burn_in=n_steps // 10,
              init=INIT_DIRECT, sigma=0.05)
    return Scene("batched", med, [Source()], sensors, pairs, run)


def gradients(n_chains: int = 65_536, n_steps: int = 10_000, cap: int = 64) -> Scene:
    """The plain geometry with MALA within-dimension moves and score gradients."""
    sc = plain(n_chains, n_steps, cap)
    sc.name = "gradients"
    sc.run = dataclasses.replace(sc.run, seed=BASE_SEED + 3, within=WITHIN_MALA,
                                 mala_step=0.02, gradients=True)
    return sc


def layered(n_sensors: int = 60, chains_per_sensor: int = 8192, n_steps: int = 10_000,
            cap: int = 1024, n_layers: int = 100, dz: float = 10.0) -> Scene:
    """Layered medium with a vertical string of sensors and one source."""
    rng = np.random.default_rng(BASE_SEED + 4)
    ls = 5.0 * np.exp(0.3 * rng.normal(size=n_layers))
    la = 100.0 * np.exp(0.3 * rng.normal(size=n_layers))
    z0 = -0.5 * n_layers * dz
    med = Medium(LAYERED, g=0.94, z0=z0, dz=dz, lambda_s_layers=ls, lambda_a_layers=la)
    z_mid = 0.0
    sensors = [Sensor((0.0, 0.0, z_mid + 17.0 * (i - (n_sensors - 1) / 2.0)), 0.165)
               for i in range(n_sensors)]
    src = Source((20.0, 0.0, z_mid))
    pairs = [Pair(0, i, chains_per_sensor, cap) for i in range(n_sensors)]
    run = Run(seed=BASE_SEED + 4, n_steps=n_steps, burn_in=n_steps // 10,
              init=INIT_DIRECT, sigma=0.05, gradients=True)
    return Scene("layered", med, [src], sensors, pairs, run)


def batched_small(n_chains: int = 1024, n_steps: int = 10_000) -> Scene:
    """A small uneven batch: four single-scatter pairs (cap 3) at 1-3 m in
    different directions and two long-cap pairs (caps 150 and 600, two more
    cap classes) at 3 m and 4 m; plain-workload medium, sensors R = 0.3 m."""
    med = Medium(HOMOGENEOUS, lambda_s=0.5, lambda_a=5.0, g=0.9)
    dirs = [(0.0, 0.0, 1.0), (1.0, 0.0, 0.0), (0.0, -0.6, 0.8), (-0.48, 0.6, -0.64), (0.0, 1.0, 0.0),
            (0.6, 0.0, -0.8)]
    dist = [1.0, 1.5, 2.0, 3.0, 3.0, 4.0]
    caps = [3, 3, 3, 3, 150, 600]
    sensors = [Sensor(tuple(d * x for x in u), 0.3) for u, d in zip(dirs, dist)]
    pairs = [Pair(0, i, n_chains, caps[i]) for i in range(6)]
    run = Run(seed=BASE_SEED + 5, n_steps=n_steps, burn_in=n_steps // 10, init=INIT_DIRECT, sigma=0.05)
    return Scene("batched_small", med, [Source()], sensors, pairs, run)


def general_small(n_chains: int = 64, n_steps: int = 400) -> Scene:
    """Exercises every general-kernel branch: layered medium, vMF emission,
    the paper's detection probability and the simplified-Liu mixture."""
    rng = np.random.default_rng(BASE_SEED + 6)
    med = Medium(LAYERED, g=0.9, f_sl=0.45, z0=-2.0, dz=0.5,
                 lambda_s_layers=0.6 * np.exp(0.3 * rng.normal(size=12)),
                 lambda_a_layers=5.0 * np.exp(0.3 * rng.normal(size=12)))
    src = Source((0.1, -0.1, -0.5), EMIT_VMF, 5.0, (0.0, 0.0, 1.0))
    sen = Sensor((0.2, 0.1, 0.9), 0.15, RHO_PAPER, (0.0, -1.0, 0.0))
    run = Run(seed=BASE_SEED + 7, n_steps=n_steps, burn_in=n_steps // 10, init=INIT_DIRECT, sigma=0.05)
    return Scene("general_small", med, [src], [sen], [Pair(0, 0, n_chains, 64)], run)


def wavelength(n_chains: int = 4096, n_steps: int = 20_000, cap: int = 64) -> Scene:
    """The plain geometry with the wavelength sampled along with the path
    (section "Discussion"): scattering and absorption lengths at 400 nm as in
    the plain workload, b ~ (l / 400 nm)^-4 (Rayleigh-like), a ~ (l / 400
    nm)^-2, and a triangular emission-times-detection spectrum over 300-600 nm
    peaking at 420 nm."""
    sc = plain(n_chains, n_steps, cap)
    sc.name = "wavelength"
    sc.medium = dataclasses.replace(sc.medium, lambda0=400.0, k_s=4.0, k_a=2.0)
    sc.run = dataclasses.replace(sc.run, seed=BASE_SEED + 8, spectrum_nm=(300.0, 420.0, 600.0),
                                 spectrum=(0.0, 1.0, 0.0), sigma_lambda=20.0)
    return sc


# Scattering coefficients b1 (1/m) of the x >= 0 half of the paper's test scene (Table tbl:results).
TWO_SENSOR_B1 = (0.1, 0.2, 0.3, 0.4, 0.5)


def to_device_frame(v):
    """Paper frame (x, y, z) -> the frame the two-region scene is built in,
    (y, z, x): a proper rotation that puts the paper's x axis (the normal of
    the plane dividing the medium) on the layer axis."""
    a = np.asarray(v, dtype=np.float64)
    return np.stack([a[..., 1], a[..., 2], a[..., 0]], axis=-1)


def to_paper_frame(v):
    """Inverse of to_device_frame: (X, Y, Z) -> (Z, X, Y)."""
    a = np.asarray(v, dtype=np.float64)
    return np.stack([a[..., 2], a[..., 0], a[..., 1]], axis=-1)


def _dev(v):
    return tuple(float(x) for x in to_device_frame(v))


def two_sensor(b1: float = 0.3, n_chains: int = 4096, n_steps: int = 200_000, cap: int = 256,
       sigma: float = 0.5, init_k: int = 30, init_jitter: float = 0.5) -> Scene:
    """The paper's two-sensor test scene (section "Implementation", Fig. setup).

    Source at the origin with vMF emission (kappa 38) along +z; the medium is
    divided by the plane x = 0: absorption 0.01/m everywhere, scattering
    0.3/m for x < 0 and ``b1`` for x >= 0; simplified-Liu / Henyey-Greenstein
    mixture with Gamma = 0.95, f_SL = 0.45; sensors of radius 0.15 m at
    (0, 0, 120) and (60, 7, 104) m, detection probability rho with rho_hat =
    (0, -1, 0).  Pair 0 ends on sensor 0, pair 1 on sensor 1.

    The two half-spaces are a two-layer medium (boundary at 0, the end layers
    extend to infinity) in the frame of to_device_frame, so positions, the
    emission axis and rho_hat are given in that frame; to_paper_frame maps
    paths back.  Chains start from straight paths with ``init_k`` jittered
    interior vertices and use Gaussian steps of ``sigma`` (m)."""
    med = Medium(LAYERED, g=0.95, f_sl=0.45, z0=-1.0, dz=1.0,
                 lambda_s_layers=np.array([1.0 / 0.3, 1.0 / float(b1)]),
                 lambda_a_layers=np.array([100.0, 100.0]))
    src = Source(_dev((0.0, 0.0, 0.0)), EMIT_VMF, 38.0, _dev((0.0, 0.0, 1.0)))
    rho_hat = _dev((0.0, -1.0, 0.0))
    sensors = [Sensor(_dev((0.0, 0.0, 120.0)), 0.15, RHO_PAPER, rho_hat),
               Sensor(_dev((60.0, 7.0, 104.0)), 0.15, RHO_PAPER, rho_hat)]
    pairs = [Pair(0, 0, n_chains, cap), Pair(0, 1, n_chains, cap)]
    run = Run(seed=BASE_SEED + 8, n_steps=n_steps, burn_in=n_steps // 10, init=INIT_STRAIGHT,
              init_k=init_k, init_jitter=init_jitter, sigma=sigma)
    return Scene("two_sensor", med, [src], sensors, pairs, run)


PRESETS = {"plain": plain, "detector": detector, "batched": batched,
           "gradients": gradients, "layered": layered}


def random_paths(source: Sequence[float], centre: Sequence[float], radius: float,
                 batch: int, cap: int, n_lo: int, n_hi: int, seed: int,
                 lateral: float = 0.3, cap_spread: float = 1.0):
    """Seeded random polylines from ``source`` to a point on the sensor sphere.

    Interior vertices sit at sorted uniform fractions of the source -> sensor
    line plus isotropic Gaussian offsets of scale ``lateral`` (m); the end
    vertex is a point of the sphere on the source-facing side, spread over a
    cap of angular scale ``cap_spread`` (rad).  Returns ``(xyz, n)`` where
    ``xyz`` is float32 of shape (3, batch, cap) (SoA, unused slots zero) and
    ``n`` is int32 vertex counts in [n_lo, n_hi].
    """
    rng = np.random.default_rng(seed)
    s = np.asarray(source, dtype=np.float64)
    c = np.asarray(centre, dtype=np.float64)
    xyz = np.zeros((3, batch, cap), dtype=np.float32)
    n = rng.integers(n_lo, n_hi + 1, size=batch).astype(np.int32)
    axis = (s - c) / np.linalg.norm(s - c)
    for i in range(batch):
        k = int(n[i])
        fr = np.sort(rng.uniform(0.05, 0.9, size=k - 2))
        pts = s[None, :] + fr[:, None] * (c - s)[None, :]
        pts = pts + lateral * rng.normal(size=pts.shape)
        nu = axis + cap_spread * rng.normal(size=3) * 0.5
        nu /= np.linalg.norm(nu)
        end = c + radius * nu
        path = np.concatenate([s[None, :], pts, end[None, :]], axis=0)
        xyz[:, i, :k] = path.T.astype(np.float32)
    return xyz, n
