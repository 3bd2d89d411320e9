"""Seeded synthetic inputs for the N-body hot path.

This module only draws initial conditions; it holds none of the force,
integration or reduction arithmetic. Both the GPU path's tests/benchmarks and
the CPU oracle receive the arrays produced here.

The paper's N-body miniapp (Sec. II-A, Sec. V-B) uses a synthetic particle set
of 10 000 bodies; this project drives the same all-pairs method with
self-gravitating Plummer spheres instead, in units G = M = a = 1:

* ``plummer``       -- one Plummer sphere, equal masses 1/N, sampled with the
                       Aarseth-Henon-Wielen (1974) inverse-CDF / rejection scheme,
                       truncated at r <= 20 a, centre of mass and its velocity
                       subtracted.
* ``two_spheres``   -- two Plummer spheres of N/2 bodies each (mass 0.5 each,
                       velocities scaled by sqrt(0.5)), centres at (-5,0,0) and
                       (+5,0,0) approaching with relative speed 0.5 along x,
                       per-body masses log-normal (sigma 0.5) normalised to a
                       total of 1.
* ``ensemble``      -- many independent Plummer systems with sizes drawn
                       log-uniformly in [n_min, n_max].
* ``kepler_pair``   -- an isolated two-body orbit with a closed-form solution.
* ``lj_gas``        -- the paper's own system (Sec. II-A): a Lennard-Jones gas in
                       reduced units, lattice start inside a cubic box, Maxwell
                       velocities.

All state is float64, shaped ``[N, 3]`` (positions, velocities) and ``[N]``
(masses), C-contiguous.
"""

from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

# Plummer model: radius truncation (in scale radii) applied when sampling.
PLUMMER_RMAX = 20.0


def _isotropic(rng: np.random.Generator, n: int) -> np.ndarray:
    """Unit vectors uniform on the sphere (z uniform in [-1,1], azimuth uniform)."""
    z = rng.uniform(-1.0, 1.0, n)
    ph = rng.uniform(0.0, 2.0 * math.pi, n)
    rho = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    return np.stack([rho * np.cos(ph), rho * np.sin(ph), z], axis=1)


def _plummer_radii(rng: np.random.Generator, n: int) -> np.ndarray:
    """Radii with cumulative mass M(<r) = r^3 / (1 + r^2)^{3/2}, truncated at PLUMMER_RMAX."""
    out = np.empty(n)
    filled = 0
    while filled < n:
        k = n - filled
        X = rng.uniform(0.0, 1.0, k)
        X = X[X > 0.0]
        r = 1.0 / np.sqrt(X ** (-2.0 / 3.0) - 1.0)
        r = r[np.isfinite(r) & (r <= PLUMMER_RMAX)]
        take = min(len(r), k)
        out[filled:filled + take] = r[:take]
        filled += take
    return out


def _plummer_q(rng: np.random.Generator, n: int) -> np.ndarray:
    """q = v / v_esc by von Neumann rejection on g(q) = q^2 (1 - q^2)^{7/2}, q in [0, 1]."""
    out = np.empty(n)
    filled = 0
    while filled < n:
        k = max(64, 2 * (n - filled))
        q = rng.uniform(0.0, 1.0, k)
        y = rng.uniform(0.0, 0.1, k)  # max g = 0.0920 at q^2 = 2/9
        q = q[y < q * q * (1.0 - q * q) ** 3.5]
        take = min(len(q), n - filled)
        out[filled:filled + take] = q[:take]
        filled += take
    return out


def plummer(n: int, seed: int, *, total_mass: float = 1.0):
    """One Plummer sphere of ``n`` equal-mass bodies (G = a = 1).

    Returns ``(x, v, m)``; centre of mass and centre-of-mass velocity are zero.
    Velocities are for a sphere of mass ``total_mass`` (speeds scale as sqrt(M)).
    """
    if n <= 0:
        return np.zeros((0, 3)), np.zeros((0, 3)), np.zeros(0)
    rng = np.random.default_rng(seed)
    r = _plummer_radii(rng, n)
    x = _isotropic(rng, n) * r[:, None]
    q = _plummer_q(rng, n)
    speed = q * math.sqrt(2.0) * (1.0 + r * r) ** (-0.25) * math.sqrt(total_mass)
    v = _isotropic(rng, n) * speed[:, None]
    m = np.full(n, total_mass / n)
    x -= x.mean(axis=0)
    v -= v.mean(axis=0)
    return np.ascontiguousarray(x), np.ascontiguousarray(v), m


def two_spheres(n: int, seed: int, *, separation: float = 10.0, rel_speed: float = 0.5,
                mass_sigma: float = 0.5):
    """Two Plummer spheres of ``n // 2`` bodies on a head-on course along x.

    Sphere A (first half of the arrays) is centred at (-separation/2, 0, 0) moving
    at +rel_speed/2; sphere B at (+separation/2, 0, 0) moving at -rel_speed/2.
    Masses are exp(sigma * Z), Z ~ N(0, 1), normalised so that they sum to 1;
    positions and velocities are then shifted so the mass-weighted centre of
    mass sits at rest at the origin.
    """
    if n % 2:
        raise ValueError("two_spheres needs an even body count")
    h = n // 2
    ss = np.random.SeedSequence(seed)
    sa, sb, sm = ss.spawn(3)
    xa, va, _ = plummer(h, int(sa.generate_state(1)[0]), total_mass=0.5)
    xb, vb, _ = plummer(h, int(sb.generate_state(1)[0]), total_mass=0.5)
    xa[:, 0] -= separation / 2
    xb[:, 0] += separation / 2
    va[:, 0] += rel_speed / 2
    vb[:, 0] -= rel_speed / 2
    x = np.concatenate([xa, xb])
    v = np.concatenate([va, vb])
    rng = np.random.default_rng(sm)
    m = np.exp(mass_sigma * rng.standard_normal(n))
    m /= m.sum()
    x -= (m[:, None] * x).sum(axis=0) / m.sum()
    v -= (m[:, None] * v).sum(axis=0) / m.sum()
    return np.ascontiguousarray(x), np.ascontiguousarray(v), m


@dataclass
class Ensemble:
    """Concatenated independent systems; system s owns rows offsets[s]:offsets[s+1]."""
    x: np.ndarray
    v: np.ndarray
    m: np.ndarray
    offsets: np.ndarray  # int64, length n_systems + 1, offsets[0] = 0

    @property
    def n_systems(self) -> int:
        return len(self.offsets) - 1

    def sizes(self) -> np.ndarray:
        return np.diff(self.offsets)


def ensemble_sizes(n_systems: int, seed: int, n_min: int = 64, n_max: int = 16384) -> np.ndarray:
    """Sizes N_s = round(exp(U(ln n_min, ln n_max))), clipped to [n_min, n_max]."""
    rng = np.random.default_rng(seed)
    u = rng.uniform(math.log(n_min), math.log(n_max), n_systems)
    return np.clip(np.rint(np.exp(u)).astype(np.int64), n_min, n_max)


def ensemble(n_systems: int, seed: int, n_min: int = 64, n_max: int = 16384,
             sizes: np.ndarray | None = None) -> Ensemble:
    """Independent Plummer spheres (each of total mass 1) with log-uniform sizes."""
    if sizes is None:
        sizes = ensemble_sizes(n_systems, seed, n_min, n_max)
    sizes = np.asarray(sizes, dtype=np.int64)
    child = np.random.SeedSequence(seed).spawn(len(sizes))
    xs, vs, ms = [], [], []
    for s, n in enumerate(sizes):
        x, v, m = plummer(int(n), int(child[s].generate_state(1)[0]))
        xs.append(x), vs.append(v), ms.append(m)
    offsets = np.zeros(len(sizes) + 1, dtype=np.int64)
    offsets[1:] = np.cumsum(sizes)
    cat = (lambda a, shape: np.ascontiguousarray(np.concatenate(a)) if a else np.zeros(shape))
    return Ensemble(cat(xs, (0, 3)), cat(vs, (0, 3)), cat(ms, (0,)), offsets)


def kepler_pair(m1: float = 0.5, m2: float = 0.5, a: float = 1.0, e: float = 0.0, G: float = 1.0):
    """Two bodies at pericentre of a Kepler orbit (semi-major axis a, eccentricity e).

    The centre of mass is at rest at the origin; the orbit lies in the x-y plane
    with pericentre along +x for body 2. Returns ``(x, v, m, period)``.
    """
    M = m1 + m2
    rp = a * (1.0 - e)
    vp = math.sqrt(G * M * (1.0 + e) / (a * (1.0 - e)))  # relative speed at pericentre
    rel_x = np.array([rp, 0.0, 0.0])
    rel_v = np.array([0.0, vp, 0.0])
    x = np.stack([-m2 / M * rel_x, m1 / M * rel_x])
    v = np.stack([-m2 / M * rel_v, m1 / M * rel_v])
    period = 2.0 * math.pi * math.sqrt(a ** 3 / (G * M))
    return np.ascontiguousarray(x), np.ascontiguousarray(v), np.array([m1, m2]), period


def sample_indices(n: int, k: int, seed: int) -> np.ndarray:
    """``k`` distinct body indices drawn uniformly without replacement (sorted)."""
    rng = np.random.default_rng(seed)
    k = min(k, n)
    return np.sort(rng.choice(n, size=k, replace=False)).astype(np.int64)


def targets(n: int, seed: int) -> np.ndarray:
    """Per-body target points t_i ~ N(0, 1)^3 for the final-position loss."""
    rng = np.random.default_rng(seed)
    return np.ascontiguousarray(rng.standard_normal((n, 3)))


def lj_gas(n: int, seed: int, *, density: float = 0.05, temperature: float = 2.0, mass: float = 1.0,
           jitter: float = 0.1):
    """A Lennard-Jones gas in reduced units (sigma = epsilon = k_B = 1) in the cube [0, box]^3.

    box = (n / density)^{1/3}. Bodies start on the first n sites of a simple
    cubic lattice of spacing box / ceil(n^{1/3}) (offset by half a spacing,
    each displaced uniformly by up to +-jitter spacings), with Maxwell
    velocities at the given temperature, the centre-of-mass velocity removed.
    Returns ``(x, v, m, box)``.
    """
    rng = np.random.default_rng(seed)
    box = (n / density) ** (1.0 / 3.0)
    k = int(math.ceil(n ** (1.0 / 3.0) - 1e-9))
    h = box / k
    g = np.arange(k)
    lat = np.stack(np.meshgrid(g, g, g, indexing="ij"), axis=-1).reshape(-1, 3)[:n].astype(np.float64)
    x = (lat + 0.5 + rng.uniform(-jitter, jitter, (n, 3))) * h
    v = rng.standard_normal((n, 3)) * math.sqrt(temperature / mass)
    v -= v.mean(axis=0)
    m = np.full(n, mass)
    return np.ascontiguousarray(x), np.ascontiguousarray(v), m, box
