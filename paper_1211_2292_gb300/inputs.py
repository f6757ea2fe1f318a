"""Seeded synthetic initial conditions for the n-body force path.

This module is shared by the tests, the benchmark and the CUDA path's users.
It holds none of the force, integrator or energy arithmetic: it only draws
initial conditions, so that the CPU oracle and the GPU library can be fed
identical inputs without sharing any of the method's code.

The paper (Sec. IV and Sec. V-C) simulates 10^5 bodies under mutual
gravitation but never states its initial conditions.  The workloads here use
Plummer spheres instead, drawn with the published rejection method of Aarseth,
Henon and Wielen (1974, A&A 37, 183):

* radius:  r = a / sqrt(X1^(-2/3) - 1), X1 ~ U(0, 1), redrawn while r > 10 a
  (a truncation the workloads fix; M(10a) = 0.985 M);
* speed:   q * v_esc(r), with v_esc = sqrt(2 G M / a) (1 + r^2/a^2)^(-1/4)
  and q drawn from g(q) ~ q^2 (1 - q^2)^(7/2) by rejection under 0.1;
* isotropic directions for both positions and velocities;
* the centre of mass is moved to the origin and brought to rest.

Draw order per sphere (fixed, so a seed is reproducible): all radii (with
their redraws), then the position directions, then the speed rejection loop,
then the velocity directions, then the masses.  Every array is float64,
positions and velocities shaped (n, 3), masses (n,).
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

R_TRUNC = 10.0  # truncation radius in units of the scale radius a


@dataclass
class Bodies:
    """A system of n bodies: positions (n,3), velocities (n,3), masses (n,)."""

    pos: np.ndarray
    vel: np.ndarray
    mass: np.ndarray

    @property
    def n(self) -> int:
        return int(self.mass.shape[0])


def _radii(rng: np.random.Generator, n: int, a: float) -> np.ndarray:
    r = np.empty(n)
    todo = np.arange(n)
    while todo.size:
        x1 = rng.random(todo.size)
        with np.errstate(divide="ignore"):
            rr = a / np.sqrt(x1 ** (-2.0 / 3.0) - 1.0)
        ok = np.isfinite(rr) & (rr <= R_TRUNC * a)
        r[todo[ok]] = rr[ok]
        todo = todo[~ok]
    return r


def _directions(rng: np.random.Generator, n: int) -> np.ndarray:
    cz = rng.uniform(-1.0, 1.0, n)
    phi = rng.uniform(0.0, 2.0 * math.pi, n)
    sz = np.sqrt(np.maximum(0.0, 1.0 - cz * cz))
    return np.stack([sz * np.cos(phi), sz * np.sin(phi), cz], axis=1)


def _speed_fractions(rng: np.random.Generator, n: int) -> np.ndarray:
    q = np.empty(n)
    todo = np.arange(n)
    while todo.size:
        x4 = rng.random(todo.size)
        x5 = rng.random(todo.size)
        ok = 0.1 * x5 < x4 * x4 * (1.0 - x4 * x4) ** 3.5
        q[todo[ok]] = x4[ok]
        todo = todo[~ok]
    return q


def _unit_plummer(rng: np.random.Generator, n: int):
    """Positions and velocities of a Plummer sphere with G = M = a = 1."""
    r = _radii(rng, n, 1.0)
    pos = r[:, None] * _directions(rng, n)
    q = _speed_fractions(rng, n)
    vesc = math.sqrt(2.0) * (1.0 + r * r) ** -0.25
    vel = (q * vesc)[:, None] * _directions(rng, n)
    return pos, vel


def _recentre(pos, vel, mass):
    mt = mass.sum()
    pos = pos - (mass[:, None] * pos).sum(0) / mt
    vel = vel - (mass[:, None] * vel).sum(0) / mt
    return pos, vel


def plummer(n: int, seed: int = 0, a: float = 1.0, total_mass: float = 1.0,
            G: float = 1.0, rng: np.random.Generator | None = None) -> Bodies:
    """Equal-mass Plummer sphere (m = M/n) with scale radius a."""
    if rng is None:
        rng = np.random.default_rng(seed)
    if n == 0:
        z = np.zeros((0, 3))
        return Bodies(z, z.copy(), np.zeros(0))
    pos, vel = _unit_plummer(rng, n)
    mass = np.full(n, total_mass / n)
    pos = pos * a
    vel = vel * math.sqrt(G * total_mass / a)
    pos, vel = _recentre(pos, vel, mass)
    return Bodies(np.ascontiguousarray(pos), np.ascontiguousarray(vel), mass)


def two_plummer(n_per: int = 524_288, seed: int = 2, sep: float = 10.0,
                v_rel: float = 0.5, sigma: float = 0.5, a: float = 1.0,
                G: float = 1.0) -> Bodies:
    """Two Plummer spheres on a head-on approach (the 2^20-body workload).

    Sphere A holds the first n_per bodies, centred at (-sep/2, 0, 0); sphere B
    the rest, at (+sep/2, 0, 0).  Masses are lognormal(0, sigma), normalised
    to a total of 1 over both spheres.  Each sphere's velocities follow a
    Plummer model of its own mass; the bulk velocities along x are
    +v_rel*M_B/M and -v_rel*M_A/M, so the pair approaches at v_rel with the
    centre of mass at rest.  Draw order: sphere A's radii, directions and
    speeds, then sphere B's, then all masses.
    """
    rng = np.random.default_rng(seed)
    pa, va = _unit_plummer(rng, n_per)
    pb, vb = _unit_plummer(rng, n_per)
    mass = rng.lognormal(0.0, sigma, 2 * n_per)
    mass /= mass.sum()
    ma, mb = mass[:n_per], mass[n_per:]
    MA, MB = ma.sum(), mb.sum()
    pa, va = _recentre(pa * a, va * math.sqrt(G * MA / a), ma)
    pb, vb = _recentre(pb * a, vb * math.sqrt(G * MB / a), mb)
    M = MA + MB
    pa[:, 0] -= 0.5 * sep
    pb[:, 0] += 0.5 * sep
    va[:, 0] += v_rel * MB / M
    vb[:, 0] -= v_rel * MA / M
    pos = np.ascontiguousarray(np.concatenate([pa, pb]))
    vel = np.ascontiguousarray(np.concatenate([va, vb]))
    return Bodies(pos, vel, mass)


def batch_sizes(nsys: int = 512, lo: int = 64, hi: int = 8192,
                rng: np.random.Generator | None = None, seed: int = 3) -> np.ndarray:
    """System sizes drawn log-uniformly from [lo, hi], rounded to integers."""
    if rng is None:
        rng = np.random.default_rng(seed)
    u = rng.uniform(math.log(lo), math.log(hi), nsys)
    return np.clip(np.rint(np.exp(u)), lo, hi).astype(np.int64)


def plummer_batch(nsys: int = 512, lo: int = 64, hi: int = 8192, seed: int = 3,
                  sizes: np.ndarray | None = None):
    """Independent Plummer systems (M = 1, a = 1, equal masses).

    Returns (Bodies of all systems concatenated, offsets[nsys + 1]).  The
    sizes are drawn first, then each system in order from the same stream.
    """
    rng = np.random.default_rng(seed)
    if sizes is None:
        sizes = batch_sizes(nsys, lo, hi, rng=rng)
    sizes = np.asarray(sizes, dtype=np.int64)
    offsets = np.zeros(sizes.size + 1, dtype=np.int64)
    offsets[1:] = np.cumsum(sizes)
    parts = [plummer(int(k), rng=rng) for k in sizes]
    if parts:
        pos = np.concatenate([p.pos for p in parts])
        vel = np.concatenate([p.vel for p in parts])
        mass = np.concatenate([p.mass for p in parts])
    else:
        pos = np.zeros((0, 3)); vel = np.zeros((0, 3)); mass = np.zeros(0)
    return Bodies(np.ascontiguousarray(pos), np.ascontiguousarray(vel), mass), offsets


def perturbation(rng: np.random.Generator, n: int, sigma: float = 1e-3) -> np.ndarray:
    """Gaussian position offsets N(0, sigma^2 I3), shaped (n, 3)."""
    return rng.normal(0.0, sigma, (n, 3))


def plummer_with_perturbation(n: int = 16_384, seed: int = 4, sigma: float = 1e-3):
    """Plummer sphere plus position offsets drawn after it from the same stream.

    Used by the differentiation workload: the target snapshot is a run from
    pos + offsets.  Returns (Bodies, offsets).
    """
    rng = np.random.default_rng(seed)
    b = plummer(n, rng=rng)
    return b, perturbation(rng, n, sigma)


def sample_rows(n: int, k: int = 4096, seed: int = 1) -> np.ndarray:
    """Indices of k distinct bodies (sorted) at which forces are checked."""
    rng = np.random.default_rng(seed)
    k = min(k, n)
    return np.sort(rng.choice(n, k, replace=False)).astype(np.int64)


def random_system(n: int, seed: int, spread: float = 1.0, mass_lo: float = 0.5,
                  mass_hi: float = 1.5) -> Bodies:
    """Uniform-in-a-cube system with uniform masses (small parity cases)."""
    rng = np.random.default_rng(seed)
    pos = rng.uniform(-spread, spread, (n, 3))
    vel = rng.uniform(-0.1, 0.1, (n, 3))
    mass = rng.uniform(mass_lo, mass_hi, n) / max(n, 1)
    return Bodies(pos, vel, mass)
