"""Seeded synthetic inputs for the direct-summation gravity pass.

This module is shared by the tests, the benchmark and the CPU oracle.  It only
draws particle sets; it contains none of the force, predictor or reduction
arithmetic of the method.  Every generator is deterministic in its seed.

Workloads (the paper measures only on synthetic star clusters, Sec. 3.2 and
Sec. 3.7, and the planetary/few-body systems motivate the small-N regime of
Sec. 2.1):

* ``plummer``            Plummer sphere in Henon units (G = M = 1, E = -1/4),
                         sampled with the Aarseth-Henon-Wielen (1974) recipe.
* ``salpeter_masses``    power-law mass function dN/dm ~ m^-2.35 on [0.1, 100].
* ``planetary_systems``  many independent star + planets systems, Kepler
                         elements converted to Cartesian coordinates.
* ``block_times``        per-particle last-update times t_j = t - k_j 2^-10.
* ``active_set``         active i-particle slots of one block step.
* ``derivative_noise``   seeded stand-in a, jerk, snap vectors.
"""
from __future__ import annotations

import math

import numpy as np

__all__ = [
    "plummer",
    "salpeter_masses",
    "planetary_systems",
    "block_times",
    "active_set",
    "derivative_noise",
    "particle_ids",
]


def _isotropic(rng: np.random.Generator, n: int) -> np.ndarray:
    """Unit vectors uniform on the sphere, shape (n, 3)."""
    cos_t = rng.uniform(-1.0, 1.0, n)
    phi = rng.uniform(0.0, 2.0 * math.pi, n)
    sin_t = np.sqrt(1.0 - cos_t * cos_t)
    return np.stack([sin_t * np.cos(phi), sin_t * np.sin(phi), cos_t], axis=1)


def plummer(n: int, seed: int, *, m_cut: float = 0.999):
    """Equal-mass Plummer sphere in Henon units.

    Aarseth, Henon & Wielen (1974): the radius comes from the cumulative mass
    fraction X ~ U(0, m_cut) as r = (X^-2/3 - 1)^-1/2 (Plummer scale length 1);
    the speed in units of the local escape speed, q, is drawn by von Neumann
    rejection from g(q) = q^2 (1 - q^2)^(7/2); directions are isotropic.  The
    model is then scaled from Plummer units to Henon units (positions by
    3 pi / 16, velocities by (16 / 3 pi)^(1/2)), and the centre of mass is moved
    to rest at the origin.

    Returns (m, x, v): m has shape (n,) and sums to 1, x and v have shape (n, 3).
    """
    if n <= 0:
        raise ValueError("n must be positive")
    rng = np.random.default_rng(seed)
    X = rng.uniform(0.0, m_cut, n)
    X = np.maximum(X, 1e-300)
    r = 1.0 / np.sqrt(X ** (-2.0 / 3.0) - 1.0)
    x = r[:, None] * _isotropic(rng, n)

    q = np.empty(n)
    todo = np.arange(n)
    gmax = 0.1  # max of q^2 (1-q^2)^3.5 is ~0.092
    while todo.size:
        qq = rng.uniform(0.0, 1.0, todo.size)
        yy = rng.uniform(0.0, gmax, todo.size)
        ok = yy < qq * qq * (1.0 - qq * qq) ** 3.5
        q[todo[ok]] = qq[ok]
        todo = todo[~ok]
    v_esc = math.sqrt(2.0) * (1.0 + r * r) ** (-0.25)
    v = (q * v_esc)[:, None] * _isotropic(rng, n)

    x *= 3.0 * math.pi / 16.0
    v *= math.sqrt(16.0 / (3.0 * math.pi))
    m = np.full(n, 1.0 / n)
    x -= (m[:, None] * x).sum(axis=0) / m.sum()
    v -= (m[:, None] * v).sum(axis=0) / m.sum()
    return m, np.ascontiguousarray(x), np.ascontiguousarray(v)


def salpeter_masses(n: int, seed: int, *, slope: float = 2.35,
                    m_lo: float = 0.1, m_hi: float = 100.0) -> np.ndarray:
    """Masses with dN/dm ~ m^-slope on [m_lo, m_hi] by inverse CDF, sum 1."""
    rng = np.random.default_rng(seed)
    u = rng.uniform(0.0, 1.0, n)
    p = 1.0 - slope
    lo, hi = m_lo ** p, m_hi ** p
    m = (lo + u * (hi - lo)) ** (1.0 / p)
    return m / m.sum()


def _solve_kepler(M: np.ndarray, e: np.ndarray) -> np.ndarray:
    """Eccentric anomaly E from the mean anomaly: E - e sin E = M (Newton)."""
    E = np.where(e < 0.8, M, np.full_like(M, math.pi))
    for _ in range(60):
        f = E - e * np.sin(E) - M
        E = E - f / (1.0 - e * np.cos(E))
    return E


def kepler_to_cartesian(mu, a, e, inc, node, peri, M):
    """Position and velocity of a Kepler orbit (vectorised over bodies)."""
    E = _solve_kepler(np.mod(M, 2.0 * math.pi), e)
    cE, sE = np.cos(E), np.sin(E)
    b = a * np.sqrt(1.0 - e * e)
    px, py = a * (cE - e), b * sE
    n_mean = np.sqrt(mu / a ** 3)
    Edot = n_mean / (1.0 - e * cE)
    vx, vy = -a * sE * Edot, b * cE * Edot
    cO, sO = np.cos(node), np.sin(node)
    cw, sw = np.cos(peri), np.sin(peri)
    ci, si = np.cos(inc), np.sin(inc)
    # rotation perifocal -> reference frame, R = Rz(node) Rx(inc) Rz(peri)
    r11 = cO * cw - sO * sw * ci
    r12 = -cO * sw - sO * cw * ci
    r21 = sO * cw + cO * sw * ci
    r22 = -sO * sw + cO * cw * ci
    r31 = sw * si
    r32 = cw * si
    pos = np.stack([r11 * px + r12 * py, r21 * px + r22 * py, r31 * px + r32 * py], axis=1)
    vel = np.stack([r11 * vx + r12 * vy, r21 * vx + r22 * vy, r31 * vx + r32 * vy], axis=1)
    return pos, vel


def planetary_systems(n_sys: int, seed: int, *, n_lo: int = 3, n_hi: int = 256):
    """Independent star + planets systems, concatenated.

    Each system has N = round(exp U(ln n_lo, ln n_hi)) bodies: a central mass 1
    at rest at the origin and N - 1 bodies with mass log-uniform in
    [1e-7, 1e-3], semi-major axis log-uniform in [0.5, 50], eccentricity
    Rayleigh(0.05) clipped below 0.99, inclination Rayleigh(0.02), and node,
    argument of pericentre and mean anomaly uniform in [0, 2 pi).  Each orbit is
    converted with mu = 1 + m.

    Returns (offsets, m, x, v): offsets has n_sys + 1 int64 entries and system s
    owns rows offsets[s]:offsets[s+1] of the concatenated arrays.
    """
    rng = np.random.default_rng(seed)
    sizes = np.rint(np.exp(rng.uniform(math.log(n_lo), math.log(n_hi), n_sys))).astype(np.int64)
    sizes = np.clip(sizes, n_lo, n_hi)
    offsets = np.zeros(n_sys + 1, dtype=np.int64)
    offsets[1:] = np.cumsum(sizes)
    total = int(offsets[-1])
    m = np.empty(total)
    x = np.zeros((total, 3))
    v = np.zeros((total, 3))
    n_pl = int((sizes - 1).sum())
    mp = np.exp(rng.uniform(math.log(1e-7), math.log(1e-3), n_pl))
    ap = np.exp(rng.uniform(math.log(0.5), math.log(50.0), n_pl))
    ep = np.minimum(rng.rayleigh(0.05, n_pl), 0.98999)
    ip = rng.rayleigh(0.02, n_pl)
    node = rng.uniform(0.0, 2.0 * math.pi, n_pl)
    peri = rng.uniform(0.0, 2.0 * math.pi, n_pl)
    M = rng.uniform(0.0, 2.0 * math.pi, n_pl)
    pos, vel = kepler_to_cartesian(1.0 + mp, ap, ep, ip, node, peri, M)
    star = offsets[:-1]
    planet_rows = np.setdiff1d(np.arange(total), star, assume_unique=True)
    m[star] = 1.0
    m[planet_rows] = mp
    x[planet_rows] = pos
    v[planet_rows] = vel
    return offsets, m, x, v


def block_times(n: int, seed: int, t: float, *, quantum: float = 2.0 ** -10, k_max: int = 63):
    """Last-update times t_j = t - k_j * quantum with k_j uniform in {0..k_max}."""
    rng = np.random.default_rng(seed)
    k = rng.integers(0, k_max + 1, n)
    return t - k.astype(np.float64) * quantum


def active_set(n: int, n_active: int, seed: int) -> np.ndarray:
    """n_active distinct slots drawn uniformly without replacement (int32, sorted)."""
    if not 0 <= n_active <= n:
        raise ValueError("need 0 <= n_active <= n")
    rng = np.random.default_rng(seed)
    if n_active == n:
        return np.arange(n, dtype=np.int32)
    return np.sort(rng.choice(n, size=n_active, replace=False)).astype(np.int32)


def derivative_noise(n: int, seed: int, *, scales=(1.0, 1.0, 1.0)):
    """Seeded isotropic-Gaussian a, jerk, snap vectors, each of shape (n, 3).

    Used where a workload needs time derivatives for the predictor but no force
    pass may produce them; the predictor's cost does not depend on their values.
    """
    rng = np.random.default_rng(seed)
    return tuple(s * rng.standard_normal((n, 3)) for s in scales)


def particle_ids(n: int, seed: int | None = None) -> np.ndarray:
    """Unique int32 particle ids: 0..n-1, or a seeded permutation of them."""
    ids = np.arange(n, dtype=np.int32)
    if seed is not None:
        ids = np.random.default_rng(seed).permutation(ids).astype(np.int32)
    return ids
