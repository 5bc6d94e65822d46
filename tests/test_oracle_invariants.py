"""Pins: conservation laws, symmetries and special cases of the oracle."""
import numpy as np
import pytest

import workloads as W

scipy_spatial = pytest.importorskip("scipy.spatial")


def _plummer_with_derivs(n, seed):
    m, x, v = W.plummer(n, seed)
    a, j, s = W.derivative_noise(n, seed + 1000)
    return m, x, v, a, j, s


def test_newton_third_law(oracle_mod):
    """All active: sum m_i acc_i = sum m_i jerk_i = sum m_i snap_i = 0."""
    n = 512
    m, x, v, a, _, _ = _plummer_with_derivs(n, 0)
    m = W.salpeter_masses(n, 5)
    ids = W.particle_ids(n, 3)
    f = oracle_mod.forces(ids, x, v, ids, m, x, v, 1e-6, 6, ai=a, aj=a)
    for key, sc in (("acc", "sc_acc"), ("jerk", "sc_jerk"), ("snap", "sc_snap")):
        tot = (m[:, None] * f[key]).sum(0)
        assert np.linalg.norm(tot) <= 1e-14 * (m * f[sc]).sum(), key


def test_potential_pair_sum(oracle_mod):
    """(1/2) sum_i m_i pot_i equals the pair sum W = -sum_{i<j} m_i m_j / sqrt(r^2 + eps^2)."""
    n = 700
    m, x, v = W.plummer(n, 1)
    eps2 = 1e-4
    ids = W.particle_ids(n)
    f = oracle_mod.forces(ids, x, v, ids, m, x, v, eps2, 4)
    d = scipy_spatial.distance.pdist(x)
    mm = np.outer(m, m)[np.triu_indices(n, 1)]
    Wpair = -np.sum(mm / np.sqrt(d * d + eps2))
    assert abs(0.5 * np.sum(m * f["pot"]) - Wpair) <= 1e-13 * abs(Wpair)


def test_plummer_energy_statistics(oracle_mod):
    """Henon units: W ~ -1/2, kinetic ~ 1/4 (statistical, N = 4096)."""
    n = 4096
    m, x, v = W.plummer(n, 2)
    ids = W.particle_ids(n)
    f = oracle_mod.forces(ids, x, v, ids, m, x, v, 0.0, 4)
    Wpot = 0.5 * np.sum(m * f["pot"])
    K = 0.5 * np.sum(m * np.sum(v * v, 1))
    assert abs(Wpot + 0.5) < 0.05 and abs(K - 0.25) < 0.03
    assert np.allclose((m[:, None] * x).sum(0), 0, atol=1e-15)


def test_permutation_of_sources(oracle_mod):
    n = 300
    m, x, v, a, _, _ = _plummer_with_derivs(n, 3)
    ids = W.particle_ids(n, 9)
    f = oracle_mod.forces(ids, x, v, ids, m, x, v, 1e-6, 6, ai=a, aj=a)
    p = np.random.default_rng(4).permutation(n)
    g = oracle_mod.forces(ids, x, v, ids[p], m[p], x[p], v[p], 1e-6, 6, ai=a, aj=a[p])
    for key, sc in (("acc", "sc_acc"), ("jerk", "sc_jerk"), ("snap", "sc_snap")):
        err = np.linalg.norm(f[key] - g[key], axis=1) / f[sc]
        assert err.max() <= 1e-14, key
    assert np.array_equal(f["nn_id"], g["nn_id"])
    assert np.allclose(f["pot"], g["pot"], rtol=1e-14, atol=0)


def test_translation(oracle_mod):
    n = 256
    m, x, v, a, _, _ = _plummer_with_derivs(n, 5)
    ids = W.particle_ids(n)
    f = oracle_mod.forces(ids, x, v, ids, m, x, v, 1e-4, 6, ai=a, aj=a)
    c = np.array([0.3, -0.7, 1.1])
    g = oracle_mod.forces(ids, x + c, v + 2 * c, ids, m, x + c, v + 2 * c, 1e-4, 6, ai=a - c, aj=a - c)
    for key, sc in (("acc", "sc_acc"), ("jerk", "sc_jerk"), ("snap", "sc_snap")):
        assert (np.linalg.norm(f[key] - g[key], axis=1) / f[sc]).max() <= 1e-12, key


def test_scaling_by_two_is_exact(oracle_mod):
    """x, v, a, eps -> 2x, 2v, 2a, 2eps: acc, jerk, snap -> /4, pot -> /2, nn_r2 -> *4, exactly."""
    n = 200
    m, x, v, a, _, _ = _plummer_with_derivs(n, 6)
    ids = W.particle_ids(n)
    eps2 = 1e-3
    f = oracle_mod.forces(ids, x, v, ids, m, x, v, eps2, 6, ai=a, aj=a)
    g = oracle_mod.forces(ids, 2 * x, 2 * v, ids, m, 2 * x, 2 * v, 4 * eps2, 6, ai=2 * a, aj=2 * a)
    assert np.array_equal(g["acc"] * 4, f["acc"])
    assert np.array_equal(g["jerk"] * 4, f["jerk"])
    assert np.array_equal(g["snap"] * 4, f["snap"])
    assert np.array_equal(g["pot"] * 2, f["pot"])
    assert np.array_equal(g["nn_r2"], 4 * f["nn_r2"])
    assert np.array_equal(g["nn_id"], f["nn_id"])


def test_single_source_textbook(oracle_mod):
    rng = np.random.default_rng(7)
    for _ in range(20):
        r = rng.uniform(-2, 2, 3)
        mj = rng.uniform(0.1, 2)
        eps2 = rng.uniform(0, 0.1)
        xs = np.array([[0.0, 0, 0], r])
        f = oracle_mod.forces(np.array([0], np.int32), xs[:1], np.zeros((1, 3)),
                              np.array([0, 1], np.int32), np.array([5.0, mj]), xs, np.zeros((2, 3)),
                              eps2, 4)
        d2 = r @ r + eps2
        assert np.allclose(f["acc"][0], mj * r / d2 ** 1.5, rtol=1e-15, atol=0)
        assert np.isclose(f["pot"][0], -mj / np.sqrt(d2), rtol=1e-15, atol=0)
        assert np.allclose(f["jerk"][0], 0, atol=0)


def test_nearest_neighbour_matches_library_argmin(oracle_mod):
    n = 1000
    m, x, v = W.plummer(n, 8)
    ids = W.particle_ids(n)
    f = oracle_mod.forces(ids, x, v, ids, m, x, v, 1e-4, 4)
    d = scipy_spatial.distance.cdist(x, x, "sqeuclidean")
    np.fill_diagonal(d, np.inf)
    assert np.array_equal(f["nn_id"], ids[np.argmin(d, axis=1)])
    assert np.allclose(f["nn_r2"], d.min(1), rtol=1e-14, atol=0)


def test_multi_rank_j_split_combines_to_full_sum(oracle_mod):
    """Splitting the sources into R shards (round-robin, as a j-distributed run
    would) and combining the partial sums (add) and nearest neighbours
    (lexicographic min of (r2, id)) reproduces the full sum."""
    n = 400
    m, x, v, a, _, _ = _plummer_with_derivs(n, 9)
    ids = W.particle_ids(n, 2)
    full = oracle_mod.forces(ids, x, v, ids, m, x, v, 1e-5, 6, ai=a, aj=a)
    R = 3
    parts = [oracle_mod.forces(ids, x, v, ids[r::R], m[r::R], x[r::R], v[r::R], 1e-5, 6,
                               ai=a, aj=a[r::R]) for r in range(R)]
    for key, sc in (("acc", "sc_acc"), ("jerk", "sc_jerk"), ("snap", "sc_snap")):
        tot = sum(p[key] for p in parts)
        assert (np.linalg.norm(tot - full[key], axis=1) / full[sc]).max() <= 1e-14
    assert np.allclose(sum(p["pot"] for p in parts), full["pot"], rtol=1e-14, atol=0)
    r2 = np.stack([p["nn_r2"] for p in parts])
    idn = np.stack([p["nn_id"] for p in parts])
    key = np.lexsort((idn, r2), axis=0)[0]
    assert np.array_equal(idn[key, np.arange(n)], full["nn_id"])
