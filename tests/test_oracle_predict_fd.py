"""Pins: the Taylor predictor, and jerk / snap against finite differences of the
oracle's own acceleration / jerk along the predicted motion."""
import numpy as np
import pytest

import workloads as W


@pytest.mark.parametrize("order", [4, 6])
def test_predictor_is_exact_on_polynomial_motion(oracle_mod, order):
    """Motion that is a polynomial of degree order-1 in t is predicted exactly
    (up to rounding) from its derivatives at t_j; compared with numpy.polyval."""
    rng = np.random.default_rng(0)
    n = 500
    deg = 3 if order == 4 else 4
    coef = rng.uniform(-1, 1, (n, 3, deg + 1))  # highest power first
    tj = W.block_times(n, 1, 0.25)
    t = 0.25

    def deriv(c, k):
        for _ in range(k):
            c = np.polyder(c)
        return c

    ev = lambda k, tt: np.array([[np.polyval(deriv(coef[i, d], k), tt[i]) for d in range(3)]  # noqa: E731
                                 for i in range(n)])
    x, v, a, jk = (ev(k, tj) for k in range(4))
    sn = ev(4, tj) if order == 6 else None
    xp, vp, ap = oracle_mod.predict(t, tj, x, v, a, jk, sn, order)
    tt = np.full(n, t)
    assert np.allclose(xp, ev(0, tt), rtol=0, atol=1e-14)
    assert np.allclose(vp, ev(1, tt), rtol=0, atol=1e-14)
    if order == 6:
        assert np.allclose(ap, ev(2, tt), rtol=0, atol=1e-14)
    # zero step is the identity, bit for bit
    xp0, vp0, ap0 = oracle_mod.predict(0.25, np.full(n, 0.25), x, v, a, jk, sn, order)
    assert np.array_equal(xp0, x) and np.array_equal(vp0, v)
    if order == 6:
        assert np.array_equal(ap0, a)


def _fd_setup(n=256, seed=4):
    m, x, v = W.plummer(n, seed)
    a, jk, sn = W.derivative_noise(n, seed + 1, scales=(1.0, 2.0, 4.0))
    return m, x, v, a, jk, sn, W.particle_ids(n)


def test_jerk_is_time_derivative_of_acc(oracle_mod):
    m, x, v, a, jk, sn, ids = _fd_setup()
    eps2 = 1e-2
    n = len(m)
    f0 = oracle_mod.forces(ids, x, v, ids, m, x, v, eps2, 4)

    def acc_at(h):
        xp, vp, _ = oracle_mod.predict(h, np.zeros(n), x, v, a, jk, None, 4)
        return oracle_mod.forces(ids, xp, vp, ids, m, xp, vp, eps2, 4)["acc"]

    errs = []
    for h in (1e-3, 5e-4):
        fd = (acc_at(h) - acc_at(-h)) / (2 * h)
        errs.append((np.linalg.norm(fd - f0["jerk"], axis=1) / f0["sc_jerk"]).max())
    assert errs[0] < 1e-4
    ratio = errs[0] / errs[1]
    assert 3.2 < ratio < 4.8, (errs, ratio)  # second-order convergence


def test_snap_is_time_derivative_of_jerk(oracle_mod):
    m, x, v, a, jk, sn, ids = _fd_setup(seed=9)
    eps2 = 1e-2
    n = len(m)
    f0 = oracle_mod.forces(ids, x, v, ids, m, x, v, eps2, 6, ai=a, aj=a)

    def jerk_at(h):
        xp, vp, ap = oracle_mod.predict(h, np.zeros(n), x, v, a, jk, sn, 6)
        return oracle_mod.forces(ids, xp, vp, ids, m, xp, vp, eps2, 6, ai=ap, aj=ap)["jerk"]

    errs = []
    for h in (1e-3, 5e-4):
        fd = (jerk_at(h) - jerk_at(-h)) / (2 * h)
        errs.append((np.linalg.norm(fd - f0["snap"], axis=1) / f0["sc_snap"]).max())
    assert errs[0] < 1e-3
    ratio = errs[0] / errs[1]
    assert 3.2 < ratio < 4.8, (errs, ratio)


def test_step_gathers_sinks_from_predicted_sources(oracle_mod):
    """step() = predict all, then sum on the chosen slots (explicit form agrees)."""
    n = 300
    m, x, v, a, jk, sn, ids = _fd_setup(n, 12)
    tj = W.block_times(n, 3, 1.0)
    idx = W.active_set(n, 40, 5)
    f = oracle_mod.step(1.0, idx, ids, m, tj, x, v, a, jk, sn, eps2=1e-4, order=6)
    xp, vp, ap = oracle_mod.predict(1.0, tj, x, v, a, jk, sn, 6)
    g = oracle_mod.forces(ids[idx], xp[idx], vp[idx], ids, m, xp, vp, 1e-4, 6, ai=ap[idx], aj=ap)
    for k in f:
        assert np.array_equal(f[k], g[k]), k
