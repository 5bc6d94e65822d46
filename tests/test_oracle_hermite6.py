"""Pins of the oracle's 6th-order Hermite integrators (Sec. 3.7 runs the
6th-order block scheme of Nitadori & Makino 2008 with an averaged time-step
criterion).

The interpolation formulas are checked on an acceleration that is exactly a
quintic in time, where the scheme is exact; the full scheme converges at
6th order on a closed Kepler orbit (5th order if the crackle term of the
predictor were dropped, 4th for the Hermite-4 scheme); the block integrator
reduces to the shared-step one bit for bit when every particle takes dt_max,
keeps its steps commensurate powers of two, and conserves energy far better
than the 4th-order block scheme at a similar number of blocks."""
import math

import numpy as np

import workloads as W


def _quintic(rng):
    """a(t) = sum_k c_k t^k / k!, k = 0..5, per component; returns the
    function giving (a, j, s, crackle, pop, 5th derivative) and the exact
    integral from 0 to t."""
    cf = rng.standard_normal((6, 3))

    def derivs(t):
        out = []
        for d in range(6):
            out.append(sum(cf[k] * t ** (k - d) / math.factorial(k - d) for k in range(d, 6)))
        return out

    def integral(t):
        return sum(cf[k] * t ** (k + 1) / math.factorial(k + 1) for k in range(6))

    return derivs, integral


def test_corrector_and_interpolation_exact_on_a_quintic(oracle_mod):
    rng = np.random.default_rng(3)
    derivs, integral = _quintic(rng)
    h = 0.37
    a0, j0, s0, _, _, _ = derivs(0.0)
    a1, j1, s1, c1, p1, q1 = derivs(h)
    v0 = rng.standard_normal(3)
    x0 = rng.standard_normal(3)
    hh = np.array([[h]])
    x1, v1, cc, pp, qq = oracle_mod._h6_correct(hh, x0[None], v0[None], a0[None], j0[None], s0[None],
                                                a1[None], j1[None], s1[None])
    # v' = a exactly a quintic: the two-point quadrature integrates it exactly
    assert np.allclose(v1[0], v0 + integral(h), rtol=0, atol=1e-13)
    # the interpolant is the quintic itself: its end derivatives are exact
    for got, want in ((cc[0], c1), (pp[0], p1), (qq[0], q1)):
        assert np.allclose(got, want, rtol=1e-10, atol=1e-10 * np.abs(want).max())


def _kepler_pair():
    m1, m2, a, e = 0.75, 0.25, 1.0, 0.5
    mu = m1 + m2
    r, vr = W.kepler_to_cartesian(mu, np.array([a]), np.array([e]), np.array([0.3]), np.array([0.2]),
                                  np.array([0.1]), np.array([0.0]))
    r, vr = r[0], vr[0]
    x = np.array([-m2 / mu * r, m1 / mu * r])
    v = np.array([-m2 / mu * vr, m1 / mu * vr])
    return np.array([m1, m2]), x, v, 2.0 * math.pi * math.sqrt(a ** 3 / mu)


def test_sixth_order_convergence_on_kepler(oracle_mod):
    """One period of an e = 0.5 orbit (eps = 0) returns to the start: the
    error falls 2^6 = 64x per halving of dt."""
    m, x, v, period = _kepler_pair()
    errs = []
    for k in (128, 256):
        xf, _ = oracle_mod.hermite6_shared(m, x, v, 0.0, period / k, k)
        errs.append(np.abs(xf - x).max())
    assert errs[1] < 1e-6
    assert 52.0 < errs[0] / errs[1] < 76.0, errs


def test_block_reduces_to_shared_steps(oracle_mod):
    n, eps2 = 64, 1e-2
    m, x, v = W.plummer(n, 4)
    dt = 2.0 ** -7
    xs, vs = oracle_mod.hermite6_shared(m, x, v, eps2, dt, 8)
    xb, vb, tb, st = oracle_mod.hermite6_block(m, x, v, eps2, 8 * dt, 1e30, 1e30, 1e30, dt)
    assert st["block_steps"] == 8 and st["active_sum"] == 8 * n
    assert np.all(tb == 8 * dt)
    assert np.array_equal(xb, xs) and np.array_equal(vb, vs)


def test_block_steps_and_energy(oracle_mod):
    n, eps2 = 128, 1e-3
    m, x, v = W.plummer(n, 8)
    e0 = oracle_mod.energy(m, x, v, eps2)
    errs = []
    for eta4, eta6 in ((0.04, 0.4), (0.01, 0.1)):
        xb, vb, t, st = oracle_mod.hermite6_block(m, x, v, eps2, 2.0 ** -3, eta4, eta6, 0.01, 2.0 ** -5)
        assert np.all(t == 2.0 ** -3)
        dt = st["dt"]
        assert np.all(np.log2(dt) == np.round(np.log2(dt)))
        assert np.all(np.fmod(t, dt) == 0.0)
        assert len(np.unique(dt)) > 1 and st["active_sum"] > st["block_steps"]
        errs.append(abs(oracle_mod.energy(m, xb, vb, eps2) / e0 - 1.0))
    assert errs[1] < 1e-10
    assert errs[1] < errs[0] / 20
    # the 4th-order block scheme at Aarseth's eta = 0.01 takes a similar number
    # of blocks here and conserves energy far less well
    x4, v4, _, st4 = oracle_mod.hermite4_block(m, x, v, eps2, 2.0 ** -3, 0.01, 0.01, 2.0 ** -5)
    e4 = abs(oracle_mod.energy(m, x4, v4, eps2) / e0 - 1.0)
    assert errs[1] < e4 / 100


def test_criterion_survives_force_noise(oracle_mod, monkeypatch):
    """Force noise of the size of double-single forces (3e-8 of the scale
    sums, added in the oracle on the CPU) costs the 6th-order block scheme
    some extra blocks but does not collapse its steps: the 4th-order half of
    the averaged criterion comes from a and jerk alone, whose interpolation
    amplifies the noise least (Sec. 3.7 warns that noisy jerk and snap can
    drive the 6th-order step to zero)."""
    n, eps2, t_end, dt_max = 256, 1e-6, 2.0 ** -4, 1.0 / 16
    m, x, v = W.plummer(n, 21)
    _, _, _, clean = oracle_mod.hermite6_block(m, x, v, eps2, t_end, 0.01, 0.1, 0.01, dt_max)
    exact = oracle_mod.forces
    rng = np.random.default_rng(5)

    def noisy(*args, **kw):
        f = exact(*args, **kw)
        for key, sc in (("acc", "sc_acc"), ("jerk", "sc_jerk"), ("snap", "sc_snap")):
            f[key] = f[key] + 3e-8 * f[sc][:, None] * rng.standard_normal(f[key].shape) / np.sqrt(3.0)
        return f

    monkeypatch.setattr(oracle_mod, "forces", noisy)
    _, _, t, st = oracle_mod.hermite6_block(m, x, v, eps2, t_end, 0.01, 0.1, 0.01, dt_max)
    assert np.all(t == t_end)
    assert clean["block_steps"] <= st["block_steps"] < 3 * clean["block_steps"], (clean["block_steps"], st)
    assert st["dt"].min() > 2.0 ** -20
