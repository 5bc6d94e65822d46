"""Pins of the oracle's time-step criteria (Sec. 3.7: Aarseth's 4th-order
criterion and its 6th-order generalisation, averaged, with eta4 = 0.01 and
eta6 = 0.1).

The criteria are pinned in closed form and the interpolation that feeds them
by exactness:

* On a circular orbit of angular frequency w every derivative of the
  acceleration has |a^(k)| = |a| w^k, so Aarseth's form gives exactly
  sqrt(eta4) / w and the 6th-order form exactly eta6 / w, whatever the radius,
  the mass or the phase (w != 1 here, so a swapped pair of norms, a wrong
  exponent or eta on the wrong side of the root changes the value).
* The cubic Hermite interpolant through (a, jerk) at both ends of a step is
  the acceleration itself when that is a cubic in time, so its 2nd derivative
  at the END of the step and its 3rd derivative are the cubic's own.
* Fed end-of-step data from a circular orbit, the whole chain (interpolation,
  then the criteria and their mean) converges to (sqrt(eta4) + eta6) / (2 w)
  as the step shrinks, and on an eccentric Kepler orbit it converges to the
  criteria evaluated on the exact derivatives at the end of the step
  (symbolic differentiation, sympy).
"""
import math

import numpy as np
import pytest


def _rotation(seed):
    q, _ = np.linalg.qr(np.random.default_rng(seed).standard_normal((3, 3)))
    return q


def _circular(R, M, phase, rot):
    """Derivatives 0..5 of the acceleration of a test particle on a circular
    orbit of radius R about a point mass M, at orbital phase `phase`:
    a(t) = -w^2 R (cos(w t), sin(w t), 0), rotated by `rot`."""
    w = math.sqrt(M / R ** 3)
    out = []
    for k in range(6):
        # the k-th derivative of (cos, sin)(w t) is w^k (cos, sin)(w t + k pi/2)
        ph = phase + k * math.pi / 2
        out.append(rot @ (-(w ** (k + 2)) * R * np.array([math.cos(ph), math.sin(ph), 0.0])))
    return w, out


@pytest.mark.parametrize("phase", [0.0, 0.9, 2.5, 4.0])
@pytest.mark.parametrize("R,M", [(1.7, 0.9), (0.31, 2.0e-3), (40.0, 1.0)])
def test_criteria_on_a_circular_orbit(oracle_mod, phase, R, M):
    w, (a, j, s, c, p, q) = _circular(R, M, phase, _rotation(4))
    assert abs(w - 1.0) > 0.05
    for eta in (0.01, 0.02, 0.3):
        assert abs(oracle_mod.aarseth4(eta, a, j, s, c) * w / math.sqrt(eta) - 1.0) < 1e-14
    for eta in (0.1, 0.05, 0.7):
        assert abs(oracle_mod.aarseth6(eta, a, j, s, c, p, q) * w / eta - 1.0) < 1e-14


def test_cubic_hermite_derivatives_exact_on_a_cubic(oracle_mod):
    """a(t) = c0 + c1 t + c2 t^2/2 + c3 t^3/6 per component: the interpolant
    through (a, a') at t0 and t1 is a itself, so a2(t1) = c2 + c3 t1 and
    a3 = c3 (the 2nd derivative at t0, c2 + c3 t0, is a different vector)."""
    rng = np.random.default_rng(17)
    c0, c1, c2, c3 = rng.standard_normal((4, 3))
    acc = lambda t: c0 + c1 * t + c2 * t * t / 2 + c3 * t ** 3 / 6  # noqa: E731
    jerk = lambda t: c1 + c2 * t + c3 * t * t / 2  # noqa: E731
    for t0, h in ((0.3, 0.4), (-1.1, 0.125), (2.0, 1.5)):
        t1 = t0 + h
        a2, a3 = oracle_mod.hermite3_derivs(h, acc(t0), jerk(t0), acc(t1), jerk(t1))
        want2 = c2 + c3 * t1
        assert np.linalg.norm(a2 - want2) < 1e-11 * np.linalg.norm(want2)
        assert np.linalg.norm(a3 - c3) < 1e-11 * np.linalg.norm(c3)
        # the same with a column of steps (the integrators' per-row form)
        A2, A3 = oracle_mod.hermite3_derivs(np.array([[h], [h]]), np.stack([acc(t0)] * 2), np.stack([jerk(t0)] * 2),
                                            np.stack([acc(t1)] * 2), np.stack([jerk(t1)] * 2))
        assert np.allclose(A2, want2, rtol=1e-11, atol=0) and np.allclose(A3, c3, rtol=1e-11, atol=0)


def test_averaged_criterion_from_end_of_step_data_on_a_circular_orbit(oracle_mod):
    """The chain the block integrators run at the end of a step -- a and jerk
    at both ends, snap at the end, the quintic interpolant's crackle, pop and
    5th derivative (_h6_correct), the cubic interpolant's a2 and a3 -- tends to
    the closed form as the step h shrinks, for the 4th-order criterion alone
    (hermite4_block) and for the mean of the two (hermite6_block)."""
    R, M, eta4, eta6 = 1.7, 0.9, 0.01, 0.1
    rot = _rotation(9)
    w = math.sqrt(M / R ** 3)
    want4 = math.sqrt(eta4) / w
    want = 0.5 * (math.sqrt(eta4) + eta6) / w
    errs4, errs = [], []
    for frac in (0.2, 0.1, 0.05, 0.025):
        h = frac / w
        _, d0 = _circular(R, M, 0.4, rot)
        _, d1 = _circular(R, M, 0.4 + w * h, rot)
        a0, j0, s0 = d0[:3]
        a1, j1, s1 = d1[:3]
        a2, a3 = oracle_mod.hermite3_derivs(h, a0, j0, a1, j1)
        errs4.append(abs(oracle_mod.aarseth4(eta4, a1, j1, a2, a3) / want4 - 1.0))
        hh = np.array([[h]])
        _, _, c1, p1, q = oracle_mod._h6_correct(hh, np.zeros((1, 3)), np.zeros((1, 3)), a0[None], j0[None],
                                                 s0[None], a1[None], j1[None], s1[None])
        got = oracle_mod._h6_step_want(eta4, eta6, h, a0, j0, a1, j1, s1, c1[0], p1[0], q[0])
        errs.append(abs(got / want - 1.0))
    assert errs4[-1] < 1e-3 and errs[-1] < 1e-3, (errs4, errs)
    # the error falls at least linearly with h (the interpolated derivatives converge)
    for e in (errs4, errs):
        assert all(e[k + 1] < 0.6 * e[k] for k in range(len(e) - 1)), e


def _eccentric_derivs(E0, n_derivs):
    """Relative acceleration of a two-body Kepler orbit (mu = 1, a = 1.3,
    e = 0.6) and its first n_derivs time derivatives at eccentric anomaly E0,
    plus the time since pericentre (Kepler's equation), at 40 digits."""
    sp = pytest.importorskip("sympy")
    E = sp.symbols("E", real=True)
    a, e, mu = sp.Rational(13, 10), sp.Rational(3, 5), sp.Integer(1)
    r = sp.Matrix([a * (sp.cos(E) - e), a * sp.sqrt(1 - e * e) * sp.sin(E), 0])
    nmean = sp.sqrt(mu / a ** 3)
    Edot = nmean / (1 - e * sp.cos(E))
    f = -mu * r / (r.dot(r)) ** sp.Rational(3, 2)
    out = []
    for _ in range(n_derivs + 1):
        out.append(np.array([float(sp.N(cpt.subs(E, E0), 40)) for cpt in f]))
        f = f.diff(E) * Edot
    t = float(sp.N(((E - e * sp.sin(E)) / nmean).subs(E, E0), 40))
    return t, out


def test_criteria_converge_to_the_exact_derivatives_on_an_eccentric_orbit(oracle_mod):
    """Away from the symmetric circular case: end-of-step data from an
    eccentric orbit.  The 4th-order criterion on the interpolated a2(t1), a3
    tends to the criterion on the exact derivatives at the end of the step;
    the 6th-order criterion on the interpolated crackle, pop and 5th
    derivative tends to the one on the exact values."""
    sp = pytest.importorskip("sympy")
    E1 = 1.1
    t1, d1 = _eccentric_derivs(E1, 5)
    a1, j1, s1, c1, p1, q1 = d1
    exact4 = oracle_mod.aarseth4(0.01, a1, j1, s1, c1)
    exact6 = oracle_mod.aarseth6(0.1, a1, j1, s1, c1, p1, q1)
    # invert Kepler's equation for the start of each step (Newton on E)
    e, nmean = 0.6, math.sqrt(1.0 / 1.3 ** 3)
    errs4, errs6 = [], []
    for h in (0.02, 0.01, 0.005, 0.0025):
        t0 = t1 - h
        E0 = E1
        for _ in range(60):
            E0 -= (E0 - e * math.sin(E0) - nmean * t0) / (1 - e * math.cos(E0))
        _, d0 = _eccentric_derivs(sp.Float(E0, 40), 2)
        a0, j0, s0 = d0
        a2, a3 = oracle_mod.hermite3_derivs(h, a0, j0, a1, j1)
        errs4.append(abs(oracle_mod.aarseth4(0.01, a1, j1, a2, a3) / exact4 - 1.0))
        _, _, c, p, q = oracle_mod._h6_correct(np.array([[h]]), np.zeros((1, 3)), np.zeros((1, 3)), a0[None],
                                               j0[None], s0[None], a1[None], j1[None], s1[None])
        errs6.append(abs(oracle_mod.aarseth6(0.1, a1, j1, s1, c[0], p[0], q[0]) / exact6 - 1.0))
    assert errs4[-1] < 2e-3 and errs6[-1] < 2e-3, (errs4, errs6)
    # first order in h (the interpolants' highest derivative is a constant);
    # at the smallest step the 5th derivative's round-off (~u / h^4) shows
    for e_ in (errs4, errs6):
        assert all(e_[k + 1] < 0.7 * e_[k] for k in range(len(e_) - 1)), e_
