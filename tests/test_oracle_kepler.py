"""Pin: the oracle against the closed-form two-body Kepler orbit (eps = 0).

For a bound pair with mu = m1 + m2 the relative vector follows
    r(E) = (a (cos E - e), a sqrt(1 - e^2) sin E),   dE/dt = n / (1 - e cos E),
n = sqrt(mu / a^3).  Body 1 feels acc1 = m2 r / |r|^3; its jerk and snap are
the first and second time derivatives of acc1 along that orbit, obtained by
symbolic differentiation (sympy) and evaluated at 40 digits.  Body 2 is the
mirror image with m1.  The orbit is rotated into a general 3-D orientation.
"""
import numpy as np
import pytest

sp = pytest.importorskip("sympy")


def _closed_form(m1, m2, a, e, E0):
    E = sp.symbols("E", real=True)
    mu = m1 + m2
    b = a * sp.sqrt(1 - e * e)
    r = sp.Matrix([a * (sp.cos(E) - e), b * sp.sin(E), 0])
    Edot = sp.sqrt(mu / a ** 3) / (1 - e * sp.cos(E))
    dt = lambda f: f.diff(E) * Edot  # noqa: E731
    rn3 = (r.dot(r)) ** sp.Rational(3, 2)
    acc1 = m2 * r / rn3
    jerk1 = dt(acc1)
    snap1 = dt(jerk1)
    vrel = dt(r)
    arel = -mu * r / rn3
    subs = {E: E0}
    ev = lambda M: np.array([float(sp.N(c.subs(subs), 40)) for c in M])  # noqa: E731
    return ev(r), ev(vrel), ev(arel), ev(acc1), ev(jerk1), ev(snap1)


def _rotation(seed):
    q, _ = np.linalg.qr(np.random.default_rng(seed).standard_normal((3, 3)))
    return q


@pytest.mark.parametrize("E0", [0.0, 0.7, 2.0, 3.1, 4.4])
@pytest.mark.parametrize("order", [4, 6])
def test_two_body_kepler(oracle_mod, E0, order):
    m1, m2, a, e = 0.75, 0.25, 1.3, 0.6
    R = _rotation(11)
    r, vrel, arel, acc1, jerk1, snap1 = (R @ q for q in _closed_form(
        sp.Rational(3, 4), sp.Rational(1, 4), sp.Rational(13, 10), sp.Rational(3, 5), E0))
    mu = m1 + m2
    x = np.array([-m2 / mu * r, m1 / mu * r])
    v = np.array([-m2 / mu * vrel, m1 / mu * vrel])
    acc = np.array([-m2 / mu * arel, m1 / mu * arel])  # a1 = m2 r / r^3, a2 = -m1 r / r^3
    ids = np.array([0, 1], dtype=np.int32)
    m = np.array([m1, m2])
    f = oracle_mod.forces(ids, x, v, ids, m, x, v, 0.0, order, ai=acc, aj=acc)
    tol = 1e-13
    assert np.linalg.norm(f["acc"][0] - acc1) <= tol * np.linalg.norm(acc1)
    assert np.linalg.norm(f["jerk"][0] - jerk1) <= tol * np.linalg.norm(jerk1)
    # body 2: everything mirrored and scaled by m1 / m2
    assert np.linalg.norm(f["acc"][1] + acc1 * m1 / m2) <= tol * np.linalg.norm(acc1) * m1 / m2
    assert np.linalg.norm(f["jerk"][1] + jerk1 * m1 / m2) <= tol * np.linalg.norm(jerk1) * m1 / m2
    if order == 6:
        assert np.linalg.norm(f["snap"][0] - snap1) <= 1e-12 * np.linalg.norm(snap1)
        assert np.linalg.norm(f["snap"][1] + snap1 * m1 / m2) <= 1e-12 * np.linalg.norm(snap1) * m1 / m2
    rr = float(r @ r)
    assert abs(f["pot"][0] + m2 / np.sqrt(rr)) <= 1e-15 * m2 / np.sqrt(rr)
    assert f["nn_id"][0] == 1 and f["nn_id"][1] == 0
    assert abs(f["nn_r2"][0] - rr) <= 1e-14 * rr
