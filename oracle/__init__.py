"""Plain FP64 CPU oracle of the direct-summation gravity pass.

TEST INFRASTRUCTURE ONLY: the test-suite, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may use it.  The
GPU library never imports, links or calls anything here, and nothing here
imports the GPU library.

Contents
--------
``predict``           Taylor predictor of the sources (Sec. 2.2), sp2_oracle.c
``forces``            direct sum of acc / jerk / snap / pot / nearest neighbour
                      with per-sink scale sums (Sec. 3), sp2_oracle.c
``neighbours``        lists of the particles within a radius of each sink
                      (Sec. 1, Sec. 3), sp2_oracle.c
``step``              predict + forces on sink slots, the block-step pass
``energy``            kinetic + potential energy
``hermite4_shared``   shared-step 4th-order Hermite integrator (test driver)
``hermite4_block``    block time-step 4th-order Hermite integrator with
                      Aarseth's criterion (Sec. 3.7; test driver)
``hermite6_shared``   shared-step 6th-order Hermite integrator (Nitadori &
                      Makino 2008; crackle in the predictor; test driver)
``hermite6_block``    block time-step 6th-order Hermite integrator with the
                      averaged 4th/6th-order criterion (Sec. 3.7; test driver)
``hermite3_derivs``   a2(t1), a3 of the cubic Hermite interpolant of a step
``aarseth4``          Aarseth's 4th-order time-step criterion
``aarseth6``          its 6th-order generalisation (Nitadori & Makino 2008)
``adjoint``           float64 torch restatement for gradient checks (adjoint.py)

Parity status: every output is pinned by the ``-m "not gpu"`` tests
(brute force in 50-digit decimal arithmetic, two-body Kepler closed form,
Newton's third law, pair-sum symmetry, finite differences along the predictor,
invariances, Hermite energy conservation, 6th-order Hermite exactness on a
quintic and 6th-order convergence on a Kepler orbit; neighbour lists against scipy's
pairwise distances on an exact integer grid, symmetry, strictness, overflow;
the time-step criteria in closed form on a circular orbit, the interpolated
derivatives exact on a cubic and convergent on an eccentric Kepler orbit).
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
from pathlib import Path

import numpy as np

_HERE = Path(__file__).resolve().parent
_SRC = _HERE / "sp2_oracle.c"
_BUILD = _HERE / "_build"
_LIB_PATH = _BUILD / "libsp2_oracle.so"
_lib = None


def build(force: bool = False) -> Path:
    """Compile sp2_oracle.c into oracle/_build/libsp2_oracle.so (gcc, OpenMP)."""
    _BUILD.mkdir(exist_ok=True)
    if force or not _LIB_PATH.exists() or _LIB_PATH.stat().st_mtime < _SRC.stat().st_mtime:
        tmp = _LIB_PATH.with_suffix(f".{os.getpid()}.tmp.so")
        cmd = ["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fno-fast-math",
               "-fPIC", "-shared", "-std=c11", str(_SRC), "-o", str(tmp), "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(str(_LIB_PATH))
        P = ctypes.c_void_p
        I64 = ctypes.c_int64
        lib.sp2o_predict.argtypes = [I64, ctypes.c_int, ctypes.c_double, P, P, P, P, P, P, P, P, P]
        lib.sp2o_predict.restype = None
        lib.sp2o_forces.argtypes = [I64, P, P, P, P, I64, P, P, P, P, P,
                                    ctypes.c_double, ctypes.c_int,
                                    P, P, P, P, P, P, P, P, P]
        lib.sp2o_forces.restype = None
        lib.sp2o_neighbours.argtypes = [I64, P, P, P, I64, P, P, ctypes.c_int32, P, P]
        lib.sp2o_neighbours.restype = None
        lib.sp2o_max_threads.restype = ctypes.c_int
        lib.sp2o_set_threads.argtypes = [ctypes.c_int]
        _lib = lib
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _f64(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None:
        a = a.reshape(shape)
    return a


def threads() -> int:
    """OpenMP threads the oracle uses."""
    return int(_load().sp2o_max_threads())


def set_threads(n: int) -> None:
    _load().sp2o_set_threads(int(n))


def predict(t, tj, x, v, a, jerk, snap=None, order: int = 4):
    """Taylor-predict sources to time t; returns (xp, vp, ap) (ap None for order 4)."""
    lib = _load()
    n = len(tj)
    tj = _f64(tj, (n,))
    x, v, a, jerk = (_f64(q, (n, 3)) for q in (x, v, a, jerk))
    xp = np.empty((n, 3))
    vp = np.empty((n, 3))
    ap = None
    sn = None
    if order == 6:
        if snap is None:
            raise ValueError("order 6 needs snap")
        sn = _f64(snap, (n, 3))
        ap = np.empty((n, 3))
    lib.sp2o_predict(n, order, float(t), _p(tj), _p(x), _p(v), _p(a), _p(jerk), _p(sn),
                     _p(xp), _p(vp), _p(ap))
    return xp, vp, ap


def forces(ids_i, xi, vi, ids_j, mj, xj, vj, eps2: float, order: int = 4, ai=None, aj=None):
    """Direct sum on explicit sinks.  Returns a dict of numpy arrays.

    Keys: acc, jerk, snap (order 6), pot, nn_id, nn_r2, sc_acc, sc_jerk, sc_snap.
    """
    lib = _load()
    n_i, n_j = len(ids_i), len(ids_j)
    ids_i = np.ascontiguousarray(ids_i, dtype=np.int32)
    ids_j = np.ascontiguousarray(ids_j, dtype=np.int32)
    xi, vi = _f64(xi, (n_i, 3)), _f64(vi, (n_i, 3))
    xj, vj = _f64(xj, (n_j, 3)), _f64(vj, (n_j, 3))
    mj = _f64(mj, (n_j,))
    if order == 6:
        if ai is None or aj is None:
            raise ValueError("order 6 needs ai and aj")
        ai, aj = _f64(ai, (n_i, 3)), _f64(aj, (n_j, 3))
    else:
        ai = aj = None
    out = {
        "acc": np.empty((n_i, 3)), "jerk": np.empty((n_i, 3)),
        "snap": np.empty((n_i, 3)) if order == 6 else None,
        "pot": np.empty(n_i), "nn_id": np.empty(n_i, dtype=np.int32), "nn_r2": np.empty(n_i),
        "sc_acc": np.empty(n_i), "sc_jerk": np.empty(n_i),
        "sc_snap": np.empty(n_i) if order == 6 else None,
    }
    lib.sp2o_forces(n_i, _p(ids_i), _p(xi), _p(vi), _p(ai),
                    n_j, _p(ids_j), _p(mj), _p(xj), _p(vj), _p(aj),
                    float(eps2), int(order),
                    _p(out["acc"]), _p(out["jerk"]), _p(out["snap"]), _p(out["pot"]),
                    _p(out["nn_id"]), _p(out["nn_r2"]),
                    _p(out["sc_acc"]), _p(out["sc_jerk"]), _p(out["sc_snap"]))
    if order != 6:
        del out["snap"], out["sc_snap"]
    return out


def neighbours(ids_i, xi, h2, ids_j, xj, nb_max: int):
    """Neighbour lists (sp2o_neighbours): count[n_i] and ids[n_i, nb_max], each
    row's first min(count, nb_max) entries ascending (the smallest ids on
    overflow); the rest of a row is -1."""
    lib = _load()
    ids_i = np.ascontiguousarray(ids_i, dtype=np.int32)
    ids_j = np.ascontiguousarray(ids_j, dtype=np.int32)
    xi = _f64(xi, (len(ids_i), 3))
    xj = _f64(xj, (len(ids_j), 3))
    h2 = _f64(h2, (len(ids_i),))
    count = np.zeros(len(ids_i), dtype=np.int32)
    out = np.full((len(ids_i), nb_max), -1, dtype=np.int32)
    lib.sp2o_neighbours(ctypes.c_int64(len(ids_i)), _p(ids_i), _p(xi), _p(h2), ctypes.c_int64(len(ids_j)), _p(ids_j),
                        _p(xj), ctypes.c_int32(nb_max), _p(count), _p(out))
    return count, out


def step(t, i_idx, ids, m, tj, x, v, a, jerk, snap=None, *, eps2: float, order: int = 4,
         j_range=None):
    """One block-step force pass: predict every source to t, then sum on sinks.

    The sinks are the predicted sources at slots ``i_idx`` (the i-particles are
    j-particles due for an update).  ``j_range=(lo, hi)`` restricts the sources
    to slots lo..hi-1 (one independent system of a batch).
    """
    xp, vp, ap = predict(t, tj, x, v, a, jerk, snap, order)
    i_idx = np.asarray(i_idx, dtype=np.int64)
    lo, hi = (0, len(ids)) if j_range is None else j_range
    sl = slice(lo, hi)
    return forces(ids[i_idx], xp[i_idx], vp[i_idx], ids[sl], m[sl], xp[sl], vp[sl],
                  eps2, order,
                  ai=None if ap is None else ap[i_idx], aj=None if ap is None else ap[sl])


def energy(m, x, v, eps2: float) -> float:
    """Total energy: sum m v^2 / 2 + (1/2) sum m_i pot_i, with the oracle's pot."""
    n = len(m)
    ids = np.arange(n, dtype=np.int32)
    f = forces(ids, x, v, ids, m, x, v, eps2, 4)
    return float(0.5 * np.sum(m * np.sum(v * v, axis=1)) + 0.5 * np.sum(m * f["pot"]))


def hermite4_shared(m, x, v, eps2: float, dt: float, n_steps: int):
    """Shared-time-step 4th-order Hermite integration (Makino & Aarseth 1992).

    Per step: predict with the Taylor polynomial, evaluate acc and jerk at the
    predicted state, then correct
        v1 = v0 + (a0 + a1) dt/2 + (j0 - j1) dt^2/12
        x1 = x0 + (v0 + v1) dt/2 + (a0 - a1) dt^2/12.
    Returns the final (x, v).  The integrator around the force pass is driver
    code of the tests; the paper leaves it to the user (Sec. 3.7).
    """
    n = len(m)
    ids = np.arange(n, dtype=np.int32)
    x = np.array(x, dtype=np.float64)
    v = np.array(v, dtype=np.float64)
    f = forces(ids, x, v, ids, m, x, v, eps2, 4)
    a0, j0 = f["acc"], f["jerk"]
    tj = np.zeros(n)
    for _ in range(n_steps):
        xp, vp, _ = predict(dt, tj, x, v, a0, j0, None, 4)
        f = forces(ids, xp, vp, ids, m, xp, vp, eps2, 4)
        a1, j1 = f["acc"], f["jerk"]
        v1 = v + (a0 + a1) * (dt / 2) + (j0 - j1) * (dt * dt / 12)
        x1 = x + (v + v1) * (dt / 2) + (a0 - a1) * (dt * dt / 12)
        x, v, a0, j0 = x1, v1, a1, j1
    return x, v


_DT_MIN = 2.0 ** -50


def _quantise(want, cap, t1):
    """Largest power-of-two step <= want (at most cap, at least 2^-50) that
    divides t1: block time-steps stay synchronised."""
    d = cap
    while d > want and d > _DT_MIN:
        d *= 0.5
    while d > _DT_MIN and math.fmod(t1, d) != 0.0:
        d *= 0.5
    return d


def hermite3_derivs(h, a0, j0, a1, j1):
    """2nd derivative at t1 and (constant) 3rd derivative of the cubic Hermite
    interpolant of the acceleration through (a0, j0) at t0 and (a1, j1) at
    t1 = t0 + h (h a column of per-row steps, or a scalar):
        a2(t0) = (-6 (a0 - a1) - h (4 j0 + 2 j1)) / h^2
        a3     = (12 (a0 - a1) + 6 h (j0 + j1)) / h^3,   a2(t1) = a2(t0) + h a3.
    Returns (a2(t1), a3)."""
    h2 = h * h
    a3 = (12.0 * (a0 - a1) + 6.0 * h * (j0 + j1)) / (h2 * h)
    a2 = (-6.0 * (a0 - a1) - h * (4.0 * j0 + 2.0 * j1)) / h2 + h * a3
    return a2, a3


def aarseth4(eta, a, j, a2, a3):
    """Aarseth's 4th-order time-step criterion (the one Sec. 3.7's averaged
    criterion starts from) for one particle, from its acceleration a, jerk j,
    2nd and 3rd derivatives a2, a3 (3-vectors):
        dt = sqrt(eta (|a||a2| + |j|^2) / (|j||a3| + |a2|^2)),
    eta inside the root.  +inf when the denominator vanishes."""
    A, J = float(np.linalg.norm(a)), float(np.linalg.norm(j))
    A2, A3 = float(np.linalg.norm(a2)), float(np.linalg.norm(a3))
    den = J * A3 + A2 * A2
    if not den > 0.0:
        return math.inf
    return math.sqrt(eta * (A * A2 + J * J) / den)


def aarseth6(eta, a, j, s, c, p, q):
    """The 6th-order generalisation of Aarseth's criterion (Nitadori & Makino
    2008) for one particle, from a, jerk j, snap s, crackle c, pop p and the
    5th derivative q of its acceleration (3-vectors):
        dt = eta ((|a||s| + |j|^2) / (|c||q| + |p|^2))^(1/6),
    eta outside the root.  +inf when the denominator vanishes."""
    A, J, S = float(np.linalg.norm(a)), float(np.linalg.norm(j)), float(np.linalg.norm(s))
    C, P, Q = float(np.linalg.norm(c)), float(np.linalg.norm(p)), float(np.linalg.norm(q))
    den = C * Q + P * P
    if not den > 0.0:
        return math.inf
    return eta * ((A * S + J * J) / den) ** (1.0 / 6.0)


def hermite4_block(m, x, v, eps2: float, t_end: float, eta: float, eta_s: float, dt_max: float):
    """Block time-step 4th-order Hermite integration (Sec. 3.7: individual
    power-of-two steps; Makino & Aarseth 1992 corrector; Aarseth's criterion).

    Start at t = 0 with a, jerk from one direct sum and steps eta_s |a|/|j|.
    Each block: t1 = min(t_i + dt_i); the particles with t_i + dt_i = t1 are
    active; every particle is predicted to t1; the active ones get a1, j1 on
    the predicted state and the corrector
        v1 = v0 + (a0 + a1) h/2 + (j0 - j1) h^2/12
        x1 = x0 + (v0 + v1) h/2 + (a0 - a1) h^2/12       (h = t1 - t_i),
    then the next step from Aarseth's criterion (aarseth4) with a2(t1) and a3
    of the cubic Hermite interpolant of the step (hermite3_derivs), quantised
    by _quantise with cap min(2h, dt_max).  Returns (x, v, t, stats).
    """
    n = len(m)
    ids = np.arange(n, dtype=np.int32)
    x = np.array(x, dtype=np.float64)
    v = np.array(v, dtype=np.float64)
    f = forces(ids, x, v, ids, m, x, v, eps2, 4)
    a, j = f["acc"].copy(), f["jerk"].copy()
    t = np.zeros(n)
    dt = np.empty(n)
    for i in range(n):
        an, jn = np.linalg.norm(a[i]), np.linalg.norm(j[i])
        dt[i] = _quantise(eta_s * an / jn if jn > 0 else dt_max, dt_max, 0.0)
    steps, active_sum = 0, 0
    while True:
        t1 = float(np.min(t + dt))
        if t1 > t_end:
            break
        act = np.flatnonzero(t + dt == t1)
        xp, vp, _ = predict(t1, t, x, v, a, j, None, 4)
        f = forces(ids[act], xp[act], vp[act], ids, m, xp, vp, eps2, 4)
        a1, j1 = f["acc"], f["jerk"]
        h = (t1 - t[act])[:, None]
        h2 = h * h
        a0, j0 = a[act], j[act]
        v1 = v[act] + (a0 + a1) * (h / 2) + (j0 - j1) * (h2 / 12)
        x1 = x[act] + (v[act] + v1) * (h / 2) + (a0 - a1) * (h2 / 12)
        a2, a3 = hermite3_derivs(h, a0, j0, a1, j1)
        x[act], v[act], a[act], j[act], t[act] = x1, v1, a1, j1, t1
        for k, i in enumerate(act):
            want = aarseth4(eta, a1[k], j1[k], a2[k], a3[k])
            dt[i] = _quantise(want if math.isfinite(want) else dt_max, min(2.0 * float(h[k, 0]), dt_max), t1)
        steps += 1
        active_sum += len(act)
    return x, v, t, {"block_steps": steps, "active_sum": active_sum, "dt": dt}


def _h6_predict(h, x, v, a, j, s, c):
    """Taylor prediction over h (per-row column vector) of the 6th-order
    scheme: x to h^5 (crackle c), v to h^4, a to h^3."""
    h2, h3 = h * h, h * h * h
    xp = x + v * h + a * (h2 / 2) + j * (h3 / 6) + s * (h2 * h2 / 24) + c * (h3 * h2 / 120)
    vp = v + a * h + j * (h2 / 2) + s * (h3 / 6) + c * (h2 * h2 / 24)
    ap = a + j * h + s * (h2 / 2) + c * (h3 / 6)
    return xp, vp, ap


def _h6_correct(h, x0, v0, a0, j0, s0, a1, j1, s1):
    """6th-order Hermite corrector (Nitadori & Makino 2008): the quintic
    Hermite interpolant of the acceleration through (a, j, s) at both ends,
    integrated once for v and (with v, a, j in place of a, j, s) for x:
        v1 = v0 + h/2 (a0 + a1) - h^2/10 (j1 - j0) + h^3/120 (s0 + s1)
        x1 = x0 + h/2 (v0 + v1) - h^2/10 (a1 - a0) + h^3/120 (j0 + j1).
    The same interpolant's 3rd, 4th and 5th derivatives at the end of the step
    (crackle, pop and its derivative), written out from the three matching
    conditions at t1:
        c1 h^3 = 60 (a1 - a0) - 24 h j0 - 36 h j1 - 3 h^2 s0 + 9 h^2 s1
        p1 h^4 = 360 (a1 - a0) - 168 h j0 - 192 h j1 - 24 h^2 s0 + 36 h^2 s1
        q  h^5 = 720 (a1 - a0) - 360 h (j0 + j1) - 60 h^2 (s0 - s1).
    Returns (x1, v1, c1, p1, q)."""
    h2 = h * h
    h3 = h2 * h
    v1 = v0 + (a0 + a1) * (h / 2) - (j1 - j0) * (h2 / 10) + (s0 + s1) * (h3 / 120)
    x1 = x0 + (v0 + v1) * (h / 2) - (a1 - a0) * (h2 / 10) + (j0 + j1) * (h3 / 120)
    da = a1 - a0
    c1 = (60.0 * da - h * (24.0 * j0 + 36.0 * j1) + h2 * (9.0 * s1 - 3.0 * s0)) / h3
    p1 = (360.0 * da - h * (168.0 * j0 + 192.0 * j1) + h2 * (36.0 * s1 - 24.0 * s0)) / (h3 * h)
    q = (720.0 * da - 360.0 * h * (j0 + j1) - 60.0 * h2 * (s0 - s1)) / (h3 * h2)
    return x1, v1, c1, p1, q


def hermite6_shared(m, x, v, eps2: float, dt: float, n_steps: int):
    """Shared-time-step 6th-order Hermite integration (Nitadori & Makino 2008).

    Per step: predict x, v, a with _h6_predict (crackle from the previous
    step's interpolation, zero on the first step), evaluate acc, jerk and snap
    at the predicted state (order-6 direct sum), correct with _h6_correct.
    Returns the final (x, v)."""
    n = len(m)
    ids = np.arange(n, dtype=np.int32)
    x = np.array(x, dtype=np.float64)
    v = np.array(v, dtype=np.float64)
    z = np.zeros((n, 3))
    f = forces(ids, x, v, ids, m, x, v, eps2, 6, ai=z, aj=z)
    a, j = f["acc"], f["jerk"]
    # snap needs the sources' accelerations: one more pass with a known
    f = forces(ids, x, v, ids, m, x, v, eps2, 6, ai=a, aj=a)
    a, j, s = f["acc"], f["jerk"], f["snap"]
    c = np.zeros((n, 3))
    h = np.full((n, 1), dt)
    for _ in range(n_steps):
        xp, vp, ap = _h6_predict(h, x, v, a, j, s, c)
        f = forces(ids, xp, vp, ids, m, xp, vp, eps2, 6, ai=ap, aj=ap)
        x, v, c, _, _ = _h6_correct(h, x, v, a, j, s, f["acc"], f["jerk"], f["snap"])
        a, j, s = f["acc"], f["jerk"], f["snap"]
    return x, v


def _h6_step_want(eta4, eta6, h, a0, j0, a1, j1, s1, c1, p1, q):
    """Next step of a particle from the end of its step: the average of
    Aarseth's 4th-order criterion, evaluated as the 4th-order scheme does
    (a and jerk at both ends; the 2nd and 3rd derivatives at t1 of their cubic
    Hermite interpolant, as in hermite4_block),
        dt4 = sqrt(eta4 (|a1||a2| + |j1|^2) / (|j1||a3| + |a2|^2)),
    and its 6th-order generalisation (Nitadori & Makino 2008) with the pass's
    snap and the quintic interpolant's crackle c1, pop p1 and 5th derivative q,
        dt6 = eta6 ((|a1||s1| + |j1|^2) / (|c1||q| + |p1|^2))^(1/6)."""
    a2, a3 = hermite3_derivs(h, a0, j0, a1, j1)
    dt4 = aarseth4(eta4, a1, j1, a2, a3)
    dt6 = aarseth6(eta6, a1, j1, s1, c1, p1, q)
    if not (math.isfinite(dt4) and math.isfinite(dt6)):
        return math.inf
    return 0.5 * (dt4 + dt6)


def hermite6_block(m, x, v, eps2: float, t_end: float, eta4: float, eta6: float, eta_s: float,
                   dt_max: float):
    """Block time-step 6th-order Hermite integration (Sec. 3.7 runs this
    scheme with the averaged criterion, eta4 = 0.01 and eta6 = 0.1).

    Start at t = 0 with a, jerk, snap from the direct sum, crackle 0 and steps
    eta_s |a|/|j|.  Each block: t1 = min(t_i + dt_i); every particle is
    predicted to t1 (_h6_predict with its own crackle); the active ones get
    a1, j1, s1 on the predicted state, _h6_correct, a new crackle, and the
    next step from _h6_step_want quantised by _quantise with cap
    min(2h, dt_max).  Returns (x, v, t, stats)."""
    n = len(m)
    ids = np.arange(n, dtype=np.int32)
    x = np.array(x, dtype=np.float64)
    v = np.array(v, dtype=np.float64)
    z = np.zeros((n, 3))
    f = forces(ids, x, v, ids, m, x, v, eps2, 6, ai=z, aj=z)
    f = forces(ids, x, v, ids, m, x, v, eps2, 6, ai=f["acc"], aj=f["acc"])
    a, j, s = f["acc"].copy(), f["jerk"].copy(), f["snap"].copy()
    c = np.zeros((n, 3))
    t = np.zeros(n)
    dt = np.empty(n)
    for i in range(n):
        an, jn = np.linalg.norm(a[i]), np.linalg.norm(j[i])
        dt[i] = _quantise(eta_s * an / jn if jn > 0 else dt_max, dt_max, 0.0)
    steps, active_sum = 0, 0
    while True:
        t1 = float(np.min(t + dt))
        if t1 > t_end:
            break
        act = np.flatnonzero(t + dt == t1)
        hh = (t1 - t)[:, None]
        xp, vp, ap = _h6_predict(hh, x, v, a, j, s, c)
        f = forces(ids[act], xp[act], vp[act], ids, m, xp, vp, eps2, 6, ai=ap[act], aj=ap)
        a1, j1, s1 = f["acc"], f["jerk"], f["snap"]
        h = hh[act]
        a0, j0 = a[act].copy(), j[act].copy()
        x1, v1, c1, p1, q = _h6_correct(h, x[act], v[act], a0, j0, s[act], a1, j1, s1)
        x[act], v[act], a[act], j[act], s[act], c[act], t[act] = x1, v1, a1, j1, s1, c1, t1
        for k, i in enumerate(act):
            hk = float(h[k, 0])
            want = _h6_step_want(eta4, eta6, hk, a0[k], j0[k], a1[k], j1[k], s1[k], c1[k], p1[k], q[k])
            dt[i] = _quantise(want, min(2.0 * hk, dt_max), t1)
        steps += 1
        active_sum += len(act)
    return x, v, t, {"block_steps": steps, "active_sum": active_sum, "dt": dt}
