"""Pin: the FP64 oracle against a 60-digit decimal brute force on tiny inputs.

The brute force uses only the textbook definitions: Newton's softened
acceleration sum_j m_j r / (r.r + eps^2)^(3/2) and potential -sum_j m_j /
(r.r + eps^2)^(1/2); jerk and snap are taken as the first and second time
derivatives of that acceleration along the predicted motion
x_k(h) = x_k + v_k h + a_k h^2 / 2 by 5-point finite differences at 60 digits
(step 1e-12, truncation and round-off both far below 1e-30).  It never writes
the jerk or snap formulas, so a dropped term, sign or index in the oracle's
expressions shows up here.  The nearest neighbour is a plain argmin over
exact decimal distances.
"""
from decimal import Decimal, getcontext

import numpy as np
import pytest

getcontext().prec = 60
D = Decimal
H = D("1e-12")


def _acc_pot(i, X, M, eps2, ids):
    ax = [D(0)] * 3
    pot = D(0)
    for j in range(len(M)):
        if ids[j] == ids[i]:
            continue
        r = [X[j][k] - X[i][k] for k in range(3)]
        d2 = sum(c * c for c in r) + eps2
        s = 1 / d2.sqrt()
        for k in range(3):
            ax[k] += M[j] * r[k] * s * s * s
        pot -= M[j] * s
    return ax, pot


def _brute(x, v, a, m, ids, eps2):
    n = len(m)
    X = [[D(float(c)) for c in row] for row in x]
    V = [[D(float(c)) for c in row] for row in v]
    A = [[D(float(c)) for c in row] for row in a]
    M = [D(float(c)) for c in m]
    E2 = D(float(eps2))

    def moved(h):
        return [[X[k][c] + V[k][c] * h + A[k][c] * h * h / 2 for c in range(3)] for k in range(n)]

    pos = {s: moved(s * H) for s in (-2, -1, 0, 1, 2)}
    out = []
    for i in range(n):
        f = {s: _acc_pot(i, pos[s], M, E2, ids) for s in pos}
        acc, pot = f[0]
        jerk = [(8 * (f[1][0][k] - f[-1][0][k]) - (f[2][0][k] - f[-2][0][k])) / (12 * H)
                for k in range(3)]
        snap = [(-f[2][0][k] + 16 * f[1][0][k] - 30 * f[0][0][k] + 16 * f[-1][0][k] - f[-2][0][k])
                / (12 * H * H) for k in range(3)]
        best, best_id = None, -1
        for j in range(n):
            if ids[j] == ids[i]:
                continue
            d2 = sum((X[j][k] - X[i][k]) ** 2 for k in range(3))
            if best is None or d2 < best or (d2 == best and ids[j] < best_id):
                best, best_id = d2, int(ids[j])
        out.append((acc, jerk, snap, pot, best_id, best))
    return out


def _case(n, seed, eps):
    rng = np.random.default_rng(seed)
    x = rng.uniform(-1, 1, (n, 3))
    v = rng.uniform(-1, 1, (n, 3))
    a = rng.uniform(-1, 1, (n, 3))
    m = rng.uniform(0.1, 1.0, n)
    ids = rng.permutation(n).astype(np.int32)
    return x, v, a, m, ids, eps * eps


@pytest.mark.parametrize("n,seed,eps", [(2, 0, 0.0), (3, 1, 0.05), (5, 2, 0.0), (8, 3, 0.1), (8, 4, 0.0)])
@pytest.mark.parametrize("order", [4, 6])
def test_oracle_matches_decimal_brute_force(oracle_mod, n, seed, eps, order):
    x, v, a, m, ids, eps2 = _case(n, seed, eps)
    f = oracle_mod.forces(ids, x, v, ids, m, x, v, eps2, order, ai=a, aj=a)
    ref = _brute(x, v, a, m, ids, eps2)
    for i, (acc, jerk, snap, pot, nn, nn2) in enumerate(ref):
        acc = np.array([float(c) for c in acc])
        jerk = np.array([float(c) for c in jerk])
        assert np.linalg.norm(f["acc"][i] - acc) <= 1e-14 * f["sc_acc"][i]
        assert np.linalg.norm(f["jerk"][i] - jerk) <= 1e-14 * f["sc_jerk"][i]
        if order == 6:
            snap = np.array([float(c) for c in snap])
            assert np.linalg.norm(f["snap"][i] - snap) <= 1e-13 * f["sc_snap"][i]
        assert abs(f["pot"][i] - float(pot)) <= 1e-14 * abs(float(pot))
        assert f["nn_id"][i] == nn
        assert abs(f["nn_r2"][i] - float(nn2)) <= 1e-15 * float(nn2)


def test_scale_sums_bound_the_terms(oracle_mod):
    """The scale sums are sums of absolute values: they bound |acc|, |jerk|, |snap|."""
    x, v, a, m, ids, eps2 = _case(8, 7, 0.01)
    f = oracle_mod.forces(ids, x, v, ids, m, x, v, eps2, 6, ai=a, aj=a)
    assert np.all(np.linalg.norm(f["acc"], axis=1) <= f["sc_acc"] * (1 + 1e-15))
    assert np.all(np.linalg.norm(f["jerk"], axis=1) <= f["sc_jerk"] * (1 + 1e-15))
    assert np.all(np.linalg.norm(f["snap"], axis=1) <= f["sc_snap"] * (1 + 1e-15))
    # single pair: the acceleration scale is exactly |A_ij|
    g = oracle_mod.forces(ids[:2], x[:2], v[:2], ids[:2], m[:2], x[:2], v[:2], eps2, 4)
    assert np.allclose(np.linalg.norm(g["acc"], axis=1), g["sc_acc"], rtol=1e-15)


def test_exact_tie_goes_to_smaller_id_and_lonely_particle(oracle_mod):
    # sink at the origin, two sources at exactly the same distance
    x = np.array([[0.0, 0, 0], [1.0, 0, 0], [-1.0, 0, 0], [0, 3.0, 0]])
    v = np.zeros((4, 3))
    m = np.ones(4)
    ids = np.array([10, 7, 5, 1], dtype=np.int32)
    f = oracle_mod.forces(ids[:1], x[:1], v[:1], ids, m, x, v, 0.0, 4)
    assert f["nn_id"][0] == 5 and f["nn_r2"][0] == 1.0
    assert np.allclose(f["acc"][0], [0.0, 1.0 / 9.0, 0.0], atol=1e-16)
    # a particle alone (only itself as a source): no neighbour, zero force
    g = oracle_mod.forces(ids[:1], x[:1], v[:1], ids[:1], m[:1], x[:1], v[:1], 0.0, 4)
    assert g["nn_id"][0] == -1 and np.isinf(g["nn_r2"][0])
    assert np.all(g["acc"] == 0) and g["pot"][0] == 0
