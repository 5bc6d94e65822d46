"""Pins: energy conservation of a shared-step Hermite-4 run driven by the oracle,
and the oracle's autograd gradient against central finite differences."""
import numpy as np
import pytest

import workloads as W


def test_hermite4_energy_conservation_fourth_order(oracle_mod):
    """Plummer N = 1024, eps = 1e-3, integrated to t = 1/8: the relative energy
    error is small and falls by ~2^4 per halving of dt (4th-order scheme)."""
    m, x, v = W.plummer(1024, 0)
    eps2 = 1e-6
    E0 = oracle_mod.energy(m, x, v, eps2)
    errs = []
    for dt in (2.0 ** -8, 2.0 ** -9):
        xf, vf = oracle_mod.hermite4_shared(m, x, v, eps2, dt, int(round(0.125 / dt)))
        errs.append(abs((oracle_mod.energy(m, xf, vf, eps2) - E0) / E0))
    assert errs[1] < 1e-5
    assert 10.0 < errs[0] / errs[1] < 40.0, errs


def test_autograd_gradient_matches_finite_differences(oracle_mod):
    """The torch restatement's gradient of L = sum w . x_final w.r.t. (x0, v0, m)
    agrees with central differences (h = 1e-6) of the C oracle's trajectory, to
    1e-6 relative (to max(|g|, 1e-3 max|g|)) above the difference's round-off."""
    torch = pytest.importorskip("torch")
    from oracle import adjoint
    n, steps, dt, eps2 = 48, 8, 1.0 / 256, 1e-4
    m, x, v = W.plummer(n, 21)
    w = np.random.default_rng(22).standard_normal((n, 3))
    L, gx, gv, gm = adjoint.loss_and_grad(x, v, m, w, eps2, dt, steps)

    def loss(xx, vv, mm):
        xf, _ = oracle_mod.hermite4_shared(mm, xx, vv, eps2, dt, steps)
        return float(np.sum(w * xf))

    assert abs(loss(x, v, m) - L) <= 1e-12 * abs(L)
    # round-off floor of a central difference: the loss is a sum of |w . x| terms,
    # each evaluated with relative error ~u, so (L+ - L-) / 2h carries ~u sum|w x| / h
    xf, _ = oracle_mod.hermite4_shared(m, x, v, eps2, dt, steps)
    noise = 8 * np.finfo(float).eps * np.sum(np.abs(w * xf)) / (2 * 1e-6)
    rng = np.random.default_rng(23)
    h = 1e-6
    for _ in range(24):
        kind = rng.integers(0, 3)
        i = int(rng.integers(0, n))
        c = int(rng.integers(0, 3))
        xx, vv, mm = x.copy(), v.copy(), m.copy()
        tgt, g = ((xx, gx[i, c]) if kind == 0 else (vv, gv[i, c]) if kind == 1 else (mm, gm[i]))
        idx = (i, c) if kind < 2 else (i,)
        base = tgt[idx]
        tgt[idx] = base + h
        lp = loss(xx, vv, mm)
        tgt[idx] = base - h
        lm = loss(xx, vv, mm)
        fd = (lp - lm) / (2 * h)
        scale = max(abs(g), 1e-3 * max(np.abs(gx).max(), np.abs(gv).max(), np.abs(gm).max()))
        assert abs(fd - g) <= 1e-6 * scale + noise, (kind, i, c, fd, g)
