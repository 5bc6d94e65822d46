"""Pins of the oracle's block time-step Hermite-4 integrator (Sec. 3.7).

With a criterion that never asks for less than dt_max, every particle steps
together and the block integrator is the shared-step one, bit for bit (a
special case pinned elsewhere); with the Aarseth criterion the steps are
powers of two that divide the particles' times, the energy is conserved and
its error shrinks when eta does."""
import numpy as np

import workloads as W


def test_reduces_to_shared_steps(oracle_mod):
    n, eps2 = 64, 1e-2
    m, x, v = W.plummer(n, 4)
    dt = 2.0 ** -7
    xs, vs = oracle_mod.hermite4_shared(m, x, v, eps2, dt, 8)
    xb, vb, tb, st = oracle_mod.hermite4_block(m, x, v, eps2, 8 * dt, 1e30, 1e30, dt)
    assert st["block_steps"] == 8 and st["active_sum"] == 8 * n
    assert np.all(tb == 8 * dt)
    assert np.array_equal(xb, xs) and np.array_equal(vb, vs)


def test_steps_are_commensurate_powers_of_two(oracle_mod):
    n, eps2 = 128, 1e-3
    m, x, v = W.plummer(n, 6)
    _, _, t, st = oracle_mod.hermite4_block(m, x, v, eps2, 2.0 ** -5, 0.01, 0.01, 2.0 ** -6)
    dt = st["dt"]
    assert np.all(np.log2(dt) == np.round(np.log2(dt)))
    assert np.all(np.fmod(t, dt) == 0.0)
    assert np.all(t <= 2.0 ** -5) and np.all(t + dt > 2.0 ** -5)
    assert st["active_sum"] > st["block_steps"]  # blocks hold several particles on average
    assert len(np.unique(dt)) > 1  # and the steps differ between particles


def test_energy_error_shrinks_with_eta(oracle_mod):
    n, eps2 = 128, 1e-3
    m, x, v = W.plummer(n, 8)
    e0 = oracle_mod.energy(m, x, v, eps2)
    errs = []
    for eta in (0.08, 0.005):
        xb, vb, t, _ = oracle_mod.hermite4_block(m, x, v, eps2, 2.0 ** -3, eta, 0.01, 2.0 ** -5)
        assert np.all(t == 2.0 ** -3)  # t_end is a multiple of dt_max: everyone arrives
        errs.append(abs(oracle_mod.energy(m, xb, vb, eps2) / e0 - 1.0))
    # a 4th-order scheme: steps ~ sqrt(eta), error ~ eta^2 -- 16x smaller eta, far smaller error
    assert errs[1] < 1e-8
    assert errs[1] < errs[0] / 20
