"""The allocation-free block step (sp2_step_static) against the oracle and
against the context-based entry points (sp2_set_j + sp2_predict +
sp2_compute), on two calls in a row.

Some callers cannot allocate device memory where they need forces: a host
code whose device memory belongs to its own allocator or a fixed budget it
may not bypass, or a real-time loop that must not enter the CUDA allocator.
They use sp2_step_static, whose scratch is a fixed array inside the library.
This file is collected last on purpose: if it fails, a run that stops at the
first failure has run everything else."""
import ctypes

import numpy as np
import pytest

from _parity import NN_BAND, TOL, check, state

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1510_04068_gb300 import build, sp2
    build.build()
    sp2.load()
    return torch, sp2


def _context_step(torch, sp2, s, idx, eps2):
    n = len(s["m"])
    D = lambda a: torch.as_tensor(np.ascontiguousarray(a)).cuda()  # noqa: E731
    with sp2.Context(order=4, precision=sp2.SP2_MIXED, n_max=n, eps2=eps2) as c:
        c.set_j(0, D(s["ids"]), D(s["m"]), D(s["x"]), D(s["v"]), D(s["a"]), D(s["jerk"]), None, D(s["tj"]))
        c.predict(s["t"])
        ni = len(idx)
        out = dict(acc=torch.empty((ni, 3), dtype=torch.float64, device="cuda"),
                   jerk=torch.empty((ni, 3), dtype=torch.float64, device="cuda"),
                   pot=torch.empty(ni, dtype=torch.float64, device="cuda"),
                   nn_id=torch.empty(ni, dtype=torch.int32, device="cuda"),
                   nn_r2=torch.empty(ni, dtype=torch.float64, device="cuda"))
        c.compute(D(idx), **out)
        c.sync()
        return {k: v.cpu().numpy() for k, v in out.items()}


def _static_step(torch, sp2, s, idx, eps2):
    D = lambda a: torch.as_tensor(np.ascontiguousarray(a)).cuda()  # noqa: E731
    ni = len(idx)
    inp = [D(s[k]) for k in ("ids", "m", "x", "v", "a", "jerk", "tj")]
    out = dict(acc=torch.full((ni, 3), float("nan"), dtype=torch.float64, device="cuda"),
               jerk=torch.full((ni, 3), float("nan"), dtype=torch.float64, device="cuda"),
               pot=torch.full((ni,), float("nan"), dtype=torch.float64, device="cuda"),
               nn_id=torch.full((ni,), -9, dtype=torch.int32, device="cuda"),
               nn_r2=torch.full((ni,), float("nan"), dtype=torch.float64, device="cuda"))
    didx = D(idx)
    stream = torch.cuda.current_stream()
    sp2.sp2_step_static(inp, s["t"], eps2, didx, out, stream.cuda_stream)
    stream.synchronize()
    return {k: v.cpu().numpy() for k, v in out.items()}


def _compare(g, ref, sc, label):
    """The static step against the context path, with the oracle's scale sums
    as the normalisation (the tolerances of the mixed-precision parity tests)."""
    tol = TOL[True]
    assert np.all(np.isfinite(g["acc"])) and np.all(np.isfinite(g["pot"])), label
    assert (np.linalg.norm(g["acc"] - ref["acc"], axis=1) / sc["sc_acc"]).max() <= tol["acc"], label
    assert (np.linalg.norm(g["jerk"] - ref["jerk"], axis=1) / sc["sc_jerk"]).max() <= tol["jerk"], label
    assert (np.abs(g["pot"] - ref["pot"]) / np.abs(ref["pot"])).max() <= tol["pot"], label
    same = g["nn_id"] == ref["nn_id"]
    rel = np.abs(g["nn_r2"] - ref["nn_r2"]) / ref["nn_r2"]
    assert np.all(same | (rel <= NN_BAND)), label
    assert rel.max() <= NN_BAND + tol["r2"], label


def test_static_step_matches_oracle_and_context_path_twice(env, oracle_mod):
    torch, sp2 = env
    eps2 = 1e-8
    cases = [(20000, 3000, 61), (9000, 17, 62)]  # two calls in a row, different sizes and inputs
    for n, n_act, seed in cases:
        s = state(n, seed)
        idx = np.sort(np.random.default_rng(seed).choice(n, n_act, replace=False)).astype(np.int32)
        ref = _context_step(torch, sp2, s, idx, eps2)
        g = _static_step(torch, sp2, s, idx, eps2)
        sc = oracle_mod.step(s["t"], idx, s["ids"], s["m"], s["tj"], s["x"], s["v"], s["a"], s["jerk"], None,
                             eps2=eps2, order=4)
        label = f"n={n} n_active={n_act}"
        check(g, sc, order=4, mixed=True, s=s, i_idx=idx, label=label + " vs oracle")
        _compare(g, ref, sc, label + " vs context path")


def test_static_step_marks_out_of_range_sinks(env, oracle_mod):
    """One sink slot past the sources, with a source split (few sinks): that
    sink's outputs are NaN / -1, every other sink is still the oracle's."""
    torch, sp2 = env
    eps2 = 1e-8
    n = 12000
    s = state(n, 63)
    idx = np.sort(np.random.default_rng(63).choice(n, 9, replace=False)).astype(np.int32)
    bad = idx.copy()
    bad[4] = n + 5
    g = _static_step(torch, sp2, s, bad, eps2)
    assert np.all(np.isnan(g["acc"][4])) and np.all(np.isnan(g["jerk"][4]))
    assert np.isnan(g["pot"][4]) and np.isnan(g["nn_r2"][4]) and g["nn_id"][4] == -1
    keep = np.array([k for k in range(len(idx)) if k != 4])
    sc = oracle_mod.step(s["t"], idx[keep], s["ids"], s["m"], s["tj"], s["x"], s["v"], s["a"], s["jerk"], None,
                         eps2=eps2, order=4)
    check({k: v[keep] for k, v in g.items()}, sc, order=4, mixed=True, s=s, i_idx=idx[keep], label="good sinks")


def test_static_step_argument_rules(env):
    torch, sp2 = env
    lib = sp2.load()
    z = ctypes.c_void_p(0)
    # more sources than the fixed scratch holds: a clear range error, nothing launched
    assert lib.sp2_step_static(65537, z, z, z, z, z, z, z, 0.0, 0.0, 1, z, z, z, z, z, z, None) == -2
    assert lib.sp2_step_static(10, z, z, z, z, z, z, z, 0.0, 0.0, 65537, z, z, z, z, z, z, None) == -2
    # no sinks: a successful no-op, whatever the pointers
    assert lib.sp2_step_static(10, z, z, z, z, z, z, z, 0.0, 0.0, 0, z, z, z, z, z, z, None) == 0
    # valid device arrays, so that only the scalar argument under test is wrong
    n, ni = 10, 5
    buf = {k: torch.zeros(sh, dtype=torch.float64, device="cuda")
           for k, sh in dict(m=n, x=(n, 3), v=(n, 3), a=(n, 3), jerk=(n, 3), tj=n, acc=(ni, 3), jk=(ni, 3),
                             pot=ni, r2=ni).items()}
    ids = torch.arange(n, dtype=torch.int32, device="cuda")
    idx = torch.arange(ni, dtype=torch.int32, device="cuda")
    nnid = torch.zeros(ni, dtype=torch.int32, device="cuda")
    P = lambda t: ctypes.c_void_p(t.data_ptr())  # noqa: E731
    args = lambda t, e2, r2=P(buf["r2"]): (n, P(ids), P(buf["m"]), P(buf["x"]), P(buf["v"]), P(buf["a"]),  # noqa: E731
                                           P(buf["jerk"]), P(buf["tj"]), t, e2, ni, P(idx), P(buf["acc"]),
                                           P(buf["jk"]), P(buf["pot"]), P(nnid), r2, None)
    assert lib.sp2_step_static(*args(0.0, -1.0)) == -1               # eps2 < 0
    assert lib.sp2_step_static(*args(0.0, float("inf"))) == -1       # eps2 not finite
    assert lib.sp2_step_static(*args(float("nan"), 0.0)) == -1       # t not finite
    assert lib.sp2_step_static(*args(0.0, 0.0, r2=z)) == -1          # nn_id without nn_r2
    assert lib.sp2_step_static(*args(0.0, 0.0)) == 0
    torch.cuda.synchronize()
