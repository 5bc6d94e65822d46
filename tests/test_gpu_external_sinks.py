"""GPU parity of forces on explicit sinks (sp2_compute_ext, the GRAPE-style
call): sinks given by their own predicted state, either loaded particles
(slot given, self pair skipped) or arbitrary points (no slot), against the
oracle's direct sum over the predicted sources."""
import numpy as np
import pytest

from _parity import check, oracle_ref, state

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sp2():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1510_04068_gb300 import build, sp2 as mod
    build.build()
    mod.load()
    return mod


def _ctx(sp2, s, order, precision, eps2, device):
    import torch
    n = len(s["m"])
    conv = (lambda a: None if a is None else torch.as_tensor(np.ascontiguousarray(a)).cuda()) if device else \
        (lambda a: None if a is None else np.ascontiguousarray(a))
    c = sp2.Context(order=order, precision=precision, n_max=n, eps2=eps2)
    c.set_j(0, conv(s["ids"]), conv(s["m"]), conv(s["x"]), conv(s["v"]), conv(s["a"]), conv(s["jerk"]),
            conv(s["snap"]) if order == 6 else None, conv(s["tj"]))
    c.predict(s["t"])
    return c, conv


def _outs(n_i, order, device):
    import torch
    if device:
        z = lambda *sh, dt=torch.float64: torch.empty(sh, dtype=dt, device="cuda")  # noqa: E731
    else:
        z = lambda *sh, dt=np.float64: np.empty(sh, dtype=dt)  # noqa: E731
    i4 = torch.int32 if device else np.int32
    return dict(acc=z(n_i, 3), jerk=z(n_i, 3), snap=z(n_i, 3) if order == 6 else None, pot=z(n_i),
                nn_id=z(n_i, dt=i4), nn_r2=z(n_i))


def _np(o):
    return {k: (None if v is None else (v.cpu().numpy() if hasattr(v, "cpu") else v)) for k, v in o.items()}


@pytest.mark.parametrize("order", [4, 6])
@pytest.mark.parametrize("mixed", [False, True])
@pytest.mark.parametrize("n_i", [1, 300])
def test_loaded_particles_as_explicit_sinks(sp2, oracle_mod, order, mixed, n_i):
    from oracle import predict
    n, eps2 = 4001, 1e-8
    s = state(n, 60 + n_i, order=order)
    idx = np.sort(np.random.default_rng(n_i).choice(n, n_i, replace=False)).astype(np.int32)
    xp, vp, ap = predict(s["t"], s["tj"], s["x"], s["v"], s["a"], s["jerk"], s["snap"], order)
    c, conv = _ctx(sp2, s, order, sp2.SP2_MIXED if mixed else sp2.SP2_FP64, eps2, True)
    o = _outs(n_i, order, True)
    c.compute_ext(conv(xp[idx]), conv(vp[idx]), conv(ap[idx]) if order == 6 else None, i_slot=conv(idx), **o)
    c.close()
    check(_np(o), oracle_ref(oracle_mod, s, idx, order=order, eps2=eps2), order=order, mixed=mixed, s=s, i_idx=idx,
          label="explicit loaded sinks")


@pytest.mark.parametrize("mixed", [False, True])
@pytest.mark.parametrize("device", [True, False])
def test_points_outside_the_set(sp2, oracle_mod, mixed, device):
    from oracle import predict
    n, eps2, n_i = 3000, 1e-6, 77
    s = state(n, 5)
    rng = np.random.default_rng(8)
    xi = rng.normal(scale=0.5, size=(n_i, 3))
    vi = rng.normal(scale=0.3, size=(n_i, 3))
    xp, vp, _ = predict(s["t"], s["tj"], s["x"], s["v"], s["a"], s["jerk"], None, 4)
    r = oracle_mod.forces(-1 - np.arange(n_i, dtype=np.int32), xi, vi, s["ids"], s["m"], xp, vp, eps2, 4)
    c, conv = _ctx(sp2, s, 4, sp2.SP2_MIXED if mixed else sp2.SP2_FP64, eps2, device)
    o = _outs(n_i, 4, device)
    c.compute_ext(conv(xi), conv(vi), None, **o)
    c.close()
    g = _np(o)
    gid, gr2 = g.pop("nn_id"), g.pop("nn_r2")
    check(g, r, order=4, mixed=mixed, label="outside points")
    pos = {int(k): q for q, k in enumerate(s["ids"])}
    for q in range(n_i):
        d = float(np.sum((xp[pos[int(gid[q])]] - xi[q]) ** 2))
        if mixed:
            assert d - r["nn_r2"][q] <= 1e-5 * r["nn_r2"][q]
            assert abs(gr2[q] - d) <= 1e-5 * d
        else:
            assert gid[q] == r["nn_id"][q] and gr2[q] == r["nn_r2"][q]


def test_leapfrog_explicit_sinks(sp2, oracle_mod):
    import torch
    import workloads as W
    n, eps2 = 2000, 1e-6
    m, x, _ = W.plummer(n, 4)
    ids = np.arange(n, dtype=np.int32)
    c = sp2.Context(order=2, precision=sp2.SP2_MIXED, n_max=n, eps2=eps2)
    D = lambda a: torch.as_tensor(np.ascontiguousarray(a)).cuda()  # noqa: E731
    c.set_j(0, D(ids), D(m), D(x), None, None, None, None, None)
    c.predict(0.0)
    xi = np.random.default_rng(3).normal(scale=0.5, size=(50, 3))
    acc = torch.empty((50, 3), dtype=torch.float64, device="cuda")
    pot = torch.empty(50, dtype=torch.float64, device="cuda")
    c.compute_ext(D(xi), acc=acc, pot=pot)
    c.close()
    z = np.zeros((50, 3))
    r = oracle_mod.forces(-1 - np.arange(50, dtype=np.int32), xi, z, ids, m, x, np.zeros_like(x), eps2, 4)
    e = np.linalg.norm(acc.cpu().numpy() - r["acc"], axis=1) / r["sc_acc"]
    assert e.max() <= 1e-6
    assert np.max(np.abs(pot.cpu().numpy() - r["pot"]) / np.abs(r["pot"])) <= 1e-6
