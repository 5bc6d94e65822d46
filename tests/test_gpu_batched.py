"""GPU parity of the batched persistent kernel: 4096 independent star + planets
systems (N log-uniform in [3, 256], eps = 0, every body active) against the
oracle system by system, in both precisions."""
import numpy as np
import pytest

import workloads as W
from _parity import check

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


def _systems(n_sys, seed):
    offsets, m, x, v = W.planetary_systems(n_sys, seed)
    total = int(offsets[-1])
    rng = np.random.default_rng(seed + 1)
    a = 1e-3 * rng.standard_normal((total, 3))
    jk = 1e-3 * rng.standard_normal((total, 3))
    return dict(offsets=offsets, m=m, x=x, v=v, a=a, jerk=jk, snap=None, ids=W.particle_ids(total, seed + 2),
                tj=np.full(total, -1.0 / 64), t=0.0)


def _run(sp2, s, prec, graph=False, order=4):
    import torch
    total = len(s["m"])
    D = lambda q: torch.as_tensor(np.ascontiguousarray(q)).cuda()  # noqa: E731
    with sp2.Context(order=order, precision=prec, n_max=total, eps2=0.0) as c:
        c.set_j(0, D(s["ids"]), D(s["m"]), D(s["x"]), D(s["v"]), D(s["a"]), D(s["jerk"]),
                D(s["snap"]) if order == 6 else None, D(s["tj"]))
        plan = c.batch_plan(s["offsets"])
        out = dict(acc=torch.empty((total, 3), dtype=torch.float64, device="cuda"),
                   jerk=torch.empty((total, 3), dtype=torch.float64, device="cuda"),
                   snap=torch.empty((total, 3), dtype=torch.float64, device="cuda") if order == 6 else None,
                   pot=torch.empty(total, dtype=torch.float64, device="cuda"),
                   nn_id=torch.empty(total, dtype=torch.int32, device="cuda"),
                   nn_r2=torch.empty(total, dtype=torch.float64, device="cuda"))
        if graph:
            sp2.sp2_graph_begin(c.ctx)
            c.predict(s["t"])
            c.compute_batched(plan, **out)
            g = sp2.sp2_graph_end(c.ctx)
            for v in out.values():
                if v is not None:
                    v.fill_(float("nan")) if v.dtype == torch.float64 else v.fill_(-7)
            sp2.sp2_graph_launch(c.ctx, g)
            sp2.sp2_graph_launch(c.ctx, g)
            c.sync()
            sp2.sp2_graph_destroy(g)
        else:
            c.predict(s["t"])
            c.compute_batched(plan, **out)
            c.sync()
        sp2.sp2_batch_plan_destroy(plan)
        return {k: (None if v is None else v.cpu().numpy()) for k, v in out.items()}


def _check_all(oracle_mod, s, g, mixed, order=4):
    off = s["offsets"]
    for sys_ in range(len(off) - 1):
        a, b = int(off[sys_]), int(off[sys_ + 1])
        idx = np.arange(a, b)
        r = oracle_mod.step(s["t"], idx, s["ids"], s["m"], s["tj"], s["x"], s["v"], s["a"], s["jerk"], s["snap"],
                            eps2=0.0, order=order, j_range=(a, b))
        gs = {k: (None if v is None else v[a:b]) for k, v in g.items()}
        check(gs, r, order=order, mixed=mixed, s=s, i_idx=idx, label=f"system {sys_}")


@pytest.mark.parametrize("mixed", [True, False])
def test_4096_planetary_systems(sp2, oracle_mod, mixed):
    s = _systems(4096, 7)
    prec = sp2.SP2_MIXED if mixed else sp2.SP2_FP64
    g = _run(sp2, s, prec, graph=True)
    _check_all(oracle_mod, s, g, mixed)


@pytest.mark.parametrize("mixed", [True, False])
def test_batched_sixth_order_small(sp2, oracle_mod, mixed):
    s = _systems(300, 11)
    s["snap"] = 1e-3 * np.random.default_rng(5).standard_normal((len(s["m"]), 3))
    prec = sp2.SP2_MIXED if mixed else sp2.SP2_FP64
    g = _run(sp2, s, prec, order=6)
    _check_all(oracle_mod, s, g, mixed, order=6)


def test_batched_equals_per_system_launches(sp2):
    """The persistent batched kernel and one compute_range launch per system
    agree (the two are the batched path and its per-system baseline)."""
    import torch
    s = _systems(200, 3)
    total = len(s["m"])
    g = _run(sp2, s, sp2.SP2_FP64)
    D = lambda q: torch.as_tensor(np.ascontiguousarray(q)).cuda()  # noqa: E731
    with sp2.Context(order=4, precision=sp2.SP2_FP64, n_max=total, eps2=0.0) as c:
        c.set_j(0, D(s["ids"]), D(s["m"]), D(s["x"]), D(s["v"]), D(s["a"]), D(s["jerk"]), None, D(s["tj"]))
        c.predict(s["t"])
        acc = torch.empty((total, 3), dtype=torch.float64, device="cuda")
        nn = torch.empty(total, dtype=torch.int32, device="cuda")
        off = s["offsets"]
        for k in range(200):
            a, b = int(off[k]), int(off[k + 1])
            c.compute(D(np.arange(a, b, dtype=np.int32)), j_range=(a, b), acc=acc[a:b], nn_id=nn[a:b])
        c.sync()
        np.testing.assert_allclose(acc.cpu().numpy(), g["acc"], rtol=0, atol=1e-13 * np.abs(g["acc"]).max())
        assert np.array_equal(nn.cpu().numpy(), g["nn_id"])


def test_plan_validation(sp2):
    import torch
    n = 5000
    with sp2.Context(order=4, precision=sp2.SP2_MIXED, n_max=n, eps2=0.0) as c:
        z = torch.zeros((n, 3), dtype=torch.float64, device="cuda")
        c.set_j(0, torch.arange(n, dtype=torch.int32, device="cuda"), torch.ones(n, dtype=torch.float64, device="cuda"),
                torch.rand((n, 3), dtype=torch.float64, device="cuda"), z, z, z, None,
                torch.zeros(n, dtype=torch.float64, device="cuda"))
        with pytest.raises(sp2.SP2Error) as e:
            c.batch_plan([0, 4097])
        assert e.value.status == -2
        with pytest.raises(sp2.SP2Error) as e:
            c.batch_plan([0, 10, 5001])
        assert e.value.status == -2
        with pytest.raises(sp2.SP2Error) as e:
            c.batch_plan([0, 10, 5])
        assert e.value.status == -2
