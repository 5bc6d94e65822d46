"""GPU parity of the order-2 (leap-frog / GRAPE-5, Sec. 1) pass: acceleration,
potential and nearest neighbour of sources at their stored positions, against
the oracle's direct sum (its acceleration and potential do not depend on the
velocities, which are zero here).  Both precisions, several sink counts and
launch shapes, the batched pass, and the argument rules of order 2."""
import numpy as np
import pytest

import workloads as W
from _parity import NN_BAND, TOL

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


def _oracle(oracle, ids, m, x, idx, eps2):
    z = np.zeros_like(x)
    return oracle.forces(ids[idx], x[idx], z[idx], ids, m, x, z, eps2, 4)


def _check(g, r, mixed, x, ids, idx):
    tol = TOL[bool(mixed)]
    e_acc = np.linalg.norm(g["acc"] - r["acc"], axis=1) / r["sc_acc"]
    e_pot = np.abs(g["pot"] - r["pot"]) / np.abs(r["pot"])
    assert e_acc.max() <= tol["acc"], e_acc.max()
    assert e_pot.max() <= tol["pot"], e_pot.max()
    bad = np.flatnonzero(g["nn_id"] != r["nn_id"])
    if not mixed:
        assert bad.size == 0
        assert np.allclose(g["nn_r2"], r["nn_r2"], rtol=1e-15, atol=0)
        return
    pos = {int(k): q for q, k in enumerate(ids)}
    for q in bad:
        d = float(np.sum((x[pos[int(g["nn_id"][q])]] - x[idx[q]]) ** 2))
        assert d - r["nn_r2"][q] <= NN_BAND * r["nn_r2"][q]


def _ctx(sp2, precision, n, eps2, ids, m, x, device, with_v=False):
    import torch
    c = sp2.Context(order=2, precision=precision, n_max=n, eps2=eps2)
    conv = (lambda a: torch.as_tensor(np.ascontiguousarray(a)).cuda()) if device else np.ascontiguousarray
    if with_v:  # velocities etc. may be given; they are not used
        rng = np.random.default_rng(0)
        v = rng.normal(size=x.shape)
        c.set_j(0, conv(ids), conv(m), conv(x), conv(v), conv(v), conv(v), None, conv(np.ones(n)))
    else:
        c.set_j(0, conv(ids), conv(m), conv(x), None, None, None, None, None)
    c.predict(0.0)
    return c


@pytest.mark.parametrize("mixed", [False, True])
@pytest.mark.parametrize("n,n_active", [(3000, 3000), (4099, 3), (5000, 257)])
def test_leapfrog_forces(sp2, oracle_mod, mixed, n, n_active):
    import torch
    eps2 = 1e-8
    m, x, _ = W.plummer(n, 40 + n_active)
    ids = W.particle_ids(n, 7)
    idx = np.sort(np.random.default_rng(n_active).choice(n, n_active, replace=False)).astype(np.int32)
    c = _ctx(sp2, sp2.SP2_MIXED if mixed else sp2.SP2_FP64, n, eps2, ids, m, x, True, with_v=(n_active == 3))
    z = lambda *sh, dt=torch.float64: torch.empty(sh, dtype=dt, device="cuda")  # noqa: E731
    out = dict(acc=z(n_active, 3), pot=z(n_active), nn_id=z(n_active, dt=torch.int32), nn_r2=z(n_active))
    c.compute(torch.as_tensor(idx).cuda(), **out)
    c.sync()
    g = {k: v.cpu().numpy() for k, v in out.items()}
    c.close()
    _check(g, _oracle(oracle_mod, ids, m, x, idx, eps2), mixed, x, ids, idx)


@pytest.mark.parametrize("launch", [dict(threads=128, i_per_thread=2, j_lanes=1, j_tile=256, split_j=5, ctas_per_sm=0),
                                    dict(threads=64, i_per_thread=1, j_lanes=8, j_tile=64, split_j=40, ctas_per_sm=0)])
def test_leapfrog_host_pointers_and_shapes(sp2, oracle_mod, launch):
    n, eps2 = 2500, 1e-6
    m, x, _ = W.plummer(n, 77)
    ids = W.particle_ids(n, 8)
    idx = np.arange(0, n, 3, dtype=np.int32)
    c = _ctx(sp2, sp2.SP2_MIXED, n, eps2, ids, m, x, False)
    c.set_launch(len(idx), launch)
    g = dict(acc=np.empty((len(idx), 3)), pot=np.empty(len(idx)), nn_id=np.empty(len(idx), np.int32),
             nn_r2=np.empty(len(idx)))
    c.compute(idx, **g)
    c.close()
    _check(g, _oracle(oracle_mod, ids, m, x, idx, eps2), True, x, ids, idx)


def test_leapfrog_batched(sp2, oracle_mod):
    import torch
    sizes = [3, 17, 64, 100, 5]
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    n = int(off[-1])
    m, x, _ = W.plummer(n, 5)
    ids = np.arange(n, dtype=np.int32)
    c = _ctx(sp2, sp2.SP2_MIXED, n, 1e-6, ids, m, x, True)
    plan = c.batch_plan(off)
    out = dict(acc=torch.empty((n, 3), dtype=torch.float64, device="cuda"),
               pot=torch.empty(n, dtype=torch.float64, device="cuda"))
    c.compute_batched(plan, **out)
    c.sync()
    for s in range(len(sizes)):
        sl = slice(off[s], off[s + 1])
        z = np.zeros((sizes[s], 3))
        r = oracle_mod.forces(ids[sl], x[sl], z, ids[sl], m[sl], x[sl], z, 1e-6, 4)
        e = np.linalg.norm(out["acc"][sl].cpu().numpy() - r["acc"], axis=1) / np.maximum(r["sc_acc"], 1e-300)
        assert e.max() <= 1e-6
    sp2.sp2_batch_plan_destroy(plan)
    c.close()


def test_leapfrog_argument_rules(sp2):
    import torch
    n = 100
    m, x, _ = W.plummer(n, 1)
    ids = np.arange(n, dtype=np.int32)
    c = _ctx(sp2, sp2.SP2_FP64, n, 1e-6, ids, m, x, True)
    idx = torch.arange(10, dtype=torch.int32, device="cuda")
    with pytest.raises(sp2.SP2Error):  # no jerk at order 2
        c.compute(idx, acc=torch.empty((10, 3), dtype=torch.float64, device="cuda"),
                  jerk=torch.empty((10, 3), dtype=torch.float64, device="cuda"))
    c.close()
    c = sp2.Context(order=4, precision=sp2.SP2_FP64, n_max=n, eps2=1e-6)
    D = lambda a: torch.as_tensor(np.ascontiguousarray(a)).cuda()  # noqa: E731
    with pytest.raises(sp2.SP2Error):  # order 4 still needs v, a, jerk, t
        c.set_j(0, D(ids), D(m), D(x), None, None, None, None, None)
    c.close()
