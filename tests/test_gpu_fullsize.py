"""GPU parity at the full workload sizes, in the autotuned launch shapes the
benchmark uses, checked on sampled sinks the oracle computes one by one.

N = 131072 Plummer, eps = 1e-4, Hermite-4, N_active in {1, 8, 64, 1024, 16384,
131072}, mixed and FP64; N = 65536 Salpeter Plummer, Hermite-6 with a, jerk,
snap from one oracle pass, N_active in {32, 4096, 65536}, mixed and FP64."""
import numpy as np
import pytest

from _parity import check, oracle_ref, state

pytestmark = pytest.mark.gpu
SAMPLE = 192


@pytest.fixture(scope="module")
def sp2():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1510_04068_gb300 import build, sp2 as mod
    build.build()
    mod.load()
    return mod


def _run_full(sp2, s, order, prec, eps2, n_active, seed):
    import torch
    n = len(s["m"])
    D = lambda a: None if a is None else torch.as_tensor(np.ascontiguousarray(a)).cuda()  # noqa: E731
    idx = np.sort(np.random.default_rng(seed).choice(n, n_active, replace=False)).astype(np.int32)
    with sp2.Context(order=order, precision=prec, n_max=n, eps2=eps2) as c:
        c.set_j(0, D(s["ids"]), D(s["m"]), D(s["x"]), D(s["v"]), D(s["a"]), D(s["jerk"]),
                D(s["snap"]) if order == 6 else None, D(s["tj"]))
        c.predict(s["t"])
        if prec == sp2.SP2_MIXED or n_active <= 4096:
            c.autotune(n_active)
        out = dict(acc=torch.empty((n_active, 3), dtype=torch.float64, device="cuda"),
                   jerk=torch.empty((n_active, 3), dtype=torch.float64, device="cuda"),
                   snap=torch.empty((n_active, 3), dtype=torch.float64, device="cuda") if order == 6 else None,
                   pot=torch.empty(n_active, dtype=torch.float64, device="cuda"),
                   nn_id=torch.empty(n_active, dtype=torch.int32, device="cuda"),
                   nn_r2=torch.empty(n_active, dtype=torch.float64, device="cuda"))
        c.compute(D(idx), **out)
        c.sync()
        g = {k: (None if v is None else v.cpu().numpy()) for k, v in out.items()}
    return idx, g


def _sample(idx, g, seed):
    q = np.sort(np.random.default_rng(seed).choice(len(idx), min(SAMPLE, len(idx)), replace=False))
    return q, {k: (None if v is None else v[q]) for k, v in g.items()}


@pytest.fixture(scope="module")
def plummer_131k():
    return state(131072, 0, t=1.0)


@pytest.mark.parametrize("mixed", [True, False])
@pytest.mark.parametrize("n_active", [1, 8, 64, 1024, 16384, 131072])
def test_plummer_131072_block_steps(sp2, oracle_mod, plummer_131k, mixed, n_active):
    s = plummer_131k
    eps2 = 1e-8
    prec = sp2.SP2_MIXED if mixed else sp2.SP2_FP64
    idx, g = _run_full(sp2, s, 4, prec, eps2, n_active, 1000 + n_active)
    q, gs = _sample(idx, g, n_active)
    r = oracle_ref(oracle_mod, s, idx[q], order=4, eps2=eps2)
    check(gs, r, order=4, mixed=mixed, s=s, i_idx=idx[q], label=f"C2/{n_active}/{mixed}")
    assert np.all(np.isfinite(g["acc"])) and np.all(g["nn_id"] >= 0)


@pytest.fixture(scope="module")
def salpeter_65k(oracle_mod):
    return state(65536, 3, order=6, salpeter=True, derivs="oracle", oracle=oracle_mod, eps2=1e-8, t=0.5)


@pytest.mark.parametrize("mixed", [True, False])
@pytest.mark.parametrize("n_active", [32, 4096, 65536])
def test_salpeter_65536_sixth_order(sp2, oracle_mod, salpeter_65k, mixed, n_active):
    s = salpeter_65k
    eps2 = 1e-8
    prec = sp2.SP2_MIXED if mixed else sp2.SP2_FP64
    idx, g = _run_full(sp2, s, 6, prec, eps2, n_active, 2000 + n_active)
    q, gs = _sample(idx, g, n_active + 1)
    r = oracle_ref(oracle_mod, s, idx[q], order=6, eps2=eps2)
    check(gs, r, order=6, mixed=mixed, s=s, i_idx=idx[q], label=f"C3/{n_active}/{mixed}")
    assert np.all(np.isfinite(g["snap"]))
