"""The source split over several devices (Sec. 2.2.3), with the devices'
shares run one after another on one GPU: each share is the force pass over a
contiguous block of sources (shards.compute_shard), the shares' outputs are
partial sums and partial nearest neighbours, and adding them (lexicographic
(r^2, id) minimum for the neighbour) gives the oracle's full result.  The
exchange between processes is covered by the two-rank CPU test."""
import numpy as np
import pytest

from _parity import check, oracle_ref, state

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1510_04068_gb300 import build, shards, sp2
    build.build()
    sp2.load()
    return torch, sp2, shards


@pytest.mark.parametrize("world", [2, 3])
@pytest.mark.parametrize("order", [4, 6])
@pytest.mark.parametrize("mixed", [False, True])
def test_shares_add_up_to_the_oracle(env, oracle_mod, world, order, mixed):
    torch, sp2, shards = env
    n, n_i, eps2 = 5003, 300, 1e-8
    s = state(n, 40 + world, order=order, salpeter=(order == 6))
    idx = np.sort(np.random.default_rng(world).choice(n, n_i, replace=False)).astype(np.int32)
    D = lambda a: None if a is None else torch.as_tensor(np.ascontiguousarray(a)).cuda()  # noqa: E731
    parts = []
    blocks = []
    with sp2.Context(order=order, precision=sp2.SP2_MIXED if mixed else sp2.SP2_FP64, n_max=n, eps2=eps2) as c:
        c.set_j(0, D(s["ids"]), D(s["m"]), D(s["x"]), D(s["v"]), D(s["a"]), D(s["jerk"]), D(s["snap"]), D(s["tj"]))
        c.predict(s["t"])
        for rank in range(world):
            out = dict(acc=torch.empty((n_i, 3), dtype=torch.float64, device="cuda"),
                       jerk=torch.empty((n_i, 3), dtype=torch.float64, device="cuda"),
                       snap=torch.empty((n_i, 3), dtype=torch.float64, device="cuda") if order == 6 else None,
                       pot=torch.empty(n_i, dtype=torch.float64, device="cuda"),
                       nn_id=torch.empty(n_i, dtype=torch.int32, device="cuda"),
                       nn_r2=torch.empty(n_i, dtype=torch.float64, device="cuda"))
            blocks.append(shards.compute_shard(c, D(idx), rank, world, **out))
            c.sync()
            parts.append({k: (None if v is None else v.cpu().numpy()) for k, v in out.items()})
    # the blocks tile the sources
    assert blocks[0][0] == 0 and blocks[-1][1] == n
    assert all(blocks[r][1] == blocks[r + 1][0] for r in range(world - 1))
    g = {k: sum(p[k] for p in parts) for k in ("acc", "jerk", "pot") + (("snap",) if order == 6 else ())}
    r2 = np.stack([p["nn_r2"] for p in parts])
    ids = np.stack([p["nn_id"] for p in parts]).astype(np.int64)
    ids_key = np.where(ids < 0, np.iinfo(np.int64).max, ids)
    best = np.lexsort((ids_key, r2), axis=0)[0]
    g["nn_r2"] = r2[best, np.arange(n_i)]
    g["nn_id"] = ids[best, np.arange(n_i)].astype(np.int32)
    # each share is itself the oracle's sum over its block
    lo, hi = blocks[1]
    rp = oracle_ref(oracle_mod, s, idx, order=order, eps2=eps2, j_range=(lo, hi))
    r = oracle_ref(oracle_mod, s, idx, order=order, eps2=eps2)
    check(g, r, order=order, mixed=mixed, s=s, i_idx=idx, label=f"world={world}")
    e = np.linalg.norm(parts[1]["acc"] - rp["acc"], axis=1) / r["sc_acc"]
    assert e.max() <= (1e-6 if mixed else 1e-12)
