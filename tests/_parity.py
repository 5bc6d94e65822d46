"""Shared helpers of the GPU parity tests: seeded inputs, the library call, and
the tolerance checks against the oracle.

Tolerances (errors of acc, jerk and snap are taken relative to the per-sink
scale sums, the sum over sources of each term's magnitude; of pot relative to
|pot|, whose terms share one sign):
  FP64 mode:   acc, jerk, snap: |d| / scale sum <= 1e-12; pot: |d| / |pot| <= 1e-12;
               nearest-neighbour id exact (ties go to the smaller id on both sides);
               nn_r2 bit-compatible (<= 1e-15 relative).
  mixed mode:  acc, pot <= 1e-6; jerk, snap <= 1e-5 (same normalisation);
               nn id exact unless the oracle's gap between best and runner-up is
               below 1e-5 relative, in which case the GPU's choice must itself lie
               within 1e-5 of the best distance; nn_r2 within 1e-6 of the exact
               distance of the chosen neighbour.
"""
from __future__ import annotations

import numpy as np

import workloads as W

TOL = {
    False: dict(acc=1e-12, jerk=1e-12, snap=1e-12, pot=1e-12, r2=1e-15),
    True: dict(acc=1e-6, jerk=1e-5, snap=1e-5, pot=1e-6, r2=1e-6),
}
NN_BAND = 1e-5


def state(n, seed, *, order=4, t=1.0, salpeter=False, ids_seed=None, quantum=2.0 ** -10, derivs="noise",
          oracle=None, eps2=None):
    """Seeded Plummer state with block times; derivatives from noise or one oracle pass."""
    m, x, v = W.plummer(n, seed)
    if salpeter:
        m = W.salpeter_masses(n, seed + 7)
    ids = W.particle_ids(n, ids_seed)
    tj = W.block_times(n, seed + 11, t, quantum=quantum)
    if derivs == "oracle":
        f4 = oracle.forces(ids, x, v, ids, m, x, v, eps2, 4)
        a, jk = f4["acc"], f4["jerk"]
        if order == 6:
            f6 = oracle.forces(ids, x, v, ids, m, x, v, eps2, 6, ai=a, aj=a)
            sn = f6["snap"]
        else:
            sn = None
    else:
        a, jk, sn = W.derivative_noise(n, seed + 13, scales=(1.0, 4.0, 16.0))
        if order == 4:
            sn = None
    return dict(m=m, x=x, v=v, a=a, jerk=jk, snap=sn, ids=ids, tj=tj, t=t)


def gpu_run(ctx_mod, s, i_idx, *, order, precision, eps2, with_nn=1, device=True, launch=None, j_range=None,
            ctx=None, keep=False):
    """set_j + predict + compute through the C ABI; returns numpy outputs."""
    import torch
    sp2 = ctx_mod
    n = len(s["m"])
    own = ctx is None
    if own:
        ctx = sp2.Context(order=order, precision=precision, n_max=n, eps2=eps2, with_nn=with_nn)
    conv = (lambda a: None if a is None else torch.as_tensor(np.ascontiguousarray(a)).cuda()) if device else \
        (lambda a: None if a is None else np.ascontiguousarray(a))
    ctx.set_j(0, conv(s["ids"]), conv(s["m"]), conv(s["x"]), conv(s["v"]), conv(s["a"]), conv(s["jerk"]),
              conv(s["snap"]) if order == 6 else None, conv(s["tj"]))
    ctx.predict(s["t"])
    if launch is not None:
        ctx.set_launch(max(len(i_idx), 1), launch)
    ni = len(i_idx)
    if device:
        out = dict(acc=torch.empty((ni, 3), dtype=torch.float64, device="cuda"),
                   jerk=torch.empty((ni, 3), dtype=torch.float64, device="cuda"),
                   snap=torch.empty((ni, 3), dtype=torch.float64, device="cuda") if order == 6 else None,
                   pot=torch.empty(ni, dtype=torch.float64, device="cuda"),
                   nn_id=torch.empty(ni, dtype=torch.int32, device="cuda") if with_nn else None,
                   nn_r2=torch.empty(ni, dtype=torch.float64, device="cuda") if with_nn else None)
        ctx.compute(conv(np.asarray(i_idx, np.int32)), j_range=j_range, **out)
        ctx.sync()
        res = {k: (None if v is None else v.cpu().numpy()) for k, v in out.items()}
    else:
        res = dict(acc=np.empty((ni, 3)), jerk=np.empty((ni, 3)), snap=np.empty((ni, 3)) if order == 6 else None,
                   pot=np.empty(ni), nn_id=np.empty(ni, np.int32) if with_nn else None,
                   nn_r2=np.empty(ni) if with_nn else None)
        ctx.compute(np.asarray(i_idx, np.int32), j_range=j_range, **res)
    if own and not keep:
        ctx.close()
    return res


def oracle_ref(oracle, s, i_idx, *, order, eps2, j_range=None):
    return oracle.step(s["t"], i_idx, s["ids"], s["m"], s["tj"], s["x"], s["v"], s["a"], s["jerk"], s["snap"],
                       eps2=eps2, order=order, j_range=j_range)


def errors(g, r, order):
    """Per-sink normalised errors (the quantities the tolerances bound)."""
    e = dict(acc=np.linalg.norm(g["acc"] - r["acc"], axis=1) / np.maximum(r["sc_acc"], 1e-300),
             jerk=np.linalg.norm(g["jerk"] - r["jerk"], axis=1) / np.maximum(r["sc_jerk"], 1e-300),
             pot=np.abs(g["pot"] - r["pot"]) / np.maximum(np.abs(r["pot"]), 1e-300))
    if order == 6:
        e["snap"] = np.linalg.norm(g["snap"] - r["snap"], axis=1) / np.maximum(r["sc_snap"], 1e-300)
    return e


def check(g, r, *, order, mixed, s=None, i_idx=None, j_range=None, label=""):
    tol = TOL[bool(mixed)]
    e = errors(g, r, order)
    for k, v in e.items():
        assert np.all(np.isfinite(v)), (label, k)
        assert v.max() <= tol[k], (label, k, float(v.max()), tol[k])
    if g.get("nn_id") is None:
        return e
    gid, rid = g["nn_id"], r["nn_id"]
    if not mixed:
        assert np.array_equal(gid, rid), (label, "nn_id", np.flatnonzero(gid != rid)[:10])
        fin = np.isfinite(r["nn_r2"])
        assert np.array_equal(np.isfinite(g["nn_r2"]), fin)
        assert np.all(np.abs(g["nn_r2"][fin] - r["nn_r2"][fin]) <= tol["r2"] * r["nn_r2"][fin]), label
        return e
    # mixed: exact unless the oracle's best and runner-up are within the band
    bad = np.flatnonzero(gid != rid)
    if bad.size:
        assert s is not None, "need the state to judge near-ties"
        from oracle import predict
        xp, _, _ = predict(s["t"], s["tj"], s["x"], s["v"], s["a"], s["jerk"], s["snap"], order)
        pos = {int(k): q for q, k in enumerate(s["ids"])}
        for q in bad:
            i = int(i_idx[q])
            assert gid[q] >= 0, (label, "missing neighbour")
            j = pos[int(gid[q])]
            d = float(np.sum((xp[j] - xp[i]) ** 2))
            d1 = float(r["nn_r2"][q])
            assert (d - d1) <= NN_BAND * d1, (label, "nn outside the tie band", i, d, d1)
    fin = np.isfinite(r["nn_r2"])
    assert np.array_equal(np.isfinite(g["nn_r2"]), fin), label
    zero = fin & (r["nn_r2"] == 0)
    assert np.all(g["nn_r2"][zero] == 0), (label, "coincident neighbour")
    pos_ = fin & ~zero
    rel = np.abs(g["nn_r2"][pos_] - r["nn_r2"][pos_]) / r["nn_r2"][pos_]
    assert rel.max(initial=0.0) <= NN_BAND + tol["r2"], (label, float(rel.max(initial=0.0)))
    return e
