"""Golden fixtures (tests/golden/, written by make_golden.py from the oracle
alone): the oracle still reproduces them, and the CUDA path matches them in
both precisions and both Hermite orders."""
import json
from pathlib import Path

import numpy as np
import pytest

from _parity import check

GOLDEN = Path(__file__).resolve().parent / "golden"


def _load(order):
    d = json.loads((GOLDEN / f"plummer32_h{order}.json").read_text())
    s = {k: np.asarray(v, dtype=np.int32 if k == "ids" else np.float64) for k, v in d["inputs"].items()}
    s.setdefault("snap", None)
    s["t"] = d["t"]
    r = {k: np.asarray(v, dtype=np.int32 if k == "nn_id" else np.float64) for k, v in d["expected"].items()}
    return d, s, r


@pytest.mark.parametrize("order", [4, 6])
def test_oracle_reproduces_golden(oracle_mod, order):
    d, s, r = _load(order)
    n = d["n"]
    got = oracle_mod.step(s["t"], np.arange(n), s["ids"], s["m"], s["tj"], s["x"], s["v"], s["a"], s["jerk"],
                          s["snap"], eps2=d["eps2"], order=order)
    assert np.array_equal(got["nn_id"], r["nn_id"])
    for k in r:
        if k == "nn_id":
            continue
        scale = {"acc": r["sc_acc"], "jerk": r["sc_jerk"], "snap": r.get("sc_snap")}.get(k)
        if scale is not None:
            err = np.linalg.norm(got[k] - r[k], axis=1) / scale
        else:
            err = np.abs(got[k] - r[k]) / np.maximum(np.abs(r[k]), 1e-300)
        assert err.max() <= 1e-15, (k, float(err.max()))


@pytest.mark.gpu
@pytest.mark.parametrize("mixed", [False, True])
@pytest.mark.parametrize("order", [4, 6])
def test_cuda_matches_golden(order, mixed):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1510_04068_gb300 import build, sp2
    from _parity import gpu_run
    build.build()
    sp2.load()
    d, s, r = _load(order)
    i_idx = np.arange(d["n"], dtype=np.int32)
    g = gpu_run(sp2, s, i_idx, order=order, precision=sp2.SP2_MIXED if mixed else sp2.SP2_FP64, eps2=d["eps2"])
    check(g, r, order=order, mixed=mixed, s=s, i_idx=i_idx, label=f"golden h{order}")
