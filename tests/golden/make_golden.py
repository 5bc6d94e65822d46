"""Writes the golden fixtures of this directory from the oracle alone.

The paper prints no worked example (its results are in figures), so the
stored expected values here are the oracle's: a fixed, seeded Plummer state
of 32 particles with block times and derivatives, Taylor-predicted to t = 1
(Sec. 2.2) and summed (Hermite-4 and Hermite-6 force law with Plummer
softening, nearest neighbour, Sec. 3), every particle a sink.  Inputs and
outputs are written in full (shortest round-trip decimals), so the fixtures
do not depend on the input generators staying the same.

    python tests/golden/make_golden.py
"""
import json
import sys
from pathlib import Path

import numpy as np

HERE = Path(__file__).resolve().parent
sys.path.insert(0, str(HERE.parent.parent))

import oracle  # noqa: E402
import workloads as W  # noqa: E402

N, SEED, EPS2, T = 32, 3, 1e-4, 1.0


def state():
    m, x, v = W.plummer(N, SEED)
    ids = W.particle_ids(N, SEED + 1)
    tj = W.block_times(N, SEED + 11, T, quantum=2.0 ** -10)
    f4 = oracle.forces(ids, x, v, ids, m, x, v, EPS2, 4)
    a, jk = f4["acc"], f4["jerk"]
    sn = oracle.forces(ids, x, v, ids, m, x, v, EPS2, 6, ai=a, aj=a)["snap"]
    return dict(ids=ids, m=m, x=x, v=v, a=a, jerk=jk, snap=sn, tj=tj)


def main():
    s = state()
    slots = np.arange(N, dtype=np.int32)
    for order in (4, 6):
        r = oracle.step(T, slots, s["ids"], s["m"], s["tj"], s["x"], s["v"], s["a"], s["jerk"],
                        s["snap"] if order == 6 else None, eps2=EPS2, order=order)
        keys = ["acc", "jerk", "pot", "nn_id", "nn_r2", "sc_acc", "sc_jerk"] + (["snap", "sc_snap"] if order == 6 else [])
        doc = {
            "about": "oracle outputs (FP64 direct sum, Sec. 2.2 predictor and Sec. 3 force law) for the "
                     "stored inputs; written by tests/golden/make_golden.py",
            "order": order, "n": N, "eps2": EPS2, "t": T,
            "inputs": {k: np.asarray(v).tolist() for k, v in s.items() if not (order == 4 and k == "snap")},
            "expected": {k: np.asarray(r[k]).tolist() for k in keys},
        }
        (HERE / f"plummer32_h{order}.json").write_text(_dump(doc))


def _dump(doc):
    """JSON with one line per array (floats as shortest round-trip decimals)."""
    out = ["{"]
    items = list(doc.items())
    for k, (key, val) in enumerate(items):
        end = "," if k + 1 < len(items) else ""
        if isinstance(val, dict):
            out.append(f"{json.dumps(key)}: {{")
            sub = list(val.items())
            for q, (sk, sv) in enumerate(sub):
                out.append(f"  {json.dumps(sk)}: {json.dumps(sv)}" + ("," if q + 1 < len(sub) else ""))
            out.append("}" + end)
        else:
            out.append(f"{json.dumps(key)}: {json.dumps(val)}{end}")
    out.append("}")
    return "\n".join(out) + "\n"


if __name__ == "__main__":
    main()
