"""GPU: the pass that predicts its sources in shared memory (mixed precision,
all sinks in one CTA) forms every source's position exactly as the sink's.

The sources of a fused pass are predicted two at a time in packed f32x2
double-single steps, the sinks one at a time by the scalar predictor; both
must round every step alike.  Here every particle has a twin with the same
position, velocity, acceleration, jerk (and snap) and block time, so each
sink's nearest neighbour is its twin at r^2 = 0 exactly -- a single differing
bit in either predictor leaves a positive distance.  The twins sit half the
set apart, so they fall in either half of a pair record, in every lane and
in other tiles and slices.  The forces are also checked against the oracle."""
import numpy as np
import pytest

from _parity import check, gpu_run, oracle_ref, state

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


def _twins(n, order, seed):
    s = state(n, seed, order=order)
    h = n // 2
    for key in ("x", "v", "a", "jerk") + (("snap",) if order == 6 else ()):
        s[key][h:2 * h] = s[key][:h]
    s["tj"][h:2 * h] = s["tj"][:h]
    return s, h


@pytest.mark.parametrize("order", [4, 6])
@pytest.mark.parametrize("n_active,shape", [
    (37, (256, 1, 4, 256, 16)),     # one CTA of 64 sink slots, 4 lanes per sink
    (37, (128, 1, 1, 256, 20)),     # one sink per thread
    (3, (128, 1, 32, 512, 64)),     # a warp per sink
    (3, (256, 1, 64, 512, 8)),      # two warps per sink
])
def test_twins_are_at_zero_distance(sp2, oracle_mod, order, n_active, shape):
    n, eps2 = 6003, 1e-6
    s, h = _twins(n, order, 40 + n_active)
    rng = np.random.default_rng(n_active + order)
    idx = np.sort(rng.choice(2 * h, n_active, replace=False)).astype(np.int32)
    launch = dict(zip(("threads", "i_per_thread", "j_lanes", "j_tile", "split_j"), shape), ctas_per_sm=0)
    ctx = sp2.Context(order=order, precision=sp2.SP2_MIXED, n_max=n, eps2=eps2, with_nn=1, profile=1)
    g = gpu_run(sp2, s, idx, order=order, precision=sp2.SP2_MIXED, eps2=eps2, launch=launch, ctx=ctx, keep=True)
    prof = ctx.profile_read()
    ctx.close()
    # the prediction ran inside the pass: no predictor launch, one force launch
    assert prof["predict"][0] == 0 and prof["force"][0] == 1, prof
    twin = np.where(idx < h, idx + h, idx - h)
    assert np.all(g["nn_r2"] == 0.0), (g["nn_r2"], idx)
    assert np.array_equal(g["nn_id"], s["ids"][twin])
    r = oracle_ref(oracle_mod, s, idx, order=order, eps2=eps2)
    check(g, r, order=order, mixed=True, s=s, i_idx=idx, label=str(shape))
