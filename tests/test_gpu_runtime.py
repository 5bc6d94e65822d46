"""GPU runtime behaviour: CUDA-graph replay, autotuner, call-order and range
errors, the bounded device-side index checks, the finite scan, profiling and
launch counting.  No test here faults, traps or hangs the GPU: bad indices are
caught by the kernels' own range checks and reported through sp2_sync."""
import numpy as np
import pytest

from _parity import check, oracle_ref, state

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


def _ctx(torch, sp2, s, prec=None, **kw):
    n = len(s["m"])
    c = sp2.Context(order=4, precision=sp2.SP2_MIXED if prec is None else prec, n_max=n, **kw)
    D = lambda a: torch.as_tensor(np.ascontiguousarray(a)).cuda()  # noqa: E731
    c.set_j(0, D(s["ids"]), D(s["m"]), D(s["x"]), D(s["v"]), D(s["a"]), D(s["jerk"]), None, D(s["tj"]))
    return c, D


def test_graph_replay_of_a_block_step(env, oracle_mod):
    torch, sp2 = env
    n, eps2 = 3000, 1e-6
    s = state(n, 21)
    c, D = _ctx(torch, sp2, s, eps2=eps2)
    idx = np.sort(np.random.default_rng(1).choice(n, 200, replace=False)).astype(np.int32)
    didx = D(idx)
    upd = {k: D(s[k][idx]) for k in ("ids", "m", "x", "v", "a", "jerk", "tj")}
    out = dict(acc=torch.empty((200, 3), dtype=torch.float64, device="cuda"),
               jerk=torch.empty((200, 3), dtype=torch.float64, device="cuda"),
               pot=torch.empty(200, dtype=torch.float64, device="cuda"),
               nn_id=torch.empty(200, dtype=torch.int32, device="cuda"),
               nn_r2=torch.empty(200, dtype=torch.float64, device="cuda"))

    def step():
        c.set_j(0, upd["ids"], upd["m"], upd["x"], upd["v"], upd["a"], upd["jerk"], None, upd["tj"], slots=didx)
        c.predict(s["t"])
        c.compute(didx, **out)

    step()  # sizes scratch outside the capture
    c.sync()
    sp2.sp2_graph_begin(c.ctx)
    step()
    g = sp2.sp2_graph_end(c.ctx)
    for v in out.values():
        v.zero_()
    before = c.kernel_launches()
    for _ in range(3):
        sp2.sp2_graph_launch(c.ctx, g)
    c.sync()
    assert c.kernel_launches() == before  # replays are not new library launches
    res = {k: v.cpu().numpy() for k, v in out.items()}
    check(res, oracle_ref(oracle_mod, s, idx, order=4, eps2=eps2), order=4, mixed=True, s=s, i_idx=idx)
    with pytest.raises(sp2.SP2Error) as e:  # host pointers are refused inside a capture
        sp2.sp2_graph_begin(c.ctx)
        try:
            c.compute(idx, acc=np.empty((200, 3)))
        finally:
            sp2.sp2_graph_destroy(sp2.sp2_graph_end(c.ctx))
    assert e.value.status == -5
    sp2.sp2_graph_destroy(g)
    c.close()


def test_autotune_picks_a_valid_shape(env, oracle_mod):
    torch, sp2 = env
    n, eps2 = 8192, 1e-6
    s = state(n, 22)
    c, D = _ctx(torch, sp2, s, eps2=eps2)
    c.predict(s["t"])
    for na in (1, 100, 4000):
        best = c.autotune(na)
        assert best == c.get_launch(na)
        idx = np.arange(0, n, n // na, dtype=np.int32)[:na]
        acc = torch.empty((na, 3), dtype=torch.float64, device="cuda")
        jerk = torch.empty((na, 3), dtype=torch.float64, device="cuda")
        pot = torch.empty(na, dtype=torch.float64, device="cuda")
        c.compute(D(idx), acc=acc, jerk=jerk, pot=pot)
        c.sync()
        r = oracle_ref(oracle_mod, s, idx, order=4, eps2=eps2)
        check(dict(acc=acc.cpu().numpy(), jerk=jerk.cpu().numpy(), pot=pot.cpu().numpy()), r, order=4, mixed=True)
    with pytest.raises(sp2.SP2Error):
        c.set_launch(10, dict(threads=96, i_per_thread=1, j_lanes=1, j_tile=64, split_j=1, ctas_per_sm=0))
    with pytest.raises(sp2.SP2Error):
        c.set_launch(10, dict(threads=64, i_per_thread=3, j_lanes=1, j_tile=64, split_j=1, ctas_per_sm=0))
    c.close()


def test_call_order_and_range_errors(env):
    torch, sp2 = env
    s = state(500, 23)
    c, D = _ctx(torch, sp2, s, eps2=1e-6)
    idx = D(np.arange(10, dtype=np.int32))
    with pytest.raises(sp2.SP2Error) as e:
        c.compute(idx, acc=torch.empty((10, 3), dtype=torch.float64, device="cuda"))
    assert e.value.status == -5  # predict first
    c.predict(1.0)
    with pytest.raises(sp2.SP2Error) as e:
        c.compute(np.array([0, 600], np.int32), acc=np.empty((2, 3)))
    assert e.value.status == -2  # host-side check of sink slots
    with pytest.raises(sp2.SP2Error) as e:
        c.compute(np.array([0], np.int32), snap=np.empty((1, 3)))
    assert e.value.status == -1  # snap from an order-4 context
    with pytest.raises(sp2.SP2Error) as e:
        c.compute(np.array([0], np.int32), acc=np.empty((1, 3)), j_range=(10, 600))
    assert e.value.status == -2
    # device-side sink slots out of range: skipped by the kernel, reported by sync
    bad = D(np.array([3, 9999, -4, 5], dtype=np.int32))
    acc = torch.zeros((4, 3), dtype=torch.float64, device="cuda")
    c.compute(bad, acc=acc)
    with pytest.raises(sp2.SP2Error) as e:
        c.sync()
    assert e.value.status == -2
    c.sync()  # the flag is cleared and the context stays usable
    ok = D(np.array([3, 5], dtype=np.int32))
    acc2 = torch.zeros((2, 3), dtype=torch.float64, device="cuda")
    c.compute(ok, acc=acc2)
    c.sync()
    assert torch.allclose(acc2, acc[[0, 3]], rtol=1e-5, atol=0)
    # a contiguous store may not leave a gap of unloaded slots
    with pytest.raises(sp2.SP2Error) as e:
        one0 = {k: D(s[k][:1]) for k in ("ids", "m", "x", "v", "a", "jerk", "tj")}
        c.set_j(501, one0["ids"], one0["m"], one0["x"], one0["v"], one0["a"], one0["jerk"], None, one0["tj"])
    assert e.value.status == -2
    # device-side scatter slots out of range
    one = {k: D(s[k][:1]) for k in ("ids", "m", "x", "v", "a", "jerk", "tj")}
    c.set_j(0, one["ids"], one["m"], one["x"], one["v"], one["a"], one["jerk"], None, one["tj"],
            slots=D(np.array([777], np.int32)))
    with pytest.raises(sp2.SP2Error) as e:
        c.sync()
    assert e.value.status == -2
    c.close()


def test_nonfinite_scan(env):
    torch, sp2 = env
    s = state(50, 24)
    for k in ("x", "v", "a", "jerk"):
        s[k][7] = s[k][3]
    s["tj"][7] = s["tj"][3]
    c, D = _ctx(torch, sp2, s, eps2=0.0, check_finite=1)
    c.predict(1.0)
    with pytest.raises(sp2.SP2Error) as e:
        c.compute(D(np.arange(50, dtype=np.int32)), acc=torch.empty((50, 3), dtype=torch.float64, device="cuda"))
    assert e.value.status == -7
    c.close()


def test_profile_and_launch_counts(env):
    torch, sp2 = env
    n = 20000
    s = state(n, 25)
    c, D = _ctx(torch, sp2, s, eps2=1e-6, profile=1)
    c.predict(1.0)
    c.profile_reset()
    l0 = c.kernel_launches()
    idx = D(np.arange(0, n, 7, dtype=np.int32))
    acc = torch.empty((len(idx), 3), dtype=torch.float64, device="cuda")
    for _ in range(3):
        c.predict(1.0)
        c.compute(idx, acc=acc)
    p = c.profile_read()
    L = c.get_launch(len(idx))
    per_step = 2 + (1 if L["split_j"] > 1 else 0)
    assert c.kernel_launches() - l0 == 3 * per_step
    assert p["predict"][0] == 3 and p["force"][0] == 3
    assert p["force"][1] > 0 and p["predict"][1] > 0
    c.close()


def test_repeated_calls_are_bit_identical():
    """The reductions have a fixed order, so the same call gives the same bits
    every time, whichever CTA finishes last; shapes with the in-pass reduction
    over few and many slices and with the separate reduction kernel."""
    import torch
    from paper_1510_04068_gb300 import build, sp2
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    sp2.load()
    import workloads as W
    n = 30000
    m, x, v = W.plummer(n, 3)
    a, jk, _ = W.derivative_noise(n, 4, scales=(1.0, 4.0, 16.0))
    ids = W.particle_ids(n, 5)
    D = lambda q: torch.as_tensor(np.ascontiguousarray(q)).cuda()  # noqa: E731
    for prec in (sp2.SP2_MIXED, sp2.SP2_FP64):
        c = sp2.Context(order=4, precision=prec, n_max=n, eps2=1e-8)
        c.set_j(0, D(ids), D(m), D(x), D(v), D(a), D(jk), None, D(W.block_times(n, 6, 1.0)))
        for n_i, shape in ((1, (64, 1, 32, 256, 100)), (3, (64, 1, 8, 64, 400)), (4000, (128, 1, 1, 128, 60))):
            idx = D(np.sort(np.random.default_rng(n_i).choice(n, n_i, replace=False)).astype(np.int32))
            c.set_launch(n_i, dict(zip(("threads", "i_per_thread", "j_lanes", "j_tile", "split_j"), shape), ctas_per_sm=0))
            outs = []
            for _ in range(3):
                c.predict(1.0)
                o = dict(acc=torch.empty((n_i, 3), dtype=torch.float64, device="cuda"),
                         jerk=torch.empty((n_i, 3), dtype=torch.float64, device="cuda"),
                         pot=torch.empty(n_i, dtype=torch.float64, device="cuda"),
                         nn_id=torch.empty(n_i, dtype=torch.int32, device="cuda"),
                         nn_r2=torch.empty(n_i, dtype=torch.float64, device="cuda"))
                c.compute(idx, **o)
                outs.append({k: t.cpu().numpy() for k, t in o.items()})
            for o2 in outs[1:]:
                for k in o2:
                    assert np.array_equal(outs[0][k].view(np.uint8), o2[k].view(np.uint8)), (prec, n_i, k)
        c.close()


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_outputs_not_written_past_their_end(precision):
    """Canary-padded outputs: for ragged sink counts and several launch shapes
    (one and many i-blocks, split and not, fused and separate reduction) the
    library writes exactly n_i entries of every output."""
    import torch
    from paper_1510_04068_gb300 import build, sp2
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    sp2.load()
    s = state(5000, 11)
    D = lambda q: torch.as_tensor(np.ascontiguousarray(q)).cuda()  # noqa: E731
    prec = sp2.SP2_MIXED if precision == "mixed" else sp2.SP2_FP64
    c = sp2.Context(order=4, precision=prec, n_max=5000, eps2=1e-8)
    c.set_j(0, D(s["ids"]), D(s["m"]), D(s["x"]), D(s["v"]), D(s["a"]), D(s["jerk"]), None, D(s["tj"]))
    pad = 64
    for n_i, shape in ((1, (32, 1, 32, 256, 16)), (37, (64, 2, 2, 64, 30)), (777, (128, 4, 1, 128, 3)),
                       (1001, (256, 1, 1, 512, 1)), (5000, (128, 2, 1, 256, 40))):
        idx = D(np.sort(np.random.default_rng(n_i).choice(5000, n_i, replace=False)).astype(np.int32))
        c.predict(1.0)
        c.set_launch(n_i, dict(zip(("threads", "i_per_thread", "j_lanes", "j_tile", "split_j"), shape), ctas_per_sm=0))
        bufs = dict(acc=torch.full(((n_i + pad) * 3,), 7.25, dtype=torch.float64, device="cuda"),
                    jerk=torch.full(((n_i + pad) * 3,), 7.25, dtype=torch.float64, device="cuda"),
                    pot=torch.full((n_i + pad,), 7.25, dtype=torch.float64, device="cuda"),
                    nn_id=torch.full((n_i + pad,), -77, dtype=torch.int32, device="cuda"),
                    nn_r2=torch.full((n_i + pad,), 7.25, dtype=torch.float64, device="cuda"))
        c.compute(idx, **bufs)
        c.sync()
        for k, b in bufs.items():
            w = 3 if k in ("acc", "jerk") else 1
            tail = b[n_i * w:].cpu().numpy()
            assert np.all(tail == (-77 if k == "nn_id" else 7.25)), (n_i, shape, k)
            assert np.all(np.isfinite(b[:n_i * w].cpu().numpy().astype(np.float64))), (n_i, k)
    c.close()


@pytest.mark.gpu
def test_pipe_peak_probe():
    """The pipe-rate probe returns finite rates in the range a GB300 can have
    (152 SMs, <= 2.1 GHz): FP32 FMA lanes 5-50 T/s in both forms, FP64 FMA
    0.05-5 T/s, rsqrt 0.5-20 T/s."""
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1510_04068_gb300 import build, sp2
    build.build()
    sp2.load()
    pk = sp2.measure_pipe_peaks()
    assert 5e12 < pk["fp32_fma_lane_ops"] < 5e13, pk
    assert 5e12 < pk["fp32x2_fma_lane_ops"] < 5e13, pk
    assert 5e10 < pk["fp64_fma_ops"] < 5e12, pk
    assert 5e11 < pk["rsqrt_ops"] < 2e13, pk
