"""GPU parity: the force pass (predict + compute) against the oracle, element by
element, at sizes the oracle finishes in seconds (several tiles, ragged tails),
over both precisions, both orders and many launch shapes."""
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


@pytest.mark.parametrize("dt_back", [0.0, 2.0 ** -8])
def test_plummer_1024_fp64_all_active(sp2, oracle_mod, dt_back):
    """N = 1024 equal-mass Plummer, eps = 1e-3, FP64 Hermite-4, every particle
    active; t_j = t (identity predictor) and t_j = t - 2^-8."""
    n, eps2 = 1024, 1e-6
    s = state(n, 0, derivs="oracle", oracle=oracle_mod, eps2=eps2)
    s["tj"] = np.full(n, s["t"] - dt_back)
    idx = np.arange(n, dtype=np.int32)
    g = gpu_run(sp2, s, idx, order=4, precision=sp2.SP2_FP64, eps2=eps2)
    r = oracle_ref(oracle_mod, s, idx, order=4, eps2=eps2)
    check(g, r, order=4, mixed=False, label="C1")


@pytest.mark.parametrize("order", [4, 6])
@pytest.mark.parametrize("mixed", [False, True])
@pytest.mark.parametrize("n,n_active", [(3000, 3000), (3001, 1), (4099, 7), (5000, 131), (2000, 2000)])
def test_block_step_parity(sp2, oracle_mod, order, mixed, n, n_active):
    eps2 = 1e-8
    s = state(n, n_active + order, order=order, salpeter=(order == 6), ids_seed=5)
    idx = np.random.default_rng(n).choice(n, n_active, replace=False).astype(np.int32)
    prec = sp2.SP2_MIXED if mixed else sp2.SP2_FP64
    g = gpu_run(sp2, s, idx, order=order, precision=prec, eps2=eps2)
    r = oracle_ref(oracle_mod, s, idx, order=order, eps2=eps2)
    check(g, r, order=order, mixed=mixed, s=s, i_idx=idx, label=f"{order}/{mixed}/{n}/{n_active}")


SHAPES = [
    dict(threads=256, i_per_thread=1, j_lanes=1, j_tile=128, split_j=1, ctas_per_sm=0),
    dict(threads=256, i_per_thread=2, j_lanes=1, j_tile=64, split_j=3, ctas_per_sm=0),
    dict(threads=128, i_per_thread=4, j_lanes=1, j_tile=256, split_j=5, ctas_per_sm=0),
    dict(threads=64, i_per_thread=1, j_lanes=4, j_tile=64, split_j=7, ctas_per_sm=2),
    dict(threads=128, i_per_thread=2, j_lanes=8, j_tile=128, split_j=40, ctas_per_sm=0),
    dict(threads=32, i_per_thread=1, j_lanes=32, j_tile=256, split_j=64, ctas_per_sm=0),
    dict(threads=256, i_per_thread=4, j_lanes=2, j_tile=32, split_j=2, ctas_per_sm=1),
    dict(threads=64, i_per_thread=2, j_lanes=16, j_tile=256, split_j=33, ctas_per_sm=0),
]


@pytest.mark.parametrize("shape", range(len(SHAPES)))
@pytest.mark.parametrize("mixed", [False, True])
def test_launch_shapes(sp2, oracle_mod, shape, mixed):
    """Every launch shape (sinks per thread, threads per sink, tile, source split,
    residency) gives the same answer within tolerance."""
    n, n_act, eps2 = 4133, 1037, 1e-6
    s = state(n, 40 + shape, order=6)
    idx = np.sort(np.random.default_rng(shape).choice(n, n_act, replace=False)).astype(np.int32)
    prec = sp2.SP2_MIXED if mixed else sp2.SP2_FP64
    g = gpu_run(sp2, s, idx, order=6, precision=prec, eps2=eps2, launch=SHAPES[shape])
    r = oracle_ref(oracle_mod, s, idx, order=6, eps2=eps2)
    check(g, r, order=6, mixed=mixed, s=s, i_idx=idx, label=str(SHAPES[shape]))


@pytest.mark.parametrize("mixed", [False, True])
def test_host_and_device_pointers_agree(sp2, oracle_mod, mixed):
    n, eps2 = 1500, 1e-6
    s = state(n, 3)
    idx = np.arange(0, n, 3, dtype=np.int32)
    prec = sp2.SP2_MIXED if mixed else sp2.SP2_FP64
    gd = gpu_run(sp2, s, idx, order=4, precision=prec, eps2=eps2, device=True)
    gh = gpu_run(sp2, s, idx, order=4, precision=prec, eps2=eps2, device=False)
    for k in gd:
        assert np.array_equal(gd[k], gh[k]), k
    check(gh, oracle_ref(oracle_mod, s, idx, order=4, eps2=eps2), order=4, mixed=mixed, s=s, i_idx=idx)


@pytest.mark.parametrize("mixed", [False, True])
def test_source_range_and_repeated_sinks(sp2, oracle_mod, mixed):
    n, eps2 = 2500, 1e-6
    s = state(n, 4, ids_seed=1)
    idx = np.array([5, 5, 17, 1999, 2400, 5, 0, 2499], dtype=np.int32)
    prec = sp2.SP2_MIXED if mixed else sp2.SP2_FP64
    for rng in [(0, n), (100, 2100), (1990, 2010)]:
        g = gpu_run(sp2, s, idx, order=4, precision=prec, eps2=eps2, j_range=rng)
        r = oracle_ref(oracle_mod, s, idx, order=4, eps2=eps2, j_range=rng)
        check(g, r, order=4, mixed=mixed, s=s, i_idx=idx, label=str(rng))


@pytest.mark.parametrize("mixed", [False, True])
def test_degenerate_sizes(sp2, oracle_mod, mixed):
    """One particle (no neighbour, zero force), two particles, coincident
    distinct particles with softening, unsoftened pairs, exact NN ties."""
    prec = sp2.SP2_MIXED if mixed else sp2.SP2_FP64
    s = state(1, 1)
    g = gpu_run(sp2, s, [0], order=4, precision=prec, eps2=0.0)
    assert g["nn_id"][0] == -1 and np.isinf(g["nn_r2"][0])
    assert np.all(g["acc"] == 0) and np.all(g["jerk"] == 0) and g["pot"][0] == 0
    s = state(2, 2)
    g = gpu_run(sp2, s, [0, 1], order=4, precision=prec, eps2=0.0)
    r = oracle_ref(oracle_mod, s, [0, 1], order=4, eps2=0.0)
    check(g, r, order=4, mixed=mixed, s=s, i_idx=np.array([0, 1]))
    # coincident distinct particles, softened
    s = state(64, 3)
    for key in ("x", "v", "a", "jerk"):
        s[key][10] = s[key][20]
    s["tj"][10] = s["tj"][20]
    idx = np.arange(64, dtype=np.int32)
    g = gpu_run(sp2, s, idx, order=4, precision=prec, eps2=1e-4)
    r = oracle_ref(oracle_mod, s, idx, order=4, eps2=1e-4)
    check(g, r, order=4, mixed=mixed, s=s, i_idx=idx)
    assert g["nn_r2"][10] == 0 and g["nn_id"][10] == s["ids"][20]
    # exact tie on a lattice: the smaller id wins on both sides
    lat = np.array([[0.0, 0, 0], [1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0], [0, 0, 2]])
    s = dict(m=np.ones(6), x=lat, v=np.zeros((6, 3)), a=np.zeros((6, 3)), jerk=np.zeros((6, 3)), snap=None,
             ids=np.array([9, 4, 7, 2, 8, 1], np.int32), tj=np.zeros(6), t=0.0)
    g = gpu_run(sp2, s, [0], order=4, precision=prec, eps2=0.0)
    assert g["nn_r2"][0] == 1.0
    # FP64 breaks exact ties by the smaller id like the oracle; in mixed mode any
    # of the tied neighbours is within the tie band
    assert g["nn_id"][0] == 2 if not mixed else g["nn_id"][0] in (4, 7, 2, 8)


def test_empty_sink_list_is_a_noop(sp2):
    import torch
    s = state(100, 5)
    with sp2.Context(order=4, precision=sp2.SP2_MIXED, n_max=100, eps2=1e-6) as c:
        conv = lambda a: torch.as_tensor(a).cuda()  # noqa: E731
        c.set_j(0, conv(s["ids"]), conv(s["m"]), conv(s["x"]), conv(s["v"]), conv(s["a"]), conv(s["jerk"]), None,
                conv(s["tj"]))
        c.predict(1.0)
        before = c.kernel_launches()
        c.compute(torch.empty(0, dtype=torch.int32, device="cuda"))
        c.sync()
        assert c.kernel_launches() == before


@pytest.mark.parametrize("order", [4, 6])
def test_fused_prediction_small_n_active(sp2, oracle_mod, order):
    """Mixed precision with few sinks: the force pass predicts its sources from
    the double-single cache (no predictor launch); a shape with several
    i-blocks writes the records first.  Both match the oracle, and a later
    consumer of the records (a large sink list) sees the same predicted state."""
    import torch
    n, eps2 = 6000, 1e-8
    s = state(n, 70 + order, order=order)
    D = lambda a: None if a is None else torch.as_tensor(np.ascontiguousarray(a)).cuda()  # noqa: E731
    with sp2.Context(order=order, precision=sp2.SP2_MIXED, n_max=n, eps2=eps2, profile=1) as c:
        c.set_j(0, D(s["ids"]), D(s["m"]), D(s["x"]), D(s["v"]), D(s["a"]), D(s["jerk"]),
                D(s["snap"]) if order == 6 else None, D(s["tj"]))
        for n_i, shape, fused in ((1, dict(threads=32, i_per_thread=1, j_lanes=32, j_tile=256, split_j=40), True),
                                  (37, dict(threads=128, i_per_thread=1, j_lanes=2, j_tile=128, split_j=20), True),
                                  (37, dict(threads=32, i_per_thread=1, j_lanes=1, j_tile=64, split_j=20), False),
                                  (300, dict(threads=256, i_per_thread=2, j_lanes=1, j_tile=128, split_j=9), True),
                                  # at most two sources per thread and tile: the next tile's cache words
                                  # are fetched while the current one is evaluated (ragged last tiles)
                                  (1, dict(threads=256, i_per_thread=1, j_lanes=32, j_tile=512, split_j=5), True),
                                  (5, dict(threads=128, i_per_thread=1, j_lanes=16, j_tile=256, split_j=3), True),
                                  (64, dict(threads=256, i_per_thread=1, j_lanes=4, j_tile=256, split_j=11), True),
                                  # several warps per sink, each on its own part of every tile
                                  (1, dict(threads=256, i_per_thread=1, j_lanes=128, j_tile=1024, split_j=3), True),
                                  (3, dict(threads=256, i_per_thread=1, j_lanes=64, j_tile=512, split_j=4), True)):
            idx = np.sort(np.random.default_rng(n_i).choice(n, n_i, replace=False)).astype(np.int32)
            c.predict(s["t"])
            c.set_launch(n_i, dict(shape, ctas_per_sm=0))
            c.profile_reset()
            out = dict(acc=torch.empty((n_i, 3), dtype=torch.float64, device="cuda"),
                       jerk=torch.empty((n_i, 3), dtype=torch.float64, device="cuda"),
                       snap=torch.empty((n_i, 3), dtype=torch.float64, device="cuda") if order == 6 else None,
                       pot=torch.empty(n_i, dtype=torch.float64, device="cuda"),
                       nn_id=torch.empty(n_i, dtype=torch.int32, device="cuda"),
                       nn_r2=torch.empty(n_i, dtype=torch.float64, device="cuda"))
            c.compute(D(idx), **out)
            prof = c.profile_read()
            assert (prof["predict"][0] == 0) == fused, (n_i, shape, prof)
            g = {k: (None if v is None else v.cpu().numpy()) for k, v in out.items()}
            r = oracle_ref(oracle_mod, s, idx, order=order, eps2=eps2)
            check(g, r, order=order, mixed=True, s=s, i_idx=idx, label=f"fused={fused} n_i={n_i}")
        # records written on demand for a consumer that needs them
        idx = np.arange(0, n, 2, dtype=np.int32)
        acc = torch.empty((len(idx), 3), dtype=torch.float64, device="cuda")
        pot = torch.empty(len(idx), dtype=torch.float64, device="cuda")
        c.compute(D(idx), acc=acc, pot=pot)
        r = oracle_ref(oracle_mod, s, idx, order=order, eps2=eps2)
        e = np.linalg.norm(acc.cpu().numpy() - r["acc"], axis=1) / r["sc_acc"]
        assert e.max() <= 1e-6


@pytest.mark.parametrize("mixed", [False, True])
@pytest.mark.parametrize("n_i,split", [(1, 300), (3, 100), (5, 64), (2, 33)])
def test_in_pass_reduction_levels(sp2, oracle_mod, mixed, n_i, split):
    """Few sinks over many slices: the last CTA of each i-block reduces the
    slices in FP64 (a warp per field), one to a few hundred of them; the result
    matches the oracle."""
    n, eps2 = 20000, 1e-8
    s = state(n, 90 + n_i, order=4)
    idx = np.sort(np.random.default_rng(split).choice(n, n_i, replace=False)).astype(np.int32)
    launch = dict(threads=64, i_per_thread=1, j_lanes=8, j_tile=64, split_j=split, ctas_per_sm=0)
    g = gpu_run(sp2, s, idx, order=4, precision=sp2.SP2_MIXED if mixed else sp2.SP2_FP64, eps2=eps2, launch=launch)
    r = oracle_ref(oracle_mod, s, idx, order=4, eps2=eps2)
    check(g, r, order=4, mixed=mixed, s=s, i_idx=idx, label=f"split={split}")


@pytest.mark.parametrize("order", [4, 6])
def test_mixed_far_from_origin(sp2, oracle_mod, order):
    """Double-single positions: a Plummer sphere moved 10^4 length units away
    (FP32 alone would keep ~3 significant digits of the close-pair
    separations) still meets the mixed-precision tolerances."""
    n, eps2 = 3000, 1e-8
    s = state(n, 33, order=order)
    s["x"] = s["x"] + np.array([1.0e4, -3.7e3, 2.2e3])
    idx = np.sort(np.random.default_rng(3).choice(n, 400, replace=False)).astype(np.int32)
    g = gpu_run(sp2, s, idx, order=order, precision=sp2.SP2_MIXED, eps2=eps2)
    r = oracle_ref(oracle_mod, s, idx, order=order, eps2=eps2)
    check(g, r, order=order, mixed=True, s=s, i_idx=idx, label="far from origin")


@pytest.mark.parametrize("mixed", [False, True])
@pytest.mark.parametrize("n,per_sm", [(24000, 1), (45000, 1)])
def test_whole_waves_and_split_tail(sp2, oracle_mod, mixed, n, per_sm):
    """Four or more waves of i-blocks (one resident CTA of 32 sinks per SM
    here): whole waves of i-blocks run over all sources and write their
    outputs directly, the last partial wave is split over the sources and
    reduced in the pass; every sink matches the oracle."""
    eps2 = 1e-8
    s = state(n, 81, order=4)
    idx = np.random.default_rng(n).permutation(n).astype(np.int32)
    launch = dict(threads=32, i_per_thread=1, j_lanes=1, j_tile=64, split_j=4, ctas_per_sm=per_sm)
    g = gpu_run(sp2, s, idx, order=4, precision=sp2.SP2_MIXED if mixed else sp2.SP2_FP64, eps2=eps2, launch=launch)
    r = oracle_ref(oracle_mod, s, idx, order=4, eps2=eps2)
    check(g, r, order=4, mixed=mixed, s=s, i_idx=idx, label=f"n={n} per_sm={per_sm}")


@pytest.mark.parametrize("n_i,shape", [
    (1, dict(threads=128, i_per_thread=1, j_lanes=128, j_tile=1024, split_j=1)),
    (5, dict(threads=128, i_per_thread=1, j_lanes=64, j_tile=512, split_j=6)),
    (700, dict(threads=256, i_per_thread=1, j_lanes=64, j_tile=512, split_j=2)),
    (3001, dict(threads=256, i_per_thread=1, j_lanes=64, j_tile=512, split_j=1)),
])
def test_several_warps_per_sink(sp2, oracle_mod, n_i, shape):
    """j_lanes above 32 (mixed precision): the warps that share a sink take
    contiguous parts of every tile and their totals and nearest neighbours are
    added in warp order; both orders, one and several i-blocks, with and
    without a source split, match the oracle.  FP64 contexts and several sinks
    per thread refuse the shape."""
    n, eps2 = 6001, 1e-8
    for order in (4, 6):
        s = state(n, 55 + n_i, order=order, salpeter=(order == 6))
        idx = np.sort(np.random.default_rng(n_i).choice(n, n_i, replace=False)).astype(np.int32)
        launch = dict(shape, ctas_per_sm=0)
        g = gpu_run(sp2, s, idx, order=order, precision=sp2.SP2_MIXED, eps2=eps2, launch=launch)
        r = oracle_ref(oracle_mod, s, idx, order=order, eps2=eps2)
        check(g, r, order=order, mixed=True, s=s, i_idx=idx, label=f"{order}/{n_i}/{shape}")
    s = state(n, 56, order=4)
    with pytest.raises(sp2.SP2Error):
        gpu_run(sp2, s, np.arange(5, dtype=np.int32), order=4, precision=sp2.SP2_FP64, eps2=eps2,
                launch=dict(threads=128, i_per_thread=1, j_lanes=64, j_tile=512, split_j=2, ctas_per_sm=0))
    with pytest.raises(sp2.SP2Error):
        gpu_run(sp2, s, np.arange(5, dtype=np.int32), order=4, precision=sp2.SP2_MIXED, eps2=eps2,
                launch=dict(threads=128, i_per_thread=2, j_lanes=64, j_tile=512, split_j=2, ctas_per_sm=0))
