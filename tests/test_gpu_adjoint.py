"""GPU parity of the adjoint: the vector-Jacobian product kernel against the
oracle's autograd gradient, one Hermite-4 step against the oracle's step, and
the checkpointed trajectory gradient against the oracle's gradient and against
FP64 central differences (h = 1e-6)."""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1510_04068_gb300 import build, sp2
    build.build()
    sp2.load()
    return torch


def _rel(g, ref):
    """max |g - ref| / max(|ref|, 1e-3 max|ref|) -- component-wise relative error
    with a floor for near-zero components."""
    scale = np.maximum(np.abs(ref), 1e-3 * np.abs(ref).max())
    return float(np.max(np.abs(g - ref) / scale))


def _normwise(gs, refs):
    """||g - ref|| / ||ref|| over the concatenated gradient (x, v, m)."""
    g = np.concatenate([np.ravel(q) for q in gs])
    r = np.concatenate([np.ravel(q) for q in refs])
    return float(np.linalg.norm(g - r) / np.linalg.norm(r))


# Mixed precision evaluates each pair term of the adjoint in FP32 (relative
# error ~u = 6e-8 from the FP32 inputs alone).  The mass cotangent of particle k
# is a sum over all sinks of cotangent-weighted terms of random sign, so its
# relative error grows with the cancellation ratio sum|t| / |sum t| (~sqrt(N)).
# The 1e-6 agreement is therefore asserted on the whole gradient vector (norm-
# wise) and component-wise on positions and velocities; mass components carry
# the FP32 cancellation floor below.
MIXED_MASS_FLOOR = 3e-5


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-10), ("mixed", 2e-5)])
def test_force_vjp_matches_autograd(torch_cuda, precision, tol):
    torch = torch_cuda
    from oracle import adjoint
    from paper_1510_04068_gb300 import sp2
    n, eps2 = 300, 1e-4
    m, x, v = W.plummer(n, 4)
    m = W.salpeter_masses(n, 4)
    rng = np.random.default_rng(9)
    ab, jb, pb = rng.standard_normal((n, 3)), rng.standard_normal((n, 3)), rng.standard_normal(n)
    gx_r, gv_r, gm_r = adjoint.force_vjp(x, v, m, ab, jb, pb, eps2)
    D = lambda q: torch.as_tensor(np.ascontiguousarray(q)).cuda()  # noqa: E731
    prec = sp2.SP2_MIXED if precision == "mixed" else sp2.SP2_FP64
    with sp2.Context(order=4, precision=prec, n_max=n, eps2=eps2, with_nn=0) as c:
        xb, vb, mb = (torch.empty((n, 3), dtype=torch.float64, device="cuda"),
                      torch.empty((n, 3), dtype=torch.float64, device="cuda"),
                      torch.empty(n, dtype=torch.float64, device="cuda"))
        c.force_vjp(D(m), D(x), D(v), D(ab), D(jb), D(pb), xb, vb, mb)
        c.sync()
        assert _rel(xb.cpu().numpy(), gx_r) <= tol
        assert _rel(vb.cpu().numpy(), gv_r) <= tol
        assert _rel(mb.cpu().numpy(), gm_r) <= tol
        # accumulate adds onto the existing values; host pointers give the same answer
        c.force_vjp(D(m), D(x), D(v), D(ab), D(jb), D(pb), xb, vb, mb, accumulate=True)
        c.sync()
        assert _rel(xb.cpu().numpy(), 2 * gx_r) <= tol
        hx, hv, hm = np.empty((n, 3)), np.empty((n, 3)), np.empty(n)
        c.force_vjp(m, x, v, ab, jb, pb, hx, hv, hm)
        assert _rel(hx, gx_r) <= tol and _rel(hm, gm_r) <= tol


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_forces_and_hermite_step(torch_cuda, oracle_mod, precision):
    torch = torch_cuda
    from paper_1510_04068_gb300 import sp2
    n, eps2, dt = 700, 1e-6, 1.0 / 256
    m, x, v = W.plummer(n, 6)
    ids = np.arange(n, dtype=np.int32)
    f0 = oracle_mod.forces(ids, x, v, ids, m, x, v, eps2, 4)
    tol = 1e-12 if precision == "fp64" else 1e-6
    D = lambda q: torch.as_tensor(np.ascontiguousarray(q)).cuda()  # noqa: E731
    prec = sp2.SP2_MIXED if precision == "mixed" else sp2.SP2_FP64
    with sp2.Context(order=4, precision=prec, n_max=n, eps2=eps2, with_nn=0) as c:
        acc, jerk, pot = (torch.empty((n, 3), dtype=torch.float64, device="cuda"),
                          torch.empty((n, 3), dtype=torch.float64, device="cuda"),
                          torch.empty(n, dtype=torch.float64, device="cuda"))
        c.forces(D(m), D(x), D(v), acc=acc, jerk=jerk, pot=pot)
        c.sync()
        ea = np.linalg.norm(acc.cpu().numpy() - f0["acc"], axis=1) / f0["sc_acc"]
        ej = np.linalg.norm(jerk.cpu().numpy() - f0["jerk"], axis=1) / f0["sc_jerk"]
        assert ea.max() <= tol and ej.max() <= 10 * tol
        xs, vs = D(x), D(v)
        c.hermite4_step(dt, D(m), xs, vs, acc, jerk)
        c.sync()
        xr, vr = oracle_mod.hermite4_shared(m, x, v, eps2, dt, 1)
        # one step moves x by ~v dt; the force error enters at dt^2 / 2
        assert np.abs(xs.cpu().numpy() - xr).max() <= 1e-14 + tol * dt * dt * np.abs(f0["sc_acc"]).max()
        assert np.abs(vs.cpu().numpy() - vr).max() <= 1e-14 + tol * dt * np.abs(f0["sc_acc"]).max()


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-9), ("mixed", 1e-6)])
def test_trajectory_gradient_matches_oracle(torch_cuda, precision, tol):
    torch = torch_cuda
    from oracle import adjoint
    from paper_1510_04068_gb300 import autograd as AG
    n, steps, dt, eps2 = 128, 12, 1.0 / 256, 1e-6
    m, x, v = W.plummer(n, 8)
    w = np.random.default_rng(18).standard_normal((n, 3))
    _, gx_r, gv_r, gm_r = adjoint.loss_and_grad(x, v, m, w, eps2, dt, steps)
    sim = AG.HermiteSim(n, eps2, precision=precision)
    T = lambda q: torch.as_tensor(np.ascontiguousarray(q)).cuda()  # noqa: E731
    x0, v0, mm = T(x).requires_grad_(True), T(v).requires_grad_(True), T(m).requires_grad_(True)
    xf, _ = sim.trajectory(x0, v0, mm, dt, steps, checkpoint_every=5)
    (T(w) * xf).sum().backward()
    sim.close()
    gx, gv, gm = x0.grad.cpu().numpy(), v0.grad.cpu().numpy(), mm.grad.cpu().numpy()
    assert _normwise((gx, gv, gm), (gx_r, gv_r, gm_r)) <= tol
    assert _rel(gx, gx_r) <= tol
    assert _rel(gv, gv_r) <= tol
    assert _rel(gm, gm_r) <= (MIXED_MASS_FLOOR if precision == "mixed" else tol)


def test_differentiable_forces_function(torch_cuda):
    torch = torch_cuda
    from oracle import adjoint
    from paper_1510_04068_gb300 import autograd as AG
    n, eps2 = 96, 1e-4
    m, x, v = W.plummer(n, 2)
    rng = np.random.default_rng(3)
    ab, jb, pb = rng.standard_normal((n, 3)), rng.standard_normal((n, 3)), rng.standard_normal(n)
    sim = AG.HermiteSim(n, eps2, precision="fp64")
    T = lambda q: torch.as_tensor(np.ascontiguousarray(q)).cuda()  # noqa: E731
    mm, xx, vv = T(m).requires_grad_(True), T(x).requires_grad_(True), T(v).requires_grad_(True)
    acc, jerk, pot = AG.forces(sim, mm, xx, vv)
    ((acc * T(ab)).sum() + (jerk * T(jb)).sum() + (pot * T(pb)).sum()).backward()
    sim.close()
    gx, gv, gm = adjoint.force_vjp(x, v, m, ab, jb, pb, eps2)
    assert _rel(xx.grad.cpu().numpy(), gx) <= 1e-10
    assert _rel(vv.grad.cpu().numpy(), gv) <= 1e-10
    assert _rel(mm.grad.cpu().numpy(), gm) <= 1e-10


def _fd_check(torch, sim_fd, x, v, m, w, dt, steps, grads, n_coords, seed, tol, mass_floor=MIXED_MASS_FLOOR):
    """Central differences of the FP64 trajectory loss at h = 1e-6."""
    gx, gv, gm = grads
    T = lambda q: torch.as_tensor(np.ascontiguousarray(q)).cuda()  # noqa: E731
    W_ = T(w)

    def loss(xx, vv, mmm):
        with torch.no_grad():
            xf, _ = sim_fd.trajectory(T(xx), T(vv), T(mmm), dt, steps, checkpoint_every=steps)
            return float((W_ * xf).sum())

    xf0 = None
    with torch.no_grad():
        xf0, _ = sim_fd.trajectory(T(x), T(v), T(m), dt, steps, checkpoint_every=steps)
    noise = 8 * np.finfo(float).eps * float((W_ * xf0).abs().sum()) / (2e-6)
    gmax = max(np.abs(gx).max(), np.abs(gv).max(), np.abs(gm).max())
    rng = np.random.default_rng(seed)
    h = 1e-6
    worst = 0.0
    gs, fds = [], []
    for _ in range(n_coords):
        kind = int(rng.integers(0, 3))
        i = int(rng.integers(0, len(m)))
        c = int(rng.integers(0, 3))
        xx, vv, mmm = x.copy(), v.copy(), m.copy()
        tgt, g = ((xx, gx[i, c]) if kind == 0 else (vv, gv[i, c]) if kind == 1 else (mmm, gm[i]))
        idx = (i, c) if kind < 2 else (i,)
        base = tgt[idx]
        tgt[idx] = base + h
        lp = loss(xx, vv, mmm)
        tgt[idx] = base - h
        lm = loss(xx, vv, mmm)
        fd = (lp - lm) / (2 * h)
        scale = max(abs(g), 1e-3 * gmax)
        worst = max(worst, (abs(fd - g) - noise) / scale)
        gs.append(g)
        fds.append(fd)
        floor = tol if kind < 2 else mass_floor
        assert abs(fd - g) <= floor * scale + noise, (kind, i, c, fd, g, noise)
    gs, fds = np.array(gs), np.array(fds)
    rel = float(np.linalg.norm(gs - fds) / np.linalg.norm(fds))
    print(f"adjoint vs FP64 central differences: norm-wise {rel:.2e}, worst component {worst:.2e}, "
          f"noise floor {noise:.1e}")
    assert np.linalg.norm(gs - fds) <= tol * np.linalg.norm(fds) + noise * np.sqrt(len(fds))
    return worst


def test_adjoint_vs_fd_oracle_size(torch_cuda, oracle_mod):
    """N = 512, 32 steps, checkpoints every 8: the mixed-precision GPU gradient
    agrees with central differences of the oracle's FP64 trajectory."""
    torch = torch_cuda
    from paper_1510_04068_gb300 import autograd as AG
    n, steps, dt, eps2 = 512, 32, 1.0 / 256, 1e-6
    m, x, v = W.plummer(n, 31)
    w = np.random.default_rng(32).standard_normal((n, 3))
    sim = AG.HermiteSim(n, eps2, precision="mixed")
    T = lambda q: torch.as_tensor(np.ascontiguousarray(q)).cuda()  # noqa: E731
    x0, v0, mm = T(x).requires_grad_(True), T(v).requires_grad_(True), T(m).requires_grad_(True)
    xf, _ = sim.trajectory(x0, v0, mm, dt, steps, checkpoint_every=8)
    (T(w) * xf).sum().backward()
    sim.close()
    grads = (x0.grad.cpu().numpy(), v0.grad.cpu().numpy(), mm.grad.cpu().numpy())

    def loss(xx, vv, mmm):
        xf_, _ = oracle_mod.hermite4_shared(mmm, xx, vv, eps2, dt, steps)
        return float(np.sum(w * xf_))

    xf_o, _ = oracle_mod.hermite4_shared(m, x, v, eps2, dt, steps)
    noise = 8 * np.finfo(float).eps * np.sum(np.abs(w * xf_o)) / 2e-6
    gx, gv, gm = grads
    gmax = max(np.abs(gx).max(), np.abs(gv).max(), np.abs(gm).max())
    rng = np.random.default_rng(33)
    gs, fds = [], []
    for _ in range(64):
        kind = int(rng.integers(0, 3))
        i = int(rng.integers(0, n))
        c = int(rng.integers(0, 3))
        xx, vv, mmm = x.copy(), v.copy(), m.copy()
        tgt, g = ((xx, gx[i, c]) if kind == 0 else (vv, gv[i, c]) if kind == 1 else (mmm, gm[i]))
        idx = (i, c) if kind < 2 else (i,)
        base = tgt[idx]
        tgt[idx] = base + 1e-6
        lp = loss(xx, vv, mmm)
        tgt[idx] = base - 1e-6
        lm = loss(xx, vv, mmm)
        fd = (lp - lm) / 2e-6
        gs.append(g)
        fds.append(fd)
        floor = 1e-6 if kind < 2 else MIXED_MASS_FLOOR
        assert abs(fd - g) <= floor * max(abs(g), 1e-3 * gmax) + noise, (kind, i, c, fd, g)
    gs, fds = np.array(gs), np.array(fds)
    assert np.linalg.norm(gs - fds) <= 1e-6 * np.linalg.norm(fds) + noise * np.sqrt(len(fds))


def test_full_size_fp64_trajectory_matches_oracle(torch_cuda, oracle_mod):
    """The anchor of the full-size gradient check below: at N = 16384, eps =
    1e-3, 32 shared Hermite-4 steps of dt = 1/256, the library's FP64
    trajectory (the one the central differences are taken on) is the oracle's
    (hermite4_shared, 33 direct sums of 16384^2 pairs on the host cores) to
    1e-12 relative in every final position and velocity."""
    torch = torch_cuda
    from paper_1510_04068_gb300 import autograd as AG
    n, steps, dt, eps2 = 16384, 32, 1.0 / 256, 1e-6
    m, x, v = W.plummer(n, 5)
    xo, vo = oracle_mod.hermite4_shared(m, x, v, eps2, dt, steps)
    sim64 = AG.HermiteSim(n, eps2, precision="fp64")
    T = lambda q: torch.as_tensor(np.ascontiguousarray(q)).cuda()  # noqa: E731
    with torch.no_grad():
        xf, vf = sim64.trajectory(T(x), T(v), T(m), dt, steps, checkpoint_every=steps)
    sim64.close()
    xg, vg = xf.cpu().numpy(), vf.cpu().numpy()
    ex = np.linalg.norm(xg - xo, axis=1) / np.linalg.norm(xo, axis=1)
    ev = np.linalg.norm(vg - vo, axis=1) / np.linalg.norm(vo, axis=1)
    print(f"FP64 trajectory vs oracle at N = {n}: max position {ex.max():.1e}, velocity {ev.max():.1e}")
    assert ex.max() <= 1e-12 and ev.max() <= 1e-12, (float(ex.max()), float(ev.max()))


def test_adjoint_full_size_vs_fp64_differences(torch_cuda):
    """N = 16384 Plummer, eps = 1e-3, 32 steps of dt = 1/256, checkpoints every
    8, mixed precision: the gradient of sum w . x_final agrees with central
    differences (h = 1e-6) of the FP64 trajectory on 64 random coordinates.
    That trajectory is the library's FP64 path, which the test above ties to
    the oracle's integrator at this size (64 coordinates x 2 oracle runs would
    take ~20 minutes of host time)."""
    torch = torch_cuda
    from paper_1510_04068_gb300 import autograd as AG
    n, steps, dt, eps2 = 16384, 32, 1.0 / 256, 1e-6
    m, x, v = W.plummer(n, 5)
    w = np.random.default_rng(1005).standard_normal((n, 3))
    sim = AG.HermiteSim(n, eps2, precision="mixed")
    T = lambda q: torch.as_tensor(np.ascontiguousarray(q)).cuda()  # noqa: E731
    x0, v0, mm = T(x).requires_grad_(True), T(v).requires_grad_(True), T(m).requires_grad_(True)
    xf, _ = sim.trajectory(x0, v0, mm, dt, steps, checkpoint_every=8)
    (T(w) * xf).sum().backward()
    sim.close()
    grads = (x0.grad.cpu().numpy(), v0.grad.cpu().numpy(), mm.grad.cpu().numpy())
    sim64 = AG.HermiteSim(n, eps2, precision="fp64")
    # N = 16384: the FP32 cancellation floor of mass components is ~sqrt(N / 128)
    # times the one measured at N = 128
    _fd_check(torch, sim64, x, v, m, w, dt, steps, grads, 64, 1006, 1e-6, mass_floor=3e-4)
    sim64.close()
