"""Differentiable gravity on the GPU library.

``forces(sim, m, x, v)``   acc, jerk, pot of all particles (every particle a
                           sink and a source), differentiable w.r.t. (m, x, v):
                           the backward pass is the library's adjoint kernel
                           (sp2_force_vjp), one pairwise pass.
``HermiteSim.trajectory``  shared-step 4th-order Hermite integration for a fixed
                           number of steps, differentiable w.r.t. the initial
                           positions, velocities and masses.  The forward pass
                           keeps the state every ``checkpoint_every`` steps; the
                           backward pass recomputes each segment from its
                           checkpoint and runs the step adjoints
                           (sp2_hermite4_step_vjp) in reverse.

Every arithmetic step runs in libsapporo_gb.so; torch provides memory,
streams and the autograd plumbing.
"""
from __future__ import annotations

import torch

from . import sp2


def _dev(t):
    return t.detach().contiguous()


class HermiteSim:
    """Owns an order-4 library context for n particles (nearest neighbour off)."""

    def __init__(self, n: int, eps2: float, precision: str = "mixed", stream=None):
        self.n = n
        self.eps2 = eps2
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        prec = sp2.SP2_MIXED if precision == "mixed" else sp2.SP2_FP64
        self.ctx = sp2.Context(order=4, precision=prec, n_max=n, eps2=eps2, with_nn=0,
                               cuda_stream=self.stream.cuda_stream)

    def close(self):
        self.ctx.close()

    def trajectory(self, x0, v0, m, dt: float, n_steps: int, checkpoint_every: int = 8):
        return _Trajectory.apply(x0, v0, m, self, float(dt), int(n_steps), int(checkpoint_every))


class _Forces(torch.autograd.Function):
    @staticmethod
    def forward(fctx, m, x, v, sim):
        with torch.cuda.stream(sim.stream):
            m_, x_, v_ = _dev(m), _dev(x), _dev(v)
            acc = torch.empty_like(x_)
            jerk = torch.empty_like(x_)
            pot = torch.empty_like(m_)
            sim.ctx.forces(m_, x_, v_, acc=acc, jerk=jerk, pot=pot)
        fctx.save_for_backward(m_, x_, v_)
        fctx.sim = sim
        return acc, jerk, pot

    @staticmethod
    def backward(fctx, ga, gj, gp):
        m, x, v = fctx.saved_tensors
        sim = fctx.sim
        with torch.cuda.stream(sim.stream):
            z3 = torch.zeros_like(x)
            ga = z3 if ga is None else ga.contiguous()
            gj = z3 if gj is None else gj.contiguous()
            gp = torch.zeros_like(m) if gp is None else gp.contiguous()
            xb, vb, mb = torch.empty_like(x), torch.empty_like(v), torch.empty_like(m)
            sim.ctx.force_vjp(m, x, v, ga, gj, gp, xb, vb, mb)
        return mb, xb, vb, None


def forces(sim: HermiteSim, m, x, v):
    """(acc, jerk, pot) with a library-computed vector-Jacobian product."""
    return _Forces.apply(m, x, v, sim)


class _Trajectory(torch.autograd.Function):
    @staticmethod
    def forward(fctx, x0, v0, m, sim, dt, n_steps, every):
        with torch.cuda.stream(sim.stream):
            m_ = _dev(m)
            x, v = _dev(x0).clone(), _dev(v0).clone()
            a, j = torch.empty_like(x), torch.empty_like(x)
            sim.ctx.forces(m_, x, v, acc=a, jerk=j)
            ckpts = []
            for k in range(n_steps):
                if k % every == 0:
                    ckpts.append((x.clone(), v.clone(), a.clone(), j.clone()))
                sim.ctx.hermite4_step(dt, m_, x, v, a, j)
        fctx.sim, fctx.dt, fctx.n_steps, fctx.every = sim, dt, n_steps, every
        fctx.ckpts = ckpts
        fctx.save_for_backward(_dev(x0), _dev(v0), m_)
        return x, v

    @staticmethod
    def backward(fctx, gxf, gvf):
        x0, v0, m = fctx.saved_tensors
        sim, dt, n_steps, every = fctx.sim, fctx.dt, fctx.n_steps, fctx.every
        with torch.cuda.stream(sim.stream):
            gx = torch.zeros_like(x0) if gxf is None else gxf.contiguous().clone()
            gv = torch.zeros_like(v0) if gvf is None else gvf.contiguous().clone()
            ga, gj = torch.zeros_like(x0), torch.zeros_like(x0)
            gm = torch.zeros_like(m)
            for seg in reversed(range(len(fctx.ckpts))):
                x, v, a, j = (t.clone() for t in fctx.ckpts[seg])
                first = seg * every
                last = min(first + every, n_steps)
                # recompute the segment's step inputs (the state after its
                # last step is the next segment's checkpoint: not needed here)
                states = [(x, v, a, j)]
                for _ in range(first + 1, last):
                    x, v, a, j = (t.clone() for t in states[-1])
                    sim.ctx.hermite4_step(dt, m, x, v, a, j)
                    states.append((x, v, a, j))
                for xs, vs, as_, js in reversed(states):
                    sim.ctx.hermite4_step_vjp(dt, m, xs, vs, as_, js, gx, gv, ga, gj, gm)
            # the initial acc / jerk are forces of (x0, v0, m)
            sim.ctx.force_vjp(m, x0, v0, ga, gj, None, gx, gv, gm, accumulate=True)
        fctx.ckpts = None
        return gx, gv, gm, None, None, None, None
