"""Source-split (j-split) runs over several processes, one GPU each (Sec. 2.2.3:
with several GPUs the work is divided over the sources, every device computes
the contributions of its sources to all sinks, and the partial results are
added).

Every rank keeps the whole particle set in its own context and runs the force
pass over its own contiguous block of source slots with ``sp2_compute_range``.
The paper's library gives each GPU only its (round-robin) subset of the
sources to save memory, transfers and prediction time; here the store is
O(N) and small next to the GPU's memory, the active particles' updates reach
every rank as the i-particles reach every device in the paper, and a pass
whose sinks fit one CTA predicts only its own block of sources, so the
prediction is divided too.  Because acc, jerk, snap and pot are sums over sources,
a rank's outputs are its partial sums; the nearest neighbour of a rank is the
best one among its sources.  One exchange then gives every rank the full
result: a sum of the force fields and a lexicographic (r^2, id) minimum of the
nearest neighbours, both as torch.distributed collectives (NCCL between GPUs,
gloo between CPU processes).  No arithmetic of the method runs outside the
library's kernels; the collectives only add the ranks' partial sums.
"""
from __future__ import annotations

from . import sp2 as _sp2

_INT32_MAX = 2 ** 31 - 1


def shard_range(n: int, rank: int, world: int) -> tuple[int, int]:
    """Source slots [lo, hi) of `rank` among `world` ranks: contiguous blocks
    whose sizes differ by at most one."""
    if world < 1 or not 0 <= rank < world or n < 0:
        raise ValueError("need 0 <= rank < world and n >= 0")
    return n * rank // world, n * (rank + 1) // world


def compute_shard(ctx, i_idx, rank: int, world: int, **out):
    """This rank's partial: the force pass on sinks i_idx (slots of the loaded
    set) over its own block of sources (outputs as for sp2_compute)."""
    c = ctx.ctx if hasattr(ctx, "ctx") else ctx
    lo, hi = shard_range(_sp2.sp2_info(c)["n_loaded"], rank, world)
    _sp2.sp2_compute(c, i_idx, j_range=(lo, hi), **out)
    return lo, hi


def combine(out: dict, group=None) -> dict:
    """Exchange of the ranks' partials, in place: acc, jerk, snap and pot
    (whichever are given, torch tensors) are summed over the ranks; nn_r2 and
    nn_id become the lexicographic (r^2, id) minimum over the ranks (id -1 and
    r^2 = +inf where no rank has a neighbour).  Tensors may live on the GPU
    (NCCL) or the CPU (gloo); every rank must pass the same keys and shapes."""
    import torch
    import torch.distributed as dist

    fields = [k for k in ("acc", "jerk", "snap", "pot") if out.get(k) is not None]
    if fields:
        n_i = out[fields[0]].shape[0]
        flat = torch.cat([out[k].reshape(n_i, -1) for k in fields], dim=1)
        dist.all_reduce(flat, op=dist.ReduceOp.SUM, group=group)
        col = 0
        for k in fields:
            w = out[k].reshape(n_i, -1).shape[1]
            out[k].copy_(flat[:, col:col + w].reshape(out[k].shape))
            col += w
    r2, nid = out.get("nn_r2"), out.get("nn_id")
    if r2 is not None and nid is not None:
        best = r2.clone()
        dist.all_reduce(best, op=dist.ReduceOp.MIN, group=group)
        cand = torch.where((r2 == best) & (nid >= 0), nid, torch.full_like(nid, _INT32_MAX))
        dist.all_reduce(cand, op=dist.ReduceOp.MIN, group=group)
        nid.copy_(torch.where(cand == _INT32_MAX, torch.full_like(cand, -1), cand))
        r2.copy_(best)
    elif r2 is not None or nid is not None:
        raise ValueError("nn_r2 and nn_id go together")
    return out

