"""GB300 (sm_103a) direct-summation gravity library (the Sapporo2 hot path).

``sp2``      -- the C-ABI binding (sp2_open, sp2_set_j, sp2_predict, sp2_compute, ...)
``autograd`` -- differentiable forces and checkpointed Hermite-4 trajectories
``shards``   -- the source split over several processes (one GPU each) and its exchange
``build``    -- in-tree nvcc build of libsapporo_gb.so
"""
from . import sp2  # noqa: F401
from .sp2 import SP2_DEVICE, SP2_FP64, SP2_HOST, SP2_MIXED, Context, SP2Error  # noqa: F401

__all__ = ["sp2", "Context", "SP2Error", "SP2_FP64", "SP2_MIXED", "SP2_HOST", "SP2_DEVICE"]
