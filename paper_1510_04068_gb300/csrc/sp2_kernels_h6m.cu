// sp2_kernels_h6m.cu -- instantiation unit: MixedForce policy, order 6 (force pass,
// split-j reduction, batched kernel).  One unit per (order, precision) so the
// variants compile in parallel.
#include "sp2_device.cuh"

SP2_DEFINE_FORCE_TU(h6m, MixedForce, 6)
