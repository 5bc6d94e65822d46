// sp2_kernels_h4m.cu -- instantiation unit: MixedForce policy, order 4 (force pass,
// split-j reduction, batched kernel).  One unit per (order, precision) so the
// variants compile in parallel.
#include "sp2_device.cuh"

SP2_DEFINE_FORCE_TU(h4m, MixedForce, 4)
