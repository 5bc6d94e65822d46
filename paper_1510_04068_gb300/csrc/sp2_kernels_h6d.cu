// sp2_kernels_h6d.cu -- instantiation unit: Fp64Force policy, order 6 (force pass,
// split-j reduction, batched kernel).  One unit per (order, precision) so the
// variants compile in parallel.
#include "sp2_device.cuh"

SP2_DEFINE_FORCE_TU(h6d, Fp64Force, Fp64Force, 6)
