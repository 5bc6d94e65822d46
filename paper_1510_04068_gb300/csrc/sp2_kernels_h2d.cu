// sp2_kernels_h2d.cu -- instantiation unit: FP64, order 2 (the leap-frog /
// GRAPE-5 kernel of Sec. 1: acceleration and potential only; force pass,
// split-j reduction, batched kernel).  One unit per (order, precision) so the
// variants compile in parallel.
#include "sp2_device.cuh"

SP2_DEFINE_FORCE_TU(h2d, Fp64Force, Fp64Force, 2)
