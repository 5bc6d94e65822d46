// sp2_kernels_h4m.cu -- instantiation unit: mixed precision, order 4 (force pass and
// split-j reduction with MixedPairForce, batched kernel with MixedPairBatch).  One
// unit per (order, precision) so the variants compile in parallel.
#include "sp2_device.cuh"

SP2_DEFINE_FORCE_TU(h4m, MixedPairForce, MixedPairBatch, 4)
