// sp2_kernels_h6m.cu -- instantiation unit: mixed precision, order 6 (force pass and
// split-j reduction with MixedPairForce, batched kernel with MixedPairBatch).  One
// unit per (order, precision) so the variants compile in parallel.
#include "sp2_device.cuh"

SP2_DEFINE_FORCE_TU(h6m, MixedPairForce, MixedPairBatch, 6)
