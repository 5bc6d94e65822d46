// sp2_kernels_h2m.cu -- instantiation unit: mixed precision, order 2 (the
// leap-frog / GRAPE-5 kernel of Sec. 1: acceleration and potential only;
// force pass and split-j reduction with MixedPairForce, batched kernel with
// MixedPairBatch).  One unit per (order, precision) so the variants compile in
// parallel.
#include "sp2_device.cuh"

SP2_DEFINE_FORCE_TU(h2m, MixedPairForce, MixedPairBatch, 2)
