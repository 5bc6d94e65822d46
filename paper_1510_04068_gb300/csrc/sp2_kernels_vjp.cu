// sp2_kernels_vjp.cu -- instantiation unit of the adjoint (VJP) pass in both
// precisions (mixed: the paired f32x2 policy MixedPairVjp).  The VJP reuses the persistent pass skeleton and the split-j
// reduction; it has no batched form.
#include "sp2_device.cuh"

namespace sp2 {

#define SP2_VJP_TU(SUFFIX, POLICY)                                                                      \
    cudaError_t launch_force_##SUFFIX(const KernelKey &k, const ForceParams &p, int grid, int threads,  \
                                      size_t tile, cudaStream_t s) {                                    \
        return dispatch_ipt<POLICY>(false, k.ipt, &p, grid, threads, tile, s, nullptr, k.fused);        \
    }                                                                                                   \
    cudaError_t occupancy_force_##SUFFIX(const KernelKey &k, int threads, size_t tile, int *blocks) {    \
        return dispatch_ipt<POLICY>(true, k.ipt, nullptr, 0, threads, tile, 0, blocks, k.fused);        \
    }                                                                                                   \
    cudaError_t launch_reduce_##SUFFIX(const KernelKey &, const ReduceParams &r, cudaStream_t s) {      \
        return launch_reduce<POLICY>(r, s);                                                             \
    }                                                                                                   \
    cudaError_t launch_batched_##SUFFIX(int, const BatchParams &, int, int, cudaStream_t) {             \
        return cudaErrorInvalidValue;                                                                   \
    }                                                                                                   \
    cudaError_t occupancy_batched_##SUFFIX(int, int, int *) { return cudaErrorInvalidValue; }

SP2_VJP_TU(vjpm, MixedPairVjp)
SP2_VJP_TU(vjpd, Fp64Vjp)
#undef SP2_VJP_TU

}  // namespace sp2
