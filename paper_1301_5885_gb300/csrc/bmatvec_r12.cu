// bmatvec_r12.cu -- instantiations of the batched product for R = 1, 2
// right-hand sides (the kernel and its shapes are in bmatvec.cuh).
#define PB_BMATVEC_KERNELS
#include "bmatvec.cuh"

namespace pb {

template <>
cudaError_t bmatvec_run<1>(int T, int acc, const BmvArgs &a, unsigned grid, cudaStream_t s, int *occ) {
    PB_BMV_SHAPES_R1(PB_BMV_SHAPE)
    return cudaErrorInvalidValue;
}

template <>
cudaError_t bmatvec_run<2>(int T, int acc, const BmvArgs &a, unsigned grid, cudaStream_t s, int *occ) {
    PB_BMV_SHAPES_R2(PB_BMV_SHAPE)
    return cudaErrorInvalidValue;
}

}  // namespace pb
