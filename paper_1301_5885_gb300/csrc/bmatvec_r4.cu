// bmatvec_r4.cu -- instantiations of the batched product for R = 4
// right-hand sides (the kernel and its shapes are in bmatvec.cuh).
#define PB_BMATVEC_KERNELS
#include "bmatvec.cuh"

namespace pb {

template <>
cudaError_t bmatvec_run<4>(int T, int acc, const BmvArgs &a, unsigned grid, cudaStream_t s, int *occ) {
    PB_BMV_SHAPES_R4(PB_BMV_SHAPE)
    return cudaErrorInvalidValue;
}

}  // namespace pb
