// Colour pass for 32 x 16 tiles .
#include "mpr_tiled_kernel.cuh"

namespace mpr {

cudaError_t launch_tiled_32x16(const SweepArgs& a, cudaStream_t s, bool setup_only) {
    return tiled::launch_shape<32, 16, 8, tiled::kModelMPR>(a, s, setup_only);
}

}  // namespace mpr
