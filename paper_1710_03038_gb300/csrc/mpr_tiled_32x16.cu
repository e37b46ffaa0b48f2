// Colour pass for 32 x 16 tiles (8 warps per block).
#include "mpr_tiled_kernel.cuh"

namespace mpr {

cudaError_t launch_tiled_32x16(const SweepArgs& a, int n_tiles, cudaStream_t s, bool setup_only) {
    return tiled::launch_shape<32, 16, 8, tiled::kModelMPR>(a, n_tiles, s, setup_only);
}

}  // namespace mpr
