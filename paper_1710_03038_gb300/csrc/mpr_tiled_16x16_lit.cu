// Colour pass for 16 x 16 tiles with the over-relaxation as printed (q = 1 field).
#include "mpr_tiled_kernel.cuh"

namespace mpr {

cudaError_t launch_tiled_16x16_lit(const SweepArgs& a, cudaStream_t s, bool setup_only) {
    return tiled::launch_shape<16, 16, 4, tiled::kModelLIT>(a, s, setup_only);
}

}  // namespace mpr
