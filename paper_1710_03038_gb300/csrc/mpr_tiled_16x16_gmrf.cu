// Colour pass for 16 x 16 tiles with the GMRF pair interaction of Sec. 4.3.
#include "mpr_tiled_kernel.cuh"

namespace mpr {

cudaError_t launch_tiled_16x16_gmrf(const SweepArgs& a, cudaStream_t s, bool setup_only) {
    return tiled::launch_shape<16, 16, 4, tiled::kModelGMRF>(a, s, setup_only);
}

}  // namespace mpr
