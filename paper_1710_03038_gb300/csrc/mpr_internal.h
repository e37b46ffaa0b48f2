// Host/device shared layout of an MPR context and the launchers that the
// translation units of the library provide to each other.
#pragma once

#include <cstddef>
#include <cstdint>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "mpr.h"

namespace mpr {

// Tile of the tiled path.  Origins are multiples of the (even) tile sizes,
// so the colour of extended-tile cell (xx, yy) is (xx + yy) & 1.  The record
// is 16 words (64 bytes) so that 16 lanes load it in one access; it repeats
// the image offsets the colour pass needs to address the tile's state.
struct TileDesc {
    int img;
    int x0, y0;
    int cp;           // floats per slot of the image's state (chains rounded up to 4)
    int off[2];       // slot offset of the colour-c gap segment inside the image's slot space
    int cnt[2];       // gap sites of colour c in the tile
    int halo_cnt[2];  // other-colour gap sites in the 1-ring seen by the colour-c pass
    long long state_off;  // float offset of the image's state
    long long slot_off;   // offset of the image in the slot arrays
    int pad[2];
};
static_assert(sizeof(TileDesc) == 64, "tile record: 16 words");

// Per image, in device memory.
struct ImgDev {
    int Lx, Ly;
    long long site_off;   // offset in concatenated [sum Lx*Ly] arrays
    long long state_off;  // float offset of chain 0, slot 0 in the state buffer
    long long stride;     // floats between consecutive chains (tiled: 1)
    long long sstride;    // floats between consecutive slots (tiled: chains rounded up to even)
    long long slot_off;   // tiled: offset in the slot arrays (acc, slot_pos); plain: site_off
    int tile0, ntiles;
    float zmin, zmax;
    float invT, pad0;
    double T, e_s, E_ss, n_bonds;
    long long n_gap, n_sp;
};

// Device-resident counters of a context.
struct Control {
    uint32_t sweep;        // Philox sweep field of the next sweep
    uint32_t equil_index;  // i of Alg. 2 step 4.2 for the next equilibration sweep
    uint32_t status;       // device-side error bits
    uint32_t ticket;       // blocks of the end-of-sweep kernel done (0 between launches)
};

// Accept counts and energy partials of a chain are spread over kSpread
// slots (indexed by thread block) to keep atomic traffic off a single address.
constexpr int kSpread = 32;

// Per-chain device arrays (length n_img * n_chains, image-major; acc_cnt and
// e_cur are kSpread times longer).
struct ChainDev {
    float* a;
    float* alpha;         // (2 pi / a) 2^-24: the proposal width in units of the 24-bit uniform
    uint32_t* acc_cnt;    // accepted proposals of the sweep in progress
    uint32_t* acc_last;   // of the last completed sweep
    double* e_cur;        // bond energy (gap-related part) reduced during the sweep
    double* e_last;       // H / N_GP after the last recorded sweep
    double* e_sum;        // sums of e over measurement sweeps (temperature estimate)
    double* e_sum2;
};

enum SweepFlags : int {
    kEnergy = 1,       // reduce the energy this pass
    kAccumulate = 2,   // add the new angles to the realisation accumulators
    kAccumulate2 = 4,  // also squares
    kAlphaOne = 8,     // a = 1 (printed Alg. 2 step 5.2)
    kLiteralOR = 16,   // printed q = 1 over-relaxation formula (plain path only)
    kGMRF = 32,        // GMRF pair interaction of Sec. 4.3 (plain path only)
};

struct SweepArgs {
    const ImgDev* img;
    const TileDesc* tiles;      // tiled path
    const uint32_t* slot_pos;   // tiled: (y << 16) | x per slot, 0xFFFFFFFF for padding
    const uint2* slot_ref;      // tiled: table entries of the slot's gap neighbours (u16 x 4)
    const float4* slot_cs;      // tiled: the slot's sample field: sum over its sample neighbours of
                                // (cos q phi, sin q phi, cos phi, sin phi); GMRF: (sum phi, number
                                // of existing neighbours, 0, 0)
    const int2* halo;           // tiled: [tile][2][cap] (slot, cs index)
    const float* samp;          // tiled: sample angle per site (>= 0) or -1 at gaps
    float* state;
    double* acc1;
    double* acc2;
    ChainDev ch;
    Control* ctl;
    uint2 key;
    uint32_t rk[20];           // Philox round keys k_i = key + i * (0x9E3779B9, 0xBB67AE85)
    float q, inv_q, two_pi_q, J;
    int n_chains;
    int chain_group;
    int chain0, chain_end;     // tiled: the launch covers chains [chain0, chain_end), chain0 even
    int colour;
    int flags;
    int halo_cap;
    int gt;                    // tiled: table entries per chain pair for this pass (largest tile)
    const int* tile_list;      // tiled: k-th tile of the launch is tile_list[tile_base + k] (null: k)
    int tile_base;
    int n_list;                // tiled: tiles in the launch
    int n_img;
    uint32_t img_tag;          // OR-ed into the image field of the counter (1 << 30: T lattices)
};

// Records the message returned by mpr_last_error() for this thread; returns s.
mpr_status set_last_error(mpr_status s, const std::string& msg);

// ---- launchers ------------------------------------------------------------
// setup_only: set the kernel's attributes without launching (before a capture)
// (chain_group: even and at most 32, or covering every chain)
cudaError_t launch_tiled_pass(const SweepArgs& a, int tile_x, int tile_y, cudaStream_t s,
                              bool setup_only = false);
cudaError_t launch_plain_pass(const SweepArgs& a, int max_Lx, int max_Ly, cudaStream_t s);
bool tiled_config_supported(int tile_x, int tile_y);
// the printed over-relaxation and the GMRF model run with 16 x 16 tiles
bool tiled_model_supported(int tile_x, int tile_y, int flags);

// tile-table construction (tiled path)
cudaError_t launch_tile_count(const ImgDev* img, const TileDesc* tiles, int n_tiles,
                              const uint8_t* gap, int tile_x, int tile_y, int* counts,
                              cudaStream_t s);
cudaError_t launch_tile_fill(const ImgDev* img, const TileDesc* tiles, int n_tiles,
                             const uint8_t* gap, int tile_x, int tile_y, uint32_t* slot_pos,
                             int* slot_map, int2* halo, int halo_cap, cudaStream_t s);
// per slot: the table entries of its gap neighbours in the pass of its own
// colour (up, down, left, right; 0 = not a gap) and its sample field
cudaError_t launch_tile_const(const ImgDev* img, const TileDesc* tiles, int n_tiles, int tile_x,
                              int tile_y, const uint32_t* slot_pos, const int2* halo, int halo_cap,
                              const float* samp, float q, int gmrf, uint2* slot_ref,
                              float4* slot_cs, cudaStream_t s);
// Dynamic shared memory of a colour-pass block of tile shape tx x ty for a
// launch whose largest tile has gt table entries; flags: the model bits of
// SweepFlags (kLiteralOR, kGMRF).
size_t tiled_pass_smem(int tx, int ty, int gt, int chain_group, int flags);
// blocks of the colour pass one SM holds by their threads and registers
int tiled_blocks_per_sm(int tx, int ty);

// float offset of gap slot k (tiled) or site k (plain) of a realisation
__host__ __device__ inline long long state_index(const ImgDev& I, int chain, long long k) {
    return I.state_off + (long long)chain * I.stride + k * I.sstride;
}

}  // namespace mpr
