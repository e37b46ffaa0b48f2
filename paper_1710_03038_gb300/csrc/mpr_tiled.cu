// Tiled path: tile tables (slot segments, ring lists) and the dispatch of
// the colour pass to its tile shape (the kernel is in mpr_tiled_kernel.cuh,
// one translation unit per tile shape).
#include "mpr_device.cuh"
#include "mpr_internal.h"
#include "mpr_tiled_kernel.cuh"

namespace mpr {

cudaError_t launch_tiled_32x16(const SweepArgs& a, cudaStream_t s, bool setup_only);
cudaError_t launch_tiled_16x16(const SweepArgs& a, cudaStream_t s, bool setup_only);
cudaError_t launch_tiled_32x32(const SweepArgs& a, cudaStream_t s, bool setup_only);
cudaError_t launch_tiled_16x16_lit(const SweepArgs& a, cudaStream_t s, bool setup_only);
cudaError_t launch_tiled_16x16_gmrf(const SweepArgs& a, cudaStream_t s, bool setup_only);

namespace {

// -------------------------------------------------------------- tile tables

__global__ void tile_count_kernel(const ImgDev* img, const TileDesc* tiles, const uint8_t* gap,
                                  int tx, int ty, int* counts) {
    const TileDesc T = tiles[blockIdx.x];
    const ImgDev& I = img[T.img];
    int c0 = 0, c1 = 0;
    for (int i = threadIdx.x; i < tx * ty; i += blockDim.x) {
        const int X = T.x0 + i % tx, Y = T.y0 + i / tx;
        if (X < I.Lx && Y < I.Ly && gap[I.site_off + (long long)Y * I.Lx + X]) {
            if ((X + Y) & 1) ++c1; else ++c0;
        }
    }
    c0 = __reduce_add_sync(0xffffffffu, c0);
    c1 = __reduce_add_sync(0xffffffffu, c1);
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(counts + 2 * blockIdx.x, c0);
        atomicAdd(counts + 2 * blockIdx.x + 1, c1);
    }
}

// One thread per tile row: row counts, an exclusive scan over rows, then each
// row writes its gap sites in order (row-major inside the tile).
__global__ void tile_fill_kernel(const ImgDev* img, const TileDesc* tiles, const uint8_t* gap,
                                 int tx, int ty, uint32_t* slot_pos, int* slot_map) {
    extern __shared__ int rowcnt[];  // [2][ty]
    const TileDesc T = tiles[blockIdx.x];
    const ImgDev& I = img[T.img];
    const int ly = threadIdx.x;
    const int Y = T.y0 + ly;
    int n0 = 0, n1 = 0;
    if (ly < ty && Y < I.Ly) {
        for (int lx = 0; lx < tx; ++lx) {
            const int X = T.x0 + lx;
            if (X >= I.Lx) break;
            if (gap[I.site_off + (long long)Y * I.Lx + X]) {
                if ((X + Y) & 1) ++n1; else ++n0;
            }
        }
    }
    if (ly < ty) { rowcnt[ly] = n0; rowcnt[ty + ly] = n1; }
    __syncthreads();
    if (threadIdx.x == 0) {
        int s0 = 0, s1 = 0;
        for (int r = 0; r < ty; ++r) {
            const int a0 = rowcnt[r], a1 = rowcnt[ty + r];
            rowcnt[r] = s0; rowcnt[ty + r] = s1;
            s0 += a0; s1 += a1;
        }
    }
    __syncthreads();
    if (ly < ty && Y < I.Ly) {
        int k0 = T.off[0] + rowcnt[ly];
        int k1 = T.off[1] + rowcnt[ty + ly];
        for (int lx = 0; lx < tx; ++lx) {
            const int X = T.x0 + lx;
            if (X >= I.Lx) break;
            const long long site = I.site_off + (long long)Y * I.Lx + X;
            if (gap[site]) {
                const int k = ((X + Y) & 1) ? k1++ : k0++;
                slot_pos[I.slot_off + k] = ((uint32_t)Y << 16) | (uint32_t)X;
                slot_map[site] = k;
            } else {
                slot_map[site] = -1;
            }
        }
    }
}

// Ring lists: for the pass of colour c, the gap cells of the other colour in
// the 1-cell ring around the tile (corners excluded), as (slot, table index).
__global__ void tile_halo_kernel(const ImgDev* img, TileDesc* tiles, const int* slot_map,
                                 int tx, int ty, int2* halo, int cap) {
    __shared__ int n[2];
    const int t = blockIdx.x;
    TileDesc T = tiles[t];
    const ImgDev& I = img[T.img];
    if (threadIdx.x < 2) n[threadIdx.x] = 0;
    __syncthreads();
    const int ring = 2 * tx + 2 * ty;
    for (int i = threadIdx.x; i < ring; i += blockDim.x) {
        int xx, yy;
        if (i < tx) { xx = i + 1; yy = 0; }
        else if (i < 2 * tx) { xx = i - tx + 1; yy = ty + 1; }
        else if (i < 2 * tx + ty) { xx = 0; yy = i - 2 * tx + 1; }
        else { xx = tx + 1; yy = i - 2 * tx - ty + 1; }
        const int X = T.x0 + xx - 1, Y = T.y0 + yy - 1;
        if (X < 0 || X >= I.Lx || Y < 0 || Y >= I.Ly) continue;
        const int slot = slot_map[I.site_off + (long long)Y * I.Lx + X];
        if (slot < 0) continue;
        const int pass = ((xx + yy) & 1) ^ 1;  // the colour whose update reads this cell
        const int k = atomicAdd(&n[pass], 1);
        if (k < cap) halo[((long long)t * 2 + pass) * cap + k] = make_int2(slot, yy * (tx + 2) + xx);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        tiles[t].halo_cnt[0] = n[0] < cap ? n[0] : cap;
        tiles[t].halo_cnt[1] = n[1] < cap ? n[1] : cap;
    }
}

// Per-slot constants of the colour passes, built once per batch: for every
// gap site of colour c, the table entries of its four neighbours in the pass
// of colour c (interior other-colour cells 1 + j, ring cells 1 + n_oth + k,
// 0 where the neighbour is a sample or outside) and its sample field, summed
// over its sample neighbours in the order up, down, left, right:
// (cos q phi, sin q phi, cos phi, sin phi), or for the GMRF model
// (sum of the sample angles, number of existing neighbours, 0, 0).
__global__ void tile_const_kernel(const ImgDev* img, const TileDesc* tiles, int tx, int ty,
                                  const uint32_t* slot_pos, const int2* halo, int halo_cap,
                                  const float* samp_all, float q, int gmrf, uint2* slot_ref,
                                  float4* slot_cs) {
    extern __shared__ uint16_t cellmap[];  // [(ty + 2) * (tx + 2)]
    const TileDesc T = tiles[blockIdx.x];
    const ImgDev& I = img[T.img];
    const int ew = tx + 2, ext = (tx + 2) * (ty + 2);
    const uint32_t* spos = slot_pos + I.slot_off;
    const float* samp = samp_all + I.site_off;
    for (int c = 0; c < 2; ++c) {
        const int oc = c ^ 1;
        for (int i = threadIdx.x; i < ext; i += blockDim.x) cellmap[i] = 0;
        __syncthreads();
        for (int j = threadIdx.x; j < T.cnt[oc]; j += blockDim.x) {
            const uint32_t p = spos[T.off[oc] + j];
            const int X = (int)(p & 0xFFFFu), Y = (int)(p >> 16);
            cellmap[(Y - T.y0 + 1) * ew + (X - T.x0 + 1)] = (uint16_t)(1 + j);
        }
        const int2* hl = halo + ((long long)blockIdx.x * 2 + c) * halo_cap;
        for (int k = threadIdx.x; k < T.halo_cnt[c]; k += blockDim.x)
            cellmap[hl[k].y] = (uint16_t)(1 + T.cnt[oc] + k);
        __syncthreads();
        for (int j = threadIdx.x; j < T.cnt[c]; j += blockDim.x) {
            const uint32_t p = spos[T.off[c] + j];
            const int X = (int)(p & 0xFFFFu), Y = (int)(p >> 16);
            const int xx = X - T.x0 + 1, yy = Y - T.y0 + 1;
            float4 f = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
            uint32_t ref[4];
#pragma unroll
            for (int m = 0; m < 4; ++m) {  // up, down, left, right
                const int dx = m < 2 ? 0 : 2 * m - 5;
                const int dy = m < 2 ? 2 * m - 1 : 0;
                const int nx = X + dx, ny = Y + dy;
                ref[m] = 0u;
                if (nx < 0 || nx >= I.Lx || ny < 0 || ny >= I.Ly) continue;
                if (gmrf) f.y += 1.0f;
                const float v = samp[(long long)ny * I.Lx + nx];
                if (v >= 0.0f) {
                    if (gmrf) {
                        f.x += v;
                    } else {
                        float sn, cs;
                        __sincosf(q * v, &sn, &cs);
                        f.x += cs;
                        f.y += sn;
                        __sincosf(v, &sn, &cs);
                        f.z += cs;
                        f.w += sn;
                    }
                } else {
                    ref[m] = cellmap[(yy + dy) * ew + (xx + dx)];
                }
            }
            slot_ref[I.slot_off + T.off[c] + j] = make_uint2(ref[0] | (ref[1] << 16), ref[2] | (ref[3] << 16));
            slot_cs[I.slot_off + T.off[c] + j] = f;
        }
        __syncthreads();
    }
}

}  // namespace

size_t tiled_pass_smem(int tx, int ty, int gt, int chain_group, int flags) {
    using namespace tiled;
    const int P = pairs_for_group(chain_group);
    if (flags & kGMRF) return Cfg<16, 16, 4, kModelGMRF>::smem_for(gt, P);
    if (flags & kLiteralOR) return Cfg<16, 16, 4, kModelLIT>::smem_for(gt, P);
    if (tx == 32 && ty == 16) return Cfg<32, 16, 8, kModelMPR>::smem_for(gt, P);
    if (tx == 32 && ty == 32) return Cfg<32, 32, 8, kModelMPR>::smem_for(gt, P);
    return Cfg<16, 16, 4, kModelMPR>::smem_for(gt, P);
}

int tiled_blocks_per_sm(int tx, int ty) {
    using namespace tiled;
    if (tx == 32) return 1024 / Cfg<32, 16, 8, kModelMPR>::NT;
    return 1024 / Cfg<16, 16, 4, kModelMPR>::NT;
}

bool tiled_config_supported(int tx, int ty) {
    return (tx == 32 && ty == 16) || (tx == 16 && ty == 16) || (tx == 32 && ty == 32);
}

bool tiled_model_supported(int tx, int ty, int flags) {
    if (flags & (kGMRF | kLiteralOR)) return tx == 16 && ty == 16;
    return tiled_config_supported(tx, ty);
}

cudaError_t launch_tiled_pass(const SweepArgs& a, int tx, int ty, cudaStream_t s,
                              bool setup_only) {
    // chain groups start on a multiple of 4 chains (16-byte aligned rows)
    if (a.chain_group < 1 || a.chain_group > 32 || (a.chain0 & 3) || a.chain0 < 0 ||
        a.chain_end <= a.chain0 || a.chain_end > a.n_chains ||
        (a.chain_group % 4 != 0 && a.chain_group < a.chain_end - a.chain0))
        return cudaErrorInvalidValue;
    if (!tiled_model_supported(tx, ty, a.flags)) return cudaErrorInvalidValue;
    if (a.flags & kGMRF) return launch_tiled_16x16_gmrf(a, s, setup_only);
    if (a.flags & kLiteralOR) return launch_tiled_16x16_lit(a, s, setup_only);
    if (tx == 32 && ty == 16) return launch_tiled_32x16(a, s, setup_only);
    if (tx == 16 && ty == 16) return launch_tiled_16x16(a, s, setup_only);
    if (tx == 32 && ty == 32) return launch_tiled_32x32(a, s, setup_only);
    return cudaErrorInvalidValue;
}

cudaError_t launch_tile_count(const ImgDev* img, const TileDesc* tiles, int n_tiles,
                              const uint8_t* gap, int tx, int ty, int* counts, cudaStream_t s) {
    tile_count_kernel<<<n_tiles, 256, 0, s>>>(img, tiles, gap, tx, ty, counts);
    return cudaGetLastError();
}

cudaError_t launch_tile_fill(const ImgDev* img, const TileDesc* tiles, int n_tiles,
                             const uint8_t* gap, int tx, int ty, uint32_t* slot_pos,
                             int* slot_map, int2* halo, int halo_cap, cudaStream_t s) {
    const int nthr = ((ty + 31) / 32) * 32;
    tile_fill_kernel<<<n_tiles, nthr, sizeof(int) * 2 * ty, s>>>(img, tiles, gap, tx, ty,
                                                                 slot_pos, slot_map);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    tile_halo_kernel<<<n_tiles, 256, 0, s>>>(img, const_cast<TileDesc*>(tiles), slot_map, tx, ty,
                                             halo, halo_cap);
    return cudaGetLastError();
}

cudaError_t launch_tile_const(const ImgDev* img, const TileDesc* tiles, int n_tiles, int tx, int ty,
                              const uint32_t* slot_pos, const int2* halo, int halo_cap,
                              const float* samp, float q, int gmrf, uint2* slot_ref,
                              float4* slot_cs, cudaStream_t s) {
    const size_t smem = sizeof(uint16_t) * (tx + 2) * (ty + 2);
    tile_const_kernel<<<n_tiles, 256, smem, s>>>(img, tiles, tx, ty, slot_pos, halo, halo_cap,
                                                 samp, q, gmrf, slot_ref, slot_cs);
    return cudaGetLastError();
}


}  // namespace mpr
