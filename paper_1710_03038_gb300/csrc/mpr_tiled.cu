// Tiled path: the batched checkerboard sweep.
//
// Layout.  Sample angles are identical in every realisation, so they are
// stored once per image (`samp`).  A realisation stores only its gap angles,
// compactly: the image is cut into TX x TY tiles and the gap sites of one
// tile and one colour form a contiguous segment of the image's slot space
// (row-major inside the tile, padded to 4 slots).  A chain's state is one
// float per slot.
//
// Work.  One thread block takes one tile and a group of chains.  It builds,
// once, a shared-memory table of (cos q phi, sin q phi) for the other-colour
// cells of the tile and its 1-cell ring, holding the sample cells; then for
// every chain of the group it writes that chain's other-colour gap cells into
// the table (interior segment + ring list), and updates its own-colour gap
// sites from the table (Alg. 1), reading and writing their segment with
// coalesced accesses.  Realisation sums stay in registers across the chain
// loop and reach global memory once per tile.
//
// Energy (black pass).  Every bond joins a red and a black site.  H is the
// sample-sample part (constant, from the initialisation) plus the bonds of
// black gap sites (-J R cos(theta - Psi) after their update) plus the bonds
// between red gap sites and black sample sites (the red site's angle against
// a per-tile constant field of its sample neighbours).
#include "mpr_device.cuh"
#include "mpr_internal.h"

namespace mpr {

namespace {

template <int TX, int TY, int NT>
struct TiledCfg {
    static constexpr int HW = TX / 2 + 1;          // other-colour cells per extended row
    static constexpr int CSN = (TY + 2) * HW;      // cells of one table buffer
    static constexpr int NMAX = TX * TY / 2;       // sites of one colour in a tile
    static constexpr int HCAP = TX + TY;           // ring cells of one colour
    static constexpr int KMAX = (NMAX + NT - 1) / NT;
    static constexpr int CGMAX = 64;               // chains per block
    static constexpr size_t smem_bytes =
        sizeof(float2) * (2 * CSN + NMAX)          // tables + energy field
        + sizeof(int) * HCAP                       // ring slots
        + sizeof(float) * CGMAX                    // alpha
        + sizeof(unsigned) * CGMAX                 // accept counts
        + sizeof(float) * CGMAX                    // energies
        + sizeof(uint16_t) * (2 * NMAX + HCAP);    // positions
};

template <int TX, int TY, int NT>
__global__ void __launch_bounds__(NT)
tiled_pass_kernel(SweepArgs a) {
    using Cfg = TiledCfg<TX, TY, NT>;
    constexpr int HW = Cfg::HW, CSN = Cfg::CSN, NMAX = Cfg::NMAX, HCAP = Cfg::HCAP;
    constexpr int KMAX = Cfg::KMAX;
    extern __shared__ __align__(16) unsigned char smem[];
    float2* cs = reinterpret_cast<float2*>(smem);
    float2* csss = cs + 2 * CSN;
    int* halo_slot = reinterpret_cast<int*>(csss + NMAX);
    float* s_alpha = reinterpret_cast<float*>(halo_slot + HCAP);
    unsigned* s_cnt = reinterpret_cast<unsigned*>(s_alpha + Cfg::CGMAX);
    float* s_e = reinterpret_cast<float*>(s_cnt + Cfg::CGMAX);
    uint16_t* own_pos = reinterpret_cast<uint16_t*>(s_e + Cfg::CGMAX);
    uint16_t* oth_idx = own_pos + NMAX;
    uint16_t* halo_idx = oth_idx + NMAX;

    const int tid = threadIdx.x;
    const int t = blockIdx.x;
    const TileDesc T = a.tiles[t];
    const ImgDev& I = a.img[T.img];
    const int c = a.colour;
    const int oc = c ^ 1;
    const int r0 = blockIdx.y * a.chain_group;
    const int ng = min(a.chain_group, a.n_chains - r0);
    const int n_own = T.cnt[c];
    const int n_oth = T.cnt[oc];
    const int n_halo = T.halo_cnt[c];
    const uint32_t* spos = a.slot_pos + I.slot_off;
    const float* samp = a.samp + I.site_off;
    const bool energy = (a.flags & kEnergy) != 0;
    const bool accum = (a.flags & kAccumulate) != 0;
    const bool accum2 = (a.flags & kAccumulate2) != 0;
    const uint32_t sweep = a.ctl->sweep;
    const uint32_t img_field = (uint32_t)T.img | a.img_tag;
    const UpdateConst uk{a.q, a.inv_q, a.two_pi_q, a.J};
    const float invT = I.invT;

    // -- prologue: sample cells of the table (both buffers) ------------------
    for (int idx = tid; idx < CSN; idx += NT) {
        const int yy = idx / HW;
        const int kk = idx - yy * HW;
        const int xx = 2 * kk + ((oc + yy) & 1);
        float2 val = make_float2(0.0f, 0.0f);
        const int X = T.x0 + xx - 1, Y = T.y0 + yy - 1;
        if (xx < TX + 2 && X >= 0 && X < I.Lx && Y >= 0 && Y < I.Ly) {
            const float v = samp[(long long)Y * I.Lx + X];
            if (v >= 0.0f) __sincosf(a.q * v, &val.y, &val.x);
        }
        cs[idx] = val;
        cs[CSN + idx] = val;
    }
    for (int j = tid; j < n_own; j += NT) {
        const uint32_t p = spos[T.off[c] + j];
        const int lx = (int)(p & 0xFFFFu) - T.x0, ly = (int)(p >> 16) - T.y0;
        own_pos[j] = (uint16_t)(lx | (ly << 8));
    }
    for (int j = tid; j < n_oth; j += NT) {
        const uint32_t p = spos[T.off[oc] + j];
        const int X = (int)(p & 0xFFFFu), Y = (int)(p >> 16);
        const int xx = X - T.x0 + 1, yy = Y - T.y0 + 1;
        oth_idx[j] = (uint16_t)(yy * HW + (xx >> 1));
        if (energy) {
            // field of the sample neighbours of this other-colour gap site
            float2 f = make_float2(0.0f, 0.0f);
            const int nx[4] = {X, X, X - 1, X + 1};
            const int ny[4] = {Y - 1, Y + 1, Y, Y};
#pragma unroll
            for (int m = 0; m < 4; ++m) {
                if (nx[m] < 0 || nx[m] >= I.Lx || ny[m] < 0 || ny[m] >= I.Ly) continue;
                const float v = samp[(long long)ny[m] * I.Lx + nx[m]];
                if (v >= 0.0f) {
                    float s, cc;
                    __sincosf(a.q * v, &s, &cc);
                    f.x += cc;
                    f.y += s;
                }
            }
            csss[j] = f;
        }
    }
    const int2* hl = a.halo + ((long long)t * 2 + c) * a.halo_cap;
    for (int j = tid; j < n_halo; j += NT) {
        const int2 h = hl[j];
        halo_slot[j] = h.x;
        halo_idx[j] = (uint16_t)h.y;
    }
    for (int j = tid; j < ng; j += NT) {
        const int chg = T.img * a.n_chains + r0 + j;
        s_alpha[j] = (a.flags & kAlphaOne) ? kTwoPi : kTwoPi / a.ch.a[chg];
        s_cnt[j] = 0u;
        s_e[j] = 0.0f;
    }
    __syncthreads();

    float accv[KMAX];
    float accq[KMAX];
#pragma unroll
    for (int k = 0; k < KMAX; ++k) { accv[k] = 0.0f; accq[k] = 0.0f; }

    for (int rr = 0; rr < ng; ++rr) {
        const int chain = r0 + rr;
        float* st = a.state + I.state_off + (long long)chain * I.stride;
        float2* CS = cs + (rr & 1) * CSN;
        float e_loc = 0.0f;
        // other-colour gap cells of this chain
        for (int j = tid; j < n_oth; j += NT) {
            const float v = st[T.off[oc] + j];
            float s, cc;
            __sincosf(a.q * v, &s, &cc);
            CS[oth_idx[j]] = make_float2(cc, s);
            if (energy) {
                const float2 f = csss[j];
                e_loc -= a.J * fmaf(f.x, cc, f.y * s);
            }
        }
        for (int j = tid; j < n_halo; j += NT) {
            const float v = st[halo_slot[j]];
            float s, cc;
            __sincosf(a.q * v, &s, &cc);
            CS[halo_idx[j]] = make_float2(cc, s);
        }
        __syncthreads();
        const float alpha = s_alpha[rr];
        unsigned cnt = 0;
#pragma unroll
        for (int k = 0; k < KMAX; ++k) {
            const int j = tid + k * NT;
            if (j < n_own) {
                const int pp = own_pos[j];
                const int lx = pp & 0xFF, ly = pp >> 8;
                const int xx = lx + 1, yy = ly + 1;
                const float2 fu = CS[(yy - 1) * HW + (xx >> 1)];
                const float2 fd = CS[(yy + 1) * HW + (xx >> 1)];
                const float2 fl = CS[yy * HW + ((xx - 1) >> 1)];
                const float2 fr = CS[yy * HW + ((xx + 1) >> 1)];
                const float C = ((fu.x + fd.x) + fl.x) + fr.x;
                const float S = ((fu.y + fd.y) + fl.y) + fr.y;
                float* sp = st + T.off[c] + j;
                const float v = *sp;
                const int X = T.x0 + lx, Y = T.y0 + ly;
                uint32_t wu, wr;
                site_uniform_words(X, Y, c, sweep, (uint32_t)chain, img_field, a.key, wu, wr);
                const UpdateOut o = hybrid_update(v, C, S, wu, wr, uk, alpha, invT);
                *sp = o.phi;
                cnt += o.accepted;
                if (energy) e_loc += site_energy_after(o, a.J);
                if (accum) {
                    accv[k] += o.phi;
                    if (accum2) accq[k] = fmaf(o.phi, o.phi, accq[k]);
                }
            }
        }
        cnt = warp_sum(cnt);
        if ((tid & 31) == 0 && cnt) atomicAdd(s_cnt + rr, cnt);
        if (energy) {
            e_loc = warp_sum(e_loc);
            if ((tid & 31) == 0) atomicAdd(s_e + rr, e_loc);
        }
    }
    __syncthreads();
    for (int j = tid; j < ng; j += NT) {
        const int chg = T.img * a.n_chains + r0 + j;
        if (s_cnt[j]) atomicAdd(a.ch.acc_cnt + chg, s_cnt[j]);
        if (energy) atomicAdd(a.ch.e_cur + chg, (double)s_e[j]);
    }
    if (accum) {
        double* acc1 = a.acc1 + I.slot_off + T.off[c];
        double* acc2 = a.acc2 + I.slot_off + T.off[c];
#pragma unroll
        for (int k = 0; k < KMAX; ++k) {
            const int j = tid + k * NT;
            if (j < n_own) {
                atomicAdd(acc1 + j, (double)accv[k]);
                if (accum2) atomicAdd(acc2 + j, (double)accq[k]);
            }
        }
    }
}

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
    const int hw = tx / 2 + 1;
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
        if (k < cap) halo[((long long)t * 2 + pass) * cap + k] = make_int2(slot, yy * hw + (xx >> 1));
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        tiles[t].halo_cnt[0] = n[0] < cap ? n[0] : cap;
        tiles[t].halo_cnt[1] = n[1] < cap ? n[1] : cap;
    }
}

template <int TX, int TY, int NT>
cudaError_t launch_cfg(const SweepArgs& a, int n_tiles, cudaStream_t s) {
    using Cfg = TiledCfg<TX, TY, NT>;
    static bool attr_set = false;
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(tiled_pass_kernel<TX, TY, NT>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)Cfg::smem_bytes);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    if (a.chain_group > Cfg::CGMAX) return cudaErrorInvalidValue;
    dim3 grid(n_tiles, (a.n_chains + a.chain_group - 1) / a.chain_group);
    tiled_pass_kernel<TX, TY, NT><<<grid, NT, Cfg::smem_bytes, s>>>(a);
    return cudaGetLastError();
}

}  // namespace

bool tiled_config_supported(int tx, int ty) {
    return (tx == 64 && ty == 64) || (tx == 64 && ty == 32) || (tx == 32 && ty == 32) ||
           (tx == 128 && ty == 32) || (tx == 32 && ty == 16);
}

cudaError_t launch_tiled_pass(const SweepArgs& a, int n_tiles, int tx, int ty, cudaStream_t s) {
    if (tx == 64 && ty == 64) return launch_cfg<64, 64, 256>(a, n_tiles, s);
    if (tx == 64 && ty == 32) return launch_cfg<64, 32, 256>(a, n_tiles, s);
    if (tx == 32 && ty == 32) return launch_cfg<32, 32, 128>(a, n_tiles, s);
    if (tx == 128 && ty == 32) return launch_cfg<128, 32, 256>(a, n_tiles, s);
    if (tx == 32 && ty == 16) return launch_cfg<32, 16, 128>(a, n_tiles, s);
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

}  // namespace mpr
