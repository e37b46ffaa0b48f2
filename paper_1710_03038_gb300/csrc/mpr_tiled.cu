// Tiled path: the batched checkerboard sweep.
//
// Layout.  Sample angles are identical in every realisation, so they are
// stored once per image (`samp`).  A realisation stores only its gap angles,
// compactly: the image is cut into TX x TY tiles and the gap sites of one
// tile and one colour form a contiguous segment of the image's slot space
// (row-major inside the tile, padded to 4 slots).  A chain's state is one
// float per slot.
//
// Work.  One thread block takes one tile and a group of chains; each warp
// takes pairs of realisations (2m, 2m + 1) of the group in turn.  Once per
// launch the block prepares, for every own-colour gap site of the tile, the
// constant part of its local field (the sines and cosines of its sample
// neighbours, summed up, down, left, right) and four references into a
// per-warp table of the other colour's gap cells (interior segment, then the
// 1-cell ring, entry 0 holding zeros for neighbours that are not gaps).  For a
// pair of realisations a warp
//  - fills its two tables from the pair's other-colour gap angles (coalesced
//    loads of the tile's segment, gathers for the ring),
//  - updates every own-colour gap site of both realisations with Alg. 1, one
//    Philox block serving the site in both (words 0-1 and 2-3), and stores
//    the new angles (coalesced).
// Warps synchronise only among their own lanes.  Realisation sums stay in
// registers across a warp's pairs and reach global memory once per tile.
//
// Energy (black pass).  Every bond joins a red and a black site.  H is the
// sample-sample part (constant, from the initialisation) plus the bonds of
// black gap sites (-J R cos(theta - Psi) after their update) plus the bonds
// between red gap sites and black sample sites (the red site's angle against
// the constant field of its sample neighbours).
#include "mpr_device.cuh"
#include "mpr_internal.h"

namespace mpr {

namespace {

template <int TX, int TY, int NW>
struct TiledCfg {
    static constexpr int NT = NW * 32;
    static constexpr int HK = (TX + TY + 31) / 32;  // ring cells per lane
    static constexpr int EW = TX + 2;              // extended tile width
    static constexpr int EXT = (TX + 2) * (TY + 2);
    static constexpr int NMAX = TX * TY / 2;       // sites of one colour in a tile
    static constexpr int HCAP = TX + TY;           // ring cells of one colour
    static constexpr int GT = NMAX + HCAP + 1;     // table entries (entry 0 = zeros)
    static constexpr int KMAX = (NMAX + 31) / 32;
    static constexpr size_t off_ref = 0;
    static constexpr size_t off_cs = off_ref + sizeof(uint2) * NMAX;
    static constexpr size_t off_csss = off_cs + sizeof(float2) * NMAX;
    static constexpr size_t off_acc = off_csss + sizeof(float2) * NMAX;
    static constexpr size_t off_c0 = off_acc + sizeof(float) * 2 * NMAX;
    static constexpr size_t off_hslot = off_c0 + sizeof(uint32_t) * NMAX;
    static constexpr size_t off_map = off_hslot + sizeof(int) * HCAP;
    // per-warp tables last, sized at launch for the largest tile of the pass
    static constexpr size_t off_tab = (off_map + sizeof(uint16_t) * EXT + 15) / 16 * 16;
    static constexpr size_t smem_for(int gt) { return off_tab + sizeof(float2) * 2 * NW * gt; }
    static constexpr size_t smem_max = smem_for(GT);
};

// K: gap sites per lane and realisation that one pass can meet (the largest
// own or other-colour count of the pass's tiles, over 32, rounded up).
// ACC: sampling pass that adds every new angle (and its square) to the
// realisation sums; equilibration passes are compiled without that code.
template <int TX, int TY, int NW, int K, bool ACC>
__global__ void __launch_bounds__(NW * 32, 1024 / (NW * 32))  // 64 registers: 32 warps per SM
tiled_pass_kernel(const __grid_constant__ SweepArgs a) {
    using Cfg = TiledCfg<TX, TY, NW>;
    constexpr int NT = Cfg::NT, EW = Cfg::EW, EXT = Cfg::EXT, NMAX = Cfg::NMAX;
    constexpr int KMAX = K, HK = Cfg::HK;
    static_assert(K * 32 <= NMAX || K == 1, "K larger than a tile's colour");
    const int GT = a.gt;  // entries of one table (entry 0 = zeros)
    extern __shared__ __align__(16) unsigned char smem[];
    uint2* own_ref = reinterpret_cast<uint2*>(smem + Cfg::off_ref);
    float2* own_cs = reinterpret_cast<float2*>(smem + Cfg::off_cs);
    float2* csss = reinterpret_cast<float2*>(smem + Cfg::off_csss);
    float2* tabs = reinterpret_cast<float2*>(smem + Cfg::off_tab);
    float* acc_s = reinterpret_cast<float*>(smem + Cfg::off_acc);
    uint32_t* own_c0 = reinterpret_cast<uint32_t*>(smem + Cfg::off_c0);
    int* halo_slot = reinterpret_cast<int*>(smem + Cfg::off_hslot);
    uint16_t* cellmap = reinterpret_cast<uint16_t*>(smem + Cfg::off_map);

    const int tid = threadIdx.x;
    const int lane = tid & 31;
    const int warp = tid >> 5;
    const TileDesc* Tp = a.tiles + blockIdx.x;
    const int c = a.colour;
    const int oc = c ^ 1;
    const int n_own = Tp->cnt[c];
    const bool energy = (a.flags & kEnergy) != 0;
    // nothing to update and no red-gap / black-sample bond energy to add
    if (n_own == 0 && !(energy && Tp->cnt[oc] > 0)) return;
    // tile descriptor as scalars (runtime-indexed struct arrays would live in local memory)
    const int t_img = Tp->img, t_x0 = Tp->x0, t_y0 = Tp->y0;
    const int off_own = Tp->off[c], off_oth = Tp->off[oc];
    const int n_oth = Tp->cnt[oc];
    const int n_halo = Tp->halo_cnt[c];
    const ImgDev& I = a.img[t_img];
    const int r0 = blockIdx.y * a.chain_group;
    const int ng = min(a.chain_group, a.n_chains - r0);
    const uint32_t* spos = a.slot_pos + I.slot_off;
    const float* samp = a.samp + I.site_off;
    constexpr bool accum = ACC;
    const bool accum2 = ACC && (a.flags & kAccumulate2) != 0;
    const uint32_t sweep = a.ctl->sweep;
    const uint32_t c3 = (uint32_t)t_img | a.img_tag | ((uint32_t)c << 31);
    const UpdateConst uk{a.q, a.inv_q, a.two_pi_q, a.J};
    const float invT = I.invT;
    const long long stride = I.stride;
    const int spread = blockIdx.x & (kSpread - 1);

    // -- prologue ---------------------------------------------------------------
    for (int i = tid; i < EXT; i += NT) cellmap[i] = 0;
    if (accum)
        for (int i = tid; i < 2 * NMAX; i += NT) acc_s[i] = 0.0f;
    for (int i = tid; i < 2 * NW; i += NT) tabs[i * GT] = make_float2(0.0f, 0.0f);
    __syncthreads();
    for (int j = tid; j < n_oth; j += NT) {
        const uint32_t p = spos[off_oth + j];
        const int X = (int)(p & 0xFFFFu), Y = (int)(p >> 16);
        cellmap[(Y - t_y0 + 1) * EW + (X - t_x0 + 1)] = (uint16_t)(1 + j);
        if (energy) {
            // field of the sample neighbours of this other-colour gap site
            float2 f = make_float2(0.0f, 0.0f);
#pragma unroll
            for (int m = 0; m < 4; ++m) {
                const int nx = m < 2 ? X : X - 1 + 2 * (m - 2);
                const int ny = m < 2 ? Y - 1 + 2 * m : Y;
                if (nx < 0 || nx >= I.Lx || ny < 0 || ny >= I.Ly) continue;
                const float v = samp[(long long)ny * I.Lx + nx];
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
    {
        const int2* hl = a.halo + ((long long)blockIdx.x * 2 + c) * a.halo_cap;
        for (int k = tid; k < n_halo; k += NT) {
            const int2 h = hl[k];
            halo_slot[k] = h.x;
            cellmap[h.y] = (uint16_t)(1 + n_oth + k);
        }
    }
    __syncthreads();
    for (int j = tid; j < n_own; j += NT) {
        const uint32_t p = spos[off_own + j];
        const int X = (int)(p & 0xFFFFu), Y = (int)(p >> 16);
        const int xx = X - t_x0 + 1, yy = Y - t_y0 + 1;
        float2 f = make_float2(0.0f, 0.0f);
        uint32_t ref[4];
#pragma unroll
        for (int m = 0; m < 4; ++m) {  // up, down, left, right
            const int dx = m < 2 ? 0 : 2 * m - 5;
            const int dy = m < 2 ? 2 * m - 1 : 0;
            const int nx = X + dx, ny = Y + dy;
            ref[m] = 0u;
            if (nx < 0 || nx >= I.Lx || ny < 0 || ny >= I.Ly) continue;
            const float v = samp[(long long)ny * I.Lx + nx];
            if (v >= 0.0f) {
                float s, cc;
                __sincosf(a.q * v, &s, &cc);
                f.x += cc;
                f.y += s;
            } else {
                ref[m] = cellmap[(yy + dy) * EW + (xx + dx)];
            }
        }
        own_ref[j] = make_uint2(ref[0] | (ref[1] << 16), ref[2] | (ref[3] << 16));
        own_cs[j] = f;
        own_c0[j] = ((uint32_t)Y << 16) | ((uint32_t)X >> 1);
    }
    __syncthreads();

    // -- chain pairs ------------------------------------------------------------
    float2* tab0 = tabs + (2 * warp) * GT;
    float2* tab1 = tab0 + GT;
    const int n_pairs = (ng + 1) >> 1;
    for (int pi = warp; pi < n_pairs; pi += NW) {
        const int ch0 = r0 + 2 * pi;
        const bool has1 = 2 * pi + 1 < ng;
        const float* st0 = a.state + I.state_off + (long long)ch0 * stride;
        const float* st1 = st0 + stride;
        // every load of this pair first (one memory latency per pair)
        float oth0[KMAX], oth1[KMAX], own0[KMAX], own1[KMAX], hal0[HK], hal1[HK];
#pragma unroll
        for (int k = 0; k < KMAX; ++k) {
            const int j = lane + k * 32;
            oth0[k] = j < n_oth ? st0[off_oth + j] : 0.0f;
            oth1[k] = (has1 && j < n_oth) ? st1[off_oth + j] : 0.0f;
            own0[k] = j < n_own ? st0[off_own + j] : 0.0f;
            own1[k] = (has1 && j < n_own) ? st1[off_own + j] : 0.0f;
        }
#pragma unroll
        for (int k = 0; k < HK; ++k) {
            const int j = lane + k * 32;
            const int hs = j < n_halo ? halo_slot[j] : 0;
            hal0[k] = j < n_halo ? st0[hs] : 0.0f;
            hal1[k] = (has1 && j < n_halo) ? st1[hs] : 0.0f;
        }
        float e0 = 0.0f, e1 = 0.0f;
        // other-colour gap cells of the two realisations (straight-line per
        // iteration: only the side effects are guarded, so independent work
        // of both realisations can interleave)
#pragma unroll
        for (int k = 0; k < KMAX; ++k) {
            if (k * 32 >= n_oth) break;
            const int j = lane + k * 32;
            const bool act = j < n_oth;
            float s0, c0, s1, c1;
            __sincosf(a.q * oth0[k], &s0, &c0);
            __sincosf(a.q * oth1[k], &s1, &c1);
            if (act) {
                tab0[1 + j] = make_float2(c0, s0);
                if (has1) tab1[1 + j] = make_float2(c1, s1);
                if (energy) {
                    const float2 f = csss[j];
                    e0 -= a.J * fmaf(f.x, c0, f.y * s0);
                    if (has1) e1 -= a.J * fmaf(f.x, c1, f.y * s1);
                }
            }
        }
#pragma unroll
        for (int k = 0; k < HK; ++k) {
            if (k * 32 >= n_halo) break;
            const int j = lane + k * 32;
            float s0, c0, s1, c1;
            __sincosf(a.q * hal0[k], &s0, &c0);
            __sincosf(a.q * hal1[k], &s1, &c1);
            if (j < n_halo) {
                tab0[1 + n_oth + j] = make_float2(c0, s0);
                if (has1) tab1[1 + n_oth + j] = make_float2(c1, s1);
            }
        }
        __syncwarp();
        const float alpha0 = (a.flags & kAlphaOne) ? kTwoPi
                                                    : kTwoPi / a.ch.a[t_img * a.n_chains + ch0];
        const float alpha1 = (a.flags & kAlphaOne) || !has1
                                 ? kTwoPi
                                 : kTwoPi / a.ch.a[t_img * a.n_chains + ch0 + 1];
        float* out0 = a.state + I.state_off + (long long)ch0 * stride + off_own;
        float* out1 = out0 + stride;
        unsigned cnt0 = 0, cnt1 = 0;
#pragma unroll
        for (int k = 0; k < KMAX; ++k) {
            if (k * 32 >= n_own) break;
            const int j = lane + k * 32;
            const bool act = j < n_own;
            const int jj = act ? j : 0;  // idle lanes recompute slot 0 and store nothing
            const uint2 rf = own_ref[jj];
            const float2 fs = own_cs[jj];
            const uint4 w = philox4x32_10_rk(make_uint4(own_c0[jj], sweep, (uint32_t)ch0 >> 1, c3),
                                             a.rk);
            const int ru = rf.x & 0xFFFFu, rd = rf.x >> 16, rl = rf.y & 0xFFFFu, rr = rf.y >> 16;
            const float2 gu0 = tab0[ru], gd0 = tab0[rd], gl0 = tab0[rl], gr0 = tab0[rr];
            const float2 gu1 = tab1[ru], gd1 = tab1[rd], gl1 = tab1[rl], gr1 = tab1[rr];
            const float C0 = (((fs.x + gu0.x) + gd0.x) + gl0.x) + gr0.x;
            const float S0 = (((fs.y + gu0.y) + gd0.y) + gl0.y) + gr0.y;
            const float C1 = (((fs.x + gu1.x) + gd1.x) + gl1.x) + gr1.x;
            const float S1 = (((fs.y + gu1.y) + gd1.y) + gl1.y) + gr1.y;
            const UpdateOut o0 = hybrid_update(own0[k], C0, S0, w.x, w.y, uk, alpha0, invT);
            const UpdateOut o1 = hybrid_update(own1[k], C1, S1, w.z, w.w, uk, alpha1, invT);
            const bool act1 = act && has1;
            if (act) out0[j] = o0.phi;
            if (act1) out1[j] = o1.phi;
            cnt0 += (act && o0.accepted) ? 1u : 0u;
            cnt1 += (act1 && o1.accepted) ? 1u : 0u;
            if (energy) {
                if (act) e0 += site_energy_after(o0, a.J);
                if (act1) e1 += site_energy_after(o1, a.J);
            }
            if (accum) {
                const float p0 = act ? o0.phi : 0.0f, p1 = act1 ? o1.phi : 0.0f;
                // one shared-memory add per site and pair of realisations
                if (act) {
                    atomicAdd(acc_s + j, p0 + p1);
                    if (accum2) atomicAdd(acc_s + NMAX + j, fmaf(p0, p0, p1 * p1));
                }
            }
        }
        cnt0 = warp_sum(cnt0);
        cnt1 = warp_sum(cnt1);
        if (energy) {
            e0 = warp_sum(e0);
            e1 = warp_sum(e1);
        }
        if (lane == 0) {
            const long long b0 = (long long)(t_img * a.n_chains + ch0) * kSpread + spread;
            if (cnt0) atomicAdd(a.ch.acc_cnt + b0, cnt0);
            if (energy) atomicAdd(a.ch.e_cur + b0, (double)e0);
            if (has1) {
                if (cnt1) atomicAdd(a.ch.acc_cnt + b0 + kSpread, cnt1);
                if (energy) atomicAdd(a.ch.e_cur + b0 + kSpread, (double)e1);
            }
        }
        __syncwarp();  // the tables are refilled by the next pair
    }
    if (accum) {
        __syncthreads();
        const bool shared_slots = gridDim.y > 1;
        double* acc1 = a.acc1 + I.slot_off + off_own;
        double* acc2 = a.acc2 + I.slot_off + off_own;
        for (int j = tid; j < n_own; j += NT) {
            if (shared_slots) {
                atomicAdd(acc1 + j, (double)acc_s[j]);
                if (accum2) atomicAdd(acc2 + j, (double)acc_s[NMAX + j]);
            } else {
                acc1[j] += (double)acc_s[j];
                if (accum2) acc2[j] += (double)acc_s[NMAX + j];
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

template <int TX, int TY, int NW, int K, bool ACC>
cudaError_t launch_one(const SweepArgs& a, int n_tiles, cudaStream_t s, bool setup_only) {
    using Cfg = TiledCfg<TX, TY, NW>;
    static_assert(Cfg::smem_max <= 227 * 1024, "shared memory");
    static bool attr_set = false;
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(tiled_pass_kernel<TX, TY, NW, K, ACC>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)Cfg::smem_max);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    if (setup_only) return cudaSuccess;
    if (a.gt < 1 || a.gt > Cfg::GT) return cudaErrorInvalidValue;
    dim3 grid(n_tiles, (a.n_chains + a.chain_group - 1) / a.chain_group);
    tiled_pass_kernel<TX, TY, NW, K, ACC><<<grid, Cfg::NT, Cfg::smem_for(a.gt), s>>>(a);
    return cudaGetLastError();
}

template <int TX, int TY, int NW, int K>
cudaError_t launch_cfg(const SweepArgs& a, int n_tiles, cudaStream_t s, bool setup_only) {
    if (setup_only) {
        cudaError_t e = launch_one<TX, TY, NW, K, false>(a, n_tiles, s, true);
        return e != cudaSuccess ? e : launch_one<TX, TY, NW, K, true>(a, n_tiles, s, true);
    }
    if (a.flags & kAccumulate) return launch_one<TX, TY, NW, K, true>(a, n_tiles, s, false);
    return launch_one<TX, TY, NW, K, false>(a, n_tiles, s, false);
}

}  // namespace

bool tiled_config_supported(int tx, int ty) {
    return (tx == 32 && ty == 16) || (tx == 16 && ty == 16) || (tx == 32 && ty == 32);
}

int tiled_max_kload(int tx, int ty) {
    return tx * ty / 64;  // every site of one colour
}

// kload = largest gap count of one colour over the pass's tiles, over 32, rounded up.
cudaError_t launch_tiled_pass(const SweepArgs& a, int n_tiles, int tx, int ty, int kload,
                              cudaStream_t s, bool setup_only) {
    if (a.chain_group % 2 != 0 && a.chain_group < a.n_chains) return cudaErrorInvalidValue;
    if (tx == 32 && ty == 16) {
        if (kload <= 3) return launch_cfg<32, 16, 4, 3>(a, n_tiles, s, setup_only);
        if (kload <= 4) return launch_cfg<32, 16, 4, 4>(a, n_tiles, s, setup_only);
        if (kload <= 5) return launch_cfg<32, 16, 4, 5>(a, n_tiles, s, setup_only);
        if (kload <= 6) return launch_cfg<32, 16, 4, 6>(a, n_tiles, s, setup_only);
        return launch_cfg<32, 16, 4, 8>(a, n_tiles, s, setup_only);
    }
    if (tx == 16 && ty == 16) {
        if (kload <= 2) return launch_cfg<16, 16, 4, 2>(a, n_tiles, s, setup_only);
        return launch_cfg<16, 16, 4, 4>(a, n_tiles, s, setup_only);
    }
    if (tx == 32 && ty == 32) {
        if (kload <= 8) return launch_cfg<32, 32, 8, 8>(a, n_tiles, s, setup_only);
        return launch_cfg<32, 32, 8, 16>(a, n_tiles, s, setup_only);
    }
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
