// Tiled path: the batched checkerboard sweep.
//
// Layout.  Sample angles are identical in every realisation, so they are
// stored once per image (`samp`).  A realisation stores only its gap angles,
// compactly: the image is cut into TX x TY tiles and the gap sites of one
// tile and one colour form a contiguous segment of the image's slot space
// (row-major inside the tile, padded to 4 slots = 16 bytes); the tile's red
// and black segments are adjacent.  A chain's state is one float per slot.
//
// Work.  One thread block takes one tile and a group of chains.  Once per
// launch it builds a shared-memory table of (cos q phi, sin q phi) for the
// other-colour cells of the tile and its 1-cell ring, holding the sample
// cells.  Then, chain after chain:
//  - the tile's two segments of that chain arrive in a shared-memory stage
//    buffer by one bulk asynchronous copy (issued two chains ahead, double
//    buffered, completion tracked by an mbarrier);
//  - the other-colour gap cells of the stage (and of the ring, whose values
//    were prefetched into registers one chain ahead) are written into the
//    table, and the own-colour angles are taken into registers;
//  - every own-colour gap site gets the hybrid update of Alg. 1 from the
//    table and its new angle is stored to global memory (coalesced).
// Realisation sums stay in registers across the chain loop and reach global
// memory once per tile.
//
// Energy (black pass).  Every bond joins a red and a black site.  H is the
// sample-sample part (constant, from the initialisation) plus the bonds of
// black gap sites (-J R cos(theta - Psi) after their update) plus the bonds
// between red gap sites and black sample sites (the red site's angle against
// a per-tile constant field of its sample neighbours).
#include "mpr_async.cuh"
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
    static constexpr int KH = (HCAP + NT - 1) / NT;
    static constexpr int SEG = TX * TY + 8;        // both padded segments of a tile
    static constexpr int CGMAX = 64;               // chains per block
    static constexpr size_t off_cs = 0;
    static constexpr size_t off_stage = off_cs + sizeof(float2) * 2 * CSN;
    static constexpr size_t off_csss = off_stage + sizeof(float) * 2 * SEG;
    static constexpr size_t off_hslot = off_csss + sizeof(float2) * NMAX;
    static constexpr size_t off_alpha = off_hslot + sizeof(int) * HCAP;
    static constexpr size_t off_cnt = off_alpha + sizeof(float) * CGMAX;
    static constexpr size_t off_e = off_cnt + sizeof(unsigned) * CGMAX;
    static constexpr size_t off_bar = (off_e + sizeof(float) * CGMAX + 15) / 16 * 16;
    static constexpr size_t off_c0 = off_bar + 16;
    static constexpr size_t off_pos = off_c0 + sizeof(uint32_t) * NMAX;
    static constexpr size_t smem_bytes = off_pos + sizeof(uint16_t) * (2 * NMAX + HCAP);
};

template <int TX, int TY, int NT>
__global__ void __launch_bounds__(NT)
tiled_pass_kernel(const __grid_constant__ SweepArgs a) {
    using Cfg = TiledCfg<TX, TY, NT>;
    constexpr int HW = Cfg::HW, CSN = Cfg::CSN, NMAX = Cfg::NMAX;
    constexpr int KMAX = Cfg::KMAX, KH = Cfg::KH, SEG = Cfg::SEG;
    extern __shared__ __align__(16) unsigned char smem[];
    float2* cs = reinterpret_cast<float2*>(smem + Cfg::off_cs);
    float* stage = reinterpret_cast<float*>(smem + Cfg::off_stage);
    float2* csss = reinterpret_cast<float2*>(smem + Cfg::off_csss);
    int* halo_slot = reinterpret_cast<int*>(smem + Cfg::off_hslot);
    float* s_alpha = reinterpret_cast<float*>(smem + Cfg::off_alpha);
    unsigned* s_cnt = reinterpret_cast<unsigned*>(smem + Cfg::off_cnt);
    float* s_e = reinterpret_cast<float*>(smem + Cfg::off_e);
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem + Cfg::off_bar);
    uint32_t* own_c0 = reinterpret_cast<uint32_t*>(smem + Cfg::off_c0);
    uint16_t* own_nb = reinterpret_cast<uint16_t*>(smem + Cfg::off_pos);
    uint16_t* oth_idx = own_nb + NMAX;
    uint16_t* halo_idx = oth_idx + NMAX;

    const int tid = threadIdx.x;
    const int t = blockIdx.x;
    // tile descriptor as scalars (runtime-indexed struct arrays would live in local memory)
    const TileDesc* Tp = a.tiles + t;
    const int c = a.colour;
    const int oc = c ^ 1;
    const int n_own = Tp->cnt[c];
    if (n_own == 0) return;  // nothing of this colour to update in this tile
    const int t_img = Tp->img, t_x0 = Tp->x0, t_y0 = Tp->y0;
    const int off_own = Tp->off[c], off_oth = Tp->off[oc];
    const int seg0 = Tp->off[0];
    const int seg_len = Tp->off[1] + ((Tp->cnt[1] + 3) & ~3) - seg0;
    const ImgDev& I = a.img[t_img];
    const int r0 = blockIdx.y * a.chain_group;
    const int ng = min(a.chain_group, a.n_chains - r0);
    const int n_oth = Tp->cnt[oc];
    const int n_halo = Tp->halo_cnt[c];
    const uint32_t* spos = a.slot_pos + I.slot_off;
    const float* samp = a.samp + I.site_off;
    const bool energy = (a.flags & kEnergy) != 0;
    const bool accum = (a.flags & kAccumulate) != 0;
    const bool accum2 = (a.flags & kAccumulate2) != 0;
    const uint32_t sweep = a.ctl->sweep;
    const uint32_t img_field = (uint32_t)t_img | a.img_tag;
    const UpdateConst uk{a.q, a.inv_q, a.two_pi_q, a.J};
    const float invT = I.invT;
    // the tile's segments: [red | black], each padded to 4 slots
    const uint32_t seg_bytes = (uint32_t)seg_len * 4u;
    const int own_in = off_own - seg0;
    const int oth_in = off_oth - seg0;
    float* state0 = a.state + I.state_off + seg0;  // chain 0, start of the tile's segments
    const long long stride = I.stride;

    if (tid == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        fence_mbar_init();
    }
    // -- prologue: sample cells of the table (both buffers) ------------------
    for (int idx = tid; idx < CSN; idx += NT) {
        const int yy = idx / HW;
        const int kk = idx - yy * HW;
        const int xx = 2 * kk + ((oc + yy) & 1);
        float2 val = make_float2(0.0f, 0.0f);
        const int X = t_x0 + xx - 1, Y = t_y0 + yy - 1;
        if (xx < TX + 2 && X >= 0 && X < I.Lx && Y >= 0 && Y < I.Ly) {
            const float v = samp[(long long)Y * I.Lx + X];
            if (v >= 0.0f) __sincosf(a.q * v, &val.y, &val.x);
        }
        cs[idx] = val;
        cs[CSN + idx] = val;
    }
    // own sites: table index of the upper neighbour with two flag bits (bit 14:
    // extended column odd, so the left neighbour shares the upper one's packed
    // column; bit 15: odd packed column, so the site takes Philox words 2-3) and
    // the first counter word (row << 16 | pair)
    for (int j = tid; j < n_own; j += NT) {
        const uint32_t p = spos[off_own + j];
        const int X = (int)(p & 0xFFFFu), Y = (int)(p >> 16);
        const int xx = X - t_x0 + 1, yy = Y - t_y0 + 1;
        own_nb[j] = (uint16_t)(((yy - 1) * HW + (xx >> 1)) | ((xx & 1) << 14) |
                               ((((uint32_t)X >> 1) & 1u) << 15));
        own_c0[j] = ((uint32_t)Y << 16) | ((uint32_t)X >> 2);
    }
    for (int j = tid; j < n_oth; j += NT) {
        const uint32_t p = spos[off_oth + j];
        const int X = (int)(p & 0xFFFFu), Y = (int)(p >> 16);
        const int xx = X - t_x0 + 1, yy = Y - t_y0 + 1;
        oth_idx[j] = (uint16_t)(yy * HW + (xx >> 1));
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
    const int2* hl = a.halo + ((long long)t * 2 + c) * a.halo_cap;
    for (int j = tid; j < n_halo; j += NT) {
        const int2 h = hl[j];
        halo_slot[j] = h.x;
        halo_idx[j] = (uint16_t)h.y;
    }
    for (int j = tid; j < ng; j += NT) {
        const int chg = t_img * a.n_chains + r0 + j;
        s_alpha[j] = (a.flags & kAlphaOne) ? kTwoPi : kTwoPi / a.ch.a[chg];
        s_cnt[j] = 0u;
        s_e[j] = 0.0f;
    }
    __syncthreads();
    if (tid == 0) {
        for (int q = 0; q < 2 && q < ng; ++q) {
            mbar_arrive_expect_tx(&bar[q], seg_bytes);
            bulk_copy_g2s(stage + q * SEG, state0 + (long long)(r0 + q) * stride, seg_bytes, &bar[q]);
        }
    }
    // ring values of the first chain
    float hv[KH];
    {
        const float* st = a.state + I.state_off + (long long)r0 * stride;
#pragma unroll
        for (int kh = 0; kh < KH; ++kh) {
            const int j = tid + kh * NT;
            hv[kh] = j < n_halo ? st[halo_slot[j]] : 0.0f;
        }
    }

    float accv[KMAX];
    float accq[KMAX];
#pragma unroll
    for (int k = 0; k < KMAX; ++k) { accv[k] = 0.0f; accq[k] = 0.0f; }

    for (int rr = 0; rr < ng; ++rr) {
        const int buf = rr & 1;
        const int chain = r0 + rr;
        float* st = a.state + I.state_off + (long long)chain * stride;
        float2* CS = cs + buf * CSN;
        const float* stg = stage + buf * SEG;
        float e_loc = 0.0f;
        // ring values of the next chain, in flight during this one
        float hn[KH];
        if (rr + 1 < ng) {
            const float* stn = st + stride;
#pragma unroll
            for (int kh = 0; kh < KH; ++kh) {
                const int j = tid + kh * NT;
                hn[kh] = j < n_halo ? stn[halo_slot[j]] : 0.0f;
            }
        }
        const bool ok = mbar_wait_bounded(&bar[buf], (uint32_t)(rr >> 1) & 1u);
        if (__syncthreads_or(!ok)) {
            // a copy did not complete in time: record it, give the copies still in
            // flight a bounded chance to land, and leave
            if (tid == 0) {
                atomicOr(&a.ctl->status, 1u);
                mbar_wait_bounded(&bar[buf], (uint32_t)(rr >> 1) & 1u);
                if (rr + 1 < ng) mbar_wait_bounded(&bar[buf ^ 1], (uint32_t)((rr + 1) >> 1) & 1u);
            }
            __syncthreads();
            return;
        }
        // other-colour gap cells of this chain
        for (int j = tid; j < n_oth; j += NT) {
            const float v = stg[oth_in + j];
            float s, cc;
            __sincosf(a.q * v, &s, &cc);
            CS[oth_idx[j]] = make_float2(cc, s);
            if (energy) {
                const float2 f = csss[j];
                e_loc -= a.J * fmaf(f.x, cc, f.y * s);
            }
        }
#pragma unroll
        for (int kh = 0; kh < KH; ++kh) {
            const int j = tid + kh * NT;
            if (j < n_halo) {
                float s, cc;
                __sincosf(a.q * hv[kh], &s, &cc);
                CS[halo_idx[j]] = make_float2(cc, s);
            }
        }
        float ov[KMAX];
#pragma unroll
        for (int k = 0; k < KMAX; ++k) {
            const int j = tid + k * NT;
            ov[k] = j < n_own ? stg[own_in + j] : 0.0f;
        }
        __syncthreads();
        // the stage buffer is free again: fetch the chain after next into it
        if (tid == 0 && rr + 2 < ng) {
            fence_proxy_async_smem();
            mbar_arrive_expect_tx(&bar[buf], seg_bytes);
            bulk_copy_g2s(stage + buf * SEG, state0 + (long long)(chain + 2) * stride, seg_bytes,
                          &bar[buf]);
        }
        const float alpha = s_alpha[rr];
        unsigned cnt = 0;
#pragma unroll
        for (int k = 0; k < KMAX; ++k) {
            const int j = tid + k * NT;
            if (j < n_own) {
                const uint32_t nb = own_nb[j];
                const int up = (int)(nb & 0x0FFFu);
                const int left = up + HW - 1 + (int)((nb >> 14) & 1u);
                const float2 fu = CS[up];
                const float2 fd = CS[up + 2 * HW];
                const float2 fl = CS[left];
                const float2 fr = CS[left + 1];
                const float C = ((fu.x + fd.x) + fl.x) + fr.x;
                const float S = ((fu.y + fd.y) + fl.y) + fr.y;
                const uint4 w = philox4x32_10_rk(
                    make_uint4(own_c0[j], sweep, (uint32_t)chain, img_field | ((uint32_t)c << 31)),
                    a.rk);
                const bool odd = (nb >> 15) != 0;
                const uint32_t wu = odd ? w.z : w.x;
                const uint32_t wr = odd ? w.w : w.y;
                const UpdateOut o = hybrid_update(ov[k], C, S, wu, wr, uk, alpha, invT);
                st[off_own + j] = o.phi;
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
        if (rr + 1 < ng) {
#pragma unroll
            for (int kh = 0; kh < KH; ++kh) hv[kh] = hn[kh];
        }
    }
    __syncthreads();
    for (int j = tid; j < ng; j += NT) {
        const int chg = t_img * a.n_chains + r0 + j;
        if (s_cnt[j]) atomicAdd(a.ch.acc_cnt + chg, s_cnt[j]);
        if (energy) atomicAdd(a.ch.e_cur + chg, (double)s_e[j]);
    }
    if (accum) {
        double* acc1 = a.acc1 + I.slot_off + off_own;
        double* acc2 = a.acc2 + I.slot_off + off_own;
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
    static_assert(TiledCfg<64, 64, 256>::smem_bytes < 227 * 1024, "shared memory");
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
