// Tiled path: the batched checkerboard pass (kernel template).
//
// Layout.  Sample angles are identical in every realisation, so they are
// stored once per image (`samp`).  A realisation stores only its gap angles:
// the image is cut into TX x TY tiles and the gap sites of one tile and one
// colour form a contiguous segment of the image's slot space (row-major
// inside the tile, padded to 4 slots).  The state is slot-major with the
// realisations interleaved: slot k of chain r sits at k * CP + r, CP being the
// chain count rounded up to even, so the pair (2m, 2m + 1) of one slot is one
// aligned float2 and the pairs of a chain group are contiguous.
//
// Work.  One thread block takes one tile and a group of 2P chains (P pairs).
// A warp lane is (site s, pair p) with p = lane mod P, so a warp step covers
// 32 / P sites of the tile for every pair of the group; the ragged end of a
// tile leaves at most one step partly idle.  Per launch the block
//  - prepares, for every own-colour gap site, the constant part of its local
//    field (sines and cosines of its sample neighbours, summed up, down, left,
//    right) and four references into the block's table of other-colour gap
//    cells (interior segment, then the 1-cell ring; entry 0 holds zeros for
//    neighbours that are not gaps);
//  - fills that table for all chains of the group: entry e, pair p holds
//    (cos, sin) of q phi for both chains of the pair (one float4); the angle
//    pairs arrive by asynchronous 8-byte copies (cp.async) that are contiguous
//    across the pairs of a slot, and are converted in place;
//  - updates every own-colour gap site of every chain with Alg. 1, one Philox
//    block serving the site in both chains of a pair (words 0-1 and 2-3), and
//    stores the new pair as one float2.
// Acceptances and energies stay in registers until the end of the block;
// realisation sums of a site are reduced across its P lanes by shuffles.
//
// Energy (black pass).  Every bond joins a red and a black site.  H is the
// sample-sample part (constant, from the initialisation) plus the bonds of
// black gap sites (-J R cos(theta - Psi) after their update) plus the bonds
// between red gap sites and black sample sites (the red site's angle against
// the constant field of its sample neighbours).
#pragma once

#include "mpr_async.cuh"
#include "mpr_device.cuh"
#include "mpr_internal.h"

namespace mpr {
namespace tiled {

template <int TX, int TY, int NW>
struct Cfg {
    static constexpr int NT = NW * 32;
    static constexpr int NMAX = TX * TY / 2;       // sites of one colour in a tile
    static constexpr int HCAP = TX + TY;           // ring cells of one colour
    static constexpr int GT = NMAX + HCAP + 1;     // table entries (entry 0 = zeros)
    static constexpr size_t a16(size_t v) { return (v + 15) / 16 * 16; }
    static constexpr size_t off_rc = 0;  // per own site: neighbour rows, sample field
    static constexpr size_t off_c0 = off_rc + sizeof(uint4) * NMAX;
    static constexpr size_t off_acc = off_c0 + sizeof(uint32_t) * NMAX;  // [2][NMAX] site sums
    static constexpr size_t off_red = a16(off_acc + sizeof(float) * 2 * NMAX);
    // the table last, sized at launch for the largest tile of the pass
    static constexpr size_t off_tab = off_red + sizeof(float4) * NW * 16;
    static constexpr size_t smem_for(int gt, int P) { return off_tab + sizeof(float4) * P * gt; }
    static constexpr size_t smem_max = smem_for(GT, 16);
};

template <int TX, int TY, int NW, int P, bool ACC>
__global__ void __launch_bounds__(NW * 32, 1024 / (NW * 32))  // 64 registers: 32 warps per SM
tiled_pass_kernel(const __grid_constant__ SweepArgs a) {
    using C = Cfg<TX, TY, NW>;
    constexpr int NT = C::NT, NMAX = C::NMAX;
    constexpr int SPW = 32 / P;  // sites per warp step
    static_assert(P >= 1 && P <= 16 && (P & (P - 1)) == 0, "pairs per site: power of two");
    extern __shared__ __align__(16) unsigned char smem[];
    uint4* own_rc = reinterpret_cast<uint4*>(smem + C::off_rc);
    uint32_t* own_c0 = reinterpret_cast<uint32_t*>(smem + C::off_c0);
    float* acc_s = reinterpret_cast<float*>(smem + C::off_acc);
    float4* red = reinterpret_cast<float4*>(smem + C::off_red);
    float4* tab = reinterpret_cast<float4*>(smem + C::off_tab);

    const int tid = threadIdx.x;
    const int lane = tid & 31;
    const int warp = tid >> 5;
    const int p = lane & (P - 1);  // pair of the group (fixed per thread: NT is a multiple of P)
    const int s = lane / P;        // site within a warp step
    const int tile = a.tile_list ? a.tile_list[a.tile_base + blockIdx.x] : (int)blockIdx.x;
    const TileDesc* Tp = a.tiles + tile;
    const int c = a.colour;
    const int oc = c ^ 1;
    const int n_own = Tp->cnt[c];
    const bool energy = (a.flags & kEnergy) != 0;
    // nothing to update and no red-gap / black-sample bond energy to add
    if (n_own == 0 && !(energy && Tp->cnt[oc] > 0)) return;
    // tile descriptor as scalars (runtime-indexed struct arrays would live in local memory)
    const int t_img = Tp->img;
    const int off_own = Tp->off[c], off_oth = Tp->off[oc];
    const int n_oth = Tp->cnt[oc];
    const int n_halo = Tp->halo_cnt[c];
    const ImgDev& I = a.img[t_img];
    const int r0 = a.chain0 + blockIdx.y * a.chain_group;
    const int ng = min(a.chain_group, a.chain_end - r0);
    const bool has0 = 2 * p < ng;      // this lane's pair exists
    const bool has1 = 2 * p + 1 < ng;  // and has a second chain
    const bool accum2 = ACC && (a.flags & kAccumulate2) != 0;
    const uint32_t sweep = a.ctl->sweep;
    const uint32_t c3 = (uint32_t)t_img | a.img_tag | ((uint32_t)c << 31);
    const uint32_t c2 = (uint32_t)(r0 >> 1) + (uint32_t)p;  // chain >> 1 of the pair
    const UpdateConst uk{a.q, a.inv_q, a.two_pi_q, a.J};
    const float invT = I.invT;
    const long long cp = I.sstride;  // floats from one slot to the next
    // this lane's pair at slot 0 (8-byte aligned: state_off, cp, r0 are even)
    float* st = a.state + I.state_off + r0 + 2 * p;
    const int spread = tile & (kSpread - 1);

    // -- table of the other colour, raw: entry 1 + e, pair p ----------------------
    // Each thread copies the angle pairs of its entries e = tid / P (mod NT / P)
    // straight into the first half of their table slots (all copies in flight
    // at once, no registers) and converts the same entries below, so its own
    // wait is enough.
    // Lanes without a pair copy nothing (their table column is never stored from).
    constexpr int NTP = NT / P;
    const int n_ent = n_oth + n_halo;
    const int e_lo = tid / P;
    float4* const tab_lo = tab + (1 + e_lo) * P + p;  // this thread's first entry
    constexpr uint32_t kDstStep = sizeof(float4) * NTP * P;
    if (has0) {
        const float* src = st + (long long)(off_oth + e_lo) * cp;
        const long long src_step = (long long)NTP * cp;
        uint32_t dst = smem_addr(tab_lo);
        for (int e = e_lo; e < n_oth; e += NTP, src += src_step, dst += kDstStep)
            cp_async8_s(dst, src);
    }
    if (tid < P) tab[tid] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);

    // -- own-colour constants of the tile (built once per batch) ---------------
    {
        const long long b = I.slot_off + off_own;
        for (int j = tid; j < n_own; j += NT) {
            const uint2 r = a.slot_ref[b + j];
            // table rows (entry * P) of the four neighbours, for the gathers
            const float2 f = a.slot_cs[b + j];
            own_rc[j] = make_uint4(((r.x & 0xFFFFu) * P) | (((r.x >> 16) * P) << 16),
                                   ((r.y & 0xFFFFu) * P) | (((r.y >> 16) * P) << 16),
                                   __float_as_uint(f.x), __float_as_uint(f.y));
            const uint32_t pos = a.slot_pos[b + j];
            own_c0[j] = (pos & 0xFFFF0000u) | ((pos & 0xFFFFu) >> 1);
        }
    }
    // ring cells (slots from the ring list), same entry residue as above
    if (has0) {
        const int k_first = (max(n_oth - e_lo, 0) + NTP - 1) / NTP;  // steps to the ring
        const int e_first = e_lo + k_first * NTP;
        const int2* h = a.halo + ((long long)tile * 2 + c) * a.halo_cap + (e_first - n_oth);
        uint32_t dst = smem_addr(tab_lo) + (uint32_t)k_first * kDstStep;
        for (int e = e_first; e < n_ent; e += NTP, h += NTP, dst += kDstStep)
            cp_async8_s(dst, st + (long long)h->x * cp);
    }
    cp_async_wait_all();

    // -- (cos, sin) of q phi in place -------------------------------------------
    float e0 = 0.0f, e1 = 0.0f;
    if (has0) {
        const float2* fcs = a.slot_cs + I.slot_off + off_oth;
        float4* t = tab_lo;
        for (int e = e_lo; e < n_ent; e += NTP, t += NTP * P) {
            const float2 v = *reinterpret_cast<const float2*>(t);
            float s0, c0, s1, c1;
            __sincosf(a.q * v.x, &s0, &c0);
            __sincosf(a.q * v.y, &s1, &c1);
            *t = make_float4(c0, s0, c1, s1);
            // bonds between this other-colour gap site and its sample neighbours
            if (energy && e < n_oth) {
                const float2 f = fcs[e];
                e0 -= a.J * fmaf(f.x, c0, f.y * s0);
                if (has1) e1 -= a.J * fmaf(f.x, c1, f.y * s1);
            }
        }
    }
    __syncthreads();

    // -- own colour: every site of every chain of the group ---------------------
    const float alpha0 = ((a.flags & kAlphaOne) || !has0)
                             ? kTwoPi
                             : kTwoPi / a.ch.a[t_img * a.n_chains + r0 + 2 * p];
    const float alpha1 = ((a.flags & kAlphaOne) || !has1)
                             ? kTwoPi
                             : kTwoPi / a.ch.a[t_img * a.n_chains + r0 + 2 * p + 1];
    unsigned cnt0 = 0, cnt1 = 0;
    const int n_steps = (n_own + SPW - 1) / SPW;
    float* sto = st + (long long)off_own * cp;  // this lane's pair at the own segment
    const int cpi = (int)cp;
    // angles of a warp step: loaded one step ahead, in flight during the step before
    float2 vn = make_float2(0.0f, 0.0f);
    {
        const int j = warp * SPW + s;
        if (has0 && j < n_own) vn = *reinterpret_cast<const float2*>(sto + j * cpi);
    }
    for (int g = warp; g < n_steps; g += NW) {  // warp-uniform
        const float2 vc = vn;
        {
            const int jn = (g + NW) * SPW + s;
            vn = make_float2(0.0f, 0.0f);
            if (has0 && jn < n_own) vn = *reinterpret_cast<const float2*>(sto + jn * cpi);
        }
        {
            const int j = g * SPW + s;
            const bool in = j < n_own;
            const bool act = in && has0;
            const int jj = in ? j : 0;  // idle lanes recompute slot 0 and store nothing
            const uint4 rc = own_rc[jj];
            const uint2 rf = make_uint2(rc.x, rc.y);
            const float2 fs = make_float2(__uint_as_float(rc.z), __uint_as_float(rc.w));
            const uint4 w = philox4x32_10_rk(make_uint4(own_c0[jj], sweep, c2, c3), a.rk);
            const float4 gu = tab[(rf.x & 0xFFFFu) + p], gd = tab[(rf.x >> 16) + p];
            const float4 gl = tab[(rf.y & 0xFFFFu) + p], gr = tab[(rf.y >> 16) + p];
            const float C0 = (((fs.x + gu.x) + gd.x) + gl.x) + gr.x;
            const float S0 = (((fs.y + gu.y) + gd.y) + gl.y) + gr.y;
            const float C1 = (((fs.x + gu.z) + gd.z) + gl.z) + gr.z;
            const float S1 = (((fs.y + gu.w) + gd.w) + gl.w) + gr.w;
            const UpdateOut o0 = hybrid_update(vc.x, C0, S0, w.x, w.y, uk, alpha0, invT);
            const UpdateOut o1 = hybrid_update(vc.y, C1, S1, w.z, w.w, uk, alpha1, invT);
            const bool act1 = act && has1;
            // a missing second chain is the padding chain of the layout: storing there is harmless
            if (act) *reinterpret_cast<float2*>(sto + j * cpi) = make_float2(o0.phi, o1.phi);
            cnt0 += (act && o0.accepted) ? 1u : 0u;
            cnt1 += (act1 && o1.accepted) ? 1u : 0u;
            if (energy) {
                if (act) e0 += site_energy_after(o0, a.J);
                if (act1) e1 += site_energy_after(o1, a.J);
            }
            if (ACC) {
                // the site's sums over the group's chains: lanes p of one site
                // hold every chain once, so one reduction gives the total
                const float p0 = act ? o0.phi : 0.0f, p1 = act1 ? o1.phi : 0.0f;
                float s1 = p0 + p1;
                if (accum2 && P > 1) {
                    // both sums in one butterfly: the upper half of the P lanes
                    // keeps the squares, the lower half the angles
                    const float s2 = fmaf(p0, p0, p1 * p1);
                    const bool up = (p & (P / 2)) != 0;
                    const float give = up ? s1 : s2;
                    s1 = (up ? s2 : s1) + __shfl_xor_sync(0xffffffffu, give, P / 2);
#pragma unroll
                    for (int o = 1; o < P / 2; o <<= 1) s1 += __shfl_xor_sync(0xffffffffu, s1, o);
                    if (in && (p & (P / 2 - 1)) == 0) acc_s[(up ? NMAX : 0) + j] = s1;
                } else {
#pragma unroll
                    for (int o = 1; o < P; o <<= 1) s1 += __shfl_xor_sync(0xffffffffu, s1, o);
                    if (in && p == 0) {
                        acc_s[j] = s1;
                        if (accum2) acc_s[NMAX + j] = fmaf(p0, p0, p1 * p1);
                    }
                }
            }
        }
    }

    // -- per-chain totals: lanes of one pair, then warps ------------------------
#pragma unroll
    for (int o = P; o < 32; o <<= 1) {
        cnt0 += __shfl_xor_sync(0xffffffffu, cnt0, o);
        cnt1 += __shfl_xor_sync(0xffffffffu, cnt1, o);
        if (energy) {
            e0 += __shfl_xor_sync(0xffffffffu, e0, o);
            e1 += __shfl_xor_sync(0xffffffffu, e1, o);
        }
    }
    if (lane < P) red[warp * P + lane] = make_float4(e0, e1, __uint_as_float(cnt0), __uint_as_float(cnt1));
    __syncthreads();
    if (ACC) {
        double* acc1 = a.acc1 + I.slot_off + off_own;
        double* acc2 = a.acc2 + I.slot_off + off_own;
        // fire-and-forget adds: no block waits for a read of the old sums (with
        // one chain group per tile each address gets one add per pass)
        for (int j = tid; j < n_own; j += NT) {
            atomicAdd(acc1 + j, (double)acc_s[j]);
            if (accum2) atomicAdd(acc2 + j, (double)acc_s[NMAX + j]);
        }
    }
    if (tid < P && 2 * tid < ng) {
        double E0 = 0.0, E1 = 0.0;
        unsigned n0 = 0, n1 = 0;
#pragma unroll
        for (int w = 0; w < NW; ++w) {
            const float4 r = red[w * P + tid];
            E0 += (double)r.x;
            E1 += (double)r.y;
            n0 += __float_as_uint(r.z);
            n1 += __float_as_uint(r.w);
        }
        const long long b0 = (long long)(t_img * a.n_chains + r0 + 2 * tid) * kSpread + spread;
        if (n0) atomicAdd(a.ch.acc_cnt + b0, n0);
        if (energy) atomicAdd(a.ch.e_cur + b0, E0);
        if (2 * tid + 1 < ng) {
            if (n1) atomicAdd(a.ch.acc_cnt + b0 + kSpread, n1);
            if (energy) atomicAdd(a.ch.e_cur + b0 + kSpread, E1);
        }
    }
}

template <int TX, int TY, int NW, int P, bool ACC>
cudaError_t launch_one(const SweepArgs& a, int n_tiles, cudaStream_t s, bool setup_only) {
    using C = Cfg<TX, TY, NW>;
    static_assert(C::smem_max <= 227 * 1024, "shared memory");
    static bool attr_set = false;
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(tiled_pass_kernel<TX, TY, NW, P, ACC>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)C::smem_max);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    if (setup_only) return cudaSuccess;
    if (a.gt < 1 || a.gt > C::GT) return cudaErrorInvalidValue;
    dim3 grid(n_tiles, (a.chain_end - a.chain0 + a.chain_group - 1) / a.chain_group);
    tiled_pass_kernel<TX, TY, NW, P, ACC><<<grid, C::NT, C::smem_for(a.gt, P), s>>>(a);
    return cudaGetLastError();
}

template <int TX, int TY, int NW, int P>
cudaError_t launch_cfg(const SweepArgs& a, int n_tiles, cudaStream_t s, bool setup_only) {
    if (setup_only) {
        cudaError_t e = launch_one<TX, TY, NW, P, false>(a, n_tiles, s, true);
        return e != cudaSuccess ? e : launch_one<TX, TY, NW, P, true>(a, n_tiles, s, true);
    }
    if (a.flags & kAccumulate) return launch_one<TX, TY, NW, P, true>(a, n_tiles, s, false);
    return launch_one<TX, TY, NW, P, false>(a, n_tiles, s, false);
}

// pairs per site for a chain group of cg chains: the next power of two of
// ceil(cg / 2), at most 16
inline int pairs_for_group(int cg) {
    const int pairs = (cg + 1) / 2;
    int P = 1;
    while (P < pairs && P < 16) P <<= 1;
    return P;
}

template <int TX, int TY, int NW>
cudaError_t launch_shape(const SweepArgs& a, int n_tiles, cudaStream_t s, bool setup_only) {
    switch (pairs_for_group(a.chain_group)) {
        case 1: return launch_cfg<TX, TY, NW, 1>(a, n_tiles, s, setup_only);
        case 2: return launch_cfg<TX, TY, NW, 2>(a, n_tiles, s, setup_only);
        case 4: return launch_cfg<TX, TY, NW, 4>(a, n_tiles, s, setup_only);
        case 8: return launch_cfg<TX, TY, NW, 8>(a, n_tiles, s, setup_only);
        default: return launch_cfg<TX, TY, NW, 16>(a, n_tiles, s, setup_only);
    }
}

}  // namespace tiled
}  // namespace mpr
