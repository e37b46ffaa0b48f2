// Tiled path: the batched checkerboard pass (kernel template).
//
// Layout.  Sample angles are identical in every realisation, so they are
// stored once per image (`samp`).  A realisation stores only its gap angles:
// the image is cut into TX x TY tiles and the gap sites of one tile and one
// colour form a contiguous segment of the image's slot space (row-major
// inside the tile, padded to 4 slots).  The state is slot-major with the
// realisations interleaved: slot k of chain r sits at k * CP + r, CP being the
// chain count rounded up to a multiple of 4, so the pair (2m, 2m + 1) of one
// slot is one aligned float2 and the pairs of a chain group are contiguous.
//
// Work.  One thread block takes one tile and a group of 2P chains (P pairs).
// A warp lane is (site s, pair p) with p = lane mod P, so a warp step covers
// 32 / P sites of the tile for every pair of the group; the ragged end of a
// tile leaves at most one step partly idle.  Per launch the block
//  - prepares, for every own-colour gap site, the constant part of its local
//    field (sines and cosines of its sample neighbours, summed up, down, left,
//    right), its random-stream counter word, and the byte offsets of its four
//    neighbours' entries in the block's table of other-colour gap cells
//    (interior segment, then the 1-cell ring; entry 0 holds zeros for
//    neighbours that are not gaps);
//  - fills that table for all chains of the group: entry e, pair p holds
//    (cos q phi_0, cos q phi_1, sin q phi_0, sin q phi_1) of the pair's two
//    chains (one float4, so the fields of both chains add as FP32x2 pairs);
//    the angle pairs arrive by asynchronous 8-byte copies (cp.async) that are
//    contiguous across the pairs of a slot, and are converted in place;
//  - updates every own-colour gap site of every chain with Alg. 1, one Philox
//    block and one packed FP32x2 instruction stream serving the site in both
//    chains of a pair, and stores the new pair as one float2;
//  - in sampling sweeps sums each site's new angles (and their squares) over
//    the chain group in shared memory, in fixed point (2^-24 rad, 2^-21 rad^2:
//    integer adds, exact and independent of their order; lanes p and p + 8
//    pre-add with one shuffle), and adds the sums to the FP64 realisation sums
//    once every site is done.
// Acceptances and energies stay in registers until the end of the block.
//
// Energy (black pass).  Every bond joins a red and a black site.  H is the
// sample-sample part (constant, from the initialisation) plus the bonds of
// black gap sites (their site energy after their update) plus the bonds
// between red gap sites and black sample sites.
//
// Models.  kModelMPR: the MPR bond with the q-consistent over-relaxation;
// kModelLIT: the over-relaxation as printed (q = 1 field; the table cell
// carries a second float4 with (cos phi, sin phi)); kModelGMRF: the GMRF bond
// of Sec. 4.3 (the table holds the raw angle pairs, the field is the
// neighbour sum).
#pragma once

#include "mpr_async.cuh"
#include "mpr_device.cuh"
#include "mpr_internal.h"

namespace mpr {
namespace tiled {

enum Model : int { kModelMPR = 0, kModelLIT = 1, kModelGMRF = 2 };


// bytes of one (entry, pair) table cell
template <int MODEL>
struct Cell {
    static constexpr int bytes = MODEL == kModelGMRF ? 8 : (MODEL == kModelLIT ? 32 : 16);
};

template <int TX, int TY, int NW, int MODEL>
struct Cfg {
    static constexpr int NT = NW * 32;
    static constexpr int NMAX = TX * TY / 2;       // sites of one colour in a tile
    static constexpr int HCAP = TX + TY;           // ring cells of one colour
    static constexpr int GT = NMAX + HCAP + 1;     // table entries (entry 0 = zeros)
    static constexpr size_t a16(size_t v) { return (v + 15) / 16 * 16; }
    // per own site: byte offsets of the four neighbour entries
    static constexpr size_t off_rows = 0;
    // per own site: sample field (x, y), counter word, unused
    static constexpr size_t off_k = off_rows + sizeof(uint4) * NMAX;
    // per own site (kModelLIT): the q = 1 sample field
    static constexpr size_t off_f1 = off_k + sizeof(uint4) * NMAX;
    static constexpr size_t off_red = off_f1 + (MODEL == kModelLIT ? sizeof(float4) * NMAX : 0);
    // the table last, sized at launch for the largest tile of the pass
    // the per-chain reduction area; sampling passes first keep the own sites'
    // fixed-point realisation sums there (two words per site)
    static constexpr size_t red_bytes =
        sizeof(float4) * NW * 16 > 8 * NMAX ? sizeof(float4) * NW * 16 : 8 * NMAX;
    static constexpr size_t off_tab = off_red + red_bytes;
    static constexpr size_t smem_for(int gt, int P) {
        return off_tab + (size_t)Cell<MODEL>::bytes * P * gt;
    }
    static constexpr size_t smem_max = smem_for(GT, 16);
};

__device__ __forceinline__ float4 tab_f4(const unsigned char* p) {
    return *reinterpret_cast<const float4*>(p);
}
__device__ __forceinline__ float2 tab_f2(const unsigned char* p) {
    return *reinterpret_cast<const float2*>(p);
}

// GMRF bonds of a pair of angles against a sample angle v.
__device__ __forceinline__ float2 gmrf_bond2(float2 phi, float v) {
    const float2 d = add2(phi, f2(-v));
    return fma2(mul2(d, d), f2(0.050660591821168885f), f2(-1.0f));
}

template <int TX, int TY, int NW, int P, bool ACC, int MODEL>
__global__ void __launch_bounds__(NW * 32, 1024 / (NW * 32))  // 64 registers: 32 warps per SM
tiled_pass_kernel(const __grid_constant__ SweepArgs a) {
    using Cf = Cfg<TX, TY, NW, MODEL>;
    constexpr int NT = Cf::NT;
    constexpr int SPW = 32 / P;  // sites per warp step
    constexpr int CB = Cell<MODEL>::bytes;
    static_assert(P >= 1 && P <= 16 && (P & (P - 1)) == 0, "pairs per site: power of two");
    extern __shared__ __align__(16) unsigned char smem[];
    uint4* own_rows = reinterpret_cast<uint4*>(smem + Cf::off_rows);
    uint4* own_k = reinterpret_cast<uint4*>(smem + Cf::off_k);
    float4* own_f1 = reinterpret_cast<float4*>(smem + Cf::off_f1);
    float4* red = reinterpret_cast<float4*>(smem + Cf::off_red);
    unsigned char* tab = smem + Cf::off_tab;
    // sampling passes: per own site, the sums over the block's chains of phi
    // (units of 2^-24 rad) and of phi^2 (units of 2^-21 rad^2), exact in 32 bits
    // for up to 32 chains
    uint32_t* accs = reinterpret_cast<uint32_t*>(smem + Cf::off_red);

    const int tid = threadIdx.x;
    const int lane = tid & 31;
    const int warp = tid >> 5;
    const int p = lane & (P - 1);  // pair of the group (fixed per thread: NT is a multiple of P)
    const int s = lane / P;        // site within a warp step
    const int tile = a.tile_list ? a.tile_list[a.tile_base + blockIdx.x] : (int)blockIdx.x;
    // the tile record carries everything the addresses need (one dependent load)
    const TileDesc T = a.tiles[tile];
    const int c = a.colour;
    const int n_own = c ? T.cnt[1] : T.cnt[0];
    const bool energy = (a.flags & kEnergy) != 0;
    const int n_oth = c ? T.cnt[0] : T.cnt[1];
    // nothing to update and no red-gap / black-sample bond energy to add
    if (n_own == 0 && !(energy && n_oth > 0)) return;
    const int t_img = T.img;
    const int off_own = c ? T.off[1] : T.off[0], off_oth = c ? T.off[0] : T.off[1];
    const int n_halo = c ? T.halo_cnt[1] : T.halo_cnt[0];
    const long long slot_off = T.slot_off;
    const ImgDev& I = a.img[t_img];
    const int r0 = a.chain0 + blockIdx.y * a.chain_group;
    const int ng = min(a.chain_group, a.chain_end - r0);
    const bool has0 = 2 * p < ng;      // this lane's pair exists
    const bool has1 = 2 * p + 1 < ng;  // and has a second chain
    const uint32_t sweep = a.ctl->sweep;
    const uint32_t c3 = (uint32_t)t_img | a.img_tag | ((uint32_t)c << 31);
    const uint32_t c2 = (uint32_t)(r0 >> 1) + (uint32_t)p;  // chain >> 1 of the pair
    const UpdateConst uk{a.q, a.inv_q, a.two_pi_q, a.J};
    const long long cp = T.cp;  // floats from one slot to the next
    // this lane's pair at slot 0 (8-byte aligned: state_off, cp, r0 are even)
    float* st = a.state + T.state_off + r0 + 2 * p;
        float* sto = st + (long long)off_own * cp;  // this lane's pair at the own segment
    const int cpi = (int)cp;
    // angles of the first warp step, in flight during the table fill
    float2 vn = make_float2(0.0f, 0.0f);
    {
        const int j = warp * SPW + s;
        if (has0 && j < n_own) vn = *reinterpret_cast<const float2*>(sto + j * cpi);
    }
    const int spread = tile & (kSpread - 1);

    // -- table of the other colour, raw: entry 1 + e, pair p ----------------------
    // Each thread copies the angle pairs of its entries e = tid / P (mod NT / P)
    // straight into the first 8 bytes of their table cells (all copies in flight
    // at once, no registers) and converts the same entries below, so its own
    // wait is enough.  Lanes without a pair copy nothing (their table column is
    // never read for a stored result).
    constexpr int NTP = NT / P;
    const int n_ent = n_oth + n_halo;
    const int e_lo = tid / P;
    const uint32_t tab_s = smem_addr(tab);
    const uint32_t cell_lo = tab_s + (uint32_t)((1 + e_lo) * P + p) * CB;  // this thread's first cell
    constexpr uint32_t kDstStep = (uint32_t)CB * NTP * P;
    if (has0) {
        const float* src = st + (long long)(off_oth + e_lo) * cp;
        const long long src_step = (long long)NTP * cp;
        uint32_t dst = cell_lo;
        for (int e = e_lo; e < n_oth; e += NTP, src += src_step, dst += kDstStep)
            cp_async8_s(dst, src);
    }
    if (tid < P) {
        float4* z = reinterpret_cast<float4*>(tab + tid * CB);
        if (CB >= 16) z[0] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        if (CB == 32) z[1] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        if (CB == 8) *reinterpret_cast<float2*>(z) = make_float2(0.0f, 0.0f);
    }

    // -- own-colour constants of the tile (built once per batch) ---------------
    {
        const long long b = slot_off + off_own;
        constexpr uint32_t kRow = (uint32_t)CB * P;  // bytes per table entry
        if (ACC)
            for (int j = tid; j < n_own; j += NT) accs[j] = accs[Cf::NMAX + j] = 0u;
        for (int j = tid; j < n_own; j += NT) {
            const uint2 r = a.slot_ref[b + j];
            const float4 f = a.slot_cs[b + j];
            own_rows[j] = make_uint4((r.x & 0xFFFFu) * kRow, (r.x >> 16) * kRow,
                                     (r.y & 0xFFFFu) * kRow, (r.y >> 16) * kRow);
            const uint32_t pos = a.slot_pos[b + j];
            own_k[j] = make_uint4(__float_as_uint(f.x), __float_as_uint(f.y),
                                  (pos & 0xFFFF0000u) | ((pos & 0xFFFFu) >> 1), 0u);
            if (MODEL == kModelLIT) own_f1[j] = make_float4(f.z, f.w, 0.0f, 0.0f);
        }
    }
    // ring cells (slots from the ring list), same entry residue as above
    if (has0) {
        const int k_first = (max(n_oth - e_lo, 0) + NTP - 1) / NTP;  // steps to the ring
        const int e_first = e_lo + k_first * NTP;
        const int2* h = a.halo + ((long long)tile * 2 + c) * a.halo_cap + (e_first - n_oth);
        uint32_t dst = cell_lo + (uint32_t)k_first * kDstStep;
        for (int e = e_first; e < n_ent; e += NTP, h += NTP, dst += kDstStep)
            cp_async8_s(dst, st + (long long)h->x * cp);
    }
    cp_async_wait_all();

    // -- conversion in place; bonds between other-colour gap cells and their
    //    sample neighbours on energy passes ------------------------------------
    float2 esum = f2(0.0f);  // energies of the pair's two chains
    if (has0) {
        const float4* fcs = a.slot_cs + slot_off + off_oth;
        unsigned char* t = tab + (size_t)((1 + e_lo) * P + p) * CB;
        for (int e = e_lo; e < n_ent; e += NTP, t += (size_t)NTP * P * CB) {
            const float2 v = *reinterpret_cast<const float2*>(t);
            if (MODEL != kModelGMRF) {
                const float2 qv = mul2(f2(a.q), v);
                float s0, c0, s1, c1;
                __sincosf(qv.x, &s0, &c0);
                __sincosf(qv.y, &s1, &c1);
                if (MODEL == kModelLIT) {
                    float u0, w0, u1, w1;
                    __sincosf(v.x, &u0, &w0);
                    __sincosf(v.y, &u1, &w1);
                    reinterpret_cast<float4*>(t)[1] = make_float4(w0, w1, u0, u1);
                }
                *reinterpret_cast<float4*>(t) = make_float4(c0, c1, s0, s1);
                if (energy && e < n_oth) {
                    const float4 f = fcs[e];
                    const float2 d = fma2(f2(f.x), make_float2(c0, c1), mul2(f2(f.y), make_float2(s0, s1)));
                    esum = fma2(f2(-a.J), d, esum);
                }
            } else if (energy && e < n_oth) {
                // GMRF: bonds to the sample neighbours from the sample plane
                const uint32_t pos = a.slot_pos[slot_off + off_oth + e];
                const int X = (int)(pos & 0xFFFFu), Y = (int)(pos >> 16);
                const float* sp = a.samp + I.site_off + (long long)Y * I.Lx + X;
                float vs[4] = {Y > 0 ? sp[-I.Lx] : -1.0f, Y + 1 < I.Ly ? sp[I.Lx] : -1.0f,
                               X > 0 ? sp[-1] : -1.0f, X + 1 < I.Lx ? sp[1] : -1.0f};
#pragma unroll
                for (int m = 0; m < 4; ++m)
                    if (vs[m] >= 0.0f) esum = fma2(f2(a.J), gmrf_bond2(v, vs[m]), esum);
            }
        }
    }
    __syncthreads();

    // -- own colour: every site of every chain of the group ---------------------
    const int ch0 = t_img * a.n_chains + r0 + 2 * p;
    const float2 alpha_s =
        (a.flags & kAlphaOne)
            ? f2(proposal_width(1.0f))
            : make_float2(has0 ? a.ch.alpha[ch0] : 0.0f, has1 ? a.ch.alpha[ch0 + 1] : 0.0f);
    const float c_acc = 1.4426950408889634f * I.invT;  // log2(e) / T
    unsigned cnt0 = 0, cnt1 = 0;
    const int n_steps = (n_own + SPW - 1) / SPW;
    const unsigned char* tabp = tab + p * CB;  // this lane's column of the table
    // angles of a warp step: loaded one step ahead, in flight during the step before
    for (int g = warp; g < n_steps; g += NW) {  // warp-uniform
        const float2 vc = vn;
        {
            const int jn = (g + NW) * SPW + s;
            vn = make_float2(0.0f, 0.0f);
            if (has0 && jn < n_own) vn = *reinterpret_cast<const float2*>(sto + jn * cpi);
        }
        const int j = g * SPW + s;
        const bool in = j < n_own;
        const bool act = in && has0;
        const int jj = in ? j : 0;  // idle lanes recompute slot 0 and store nothing
        const uint4 rw = own_rows[jj];
        const uint4 kk = own_k[jj];
        const uint4 w = philox4x32_10_rk(make_uint4(kk.z, sweep, c2, c3), a.rk);
        const PairRand u = pair_uniforms(w);
        PairOut o;
        if (MODEL == kModelGMRF) {
            const float2 gu = tab_f2(tabp + rw.x), gd = tab_f2(tabp + rw.y);
            const float2 gl = tab_f2(tabp + rw.z), gr = tab_f2(tabp + rw.w);
            const float2 sum = add2(add2(add2(add2(f2(__uint_as_float(kk.x)), gu), gd), gl), gr);
            o = gmrf_pair<false>(vc, sum, __uint_as_float(kk.y), u, a.J, alpha_s, c_acc);
            if (energy) {
                // the site's bonds after its update: gap neighbours from the table,
                // sample neighbours from the sample plane
                const int Y = (int)(kk.z >> 16);
                const int X = 2 * (int)(kk.z & 0xFFFFu) + ((Y ^ c) & 1);
                const float* sp = a.samp + I.site_off + (long long)Y * I.Lx + X;
                const bool hn[4] = {Y > 0, Y + 1 < I.Ly, X > 0, X + 1 < I.Lx};
                const long long dn[4] = {-(long long)I.Lx, (long long)I.Lx, -1, 1};
                const float2 gv[4] = {gu, gd, gl, gr};
                const uint32_t rr[4] = {rw.x, rw.y, rw.z, rw.w};
                float2 es = f2(0.0f);
#pragma unroll
                for (int m = 0; m < 4; ++m) {
                    if (!hn[m]) continue;
                    const float vs = sp[dn[m]];
                    if (vs >= 0.0f) es = add2(es, gmrf_bond2(o.phi, vs));
                    else if (rr[m] != 0u) {
                        const float2 d = add2(o.phi, mul2(gv[m], f2(-1.0f)));
                        es = add2(es, fma2(mul2(d, d), f2(0.050660591821168885f), f2(-1.0f)));
                    }
                }
                o.e = mul2(f2(a.J), es);
            }
        } else {
            const float4 gu = tab_f4(tabp + rw.x), gd = tab_f4(tabp + rw.y);
            const float4 gl = tab_f4(tabp + rw.z), gr = tab_f4(tabp + rw.w);
            const float fsx = __uint_as_float(kk.x), fsy = __uint_as_float(kk.y);
            const float2 C = add2(add2(add2(add2(f2(fsx), make_float2(gu.x, gu.y)),
                                            make_float2(gd.x, gd.y)),
                                       make_float2(gl.x, gl.y)),
                                  make_float2(gr.x, gr.y));
            const float2 S = add2(add2(add2(add2(f2(fsy), make_float2(gu.z, gu.w)),
                                            make_float2(gd.z, gd.w)),
                                       make_float2(gl.z, gl.w)),
                                  make_float2(gr.z, gr.w));
            if (MODEL == kModelLIT) {
                const float4 f1 = own_f1[jj];
                const float4 hu = tab_f4(tabp + rw.x + 16), hd = tab_f4(tabp + rw.y + 16);
                const float4 hl = tab_f4(tabp + rw.z + 16), hr = tab_f4(tabp + rw.w + 16);
                const float2 C1 = add2(add2(add2(add2(f2(f1.x), make_float2(hu.x, hu.y)),
                                                 make_float2(hd.x, hd.y)),
                                            make_float2(hl.x, hl.y)),
                                       make_float2(hr.x, hr.y));
                const float2 S1 = add2(add2(add2(add2(f2(f1.y), make_float2(hu.z, hu.w)),
                                                 make_float2(hd.z, hd.w)),
                                            make_float2(hl.z, hl.w)),
                                       make_float2(hr.z, hr.w));
                if (energy) o = literal_pair<true>(vc, C, S, C1, S1, u, uk, alpha_s, c_acc);
                else o = literal_pair<false>(vc, C, S, C1, S1, u, uk, alpha_s, c_acc);
            } else {
                if (energy) o = hybrid_pair<true>(vc, C, S, u, uk, alpha_s, c_acc);
                else o = hybrid_pair<false>(vc, C, S, u, uk, alpha_s, c_acc);
            }
        }
        const bool act1 = act && has1;
        // a missing second chain is the padding chain of the layout: storing there is harmless
        if (act) *reinterpret_cast<float2*>(sto + j * cpi) = o.phi;
        if (ACC) {
            // this pair's part of the site's realisation sums, added to that of
            // pair p + 8 first (half the lanes on each shared-memory word), then
            // in fixed point
            const float x0 = act ? o.phi.x : 0.0f, x1 = act1 ? o.phi.y : 0.0f;
            float sa = x0 + x1, sb = fmaf(x0, x0, x1 * x1);
            constexpr int kAdders = P >= 16 ? 8 : P;
            if (P >= 16) {
                sa += __shfl_xor_sync(0xffffffffu, sa, 8);
                sb += __shfl_xor_sync(0xffffffffu, sb, 8);
            }
            if (in && p < kAdders) {
                atomicAdd(&accs[j], __float2uint_rn(sa * 16777216.0f));
                atomicAdd(&accs[Cf::NMAX + j], __float2uint_rn(sb * 2097152.0f));
            }
        }
        cnt0 += (act && o.acc0) ? 1u : 0u;
        cnt1 += (act1 && o.acc1) ? 1u : 0u;
        if (energy) esum = add2(esum, make_float2(act ? o.e.x : 0.0f, act1 ? o.e.y : 0.0f));
    }

    if (ACC) {
        // the block's sums go to the FP64 realisation sums (fire-and-forget adds;
        // one add per site and block)
        __syncthreads();
        const bool accum2 = (a.flags & kAccumulate2) != 0;
        for (int j = tid; j < n_own; j += NT) {
            atomicAdd(a.acc1 + slot_off + off_own + j, (double)accs[j] * 0x1p-24);
            if (accum2)
                atomicAdd(a.acc2 + slot_off + off_own + j, (double)accs[Cf::NMAX + j] * 0x1p-21);
        }
        __syncthreads();  // the per-chain reduction below reuses the area
    }

    // -- per-chain totals: lanes of one pair, then warps ------------------------
    float e0 = esum.x, e1 = esum.y;
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

template <int TX, int TY, int NW, int P, bool ACC, int MODEL>
cudaError_t launch_one(const SweepArgs& a, cudaStream_t s, bool setup_only) {
    using Cf = Cfg<TX, TY, NW, MODEL>;
    static_assert(Cf::smem_max <= 227 * 1024, "shared memory");
    static bool attr_set = false;
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(tiled_pass_kernel<TX, TY, NW, P, ACC, MODEL>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)Cf::smem_max);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    if (setup_only) return cudaSuccess;
    if (a.gt < 1 || a.gt > Cf::GT) return cudaErrorInvalidValue;
    dim3 grid(a.n_list, (a.chain_end - a.chain0 + a.chain_group - 1) / a.chain_group);
    tiled_pass_kernel<TX, TY, NW, P, ACC, MODEL><<<grid, Cf::NT, Cf::smem_for(a.gt, P), s>>>(a);
    return cudaGetLastError();
}

template <int TX, int TY, int NW, int P, int MODEL>
cudaError_t launch_cfg(const SweepArgs& a, cudaStream_t s, bool setup_only) {
    if (setup_only) {
        cudaError_t e = launch_one<TX, TY, NW, P, false, MODEL>(a, s, true);
        return e != cudaSuccess ? e : launch_one<TX, TY, NW, P, true, MODEL>(a, s, true);
    }
    if (a.flags & kAccumulate) return launch_one<TX, TY, NW, P, true, MODEL>(a, s, false);
    return launch_one<TX, TY, NW, P, false, MODEL>(a, s, false);
}

// pairs per site for a chain group of cg chains: the next power of two of
// ceil(cg / 2), at most 16
inline int pairs_for_group(int cg) {
    const int pairs = (cg + 1) / 2;
    int P = 1;
    while (P < pairs && P < 16) P <<= 1;
    return P;
}

template <int TX, int TY, int NW, int MODEL>
cudaError_t launch_shape(const SweepArgs& a, cudaStream_t s, bool setup_only) {
    switch (pairs_for_group(a.chain_group)) {
        case 1: return launch_cfg<TX, TY, NW, 1, MODEL>(a, s, setup_only);
        case 2: return launch_cfg<TX, TY, NW, 2, MODEL>(a, s, setup_only);
        case 4: return launch_cfg<TX, TY, NW, 4, MODEL>(a, s, setup_only);
        case 8: return launch_cfg<TX, TY, NW, 8, MODEL>(a, s, setup_only);
        default: return launch_cfg<TX, TY, NW, 16, MODEL>(a, s, setup_only);
    }
}

}  // namespace tiled
}  // namespace mpr
