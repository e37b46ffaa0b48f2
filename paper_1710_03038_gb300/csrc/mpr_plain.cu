// Plain path: the straightforward GPU form of the checkerboard sweep.
//
// Every realisation keeps a dense [Ly][Lx] angle plane (sample sites carry
// their fixed angle with the sign bit set).  One thread per site of the
// colour being updated and per realisation pair reads the four neighbours of
// both realisations from global memory, takes their sines and cosines, and
// applies the hybrid update of Alg. 1 to the pair (the same pair update and
// the same order of the field sums as the tiled path, so both paths give
// identical bits); one launch per colour (Sec. 5.2: a sweep in two
// checkerboard steps).  This is the baseline the tiled path is measured
// against.
#include "mpr_device.cuh"
#include "mpr_internal.h"

namespace mpr {

namespace {

constexpr int kPlainBX = 128;

__global__ void __launch_bounds__(kPlainBX)
plain_pass_kernel(SweepArgs a) {
    const int np = (a.n_chains + 1) / 2;  // realisation pairs per image
    const int ip = blockIdx.z;
    const int img = ip / np;
    const int m = ip - img * np;
    const int ch0 = 2 * m;
    const bool has1 = ch0 + 1 < a.n_chains;
    const ImgDev& I = a.img[img];
    const int colour = a.colour;
    const int y = blockIdx.y;
    const int xm = blockIdx.x * kPlainBX + threadIdx.x;
    const int x = 2 * xm + ((y + colour) & 1);
    const bool inside = (y < I.Ly) && (x < I.Lx);
    float* P0 = a.state + state_index(I, ch0, 0);
    float* P1 = has1 ? a.state + state_index(I, ch0 + 1, 0) : P0;
    const uint32_t sweep = a.ctl->sweep;

    unsigned n0 = 0, n1 = 0;
    float2 e_site = f2(0.0f);
    if (inside) {
        const long long i = (long long)y * I.Lx + x;
        const float v0 = P0[i];
        // neighbours in the order up, down, left, right
        const bool has[4] = {y > 0, y + 1 < I.Ly, x > 0, x + 1 < I.Lx};
        const long long off[4] = {-(long long)I.Lx, (long long)I.Lx, -1, 1};
        float2 nb[4];
        bool fixed_nb[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const float w0 = has[j] ? P0[i + off[j]] : 0.0f;
            const float w1 = has[j] ? P1[i + off[j]] : 0.0f;
            fixed_nb[j] = has[j] && is_fixed(w0);
            nb[j] = make_float2(angle_of(w0), angle_of(w1));
        }
        float2 phi_now = make_float2(angle_of(v0), angle_of(P1[i]));
        if (!is_fixed(v0)) {
            const int cg = img * a.n_chains + ch0;
            const float2 alpha_s =
                (a.flags & kAlphaOne)
                    ? f2(proposal_width(1.0f))
                    : make_float2(a.ch.alpha[cg], has1 ? a.ch.alpha[cg + 1] : 0.0f);
            const float c_acc = 1.4426950408889634f * I.invT;
            const uint4 w = philox4x32_10(
                site_counter(x, y, colour, sweep, (uint32_t)ch0, (uint32_t)img | a.img_tag), a.key);
            const PairRand u = pair_uniforms(w);
            const UpdateConst k{a.q, a.inv_q, a.two_pi_q, a.J};
            PairOut o;
            if (a.flags & kGMRF) {
                // neighbour sum: sample neighbours first, then gap neighbours,
                // each in the order up, down, left, right (the tiled path's order)
                float2 sum = f2(0.0f);
                float n = 0.0f;
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    if (fixed_nb[j]) sum = add2(sum, nb[j]);
                    n += has[j] ? 1.0f : 0.0f;
                }
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    if (has[j] && !fixed_nb[j]) sum = add2(sum, nb[j]);
                o = gmrf_pair<false>(phi_now, sum, n, u, a.J, alpha_s, c_acc);
            } else {
                float2 cn[4], sn[4];
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const float2 qn = mul2(f2(a.q), nb[j]);
                    __sincosf(qn.x, &sn[j].x, &cn[j].x);
                    __sincosf(qn.y, &sn[j].y, &cn[j].y);
                }
                // the local field: sample neighbours first, then gap neighbours
                float2 C = f2(0.0f), S = f2(0.0f);
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    if (fixed_nb[j]) { C = add2(C, cn[j]); S = add2(S, sn[j]); }
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    if (has[j] && !fixed_nb[j]) { C = add2(C, cn[j]); S = add2(S, sn[j]); }
                if (a.flags & kLiteralOR) {
                    float2 c1[4], s1[4];
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        __sincosf(nb[j].x, &s1[j].x, &c1[j].x);
                        __sincosf(nb[j].y, &s1[j].y, &c1[j].y);
                    }
                    float2 C1 = f2(0.0f), S1 = f2(0.0f);
#pragma unroll
                    for (int j = 0; j < 4; ++j)
                        if (fixed_nb[j]) { C1 = add2(C1, c1[j]); S1 = add2(S1, s1[j]); }
#pragma unroll
                    for (int j = 0; j < 4; ++j)
                        if (has[j] && !fixed_nb[j]) { C1 = add2(C1, c1[j]); S1 = add2(S1, s1[j]); }
                    o = literal_pair<false>(phi_now, C, S, C1, S1, u, k, alpha_s, c_acc);
                } else {
                    o = hybrid_pair<false>(phi_now, C, S, u, k, alpha_s, c_acc);
                }
            }
            P0[i] = o.phi.x;
            if (has1) P1[i] = o.phi.y;
            phi_now = o.phi;
            n0 = o.acc0;
            n1 = has1 && o.acc1;
            if (a.flags & kAccumulate) {
                atomicAdd(a.acc1 + I.slot_off + i, (double)o.phi.x);
                if (has1) atomicAdd(a.acc1 + I.slot_off + i, (double)o.phi.y);
                if (a.flags & kAccumulate2) {
                    atomicAdd(a.acc2 + I.slot_off + i, (double)o.phi.x * o.phi.x);
                    if (has1) atomicAdd(a.acc2 + I.slot_off + i, (double)o.phi.y * o.phi.y);
                }
            }
        }
        if (a.flags & kEnergy) {
            // every bond has exactly one end of the second colour
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                if (!has[j]) continue;
                if (a.flags & kGMRF) {
                    e_site.x += a.J * gmrf_bond(phi_now.x - nb[j].x);
                    e_site.y += a.J * gmrf_bond(phi_now.y - nb[j].y);
                } else {
                    e_site.x += -a.J * __cosf(a.q * (phi_now.x - nb[j].x));
                    e_site.y += -a.J * __cosf(a.q * (phi_now.y - nb[j].y));
                }
            }
        }
    }
    const long long slot =
        (long long)(img * a.n_chains + ch0) * kSpread + ((blockIdx.x + blockIdx.y) & (kSpread - 1));
    n0 = warp_sum(n0);
    n1 = warp_sum(n1);
    if ((threadIdx.x & 31) == 0) {
        if (n0) atomicAdd(a.ch.acc_cnt + slot, n0);
        if (n1) atomicAdd(a.ch.acc_cnt + slot + kSpread, n1);
    }
    if (a.flags & kEnergy) {
        const double e0 = warp_sum((double)e_site.x);
        const double e1 = warp_sum((double)e_site.y);
        if ((threadIdx.x & 31) == 0) {
            if (e0 != 0.0) atomicAdd(a.ch.e_cur + slot, e0);
            if (has1 && e1 != 0.0) atomicAdd(a.ch.e_cur + slot + kSpread, e1);
        }
    }
}

}  // namespace

cudaError_t launch_plain_pass(const SweepArgs& a, int max_Lx, int max_Ly, cudaStream_t s) {
    const int half = (max_Lx + 1) / 2;
    dim3 grid((half + kPlainBX - 1) / kPlainBX, max_Ly, a.n_img * ((a.n_chains + 1) / 2));
    plain_pass_kernel<<<grid, kPlainBX, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace mpr
