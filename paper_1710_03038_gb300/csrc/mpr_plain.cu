// Plain path: the straightforward GPU form of the checkerboard sweep.
//
// Every realisation keeps a dense [Ly][Lx] angle plane (sample sites carry
// their fixed angle with the sign bit set).  One thread per site of the
// colour being updated reads its four neighbours from global memory, takes
// their sines and cosines, and applies the hybrid update of Alg. 1; one
// launch per colour (Sec. 5.2: a sweep in two checkerboard steps).  This is
// the baseline the tiled path is measured against.
#include "mpr_device.cuh"
#include "mpr_internal.h"

namespace mpr {

namespace {

constexpr int kPlainBX = 128;

__global__ void __launch_bounds__(kPlainBX)
plain_pass_kernel(SweepArgs a) {
    const int ic = blockIdx.z;
    const int img = ic / a.n_chains;
    const int chain = ic - img * a.n_chains;
    const ImgDev& I = a.img[img];
    const int colour = a.colour;
    const int y = blockIdx.y;
    const int m = blockIdx.x * kPlainBX + threadIdx.x;
    const int x = 2 * m + ((y + colour) & 1);
    const bool inside = (y < I.Ly) && (x < I.Lx);
    float* P = a.state + state_index(I, chain, 0);
    const uint32_t sweep = a.ctl->sweep;

    unsigned n_acc = 0;
    float e_site = 0.0f;
    if (inside) {
        const long long i = (long long)y * I.Lx + x;
        const float v = P[i];
        // neighbours in the order up, down, left, right
        float nb[4];
        bool has[4] = {y > 0, y + 1 < I.Ly, x > 0, x + 1 < I.Lx};
        nb[0] = has[0] ? angle_of(P[i - I.Lx]) : 0.0f;
        nb[1] = has[1] ? angle_of(P[i + I.Lx]) : 0.0f;
        nb[2] = has[2] ? angle_of(P[i - 1]) : 0.0f;
        nb[3] = has[3] ? angle_of(P[i + 1]) : 0.0f;
        // local field: sample neighbours first, then gap neighbours, each in the
        // order up, down, left, right (the tiled path sums in the same order)
        bool fixed_nb[4];
        fixed_nb[0] = has[0] && is_fixed(P[i - I.Lx]);
        fixed_nb[1] = has[1] && is_fixed(P[i + I.Lx]);
        fixed_nb[2] = has[2] && is_fixed(P[i - 1]);
        fixed_nb[3] = has[3] && is_fixed(P[i + 1]);
        float sn[4], cn[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) __sincosf(a.q * nb[j], &sn[j], &cn[j]);
        float C = 0.0f, S = 0.0f;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            C += fixed_nb[j] ? cn[j] : 0.0f;
            S += fixed_nb[j] ? sn[j] : 0.0f;
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const bool g = has[j] && !fixed_nb[j];
            C += g ? cn[j] : 0.0f;
            S += g ? sn[j] : 0.0f;
        }
        float phi_now = angle_of(v);
        if (!is_fixed(v)) {
            const int ch_global = img * a.n_chains + chain;
            const float alpha = (a.flags & kAlphaOne) ? kTwoPi : kTwoPi / a.ch.a[ch_global];
            uint32_t wu, wr;
            site_uniform_words(x, y, colour, sweep, (uint32_t)chain, (uint32_t)img | a.img_tag,
                               a.key, wu, wr);
            UpdateConst k{a.q, a.inv_q, a.two_pi_q, a.J};
            UpdateOut o;
            if (a.flags & kGMRF) {
                float sum = 0.0f, cnt = 0.0f;
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    sum += has[j] ? nb[j] : 0.0f;
                    cnt += has[j] ? 1.0f : 0.0f;
                }
                o = gmrf_update(phi_now, sum / cnt, cnt, wu, wr, a.J, alpha, I.invT);
            } else if (a.flags & kLiteralOR) {
                float C1 = 0.0f, S1 = 0.0f;
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    float s1, c1;
                    sincosf(nb[j], &s1, &c1);
                    C1 += has[j] ? c1 : 0.0f;
                    S1 += has[j] ? s1 : 0.0f;
                }
                o = literal_update(phi_now, C, S, C1, S1, wu, wr, k, alpha, I.invT);
            } else {
                o = hybrid_update(phi_now, C, S, wu, wr, k, alpha, I.invT);
            }
            P[i] = o.phi;
            phi_now = o.phi;
            n_acc = o.accepted;
            if (a.flags & kAccumulate) {
                atomicAdd(a.acc1 + I.slot_off + i, (double)o.phi);
                if (a.flags & kAccumulate2) atomicAdd(a.acc2 + I.slot_off + i, (double)o.phi * o.phi);
            }
        }
        if (a.flags & kEnergy) {
            // every bond has exactly one end of the second colour
            if (a.flags & kGMRF) {
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    e_site += has[j] ? a.J * gmrf_bond(phi_now - nb[j]) : 0.0f;
            } else {
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    e_site += has[j] ? -a.J * __cosf(a.q * (phi_now - nb[j])) : 0.0f;
            }
        }
    }
    const long long slot =
        (long long)(img * a.n_chains + chain) * kSpread + ((blockIdx.x + blockIdx.y) & (kSpread - 1));
    n_acc = warp_sum(n_acc);
    if ((threadIdx.x & 31) == 0 && n_acc) atomicAdd(a.ch.acc_cnt + slot, n_acc);
    if (a.flags & kEnergy) {
        const double e = warp_sum((double)e_site);
        if ((threadIdx.x & 31) == 0 && e != 0.0) atomicAdd(a.ch.e_cur + slot, e);
    }
}

}  // namespace

cudaError_t launch_plain_pass(const SweepArgs& a, int max_Lx, int max_Ly, cudaStream_t s) {
    const int half = (max_Lx + 1) / 2;
    dim3 grid((half + kPlainBX - 1) / kPlainBX, max_Ly, a.n_img * a.n_chains);
    plain_pass_kernel<<<grid, kPlainBX, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace mpr
