// Device-side building blocks shared by the MPR kernels: the counter-based
// random stream, the hybrid single-site update of Alg. 1 and small math
// helpers.  Everything here is single precision except where noted.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace mpr {

constexpr float kTwoPi = 6.28318530717958647692f;    // rounds up: 6.2831855f
constexpr float kInvTwoPi = 0.15915494309189533577f;
constexpr float kPi = 3.14159265358979323846f;
constexpr float kFieldEps2 = 1e-24f;                   // |field| < 1e-12: no reflection

// --------------------------------------------------------------- Philox
// Philox4x32-10 (Salmon et al., SC'11): ten rounds of two 32x32 -> 64-bit
// products, Weyl key schedule.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
    for (int i = 0; i < 10; ++i) {
        // one 32 x 32 -> 64-bit multiply each (both halves at once)
        const unsigned long long p0 = (unsigned long long)0xD2511F53u * c.x;
        const unsigned long long p1 = (unsigned long long)0xCD9E8D57u * c.z;
        c = make_uint4((uint32_t)(p1 >> 32) ^ c.y ^ k.x, (uint32_t)p1,
                       (uint32_t)(p0 >> 32) ^ c.w ^ k.y, (uint32_t)p0);
        k.x += 0x9E3779B9u;
        k.y += 0xBB67AE85u;
    }
    return c;
}

// The same generator with the ten round keys precomputed (rk[2i], rk[2i+1]);
// with rk in kernel parameters the XORs take them straight from the
// constant bank.
__device__ __forceinline__ uint4 philox4x32_10_rk(uint4 c, const uint32_t* __restrict__ rk) {
#pragma unroll
    for (int i = 0; i < 10; ++i) {
        const unsigned long long p0 = (unsigned long long)0xD2511F53u * c.x;
        const unsigned long long p1 = (unsigned long long)0xCD9E8D57u * c.z;
        c = make_uint4((uint32_t)(p1 >> 32) ^ c.y ^ rk[2 * i], (uint32_t)p1,
                       (uint32_t)(p0 >> 32) ^ c.w ^ rk[2 * i + 1], (uint32_t)p0);
    }
    return c;
}

// 24-bit uniform in [0, 1), exact in FP32.
__device__ __forceinline__ float u24(uint32_t w) { return (float)(w >> 8) * 0x1p-24f; }

// The random stream's counter for site (x, y) of colour `colour`: one Philox
// call per site (packed column k = x >> 1 of its row) and per pair of
// realisations (chain >> 1).  sweep = 0xFFFFFFFF is the hot start.
__device__ __forceinline__ uint4 site_counter(int x, int y, int colour, uint32_t sweep,
                                              uint32_t chain, uint32_t img) {
    return make_uint4(((uint32_t)y << 16) | ((uint32_t)x >> 1), sweep, chain >> 1,
                      img | ((uint32_t)colour << 31));
}

// (u, r) of a site in realisation `chain`: words 0-1 for an even chain, 2-3
// for an odd one.
__device__ __forceinline__ void site_uniform_words(int x, int y, int colour, uint32_t sweep,
                                                   uint32_t chain, uint32_t img, uint2 key,
                                                   uint32_t& wu, uint32_t& wr) {
    const uint4 w = philox4x32_10(site_counter(x, y, colour, sweep, chain, img), key);
    const bool odd = chain & 1u;
    wu = odd ? w.z : w.x;
    wr = odd ? w.w : w.y;
}

// ---------------------------------------------------------- small math
// sin(t) for |t| <= pi/2 from its Taylor series through t^13 (relative error
// below one ulp on that interval); used for the half proposal step where the
// hardware sine's absolute error would dominate.
__device__ __forceinline__ float sin_taylor(float t) {
    const float t2 = t * t;
    float p = -1.0f / 6227020800.0f;          // -1/13!
    p = fmaf(p, t2, 1.0f / 39916800.0f);       //  1/11!
    p = fmaf(p, t2, -1.0f / 362880.0f);        // -1/9!
    p = fmaf(p, t2, 1.0f / 5040.0f);           //  1/7!  (sign pattern of sin)
    p = fmaf(p, t2, -1.0f / 120.0f);
    p = fmaf(p, t2, 1.0f / 6.0f);
    // sin t = t - t^3/3! + t^5/5! - ...  = t * (1 - t2 * (1/3! - t2 * (1/5! - ...)))
    return t * fmaf(-t2, p, 1.0f);
}

// atan2(y, x) for |x| + |y| > 0: octant reduction to t = min/max in [0, 1]
// and an odd degree-15 polynomial t P(t^2) for atan(t) whose coefficients
// were fitted here (minimax in the absolute error on [0, 1], 3.8e-8 in exact
// arithmetic; about 1.2e-7 rad in FP32 including the approximate reciprocal).
__device__ __forceinline__ float atan2_poly(float y, float x) {
    const float ax = fabsf(x), ay = fabsf(y);
    const float mx = fmaxf(ax, ay), mn = fminf(ax, ay);
    const float t = __fdividef(mn, mx);
    const float t2 = t * t;
    float p = -0.004054575f;
    p = fmaf(p, t2, 0.021862987f);
    p = fmaf(p, t2, -0.05591237f);
    p = fmaf(p, t2, 0.09642201f);
    p = fmaf(p, t2, -0.1390863f);
    p = fmaf(p, t2, 0.19946566f);
    p = fmaf(p, t2, -0.3332986f);
    p = fmaf(p, t2, 0.99999934f);
    float r = p * t;
    if (ay > ax) r = 1.57079632679489662f - r;
    if (x < 0.0f) r = kPi - r;
    return copysignf(r, y);
}

// Wraps an angle from (-3 pi, 3 pi) into [-pi, pi].
__device__ __forceinline__ float wrap_pi(float v) {
    if (v > kPi) v -= kTwoPi;
    else if (v < -kPi) v += kTwoPi;
    return v;
}

// ------------------------------------------------------ hybrid update
struct UpdateConst {
    float q, inv_q, two_pi_q, J;
};

struct UpdateOut {
    float phi;      // new angle
    float R;        // local field length |sum_j exp(i q phi_j)|
    float x_new;    // q * phi_new - Psi (site energy = -J R cos(x_new))
    bool accepted;
};

// The restricted Metropolis half of Alg. 1 (steps 2-6) for a spin at phi1
// (after over-relaxation) in the field of length R and angle Psi:
//  2-3. proposal phi'' = (phi1 + alpha (u - 1/2)) mod 2 pi, alpha = 2 pi / a;
//  4. dH = -J R [cos(q phi'' - Psi) - cos(q phi1 - Psi)]
//        = 2 J R sin(x + h) sin(h), x = q phi1 - Psi, h = q (phi'' - phi1) / 2
//     (product form: no cancellation for small steps);
//  5-6. accept iff r < exp(-dH / T) (always when dH <= 0).
__device__ __forceinline__ UpdateOut metropolis_step(float phi1, float Psi, float R, uint32_t wu,
                                                     uint32_t wr, const UpdateConst& k,
                                                     float alpha, float invT) {
    const float u = u24(wu);
    const float r = u24(wr);
    float phi2 = fmaf(alpha, u - 0.5f, phi1);
    if (phi2 < 0.0f) phi2 += kTwoPi;
    else if (phi2 >= kTwoPi) phi2 -= kTwoPi;
    const float x = fmaf(k.q, phi1, -Psi);
    const float h = 0.5f * k.q * (phi2 - phi1);
    // x + h lies in (-3 pi/2, 5 pi/2): the hardware sine reduces that range itself
    const float s1 = __sinf(x + h);
    const float s2 = sin_taylor(h);
    const float dH = 2.0f * k.J * R * s1 * s2;
    const bool acc = (dH <= 0.0f) || (r < __expf(-dH * invT));
    UpdateOut o;
    o.phi = acc ? phi2 : phi1;
    o.R = R;
    o.x_new = acc ? x + 2.0f * h : x;
    o.accepted = acc;
    return o;
}

// One application of Alg. 1 to a gap site with angle phi whose neighbours
// give the field (C, S) = sum_j (cos q phi_j, sin q phi_j): over-relaxation
// (Eq. over-relax, q-consistent): Psi = atan2(S, C), theta' = (2 Psi - q phi)
// mod 2 pi, phi' = theta'/q if theta' < 2 pi q (else phi' = phi); then the
// restricted Metropolis step.
__device__ __forceinline__ UpdateOut hybrid_update(float phi, float C, float S, uint32_t wu,
                                                   uint32_t wr, const UpdateConst& k,
                                                   float alpha, float invT) {
    const float R2 = fmaf(C, C, S * S);
    float Psi = 0.0f;
    float phi1 = phi;
    float R = 0.0f;
    if (R2 > kFieldEps2) {
        Psi = atan2_poly(S, C);
        R = R2 * rsqrtf(R2);
        float t = fmaf(2.0f, Psi, -k.q * phi);
        t = fmaf(-kTwoPi, floorf(t * kInvTwoPi), t);
        if (t >= 0.0f && t < k.two_pi_q) phi1 = t * k.inv_q;
    }
    return metropolis_step(phi1, Psi, R, wu, wr, k, alpha, invT);
}

// Alg. 1 with the over-relaxation formula as printed (Eq. over-relax with the
// q = 1 field (C1, S1) = sum_j (cos phi_j, sin phi_j)): phi' = (2 Phi - phi)
// mod 2 pi, Phi = atan2(S1, C1), always applied; the Metropolis step still
// uses the MPR energy through its field (C, S).
__device__ __forceinline__ UpdateOut literal_update(float phi, float C, float S, float C1, float S1,
                                                    uint32_t wu, uint32_t wr, const UpdateConst& k,
                                                    float alpha, float invT) {
    const float R2 = fmaf(C, C, S * S);
    float Psi = 0.0f, R = 0.0f;
    if (R2 > kFieldEps2) {
        Psi = atan2_poly(S, C);
        R = R2 * rsqrtf(R2);
    }
    float phi1 = phi;
    if (fmaf(C1, C1, S1 * S1) > kFieldEps2) {
        float t = fmaf(2.0f, atan2_poly(S1, C1), -phi);
        phi1 = fmaf(-kTwoPi, floorf(t * kInvTwoPi), t);
        if (phi1 >= kTwoPi || phi1 < 0.0f) phi1 = 0.0f;
    }
    return metropolis_step(phi1, Psi, R, wu, wr, k, alpha, invT);
}

// Alg. 1 with the GMRF pair interaction of Sec. 4.3 (every bond costs
// J (dphi^2 / (2 pi^2) - 1)): the site energy is quadratic with its minimum at
// the mean m of the n existing neighbours, so over-relaxation reflects about
// it, phi' = 2m - phi, kept inside [0, 2 pi); the proposal and acceptance are
// those of the MPR step, with
// dH = J n (phi'' - phi')(phi'' + phi' - 2m) / (2 pi^2) (a product: no cancellation).
__device__ __forceinline__ UpdateOut gmrf_update(float phi, float m, float n, uint32_t wu,
                                                 uint32_t wr, float J, float alpha, float invT) {
    const float t = fmaf(2.0f, m, -phi);
    const float phi1 = (t >= 0.0f && t < kTwoPi) ? t : phi;
    const float u = u24(wu);
    const float r = u24(wr);
    float phi2 = fmaf(alpha, u - 0.5f, phi1);
    if (phi2 < 0.0f) phi2 += kTwoPi;
    else if (phi2 >= kTwoPi) phi2 -= kTwoPi;
    constexpr float kInvTwoPi2 = 0.050660591821168885f;  // 1 / (2 pi^2)
    const float dH = J * n * kInvTwoPi2 * (phi2 - phi1) * ((phi2 + phi1) - 2.0f * m);
    const bool acc = (dH <= 0.0f) || (r < __expf(-dH * invT));
    UpdateOut o;
    o.phi = acc ? phi2 : phi1;
    o.R = 0.0f;
    o.x_new = 0.0f;
    o.accepted = acc;
    return o;
}

__device__ __forceinline__ float gmrf_bond(float d) {
    return fmaf(d * d, 0.050660591821168885f, -1.0f);
}

// Energy of a site after its update: -J R cos(x_new).
__device__ __forceinline__ float site_energy_after(const UpdateOut& o, float J) {
    return -J * o.R * __cosf(wrap_pi(o.x_new));
}

// --------------------------------------------------------- reductions
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ unsigned warp_sum(unsigned v) {
    return __reduce_add_sync(0xffffffffu, v);
}
__device__ __forceinline__ float warp_min(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fminf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}
__device__ __forceinline__ float warp_max(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// Sample sites are stored with the sign bit set (-0.0f encodes angle 0).
__device__ __forceinline__ bool is_fixed(float v) { return __float_as_uint(v) >> 31; }
__device__ __forceinline__ float angle_of(float v) { return fabsf(v); }
__device__ __forceinline__ float as_fixed(float phi) {
    return __uint_as_float(__float_as_uint(phi) | 0x80000000u);
}

}  // namespace mpr
