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
constexpr float kFieldEps2 = 1e-12f;                   // |field| < 1e-6: vanishing field

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
// Every realisation pair (2m, 2m + 1) is updated by one thread: both updates
// run the same instruction sequence on different data, so the FP32 adds,
// multiplies and FMAs of the pair are issued as packed FP32x2 instructions
// (sm_100 and later), one issue slot for both realisations.  Each component
// is rounded exactly as the scalar operation would be.
__device__ __forceinline__ float2 f2(float v) { return make_float2(v, v); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
// c - a (one rounding, as the scalar subtraction)
__device__ __forceinline__ float2 rsub2(float2 a, float2 c) { return __ffma2_rn(a, f2(-1.0f), c); }
__device__ __forceinline__ float2 floor2(float2 a) { return make_float2(floorf(a.x), floorf(a.y)); }
__device__ __forceinline__ float2 sel2(bool p0, bool p1, float2 a, float2 b) {
    return make_float2(p0 ? a.x : b.x, p1 ? a.y : b.y);
}

// The hardware approximations, named explicitly.
__device__ __forceinline__ float rcp_approx(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ float rsqrt_approx(float x) {
    float r;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ float ex2_approx(float x) {
    float r;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ float sin_approx(float x) {
    float r;
    asm("sin.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ float cos_approx(float x) {
    float r;
    asm("cos.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// sin(t) for |t| <= 3 pi / 4 from its Taylor series through t^13 (relative
// error below 3e-7 there, one ulp near 0); used for the half proposal step,
// where the hardware sine's absolute error would dominate small steps.
__device__ __forceinline__ float2 sin_taylor2(float2 t) {
    const float2 t2 = mul2(t, t);
    float2 p = f2(-1.0f / 6227020800.0f);          // -1/13!
    p = fma2(p, t2, f2(1.0f / 39916800.0f));       //  1/11!
    p = fma2(p, t2, f2(-1.0f / 362880.0f));        // -1/9!
    p = fma2(p, t2, f2(1.0f / 5040.0f));           //  1/7!
    p = fma2(p, t2, f2(-1.0f / 120.0f));
    p = fma2(p, t2, f2(1.0f / 6.0f));
    // sin t = t (1 - t^2 (1/3! - t^2 (1/5! - ...)))
    return mul2(t, fma2(mul2(t2, f2(-1.0f)), p, f2(1.0f)));
}

// atan2(y, x) of both components (finite for x = y = 0): octant reduction to
// t = min/max in [0, 1] and an odd degree-15 polynomial t P(t^2) for atan(t):
// the minimax fit of the absolute error on [0, 1] (Remez exchange; levelled
// error 3.8e-8), its coefficients rounded to FP32 (6.2e-8 in exact
// arithmetic, 1.3e-7 rad in FP32 Horner arithmetic; tests/test_atan2_fit.py
// repeats the fit and both bounds).
__device__ __forceinline__ float2 atan2_pair(float2 y, float2 x) {
    const float ax0 = fabsf(x.x), ay0 = fabsf(y.x), ax1 = fabsf(x.y), ay1 = fabsf(y.y);
    // the floor keeps t finite (0) for a vanishing field
    const float2 mx = make_float2(fmaxf(fmaxf(ax0, ay0), 1e-30f), fmaxf(fmaxf(ax1, ay1), 1e-30f));
    const float2 mn = make_float2(fminf(ax0, ay0), fminf(ax1, ay1));
    const float2 t = mul2(mn, make_float2(rcp_approx(mx.x), rcp_approx(mx.y)));
    const float2 t2 = mul2(t, t);
    // coefficients of t^15, t^13, ..., t^1
    float2 p = f2(-0.004054575f);
    p = fma2(p, t2, f2(0.021862987f));
    p = fma2(p, t2, f2(-0.05591237f));
    p = fma2(p, t2, f2(0.09642201f));
    p = fma2(p, t2, f2(-0.1390863f));
    p = fma2(p, t2, f2(0.19946566f));
    p = fma2(p, t2, f2(-0.3332986f));
    p = fma2(p, t2, f2(0.99999934f));
    float2 r = mul2(p, t);
    r = sel2(ay0 > ax0, ay1 > ax1, rsub2(r, f2(1.57079632679489662f)), r);
    r = sel2(x.x < 0.0f, x.y < 0.0f, rsub2(r, f2(kPi)), r);
    return make_float2(copysignf(r.x, y.x), copysignf(r.y, y.y));
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

// Per pair: the uniforms of Alg. 1 steps 2 and 6 come from one Philox block,
// words (0, 1) for the even realisation and (2, 3) for the odd one, as
// u = (w >> 8) 2^-24.  The proposal uses (u - 1/2) alpha = (w >> 8 - 2^23)
// (alpha 2^-24) (the same product, the power of two being exact).
// (2 pi / a) 2^-24: the proposal half-range alpha = 2 pi / a of Alg. 1 step 3
// in units of the 24-bit uniform (the power of two is exact)
__host__ __device__ __forceinline__ float proposal_width(float a) {
    return (6.28318530717958647692f / a) * 0x1p-24f;
}

struct PairRand {
    float2 um;  // (w >> 8) - 2^23 of both realisations (exact integers)
    float2 r;   // acceptance uniforms
};
__device__ __forceinline__ PairRand pair_uniforms(uint4 w) {
    PairRand o;
    o.um = add2(make_float2((float)(w.x >> 8), (float)(w.z >> 8)), f2(-8388608.0f));
    o.r = mul2(make_float2((float)(w.y >> 8), (float)(w.w >> 8)), f2(0x1p-24f));
    return o;
}

struct PairOut {
    float2 phi;     // new angles
    float2 e;       // site energies after the update (when requested)
    bool acc0, acc1;
};

// Alg. 1 steps 2-6 for both realisations of a pair whose spins sit at phi1
// (after over-relaxation):
//  2-3. proposal phi'' = (phi1 + alpha (u - 1/2)) mod 2 pi, alpha = 2 pi / a;
//  4. dH = -J R [cos(q phi'' - Psi) - cos(q phi1 - Psi)]
//        = 2 J R sin(x + h) sin(h), x = q phi1 - Psi, h = q (phi'' - phi1) / 2
//     (product form: no cancellation for small steps);
//  5-6. accept iff r < exp(-dH / T) (dH <= 0 gives exp >= 1 > r: always).
// alpha_s = alpha 2^-24; c_acc = log2(e) / T (so that exp(-dH/T) = 2^(-dH c_acc)).
template <bool ENERGY>
__device__ __forceinline__ PairOut metropolis_pair(float2 phi1, float2 mPsi, float2 R,
                                                   const PairRand& u, const UpdateConst& k,
                                                   float2 alpha_s, float c_acc) {
    float2 phi2 = fma2(alpha_s, u.um, phi1);
    // mod 2 pi for phi2 in (-pi, 3 pi): phi2 - 2 pi floor(phi2 / 2 pi) gives the
    // same bits as adding or subtracting 2 pi below 0 or from 2 pi up (checked
    // for every FP32 value of the range; they differ only at -0 and negative
    // denormals, which this update cannot produce)
    phi2 = fma2(f2(-kTwoPi), floor2(mul2(phi2, f2(kInvTwoPi))), phi2);
    const float2 x = fma2(f2(k.q), phi1, mPsi);
    const float2 h = mul2(f2(0.5f * k.q), rsub2(phi1, phi2));
    // x + h lies in (-3 pi/2, 5 pi/2): the hardware sine reduces that range itself
    const float2 xh = add2(x, h);
    const float2 s1 = make_float2(sin_approx(xh.x), sin_approx(xh.y));
    const float2 s2 = sin_taylor2(h);
    const float2 dH = mul2(mul2(mul2(f2(2.0f * k.J), R), s1), s2);
    const float2 arg = mul2(dH, f2(-c_acc));
    PairOut o;
    o.acc0 = u.r.x < ex2_approx(arg.x);
    o.acc1 = u.r.y < ex2_approx(arg.y);
    o.phi = sel2(o.acc0, o.acc1, phi2, phi1);
    if (ENERGY) {
        // site energy -J R cos(x_new), x_new = x + 2h if accepted
        const float2 xn = sel2(o.acc0, o.acc1, fma2(f2(2.0f), h, x), x);
        o.e = mul2(mul2(f2(-k.J), R),
                   make_float2(cos_approx(wrap_pi(xn.x)), cos_approx(wrap_pi(xn.y))));
    }
    return o;
}

// One application of Alg. 1 to the gap site of both realisations of a pair,
// with angles phi and neighbour fields (C, S) = sum_j (cos q phi_j, sin q phi_j):
// over-relaxation (Eq. over-relax, q-consistent): Psi = atan2(S, C),
// theta' = (2 Psi - q phi) mod 2 pi, phi' = theta'/q if theta' < 2 pi q (else
// phi' = phi; a field shorter than 1e-6 vanishes: no reflection and no energy
// change); then the restricted
// Metropolis step.
template <bool ENERGY>
__device__ __forceinline__ PairOut hybrid_pair(float2 phi, float2 C, float2 S, const PairRand& u,
                                               const UpdateConst& k, float2 alpha_s, float c_acc) {
    const float2 R2 = fma2(C, C, mul2(S, S));
    const bool f0 = R2.x > kFieldEps2, f1 = R2.y > kFieldEps2;
    const float2 Psi = atan2_pair(S, C);  // finite for any field; unused when it vanishes
    const float2 R = sel2(f0, f1, mul2(R2, make_float2(rsqrt_approx(fmaxf(R2.x, 1e-30f)),
                                                       rsqrt_approx(fmaxf(R2.y, 1e-30f)))),
                          f2(0.0f));
    float2 t = fma2(f2(2.0f), Psi, mul2(f2(-k.q), phi));
    t = fma2(f2(-kTwoPi), floor2(mul2(t, f2(kInvTwoPi))), t);
    const float2 ref = mul2(t, f2(k.inv_q));
    const float2 phi1 = sel2(f0 && t.x >= 0.0f && t.x < k.two_pi_q,
                             f1 && t.y >= 0.0f && t.y < k.two_pi_q, ref, phi);
    return metropolis_pair<ENERGY>(phi1, mul2(Psi, f2(-1.0f)), R, u, k, alpha_s, c_acc);
}

// Alg. 1 with the over-relaxation formula as printed (Eq. over-relax with the
// q = 1 field (C1, S1) = sum_j (cos phi_j, sin phi_j)): phi' = (2 Phi - phi)
// mod 2 pi, Phi = atan2(S1, C1), always applied; the Metropolis step still
// uses the MPR energy through its field (C, S).
template <bool ENERGY>
__device__ __forceinline__ PairOut literal_pair(float2 phi, float2 C, float2 S, float2 C1,
                                                float2 S1, const PairRand& u, const UpdateConst& k,
                                                float2 alpha_s, float c_acc) {
    const float2 R2 = fma2(C, C, mul2(S, S));
    const bool f0 = R2.x > kFieldEps2, f1 = R2.y > kFieldEps2;
    const float2 Psi = sel2(f0, f1, atan2_pair(S, C), f2(0.0f));
    const float2 R = sel2(f0, f1, mul2(R2, make_float2(rsqrt_approx(R2.x), rsqrt_approx(R2.y))),
                          f2(0.0f));
    const float2 Q2 = fma2(C1, C1, mul2(S1, S1));
    const bool g0 = Q2.x > kFieldEps2, g1 = Q2.y > kFieldEps2;
    float2 t = fma2(f2(2.0f), atan2_pair(S1, C1), mul2(f2(-1.0f), phi));
    t = fma2(f2(-kTwoPi), floor2(mul2(t, f2(kInvTwoPi))), t);
    t = sel2(t.x >= kTwoPi || t.x < 0.0f, t.y >= kTwoPi || t.y < 0.0f, f2(0.0f), t);
    const float2 phi1 = sel2(g0, g1, t, phi);
    return metropolis_pair<ENERGY>(phi1, mul2(Psi, f2(-1.0f)), R, u, k, alpha_s, c_acc);
}

// Alg. 1 with the GMRF pair interaction of Sec. 4.3 (every bond costs
// J (dphi^2 / (2 pi^2) - 1)): the site energy is quadratic with its minimum at
// the mean m of the n existing neighbours, so over-relaxation reflects about
// it, phi' = 2m - phi, kept inside [0, 2 pi); the proposal and acceptance are
// those of the MPR step, with
// dH = J n (phi'' - phi')(phi'' + phi' - 2m) / (2 pi^2) (a product: no cancellation).
// sum = sum of the neighbour angles, n their number (m = sum (1/n)).
template <bool ENERGY>
__device__ __forceinline__ PairOut gmrf_pair(float2 phi, float2 sum, float n, const PairRand& u,
                                             float J, float2 alpha_s, float c_acc) {
    const float2 m = mul2(sum, f2(__frcp_rn(n)));
    const float2 t = fma2(f2(2.0f), m, mul2(f2(-1.0f), phi));
    const float2 phi1 = sel2(t.x >= 0.0f && t.x < kTwoPi, t.y >= 0.0f && t.y < kTwoPi, t, phi);
    float2 phi2 = fma2(alpha_s, u.um, phi1);
    phi2 = fma2(f2(-kTwoPi), floor2(mul2(phi2, f2(kInvTwoPi))), phi2);  // mod 2 pi
    constexpr float kInvTwoPi2 = 0.050660591821168885f;  // 1 / (2 pi^2)
    const float2 d = rsub2(phi1, phi2);
    const float2 s = fma2(f2(-2.0f), m, add2(phi2, phi1));
    const float2 dH = mul2(mul2(f2(J * n * kInvTwoPi2), d), s);
    const float2 arg = mul2(dH, f2(-c_acc));
    PairOut o;
    o.acc0 = u.r.x < ex2_approx(arg.x);
    o.acc1 = u.r.y < ex2_approx(arg.y);
    o.phi = sel2(o.acc0, o.acc1, phi2, phi1);
    if (ENERGY) o.e = f2(0.0f);  // GMRF bond energies are summed by the caller
    return o;
}

__device__ __forceinline__ float gmrf_bond(float d) {
    return fmaf(d * d, 0.050660591821168885f, -1.0f);
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
