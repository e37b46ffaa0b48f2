// Context-free kernels: lattice energy and its gradient for dense angle
// grids (the forward and backward of the energy as a differentiable
// function), and direct access to the random stream's Philox blocks.
#include <curand_philox4x32_x.h>

#include <algorithm>
#include <vector>

#include "mpr_device.cuh"
#include "mpr_internal.h"

using namespace mpr;

namespace {

struct GridTable {
    int Lx, Ly;
    long long off;
};

// Shapes travel in the kernel parameters (no device allocation): up to
// kMaxGrids grids per launch, more are launched in chunks.
constexpr int kMaxGrids = 256;
struct Grids {
    GridTable g[kMaxGrids];
};

// H_k = -J sum_<ij> cos(q (phi_i - phi_j)) over the right and down bonds of
// grid k; FP32 bond terms, FP64 sums.
__global__ void lattice_energy_kernel(const __grid_constant__ Grids G, int k0, const float* phi,
                                      float q, float J, double* H) {
    const GridTable g = G.g[blockIdx.y];
    const long long n = (long long)g.Lx * g.Ly;
    const float* p = phi + g.off;
    double s = 0.0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(i % g.Lx), y = (int)(i / g.Lx);
        const float v = p[i];
        float e = 0.0f;
        if (x + 1 < g.Lx) e -= J * cosf(q * (v - p[i + 1]));
        if (y + 1 < g.Ly) e -= J * cosf(q * (v - p[i + g.Lx]));
        s += (double)e;
    }
    s = warp_sum(s);
    if ((threadIdx.x & 31) == 0 && s != 0.0) atomicAdd(H + k0 + blockIdx.y, s);
}

// grad_i = g_k J q sum_j sin(q (phi_i - phi_j)): the torque on spin i (the
// same local field the sweep uses) as dH/dphi_i, weighted by dL/dH_k.
__global__ void lattice_torque_kernel(const __grid_constant__ Grids G, int k0, const float* phi,
                                      float q, float J, const double* up, float* grad) {
    const GridTable g = G.g[blockIdx.y];
    const long long n = (long long)g.Lx * g.Ly;
    const float* p = phi + g.off;
    const float w = (float)up[k0 + blockIdx.y] * J * q;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(i % g.Lx), y = (int)(i / g.Lx);
        const float v = p[i];
        float s = 0.0f;
        if (y > 0) s += sinf(q * (v - p[i - g.Lx]));
        if (y + 1 < g.Ly) s += sinf(q * (v - p[i + g.Lx]));
        if (x > 0) s += sinf(q * (v - p[i - 1]));
        if (x + 1 < g.Lx) s += sinf(q * (v - p[i + 1]));
        grad[g.off + i] = w * s;
    }
}

// Both gradients of L = sum_k g_k H_k: the torque of every site (when grad is
// non-null) and dL/dJ = -sum_k g_k sum over the right and down bonds of
// cos(q dphi) (when gJ is non-null; FP32 bond terms, FP64 sums).
__global__ void lattice_grad_kernel(const __grid_constant__ Grids G, int k0, const float* phi,
                                    float q, float J, const double* up, float* grad,
                                    double* gJ) {
    const GridTable g = G.g[blockIdx.y];
    const long long n = (long long)g.Lx * g.Ly;
    const float* p = phi + g.off;
    const double uk = up[k0 + blockIdx.y];
    const float w = (float)uk * J * q;
    double sJ = 0.0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(i % g.Lx), y = (int)(i / g.Lx);
        const float v = p[i];
        if (grad) {
            float s = 0.0f;
            if (y > 0) s += sinf(q * (v - p[i - g.Lx]));
            if (y + 1 < g.Ly) s += sinf(q * (v - p[i + g.Lx]));
            if (x > 0) s += sinf(q * (v - p[i - 1]));
            if (x + 1 < g.Lx) s += sinf(q * (v - p[i + 1]));
            grad[g.off + i] = w * s;
        }
        if (gJ) {
            float e = 0.0f;
            if (x + 1 < g.Lx) e -= cosf(q * (v - p[i + 1]));
            if (y + 1 < g.Ly) e -= cosf(q * (v - p[i + g.Lx]));
            sJ += (double)e;
        }
    }
    if (gJ) {
        sJ = warp_sum(sJ) * uk;
        if ((threadIdx.x & 31) == 0 && sJ != 0.0) atomicAdd(gJ, sJ);
    }
}

__global__ void philox_kernel(int n, const uint32_t* ctr, uint2 key, uint32_t* out, int reference) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint4 c = make_uint4(ctr[4 * i], ctr[4 * i + 1], ctr[4 * i + 2], ctr[4 * i + 3]);
    const uint4 w = reference ? curand_Philox4x32_10(c, key) : philox4x32_10(c, key);
    out[4 * i] = w.x;
    out[4 * i + 1] = w.y;
    out[4 * i + 2] = w.z;
    out[4 * i + 3] = w.w;
}

__global__ void math_probe_kernel(int fn, int n, const float* a, const float* b, float* out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float v = 0.0f;
    switch (fn) {
        case 0: v = atan2_pair(f2(a[i]), f2(b[i])).x; break;
        case 1: v = atan2f(a[i], b[i]); break;
        case 2: v = sin_taylor2(f2(a[i])).x; break;
        default: v = sinf(a[i]); break;
    }
    out[i] = v;
}

template <typename F>
mpr_status for_chunks(int n, const int* Lx, const int* Ly, F launch) {
    if (n < 1 || !Lx || !Ly) return MPR_ERR_INVALID_ARG;
    long long off = 0;
    for (int k0 = 0; k0 < n; k0 += kMaxGrids) {
        Grids G;
        const int m = std::min(kMaxGrids, n - k0);
        long long mx = 1;
        for (int j = 0; j < m; ++j) {
            const int i = k0 + j;
            if (Lx[i] < 1 || Ly[i] < 1) return MPR_ERR_INVALID_ARG;
            G.g[j] = GridTable{Lx[i], Ly[i], off};
            off += (long long)Lx[i] * Ly[i];
            mx = std::max(mx, (long long)Lx[i] * Ly[i]);
        }
        const int blocks = (int)std::min<long long>((mx + 255) / 256, 1024);
        if (launch(G, k0, m, blocks) != cudaSuccess) return MPR_ERR_CUDA;
    }
    return MPR_OK;
}

}  // namespace

extern "C" {

mpr_status mpr_lattice_energy(int n, const int* Lx, const int* Ly, const float* phi, double q,
                              double J, double* H_out, mpr_stream stream) {
    if (!phi || !H_out) return MPR_ERR_INVALID_ARG;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if (cudaMemsetAsync(H_out, 0, sizeof(double) * (n > 0 ? n : 0), s) != cudaSuccess)
        return MPR_ERR_CUDA;
    return for_chunks(n, Lx, Ly, [&](const Grids& G, int k0, int m, int blocks) {
        lattice_energy_kernel<<<dim3(blocks, m), 256, 0, s>>>(G, k0, phi, (float)q, (float)J, H_out);
        return cudaGetLastError();
    });
}

mpr_status mpr_lattice_torque(int n, const int* Lx, const int* Ly, const float* phi, double q,
                              double J, const double* g, float* grad, mpr_stream stream) {
    if (!phi || !g || !grad) return MPR_ERR_INVALID_ARG;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    return for_chunks(n, Lx, Ly, [&](const Grids& G, int k0, int m, int blocks) {
        lattice_torque_kernel<<<dim3(blocks, m), 256, 0, s>>>(G, k0, phi, (float)q, (float)J, g, grad);
        return cudaGetLastError();
    });
}

mpr_status mpr_lattice_grad(int n, const int* Lx, const int* Ly, const float* phi, double q,
                            double J, const double* g, float* grad_phi, double* grad_J,
                            mpr_stream stream) {
    if (!phi || !g || (!grad_phi && !grad_J)) return MPR_ERR_INVALID_ARG;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if (grad_J && cudaMemsetAsync(grad_J, 0, sizeof(double), s) != cudaSuccess) return MPR_ERR_CUDA;
    return for_chunks(n, Lx, Ly, [&](const Grids& G, int k0, int m, int blocks) {
        lattice_grad_kernel<<<dim3(blocks, m), 256, 0, s>>>(G, k0, phi, (float)q, (float)J, g,
                                                            grad_phi, grad_J);
        return cudaGetLastError();
    });
}

mpr_status mpr_philox(int n, const uint32_t* ctr, const uint32_t* key, uint32_t* out, int reference,
                      mpr_stream stream) {
    if (n < 0 || !ctr || !key || !out) return MPR_ERR_INVALID_ARG;
    if (n == 0) return MPR_OK;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    philox_kernel<<<(n + 255) / 256, 256, 0, s>>>(n, ctr, make_uint2(key[0], key[1]), out, reference);
    return cudaGetLastError() == cudaSuccess ? MPR_OK : MPR_ERR_CUDA;
}

mpr_status mpr_math_probe(int fn, int n, const float* a, const float* b, float* out,
                          mpr_stream stream) {
    if (fn < 0 || fn > 3 || n < 0 || !a || !out || (fn < 2 && !b)) return MPR_ERR_INVALID_ARG;
    if (n == 0) return MPR_OK;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    math_probe_kernel<<<(n + 255) / 256, 256, 0, s>>>(fn, n, a, b, out);
    return cudaGetLastError() == cudaSuccess ? MPR_OK : MPR_ERR_CUDA;
}

}  // extern "C"
