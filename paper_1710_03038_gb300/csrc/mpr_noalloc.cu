// Sample specific energy without any allocation, for callers that cannot
// call cudaMalloc (or any allocator): the per-block partial results live in
// a fixed array in this library's device memory instead of a workspace.
//
// The array is file scope and shared by every call on a device; it holds the
// last call's partials.  Nothing in it has to start at zero (every partial is
// written before it is read), but two calls that overlap on the GPU (in
// different streams, or in a graph) would overwrite each other's partials.
#include <cmath>
#include <cstring>
#include <mutex>
#include <string>

#include "mpr_device.cuh"
#include "mpr_internal.h"

using namespace mpr;

namespace {

constexpr int kNoAllocMaxImages = 64;   // images per call
constexpr int kNoAllocBlocks = 256;     // partials per image and phase
constexpr double kPiD = 3.14159265358979323846;

struct Partial {        // one thread block's share of one image
    uint32_t zlo, zhi;  // order-preserving encodings of the sample extremes
    unsigned long long n_gap;
    double sum;         // -J sum cos(q dphi) over sample-sample bonds
    unsigned long long n_pair;
};

struct ImgStat {
    float zmin, zmax;
    unsigned long long n_gap;
};

// The scratch: two phases of partials plus per-image extremes.
constexpr size_t kScratchBytes =
    sizeof(Partial) * kNoAllocMaxImages * kNoAllocBlocks + sizeof(ImgStat) * kNoAllocMaxImages;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

struct Shapes {
    int n;
    int Lx[kNoAllocMaxImages], Ly[kNoAllocMaxImages];
    long long off[kNoAllocMaxImages];
};

__device__ __forceinline__ uint32_t ordered_f(float f) {
    const uint32_t b = __float_as_uint(f);
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}
__device__ __forceinline__ float unordered_f(uint32_t u) {
    return __uint_as_float((u & 0x80000000u) ? (u & 0x7FFFFFFFu) : ~u);
}

template <typename T, typename F>
__device__ T block_reduce(T v, F op, T* sh, T identity) {
    for (int o = 16; o > 0; o >>= 1) v = op(v, __shfl_xor_sync(0xffffffffu, v, o));
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) sh[w] = v;
    __syncthreads();
    if (w == 0) {
        v = l < (int)(blockDim.x >> 5) ? sh[l] : identity;
        for (int o = 16; o > 0; o >>= 1) v = op(v, __shfl_xor_sync(0xffffffffu, v, o));
    }
    __syncthreads();
    return v;  // valid in thread 0
}

// Phase 1: per-block sample extremes and gap counts.
__global__ void noalloc_extremes_kernel(const __grid_constant__ Shapes S, const float* z,
                                        const uint8_t* gap, Partial* part) {
    __shared__ unsigned long long sh[32];
    const int im = blockIdx.y;
    const long long n = (long long)S.Lx[im] * S.Ly[im];
    const float* zi = z + S.off[im];
    const uint8_t* gi = gap + S.off[im];
    uint32_t lo = 0xFFFFFFFFu, hi = 0u;
    unsigned long long cnt = 0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        if (gi[i]) { ++cnt; continue; }
        const uint32_t o = ordered_f(zi[i]);
        lo = min(lo, o);
        hi = max(hi, o);
    }
    auto mn = [](unsigned long long a, unsigned long long b) { return a < b ? a : b; };
    auto mx = [](unsigned long long a, unsigned long long b) { return a > b ? a : b; };
    auto ad = [](unsigned long long a, unsigned long long b) { return a + b; };
    const unsigned long long rlo = block_reduce<unsigned long long>(lo, mn, sh, 0xFFFFFFFFull);
    const unsigned long long rhi = block_reduce<unsigned long long>(hi, mx, sh, 0ull);
    const unsigned long long rc = block_reduce<unsigned long long>(cnt, ad, sh, 0ull);
    if (threadIdx.x == 0) {
        Partial& p = part[im * kNoAllocBlocks + blockIdx.x];
        p.zlo = (uint32_t)rlo;
        p.zhi = (uint32_t)rhi;
        p.n_gap = rc;
    }
}

// Phase 2: per image, combine the partials in a fixed order.
__global__ void noalloc_extremes_final_kernel(const Partial* part, ImgStat* stat) {
    if (threadIdx.x != 0) return;
    const int im = blockIdx.x;
    uint32_t lo = 0xFFFFFFFFu, hi = 0u;
    unsigned long long cnt = 0;
    for (int b = 0; b < kNoAllocBlocks; ++b) {
        const Partial& p = part[im * kNoAllocBlocks + b];
        lo = min(lo, p.zlo);
        hi = max(hi, p.zhi);
        cnt += p.n_gap;
    }
    stat[im].zmin = lo == 0xFFFFFFFFu ? __int_as_float(0x7FC00000) : unordered_f(lo);
    stat[im].zmax = lo == 0xFFFFFFFFu ? __int_as_float(0x7FC00000) : unordered_f(hi);
    stat[im].n_gap = cnt;
}

// Phase 3: sample-sample bond sums with the angles of Eq. map computed on the
// fly exactly as the context's initialisation computes them (FP64 map,
// rounded to FP32 once; FP32 bond terms -J cos(q (v - w)) summed in FP64).
__global__ void noalloc_pairs_kernel(const __grid_constant__ Shapes S, const float* z,
                                     const uint8_t* gap, const ImgStat* stat, double q, double J,
                                     Partial* part) {
    __shared__ double shd[32];
    __shared__ unsigned long long shu[32];
    const int im = blockIdx.y;
    const int Lx = S.Lx[im], Ly = S.Ly[im];
    const long long n = (long long)Lx * Ly;
    const float* zi = z + S.off[im];
    const uint8_t* gi = gap + S.off[im];
    const double zmin = stat[im].zmin;
    const double scale = 2.0 * kPiD / ((double)stat[im].zmax - zmin);
    const bool ok = stat[im].zmax > stat[im].zmin;
    double s = 0.0;
    unsigned long long cnt = 0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; ok && i < n;
         i += (long long)gridDim.x * blockDim.x) {
        if (gi[i]) continue;
        const int x = (int)(i % Lx), y = (int)(i / Lx);
        const float v = (float)(((double)zi[i] - zmin) * scale);
        if (x + 1 < Lx && !gi[i + 1]) {
            const float w = (float)(((double)zi[i + 1] - zmin) * scale);
            s -= (double)((float)J * cosf((float)q * (v - w)));
            ++cnt;
        }
        if (y + 1 < Ly && !gi[i + Lx]) {
            const float w = (float)(((double)zi[i + Lx] - zmin) * scale);
            s -= (double)((float)J * cosf((float)q * (v - w)));
            ++cnt;
        }
    }
    auto add_d = [](double a, double b) { return a + b; };
    auto add_u = [](unsigned long long a, unsigned long long b) { return a + b; };
    const double rs = block_reduce<double>(s, add_d, shd, 0.0);
    const unsigned long long rc = block_reduce<unsigned long long>(cnt, add_u, shu, 0ull);
    if (threadIdx.x == 0) {
        Partial& p = part[im * kNoAllocBlocks + blockIdx.x];
        p.sum = rs;
        p.n_pair = rc;
    }
}

__global__ void noalloc_final_kernel(const Partial* part, const ImgStat* stat, double* e_s,
                                     long long* n_sp, float* zmin, float* zmax) {
    if (threadIdx.x != 0) return;
    const int im = blockIdx.x;
    double s = 0.0;
    unsigned long long c = 0;
    for (int b = 0; b < kNoAllocBlocks; ++b) {
        s += part[im * kNoAllocBlocks + b].sum;
        c += part[im * kNoAllocBlocks + b].n_pair;
    }
    const bool ok = stat[im].zmax > stat[im].zmin;
    e_s[im] = (ok && c > 0) ? s / (double)c : __longlong_as_double(0x7FF8000000000000LL);
    if (n_sp) n_sp[im] = ok ? (long long)c : 0;
    if (zmin) zmin[im] = stat[im].zmin;
    if (zmax) zmax[im] = stat[im].zmax;
}

// Per-device address of the scratch array, looked up once per device.
std::mutex g_mu;
void* g_scratch_ptr[64] = {nullptr};

}  // namespace

extern "C" mpr_status mpr_sample_energy_noalloc(int n_img, const int* Lx, const int* Ly,
                                                const float* z, const uint8_t* gap, double q,
                                                double J, double* e_s, int64_t* n_sp,
                                                float* z_min, float* z_max, mpr_stream stream) {
    static_assert(kNoAllocMaxImages == MPR_NOALLOC_MAX_IMAGES, "header and scratch disagree");
    if (n_img < 1 || n_img > kNoAllocMaxImages)
        return set_last_error(MPR_ERR_INVALID_ARG,
                              "mpr_sample_energy_noalloc: n_img = " + std::to_string(n_img) +
                                  " is outside [1, " + std::to_string(kNoAllocMaxImages) +
                                  "], the capacity of its fixed scratch array");
    if (!Lx || !Ly || !z || !gap || !e_s)
        return set_last_error(MPR_ERR_INVALID_ARG, "mpr_sample_energy_noalloc: NULL argument");
    if (!(q > 0.0) || !(J > 0.0))
        return set_last_error(MPR_ERR_INVALID_ARG, "mpr_sample_energy_noalloc: q and J must be positive");
    Shapes S;
    std::memset(&S, 0, sizeof(S));
    S.n = n_img;
    long long off = 0;
    for (int i = 0; i < n_img; ++i) {
        if (Lx[i] < 2 || Ly[i] < 2 || Lx[i] > 65535 || Ly[i] > 65535)
            return set_last_error(MPR_ERR_INVALID_ARG,
                                  "mpr_sample_energy_noalloc: image sides must lie in [2, 65535]");
        S.Lx[i] = Lx[i];
        S.Ly[i] = Ly[i];
        S.off[i] = off;
        off += (long long)Lx[i] * Ly[i];
    }
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64)
        return set_last_error(MPR_ERR_CUDA, "mpr_sample_energy_noalloc: no current device");
    void* base = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        if (!g_scratch_ptr[dev]) {
            void* p = nullptr;
            const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
            if (e != cudaSuccess || !p)
                return set_last_error(MPR_ERR_CUDA, std::string("mpr_sample_energy_noalloc: "
                                                                "cudaGetSymbolAddress: ") +
                                                        cudaGetErrorString(e));
            g_scratch_ptr[dev] = p;
        }
        base = g_scratch_ptr[dev];
    }
    Partial* part = static_cast<Partial*>(base);
    ImgStat* stat = reinterpret_cast<ImgStat*>(part + kNoAllocMaxImages * kNoAllocBlocks);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    dim3 grid(kNoAllocBlocks, n_img);
    noalloc_extremes_kernel<<<grid, 256, 0, s>>>(S, z, gap, part);
    noalloc_extremes_final_kernel<<<n_img, 32, 0, s>>>(part, stat);
    noalloc_pairs_kernel<<<grid, 256, 0, s>>>(S, z, gap, stat, q, J, part);
    noalloc_final_kernel<<<n_img, 32, 0, s>>>(part, stat, e_s, reinterpret_cast<long long*>(n_sp),
                                              z_min, z_max);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess)
        return set_last_error(MPR_ERR_CUDA, std::string("mpr_sample_energy_noalloc: ") +
                                                cudaGetErrorString(e));
    return MPR_OK;
}
