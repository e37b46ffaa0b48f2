// Cross-validated choice of the modification factor q.  The paper names the
// selection of q in (0, 1/2] by cross-validation as an extension of the method
// (conclusions) without fixing a procedure; this one follows the validation
// design of Sec. 3: a set-aside portion of the samples is the validation set and
// the absolute error averaged over it (AAE) scores a prediction.  For every
// candidate q the whole gap fill of Alg. 2 runs through the library's own entry
// points (init with the validation points as extra gaps, SEM temperature,
// equilibration, sampling, prediction); two small kernels here build the
// cross-validation mask and reduce the validation error.

#include <cmath>
#include <string>

#include "mpr_internal.h"

namespace {

using mpr::set_last_error;

#define MPR_TRY_Q(call)              \
    do {                             \
        const mpr_status s_ = (call); \
        if (s_ != MPR_OK) return s_; \
    } while (0)

constexpr size_t kQcvAlign = 256;
size_t qcv_align(size_t v) { return (v + kQcvAlign - 1) / kQcvAlign * kQcvAlign; }

struct QcvLayout {
    size_t ctx_bytes;  // the per-candidate context's workspace
    size_t z, gcv, hold, zhat, acc, total;
};

QcvLayout qcv_layout(size_t ctx_bytes, long long N) {
    QcvLayout L;
    L.ctx_bytes = qcv_align(ctx_bytes);
    L.z = L.ctx_bytes;
    L.gcv = L.z + qcv_align(sizeof(float) * N);
    L.hold = L.gcv + qcv_align(N);
    L.zhat = L.hold + qcv_align(N);
    L.acc = L.zhat + qcv_align(sizeof(float) * N);
    L.total = L.acc + qcv_align(2 * sizeof(double));
    return L;
}

// gcv = gap or (held out and not a gap); hold keeps only held-out samples;
// acc[1] counts them.
// gap and gcv may be the same buffer (no __restrict__ on them).
__global__ void qcv_mask_kernel(long long N, const uint8_t* gap, uint8_t* __restrict__ hold,
                                uint8_t* gcv, double* __restrict__ acc) {
    long long n = 0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N;
         i += (long long)gridDim.x * blockDim.x) {
        const bool g = gap[i] != 0;
        const bool h = hold[i] != 0 && !g;
        hold[i] = h ? 1 : 0;
        gcv[i] = (g || h) ? 1 : 0;
        n += h;
    }
    for (int o = 16; o > 0; o >>= 1) n += __shfl_xor_sync(0xffffffffu, n, o);
    if ((threadIdx.x & 31) == 0 && n) atomicAdd(acc + 1, (double)n);
}

// acc[0] += sum over held-out pixels of |z_hat - z| (FP64).
__global__ void qcv_abs_error_kernel(long long N, const float* __restrict__ z,
                                     const float* __restrict__ zhat, const uint8_t* __restrict__ hold,
                                     double* __restrict__ acc) {
    double s = 0.0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N;
         i += (long long)gridDim.x * blockDim.x)
        if (hold[i]) s += fabs((double)zhat[i] - (double)z[i]);
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0 && s != 0.0) atomicAdd(acc, s);
}

int qcv_blocks(long long N) {
    const long long b = (N + 255) / 256;
    return (int)(b < 1 ? 1 : (b > 4 * 152 ? 4 * 152 : b));
}

mpr_status copy_in(void* dst, const void* src, size_t bytes, mpr_mem where, cudaStream_t s) {
    const cudaMemcpyKind k = where == MPR_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
    const cudaError_t e = cudaMemcpyAsync(dst, src, bytes, k, s);
    if (e != cudaSuccess)
        return set_last_error(MPR_ERR_CUDA, std::string("mpr_select_q: copy-in: ") + cudaGetErrorString(e));
    return MPR_OK;
}

}  // namespace

extern "C" {

mpr_status mpr_select_q_workspace_size(int Lx, int Ly, int n_chains, const mpr_params* p,
                                       const mpr_T_opts* T_opts, size_t* bytes) {
    if (!bytes || !p) return set_last_error(MPR_ERR_INVALID_ARG, "mpr_select_q_workspace_size: NULL argument");
    size_t ctx = 0;
    const mpr_status st = mpr_workspace_size(1, &Lx, &Ly, nullptr, n_chains, p, T_opts, &ctx);
    if (st != MPR_OK) return st;
    *bytes = qcv_layout(ctx, (long long)Lx * Ly).total;
    return MPR_OK;
}

mpr_status mpr_select_q(int Lx, int Ly, const float* z, const uint8_t* gap, const uint8_t* holdout,
                        mpr_mem where, int n_q, const double* q, int n_chains, int n_equil,
                        int n_meas, const mpr_params* p, const mpr_T_opts* T_opts, void* workspace,
                        size_t ws_bytes, double* scores, double* T_out, double* q_best,
                        mpr_stream stream) {
    if (!z || !gap || !holdout || !q || !p || !scores || !workspace)
        return set_last_error(MPR_ERR_INVALID_ARG, "mpr_select_q: NULL argument");
    if (where != MPR_HOST && where != MPR_DEVICE)
        return set_last_error(MPR_ERR_INVALID_ARG, "mpr_select_q: bad memory kind");
    if (n_q < 1 || n_chains < 1 || n_equil < 0 || n_meas < 1)
        return set_last_error(MPR_ERR_INVALID_ARG,
                              "mpr_select_q: need n_q >= 1, n_chains >= 1, n_equil >= 0, n_meas >= 1");
    for (int k = 0; k < n_q; ++k)
        if (!(q[k] > 0.0 && q[k] <= 0.5))
            return set_last_error(MPR_ERR_INVALID_ARG, "mpr_select_q: every candidate q must lie in (0, 1/2]");
    if (p->model != MPR_MODEL_MPR || p->literal_or)
        return set_last_error(MPR_ERR_INVALID_ARG, "mpr_select_q: q belongs to the MPR bond (model MPR, literal_or 0)");
    size_t ctx_bytes = 0;
    mpr_status st = mpr_workspace_size(1, &Lx, &Ly, nullptr, n_chains, p, T_opts, &ctx_bytes);
    if (st != MPR_OK) return st;
    const long long N = (long long)Lx * Ly;
    const QcvLayout L = qcv_layout(ctx_bytes, N);
    if (ws_bytes < L.total || reinterpret_cast<uintptr_t>(workspace) % kQcvAlign)
        return set_last_error(MPR_ERR_WORKSPACE, "mpr_select_q: workspace too small or not 256-byte aligned: need " +
                                                     std::to_string(L.total) + " bytes");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    char* ws = static_cast<char*>(workspace);
    float* dz = reinterpret_cast<float*>(ws + L.z);
    uint8_t* dgcv = reinterpret_cast<uint8_t*>(ws + L.gcv);
    uint8_t* dhold = reinterpret_cast<uint8_t*>(ws + L.hold);
    float* dzhat = reinterpret_cast<float*>(ws + L.zhat);
    double* dacc = reinterpret_cast<double*>(ws + L.acc);

    // stage the inputs: z, the image's gaps (into gcv, rewritten below), the holdout flags
    MPR_TRY_Q(copy_in(dz, z, sizeof(float) * N, where, s));
    MPR_TRY_Q(copy_in(dgcv, gap, N, where, s));
    MPR_TRY_Q(copy_in(dhold, holdout, N, where, s));
    if (cudaMemsetAsync(dacc, 0, 2 * sizeof(double), s) != cudaSuccess)
        return set_last_error(MPR_ERR_CUDA, "mpr_select_q: memset");
    // gcv is both the image's gap input and the merged output: each element is read
    // and written by the same thread
    qcv_mask_kernel<<<qcv_blocks(N), 256, 0, s>>>(N, dgcv, dhold, dgcv, dacc);
    if (cudaGetLastError() != cudaSuccess) return set_last_error(MPR_ERR_CUDA, "mpr_select_q: mask kernel");
    double acc[2];
    if (cudaMemcpyAsync(acc, dacc, sizeof(acc), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return set_last_error(MPR_ERR_CUDA, "mpr_select_q: reading the holdout count");
    const double n_hold = acc[1];
    if (!(n_hold > 0.0)) return set_last_error(MPR_ERR_INVALID_ARG, "mpr_select_q: no held-out sample");

    int best = -1;
    for (int k = 0; k < n_q; ++k) {
        mpr_params pk = *p;
        pk.q = q[k];
        mpr_ctx* ctx = nullptr;
        st = mpr_init_grid(&ctx, 1, &Lx, &Ly, n_chains, &pk, T_opts, dz, dgcv, MPR_DEVICE, ws,
                           L.ctx_bytes, stream);
        if (st != MPR_OK) return st;
        double T = NAN;
        st = mpr_estimate_T(ctx, &T, stream);
        if (st == MPR_ERR_T_OUT_OF_RANGE) {
            // no SEM temperature at this q: the candidate is out
            mpr_destroy(ctx);
            scores[k] = INFINITY;
            if (T_out) T_out[k] = NAN;
            continue;
        }
        if (st == MPR_OK) st = mpr_sweep(ctx, n_equil, MPR_EQUIL, 0, stream);
        if (st == MPR_OK) st = mpr_sweep(ctx, n_meas, MPR_MEASURE, 0, stream);
        if (st == MPR_OK) st = mpr_predict(ctx, dzhat, nullptr, MPR_DEVICE, stream);
        if (st == MPR_OK && cudaMemsetAsync(dacc, 0, sizeof(double), s) != cudaSuccess)
            st = set_last_error(MPR_ERR_CUDA, "mpr_select_q: memset");
        if (st == MPR_OK) {
            qcv_abs_error_kernel<<<qcv_blocks(N), 256, 0, s>>>(N, dz, dzhat, dhold, dacc);
            if (cudaGetLastError() != cudaSuccess ||
                cudaMemcpyAsync(acc, dacc, sizeof(double), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
                cudaStreamSynchronize(s) != cudaSuccess)
                st = set_last_error(MPR_ERR_CUDA, "mpr_select_q: validation error");
        }
        mpr_destroy(ctx);
        if (st != MPR_OK) return st;
        scores[k] = acc[0] / n_hold;
        if (T_out) T_out[k] = T;
        if (best < 0 || scores[k] < scores[best]) best = k;
    }
    if (best < 0)
        return set_last_error(MPR_ERR_T_OUT_OF_RANGE, "mpr_select_q: no candidate q has a SEM temperature");
    if (q_best) *q_best = q[best];
    return MPR_OK;
}

}  // extern "C"
