// C ABI of the MPR library: context, workspace layout, initialisation,
// sweeps, temperature estimate, prediction and state access.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "mpr_device.cuh"
#include "mpr_internal.h"

using namespace mpr;

// ============================================================== errors

namespace {

thread_local std::string g_last_error;

mpr_status fail(mpr_status s, const std::string& msg) {
    g_last_error = msg;
    return s;
}

#define MPR_CUDA(call)                                                                   \
    do {                                                                                 \
        cudaError_t e_ = (call);                                                         \
        if (e_ != cudaSuccess)                                                           \
            return fail(MPR_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

#define MPR_TRY(call)                      \
    do {                                   \
        mpr_status s_ = (call);            \
        if (s_ != MPR_OK) return s_;       \
    } while (0)

constexpr size_t kAlign = 256;
constexpr int kHist = 512;  // chain-mean energies kept per image for the equilibration test
size_t align_up(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }
constexpr double kPiD = 3.14159265358979323846;

// ============================================================ layout

// Byte offsets of the workspace regions of one context.
struct Layout {
    size_t img, ctl, ch_a, ch_alpha, ch_cnt, ch_last, ch_ecur, ch_elast, ch_esum, ch_esum2;
    size_t zst, gst, outst, eout, samp, slot_map, tiles, counts, halo, tile_list, scratch;
    size_t slot_pos, slot_ref, slot_cs, acc1, acc2, state, newton, hist, sub;
    size_t total;
    long long n_slots;   // slot space over all images
    long long n_state;   // floats of the state buffer
};

struct Geometry {
    int n_img = 0, n_chains = 0, path = 0, tx = 64, ty = 64, halo_cap = 128;
    std::vector<int> Lx, Ly;
    std::vector<long long> site_off;
    std::vector<int> tile0, ntiles;
    long long n_sites = 0;
    int n_tiles = 0;
    int max_Lx = 0, max_Ly = 0;
};

// Floats per slot of the state buffer: the tiled layout interleaves the
// chains, rounded up to a multiple of 4 so that every chain group's part of a
// slot is a 16-byte aligned row (bulk copies) and chain pairs are float2.
long long state_chains(const Geometry& g) {
    return g.path == MPR_PATH_TILED ? (long long)((g.n_chains + 3) & ~3) : (long long)g.n_chains;
}

void make_geometry(Geometry& g, int n_img, const int* Lx, const int* Ly, int n_chains, int path,
                   int tx, int ty) {
    g.n_img = n_img;
    g.n_chains = n_chains;
    g.path = path;
    g.tx = tx;
    g.ty = ty;
    g.halo_cap = tx + ty;
    g.Lx.assign(Lx, Lx + n_img);
    g.Ly.assign(Ly, Ly + n_img);
    g.site_off.resize(n_img);
    g.tile0.resize(n_img);
    g.ntiles.resize(n_img);
    g.n_sites = 0;
    g.n_tiles = 0;
    g.max_Lx = g.max_Ly = 0;
    for (int i = 0; i < n_img; ++i) {
        g.site_off[i] = g.n_sites;
        g.n_sites += (long long)Lx[i] * Ly[i];
        const int nt = ((Lx[i] + tx - 1) / tx) * ((Ly[i] + ty - 1) / ty);
        g.tile0[i] = g.n_tiles;
        g.ntiles[i] = path == MPR_PATH_TILED ? nt : 0;
        if (path == MPR_PATH_TILED) g.n_tiles += nt;
        g.max_Lx = std::max(g.max_Lx, Lx[i]);
        g.max_Ly = std::max(g.max_Ly, Ly[i]);
    }
}

// Per image slot counts: tiled path = padded gap segments, plain = sites.
Layout make_layout(const Geometry& g, const std::vector<long long>& slots_per_img,
                   size_t sub_bytes, bool staging) {
    Layout L{};
    size_t o = 0;
    auto take = [&](size_t bytes) { size_t r = o; o = align_up(o + bytes); return r; };
    const size_t NC = (size_t)g.n_img * g.n_chains;
    const size_t N = (size_t)g.n_sites;
    L.img = take(sizeof(ImgDev) * g.n_img);
    L.ctl = take(sizeof(Control));
    L.ch_a = take(sizeof(float) * NC);
    L.ch_alpha = take(sizeof(float) * NC);
    L.ch_cnt = take(sizeof(uint32_t) * NC * kSpread);
    L.ch_last = take(sizeof(uint32_t) * NC);
    L.ch_ecur = take(sizeof(double) * NC * kSpread);
    L.ch_elast = take(sizeof(double) * NC);
    L.ch_esum = take(sizeof(double) * NC);
    L.ch_esum2 = take(sizeof(double) * NC);
    L.zst = take(staging ? sizeof(float) * N : 0);
    L.gst = take(sizeof(uint8_t) * N);
    L.outst = take(staging ? 2 * sizeof(float) * N : 0);
    L.eout = take(sizeof(double) * NC);
    L.samp = take(sizeof(float) * N);
    const bool tiled = g.path == MPR_PATH_TILED;
    L.slot_map = take(tiled ? sizeof(int) * N : 0);
    L.tiles = take(sizeof(TileDesc) * g.n_tiles);
    L.counts = take(sizeof(int) * 2 * g.n_tiles);
    L.halo = take(sizeof(int2) * (size_t)g.n_tiles * 2 * g.halo_cap);
    L.tile_list = take(sizeof(int) * 2 * (size_t)g.n_tiles);
    L.scratch = take(sizeof(double) * 4 * g.n_img);
    L.n_slots = 0;
    L.n_state = 0;
    for (int i = 0; i < g.n_img; ++i) {
        L.n_slots += slots_per_img[i];
        L.n_state += slots_per_img[i] * state_chains(g);
    }
    L.slot_pos = take(tiled ? sizeof(uint32_t) * L.n_slots : 0);
    L.slot_ref = take(tiled ? sizeof(uint2) * L.n_slots : 0);
    L.slot_cs = take(tiled ? sizeof(float4) * L.n_slots : 0);
    L.acc1 = take(sizeof(double) * L.n_slots);
    L.acc2 = take(sizeof(double) * L.n_slots);
    L.state = take(sizeof(float) * L.n_state);
    L.newton = take(sizeof(double) * 4 * g.n_img);
    L.hist = take(sizeof(double) * kHist * g.n_img + sizeof(int) * (g.n_img + 3));
    L.sub = take(sub_bytes);
    L.total = o;
    return L;
}

long long slot_bound(const Geometry& g, int i, long long n_gap) {
    if (g.path != MPR_PATH_TILED) return (long long)g.Lx[i] * g.Ly[i];
    return n_gap + 8LL * g.ntiles[i];
}

int default_T_side(int Lx, int Ly, const mpr_T_opts& o) {
    if (o.L > 0) return o.L;
    return std::min(256, std::max(Lx, Ly));
}

}  // namespace

mpr_status mpr::set_last_error(mpr_status s, const std::string& msg) { return fail(s, msg); }

// ============================================================== context

struct mpr_ctx {
    mpr_params p{};
    mpr_T_opts topt{};
    Geometry g;
    Layout L{};
    unsigned char* ws = nullptr;
    bool unconditional = false;   // the temperature lattices (no samples)
    uint32_t img_tag = 0;
    // device views
    ImgDev* d_img = nullptr;
    Control* d_ctl = nullptr;
    ChainDev ch{};
    float* d_samp = nullptr;
    int* d_slot_map = nullptr;
    TileDesc* d_tiles = nullptr;
    int2* d_halo = nullptr;
    int* d_tile_list = nullptr;  // per colour: the tiles of the light launch, then the heavy ones
    uint32_t* d_slot_pos = nullptr;
    uint2* d_slot_ref = nullptr;
    float4* d_slot_cs = nullptr;
    double* d_acc1 = nullptr;
    double* d_acc2 = nullptr;
    float* d_state = nullptr;
    float* d_zst = nullptr;
    uint8_t* d_gst = nullptr;
    float* d_out = nullptr;
    double* d_eout = nullptr;
    double* d_newton = nullptr;
    double* d_hist = nullptr;     // [n_img][kHist] chain-mean specific energy per sweep (ring)
    int* d_sg = nullptr;          // [n_img] image settled; then images still settling after the
                                  // last check, sweeps done, 1 once every image settled
    // host mirrors
    std::vector<ImgDev> h_img;
    std::vector<long long> slots;
    int gt[2] = {1, 1};           // tiled: table entries for the pass of colour c (largest tile)
    // tiled: tiles whose table fits the shared memory of a full SM of blocks run
    // in one launch (gt_light entries), the rest in a second one (gt entries)
    int gt_light[2] = {1, 1};
    int n_light[2] = {0, 0};
    uint32_t sweep = 0, equil_index = 0;
    long long n_meas_done = 0;
    bool T_set = false;
    mpr_ctx* sub = nullptr;   // unconditional lattices of the temperature estimate
    // instantiated CUDA graphs of sweep sequences, keyed by (n, phase, flags, stats, accumulate)
    std::vector<std::pair<long long, cudaGraphExec_t>> graphs;
    // the equilibration with its stop rule as one device-side while loop, keyed by
    // (n_f, n_fit, i_max)
    cudaGraphExec_t eq_exec = nullptr;
    long long eq_key = -1;
    // tiled path: a second stream and two events, so that a colour pass's launch
    // for its heavy tiles and the one for the chains left over by the chain
    // groups run beside the main launch (they touch other tiles or chains)
    cudaStream_t side = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    ~mpr_ctx() {
        for (auto& g : graphs) cudaGraphExecDestroy(g.second);
        if (eq_exec) cudaGraphExecDestroy(eq_exec);
        if (ev_fork) cudaEventDestroy(ev_fork);
        if (ev_join) cudaEventDestroy(ev_join);
        if (side) cudaStreamDestroy(side);
        delete sub;
    }
};

namespace {

template <typename T>
T* at(unsigned char* base, size_t off) { return reinterpret_cast<T*>(base + off); }

void bind_views(mpr_ctx* c) {
    unsigned char* w = c->ws;
    const Layout& L = c->L;
    c->d_img = at<ImgDev>(w, L.img);
    c->d_ctl = at<Control>(w, L.ctl);
    c->ch.a = at<float>(w, L.ch_a);
    c->ch.alpha = at<float>(w, L.ch_alpha);
    c->ch.acc_cnt = at<uint32_t>(w, L.ch_cnt);
    c->ch.acc_last = at<uint32_t>(w, L.ch_last);
    c->ch.e_cur = at<double>(w, L.ch_ecur);
    c->ch.e_last = at<double>(w, L.ch_elast);
    c->ch.e_sum = at<double>(w, L.ch_esum);
    c->ch.e_sum2 = at<double>(w, L.ch_esum2);
    c->d_zst = at<float>(w, L.zst);
    c->d_gst = at<uint8_t>(w, L.gst);
    c->d_out = at<float>(w, L.outst);
    c->d_eout = at<double>(w, L.eout);
    c->d_samp = at<float>(w, L.samp);
    c->d_slot_map = at<int>(w, L.slot_map);
    c->d_tiles = at<TileDesc>(w, L.tiles);
    c->d_halo = at<int2>(w, L.halo);
    c->d_tile_list = at<int>(w, L.tile_list);
    c->d_slot_pos = at<uint32_t>(w, L.slot_pos);
    c->d_slot_ref = at<uint2>(w, L.slot_ref);
    c->d_slot_cs = at<float4>(w, L.slot_cs);
    c->d_acc1 = at<double>(w, L.acc1);
    c->d_acc2 = at<double>(w, L.acc2);
    c->d_state = at<float>(w, L.state);
    c->d_newton = at<double>(w, L.newton);
    c->d_hist = at<double>(w, L.hist);
    c->d_sg = reinterpret_cast<int*>(c->d_hist + (size_t)kHist * c->g.n_img);
}

// ======================================================= init kernels

__device__ __forceinline__ uint32_t ordered(float f) {
    const uint32_t b = __float_as_uint(f);
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}

// Extremes over sample sites and gap counts, per image (blockIdx.y).
__global__ void minmax_kernel(const ImgDev* img, const float* z, const uint8_t* gap,
                              uint32_t* mm, unsigned long long* ngap) {
    const ImgDev& I = img[blockIdx.y];
    const long long n = (long long)I.Lx * I.Ly;
    uint32_t lo = 0xFFFFFFFFu, hi = 0u;
    unsigned long long cnt = 0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        if (gap[I.site_off + i]) { ++cnt; continue; }
        const uint32_t o = ordered(z[I.site_off + i]);
        lo = min(lo, o);
        hi = max(hi, o);
    }
    lo = __reduce_min_sync(0xffffffffu, lo);
    hi = __reduce_max_sync(0xffffffffu, hi);
    for (int off = 16; off > 0; off >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, off);
    if ((threadIdx.x & 31) == 0) {
        atomicMin(mm + 2 * blockIdx.y, lo);
        atomicMax(mm + 2 * blockIdx.y + 1, hi);
        if (cnt) atomicAdd(ngap + blockIdx.y, cnt);
    }
}

// Eq. map into the per-image sample plane (FP64 arithmetic, rounded once);
// gap sites hold -1.
__global__ void map_kernel(const ImgDev* img, const float* z, const uint8_t* gap, float* samp,
                           int unconditional) {
    const ImgDev& I = img[blockIdx.y];
    const long long n = (long long)I.Lx * I.Ly;
    const double zmin = I.zmin, scale = 2.0 * kPiD / ((double)I.zmax - (double)I.zmin);
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const long long s = I.site_off + i;
        samp[s] = (unconditional || gap[s]) ? -1.0f : (float)(((double)z[s] - zmin) * scale);
    }
}

// Sample specific energy (Eq. mpr-sse) sums: -J sum cos(q dphi) over sample
// pairs (right and down bonds), FP64.
// One bond's energy in FP32 (summed in FP64 by the caller); the same
// expression as the allocation-free entry point's.
__device__ __forceinline__ float bond_energy(float d, float q, float J, int gmrf) {
    return gmrf ? J * (d * d * (float)(0.5 / (kPiD * kPiD)) - 1.0f) : -J * cosf(q * d);
}

__global__ void sample_energy_kernel(const ImgDev* img, const float* samp, double q, double J,
                                     int gmrf, double* sums, unsigned long long* npairs) {
    const ImgDev& I = img[blockIdx.y];
    const long long n = (long long)I.Lx * I.Ly;
    double s = 0.0;
    unsigned long long cnt = 0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const float v = samp[I.site_off + i];
        if (v < 0.0f) continue;
        const int x = (int)(i % I.Lx), y = (int)(i / I.Lx);
        if (x + 1 < I.Lx) {
            const float w = samp[I.site_off + i + 1];
            if (w >= 0.0f) { s += (double)bond_energy(v - w, (float)q, (float)J, gmrf); ++cnt; }
        }
        if (y + 1 < I.Ly) {
            const float w = samp[I.site_off + i + I.Lx];
            if (w >= 0.0f) { s += (double)bond_energy(v - w, (float)q, (float)J, gmrf); ++cnt; }
        }
    }
    s = warp_sum(s);
    for (int off = 16; off > 0; off >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, off);
    if ((threadIdx.x & 31) == 0) {
        if (s != 0.0) atomicAdd(sums + blockIdx.y, s);
        if (cnt) atomicAdd(npairs + blockIdx.y, cnt);
    }
}

// Start of the tiled state: hot (slot -> 2 pi u with the site's first uniform
// at sweep 0xFFFFFFFF) or cold (every gap angle pi); padding slots and the
// padding chain of an odd chain count hold 0.  One thread per (slot, chain
// pair): the pair shares its Philox block (words 0 and 2) and one float2 store.
__global__ void hot_start_tiled_kernel(const ImgDev* img, const uint32_t* slot_pos, float* state,
                                       long long slots_img, int img_i, int n_chains, uint2 key,
                                       uint32_t img_tag, int cold) {
    const ImgDev& I = img[img_i];
    const long long np = I.sstride / 2;  // chain pairs per slot
    const long long total = slots_img * np;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        const long long k = t / np;
        const int c0 = 2 * (int)(t - k * np);
        const uint32_t p = slot_pos[I.slot_off + k];
        float2 v = make_float2(0.0f, 0.0f);
        if (p != 0xFFFFFFFFu) {
            if (cold) {
                v = make_float2(kPi, c0 + 1 < n_chains ? kPi : 0.0f);
            } else {
                const int X = (int)(p & 0xFFFFu), Y = (int)(p >> 16);
                const uint4 w = philox4x32_10(site_counter(X, Y, (X + Y) & 1, 0xFFFFFFFFu,
                                                           (uint32_t)c0, (uint32_t)img_i | img_tag),
                                              key);
                v = make_float2(kTwoPi * u24(w.x), c0 + 1 < n_chains ? kTwoPi * u24(w.z) : 0.0f);
            }
        }
        *reinterpret_cast<float2*>(state + state_index(I, c0, k)) = v;
    }
}

// Dense planes of the plain path: fixed angle with the sign bit at samples,
// hot start at gaps.
__global__ void init_plain_kernel(const ImgDev* img, const float* samp, float* state,
                                  int img_i, int n_chains, uint2 key, uint32_t img_tag) {
    const ImgDev& I = img[img_i];
    const long long n = (long long)I.Lx * I.Ly;
    const long long total = n * n_chains;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        const int chain = (int)(t / n);
        const long long i = t - (long long)chain * n;
        const float v = samp[I.site_off + i];
        float out;
        if (v >= 0.0f) {
            out = as_fixed(v);
        } else {
            const int X = (int)(i % I.Lx), Y = (int)(i / I.Lx);
            uint32_t wu, wr;
            site_uniform_words(X, Y, (X + Y) & 1, 0xFFFFFFFFu, (uint32_t)chain,
                               (uint32_t)img_i | img_tag, key, wu, wr);
            out = kTwoPi * u24(wu);
        }
        state[state_index(I, chain, i)] = out;
    }
}

__global__ void init_chains_kernel(ChainDev ch, int nc) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nc * kSpread;
         i += gridDim.x * blockDim.x) {
        ch.acc_cnt[i] = 0;
        ch.e_cur[i] = 0.0;
    }
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nc; i += gridDim.x * blockDim.x) {
        ch.a[i] = 1.0f;
        ch.alpha[i] = proposal_width(1.0f);
        ch.acc_last[i] = 0;
        ch.e_last[i] = __longlong_as_double(0x7FF8000000000000LL);
        ch.e_sum[i] = 0.0;
        ch.e_sum2[i] = 0.0;
    }
}

// ======================================================= sweep kernels

__global__ void set_alpha_kernel(ChainDev ch, int nc) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < nc) ch.alpha[i] = proposal_width(ch.a[i]);
}

// Bookkeeping after every sweep: acceptance -> a (Alg. 2 step 4.2), energy
// record (step 4.3), counters.  One warp per chain sums the chain's kSpread
// partial slots; the warps of all blocks share the chains.
__global__ void end_sweep_kernel(const ImgDev* img, ChainDev ch, Control* ctl, int n_img,
                                 int n_chains, int equil, int record, int stats, int add_ess,
                                 double A_targ, double k_a) {
    static_assert(kSpread == 32, "one lane per spread slot");
    const uint32_t i = ctl->equil_index;
    const int nc = n_img * n_chains;
    const int lane = threadIdx.x & 31;
    const int wpb = blockDim.x >> 5;
    for (int c = blockIdx.x * wpb + (threadIdx.x >> 5); c < nc; c += gridDim.x * wpb) {
        const ImgDev& I = img[c / n_chains];
        uint32_t cnt = ch.acc_cnt[c * kSpread + lane];
        double e_gap = ch.e_cur[c * kSpread + lane];
        ch.acc_cnt[c * kSpread + lane] = 0;
        ch.e_cur[c * kSpread + lane] = 0.0;
        cnt = __reduce_add_sync(0xffffffffu, cnt);
        e_gap = warp_sum(e_gap);
        if (lane != 0) continue;
        ch.acc_last[c] = cnt;
        if (equil && (double)cnt < A_targ * (double)I.n_gap) {
            ch.a[c] = (float)(1.0 + (double)(i + 1) / k_a);
            ch.alpha[c] = proposal_width(ch.a[c]);
        }
        if (record) {
            const double e = (e_gap + (add_ess ? I.E_ss : 0.0)) / I.n_bonds;
            ch.e_last[c] = e;
            if (stats) {
                ch.e_sum[c] += e;
                ch.e_sum2[c] += e * e;
            }
        } else {
            ch.e_last[c] = __longlong_as_double(0x7FF8000000000000LL);
        }
    }
    // the last block to finish advances the counters: every block has read
    // equil_index before it takes its ticket
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        if (atomicAdd(&ctl->ticket, 1u) == gridDim.x - 1) {
            ctl->ticket = 0;
            ctl->sweep += 1;
            if (equil) ctl->equil_index += 1;
        }
    }
}

// One Newton step of the specific energy matching per image (thread):
// <e>, Var(e) over the chains' measurement sweeps, bracket update, then
// T <- T - (<e> - e_s) T^2 / (N_GP Var(e)), or the geometric bisection of the
// bracket when the step leaves it.
__global__ void newton_kernel(ImgDev* sub_img, ImgDev* main_img, ChainDev sub_ch, double* nst,
                              int n_img, int K, int n_meas) {
    const int im = blockIdx.x * blockDim.x + threadIdx.x;
    if (im >= n_img) return;
    double s = 0.0, s2 = 0.0;
    for (int k = 0; k < K; ++k) {
        s += sub_ch.e_sum[im * K + k];
        s2 += sub_ch.e_sum2[im * K + k];
        sub_ch.e_sum[im * K + k] = 0.0;
        sub_ch.e_sum2[im * K + k] = 0.0;
    }
    const double n = (double)K * n_meas;
    const double mean = s / n;
    const double var = fmax(s2 / n - mean * mean, 1e-300);
    double* st = nst + 4 * im;
    double lo = st[0], hi = st[1];
    const double T = st[2];
    const double e_s = main_img[im].e_s;
    if (mean > e_s) hi = fmin(hi, T); else lo = fmax(lo, T);
    const double slope = sub_img[im].n_bonds * var / (T * T);
    double Tn = T - (mean - e_s) / slope;
    if (!(Tn > lo && Tn < hi)) Tn = sqrt(lo * hi);
    st[0] = lo;
    st[1] = hi;
    st[2] = Tn;
    st[3] = mean;
    sub_img[im].T = Tn;
    sub_img[im].invT = (float)(1.0 / Tn);
    main_img[im].T = Tn;
    main_img[im].invT = (float)(1.0 / Tn);
}

__global__ void newton_init_kernel(ImgDev* sub_img, const ImgDev* main_img, double* nst,
                                   int n_img, double T_lo, double T_hi, double J) {
    const int im = blockIdx.x * blockDim.x + threadIdx.x;
    if (im >= n_img) return;
    // harmonic guess e ~ -J + T/4 (each site carries T/2 over two bonds)
    double T0 = 4.0 * (main_img[im].e_s + J);
    T0 = fmin(fmax(T0, T_lo * 4.0), T_hi / 4.0);
    nst[4 * im + 0] = T_lo;
    nst[4 * im + 1] = T_hi;
    nst[4 * im + 2] = T0;
    nst[4 * im + 3] = 0.0;
    sub_img[im].T = T0;
    sub_img[im].invT = (float)(1.0 / T0);
}

// ======================================================= dense views

__device__ __forceinline__ float site_value(const ImgDev& I, const float* state, const float* samp,
                                            const int* slot_map, int tiled, int chain,
                                            long long i) {
    if (tiled) {
        const int s = slot_map[I.site_off + i];
        return s >= 0 ? state[state_index(I, chain, s)] : samp[I.site_off + i];
    }
    return fabsf(state[state_index(I, chain, i)]);
}

// H of every (image, chain) (blockIdx.y), FP64 sums of FP32 bond terms.
__global__ void energy_kernel(const ImgDev* img, const float* state, const float* samp,
                              const int* slot_map, int tiled, int n_chains, float q, float J,
                              int gmrf, double* out) {
    const int ic = blockIdx.y;
    const int im = ic / n_chains, chain = ic - im * n_chains;
    const ImgDev& I = img[im];
    const long long n = (long long)I.Lx * I.Ly;
    double s = 0.0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(i % I.Lx), y = (int)(i / I.Lx);
        const float v = site_value(I, state, samp, slot_map, tiled, chain, i);
        float e = 0.0f;
        if (x + 1 < I.Lx) {
            const float d = v - site_value(I, state, samp, slot_map, tiled, chain, i + 1);
            e += gmrf ? J * gmrf_bond(d) : -J * cosf(q * d);
        }
        if (y + 1 < I.Ly) {
            const float d = v - site_value(I, state, samp, slot_map, tiled, chain, i + I.Lx);
            e += gmrf ? J * gmrf_bond(d) : -J * cosf(q * d);
        }
        s += (double)e;
    }
    s = warp_sum(s);
    if ((threadIdx.x & 31) == 0 && s != 0.0) atomicAdd(out + ic, s);
}

__global__ void energy_finish_kernel(const ImgDev* img, double* out, int n_chains, int nc) {
    const int ic = blockIdx.x * blockDim.x + threadIdx.x;
    if (ic < nc) out[ic] /= img[ic / n_chains].n_bonds;
}

// state <-> dense [chain][Ly][Lx] per image (dir 0: get, 1: set gap sites).
__global__ void state_copy_kernel(const ImgDev* img, float* state, const float* samp,
                                  const int* slot_map, int tiled, int n_chains, float* dense,
                                  int dir, int ic0, float* plane) {
    const int ic = ic0 + blockIdx.y;
    const int im = ic / n_chains, chain = ic - im * n_chains;
    const ImgDev& I = img[im];
    const long long n = (long long)I.Lx * I.Ly;
    float* d = plane ? plane : dense + I.site_off * n_chains + (long long)chain * n;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        if (tiled) {
            const int s = slot_map[I.site_off + i];
            if (dir == 0) d[i] = s >= 0 ? state[state_index(I, chain, s)] : samp[I.site_off + i];
            else if (s >= 0) state[state_index(I, chain, s)] = d[i];
        } else {
            float* st = state + state_index(I, chain, 0);
            const float v = st[i];
            if (dir == 0) d[i] = fabsf(v);
            else if (!is_fixed(v)) st[i] = d[i];
        }
    }
}

// Conditional mean and standard deviation over realisations (Alg. 2 step 6).
__global__ void predict_kernel(const ImgDev* img, const double* acc1, const double* acc2,
                               const float* zin, const int* slot_map, const float* samp,
                               int tiled, double n_samples, float* zhat, float* zstd) {
    const ImgDev& I = img[blockIdx.y];
    const long long n = (long long)I.Lx * I.Ly;
    const double range = (double)I.zmax - (double)I.zmin;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const long long s = I.site_off + i;
        long long slot = -1;
        if (tiled) slot = slot_map[s];
        else if (samp[s] < 0.0f) slot = i;
        if (slot < 0) {
            zhat[s] = zin[s];
            if (zstd) zstd[s] = 0.0f;
        } else {
            const double m = acc1[I.slot_off + slot] / n_samples;
            zhat[s] = (float)(I.zmin + range * m / (2.0 * kPiD));
            if (zstd) {
                const double v = fmax(acc2[I.slot_off + slot] / n_samples - m * m, 0.0);
                zstd[s] = (float)(range * sqrt(v) / (2.0 * kPiD));
            }
        }
    }
}

// Realisation sums <-> dense per-pixel arrays (dir 0: get, 1: set gap pixels).
__global__ void acc_dense_kernel(const ImgDev* img, double* acc, const int* slot_map,
                                 const float* samp, int tiled, double* dense, int dir) {
    const ImgDev& I = img[blockIdx.y];
    const long long n = (long long)I.Lx * I.Ly;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const long long s = I.site_off + i;
        long long slot = -1;
        if (tiled) slot = slot_map[s];
        else if (samp[s] < 0.0f) slot = i;
        if (dir == 0) dense[s] = slot < 0 ? 0.0 : acc[I.slot_off + slot];
        else if (slot >= 0) acc[I.slot_off + slot] = dense[s];
    }
}

// Chain-mean specific energy of every image after sweep i, into its ring.
// Alg. 2 step 4.4 after the equilibration sweep i that just ran (i read from
// sg[n_img + 1]): records the chain-mean specific energy of every image in the
// ring hist; at a check sweep (i >= n_fit and i mod n_f == 0) fits the
// least-squares line (a degree-1 Savitzky-Golay filter) through the last n_fit
// entries of every image still settling and marks an image settled once its
// slope is no longer negative.  sg: [n_img] settled flags (sticky), then the
// images still settling after the last check, the sweeps done, and 1 once every
// image settled.  With use_h the kernel also sets the conditional handle h to
// whether another sweep follows (not once every image settled, nor after sweep
// i_max); h ends the device-side while loop, which therefore runs at most
// i_max + 1 times.  One block.
__global__ void sg_step_kernel(const ChainDev ch, double* hist, int* sg, int n_img, int n_chains,
                               int n_fit, int n_f, int i_max, cudaGraphConditionalHandle h,
                               int use_h) {
    __shared__ int unsettled;
    const uint32_t i = (uint32_t)sg[n_img + 1];
    if (threadIdx.x == 0) unsettled = 0;
    for (int im = threadIdx.x; im < n_img; im += blockDim.x) {
        double s = 0.0;
        for (int k = 0; k < n_chains; ++k) s += ch.e_last[(size_t)im * n_chains + k];
        hist[(size_t)im * kHist + (i % kHist)] = s / n_chains;
    }
    __syncthreads();
    const bool check = i >= (uint32_t)n_fit && i % (uint32_t)n_f == 0;
    if (check) {
        for (int im = threadIdx.x; im < n_img; im += blockDim.x) {
            if (sg[im]) continue;
            const double xm = 0.5 * (n_fit - 1);
            double ym = 0.0;
            for (int k = 0; k < n_fit; ++k)
                ym += hist[(size_t)im * kHist + ((i + 1 + k - n_fit) % kHist)];
            ym /= n_fit;
            double sxy = 0.0, sxx = 0.0;
            for (int k = 0; k < n_fit; ++k) {
                const double y = hist[(size_t)im * kHist + ((i + 1 + k - n_fit) % kHist)];
                sxy += (k - xm) * (y - ym);
                sxx += (k - xm) * (k - xm);
            }
            if (sxy / sxx >= 0.0) sg[im] = 1;
            else atomicAdd(&unsettled, 1);
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const bool stop = check && unsettled == 0;
        if (check) sg[n_img] = unsettled;
        sg[n_img + 1] = (int)(i + 1);
        sg[n_img + 2] = stop ? 1 : 0;
        if (use_h) cudaGraphSetConditional(h, (!stop && i + 1 <= (uint32_t)i_max) ? 1u : 0u);
    }
}

__global__ void set_T_kernel(ImgDev* img, const double* T, int n) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) { img[i].T = T[i]; img[i].invT = (float)(1.0 / T[i]); }
}

int grid_for(long long n, int block = 256, int cap = 4096) {
    long long b = (n + block - 1) / block;
    return (int)std::max<long long>(1, std::min<long long>(b, cap));
}

// ======================================================= host helpers

mpr_status check_params(const mpr_params* p) {
    if (!p) return fail(MPR_ERR_INVALID_ARG, "params is NULL");
    if (!(p->q > 0.0 && p->q <= 0.5 + 1e-12) && !(p->q == 1.0))
        return fail(MPR_ERR_INVALID_ARG, "q must lie in (0, 1/2] (or equal 1)");
    if (!(p->J > 0.0)) return fail(MPR_ERR_INVALID_ARG, "J must be positive");
    if (!(p->A_targ >= 0.0 && p->A_targ <= 1.0)) return fail(MPR_ERR_INVALID_ARG, "A_targ in [0,1]");
    if (!(p->k_a > 0.0)) return fail(MPR_ERR_INVALID_ARG, "k_a must be positive");
    if (p->path != MPR_PATH_TILED && p->path != MPR_PATH_PLAIN)
        return fail(MPR_ERR_INVALID_ARG, "unknown path");
    if (p->chain_group < 0) return fail(MPR_ERR_INVALID_ARG, "chain_group < 0");
    if (p->model != MPR_MODEL_MPR && p->model != MPR_MODEL_GMRF)
        return fail(MPR_ERR_INVALID_ARG, "unknown model");
    if (p->model == MPR_MODEL_GMRF && p->literal_or)
        return fail(MPR_ERR_INVALID_ARG, "the printed over-relaxation belongs to the MPR model");
    if (p->path == MPR_PATH_TILED && (p->model == MPR_MODEL_GMRF || p->literal_or) &&
        !((p->tile_x == 0 && p->tile_y == 0) || (p->tile_x == 16 && p->tile_y == 16)))
        return fail(MPR_ERR_INVALID_ARG,
                    "the GMRF model and the printed over-relaxation run with 16 x 16 tiles");
    return MPR_OK;
}

void pick_tiles(const mpr_params& p, int n_img, const int* Lx, const int* Ly, int n_chains,
                int& tx, int& ty) {
    tx = p.tile_x;
    ty = p.tile_y;
    if (tx > 0 && ty > 0) return;
    (void)n_img;
    (void)Lx;
    (void)Ly;
    (void)n_chains;
    // 16 x 16: the shortest block life per chain group of 32 (measured fastest
    // of the three shapes on 4096^2 images at 40 % gaps)
    tx = 16;
    ty = 16;
}

// Model bits of the sweep flags (SweepFlags) for a parameter set.
int model_flags(const mpr_params& p) {
    return (p.literal_or ? kLiteralOR : 0) | (p.model == MPR_MODEL_GMRF ? kGMRF : 0);
}

// Chains per thread block of the tiled pass (a multiple of 4, or covering
// every chain; at most 32).  Automatic: the largest power of two from 4 up to
// 32 that still gives at least four blocks per SM (152 SMs); on the
// 256^2 x 16 temperature lattices that is 4.
int pick_chain_group(const mpr_ctx* c) {
    if (c->g.path != MPR_PATH_TILED) return 1;
    const int n = c->g.n_chains;
    if (c->p.chain_group > 0) return std::min(c->p.chain_group, 32);
    const long long target = 152LL * 4;
    const long long tiles = std::max(1, c->g.n_tiles);
    int cg = 4;
    while (cg < 32 && cg < n && tiles * ((n + 2 * cg - 1) / (2 * cg)) >= target) cg *= 2;
    return cg >= n ? n : cg;
}

// Chain ranges of a tiled pass: whole groups of the automatic (or requested)
// size, then, when the chain count is not a multiple of it, the remaining
// chains as one smaller group in a launch of their own, so that they do not
// occupy a full group's lanes (100 chains: 3 x 32, then 4).
struct ChainRange {
    int chain0, chain_end, group;
};

int chain_ranges(const mpr_ctx* c, ChainRange out[2]) {
    const int n = c->g.n_chains, cg = pick_chain_group(c);
    const int rem = cg < n ? n % cg : 0;
    if (rem == 0) {
        out[0] = {0, n, cg};
        return 1;
    }
    out[0] = {0, n - rem, cg};
    out[1] = {n - rem, n, rem};
    return 2;
}

// Sorts the tiles of each colour pass into a light launch, whose tables let
// an SM hold as many blocks as its threads allow, and a heavy launch with the
// rest (tiles inside large gap blocks, say), so that a few dense tiles do not
// cut the occupancy of every block.  Without heavy tiles a pass is one launch.
mpr_status split_tiles(mpr_ctx* c, const std::vector<TileDesc>& tiles, cudaStream_t s) {
    const Geometry& g = c->g;
    const int cg = pick_chain_group(c), flags = model_flags(c->p);
    int dev = 0, sm_bytes = 0, reserved = 0;
    MPR_CUDA(cudaGetDevice(&dev));
    MPR_CUDA(cudaDeviceGetAttribute(&sm_bytes, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev));
    MPR_CUDA(cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev));
    const size_t budget = (size_t)sm_bytes / tiled_blocks_per_sm(g.tx, g.ty) - (size_t)reserved;
    const int n = g.n_tiles;
    std::vector<int> list(2 * (size_t)n);
    bool split = false;
    for (int col = 0; col < 2; ++col) {
        int gmax = 1, glight = 1, nl = 0;
        std::vector<int> heavy;
        for (int t = 0; t < n; ++t) {
            const int e = tiles[t].cnt[col ^ 1] + tiles[t].halo_cnt[col] + 1;
            gmax = std::max(gmax, e);
            if (tiled_pass_smem(g.tx, g.ty, e, cg, flags) <= budget) {
                list[(size_t)col * n + nl++] = t;
                glight = std::max(glight, e);
            } else {
                heavy.push_back(t);
            }
        }
        for (size_t k = 0; k < heavy.size(); ++k) list[(size_t)col * n + nl + k] = heavy[k];
        c->gt[col] = gmax;
        c->gt_light[col] = glight;
        c->n_light[col] = nl;
        split = split || nl < n;
    }
    if (split) {
        MPR_CUDA(cudaMemcpyAsync(c->d_tile_list, list.data(), sizeof(int) * list.size(),
                                 cudaMemcpyHostToDevice, s));
        MPR_CUDA(cudaStreamSynchronize(s));
    }
    return MPR_OK;
}

mpr_status sub_workspace_size(const mpr_params& p, const mpr_T_opts& o, int n_img, const int* Lx,
                              const int* Ly, size_t* bytes);

mpr_status workspace_size_impl(int n_img, const int* Lx, const int* Ly, const int64_t* n_gap,
                               int n_chains, const mpr_params& p, const mpr_T_opts& o,
                               bool with_sub, bool staging, size_t* bytes) {
    int tx, ty;
    pick_tiles(p, n_img, Lx, Ly, n_chains, tx, ty);
    if (p.path == MPR_PATH_TILED && !tiled_config_supported(tx, ty))
        return fail(MPR_ERR_INVALID_ARG, "unsupported tile shape");
    Geometry g;
    make_geometry(g, n_img, Lx, Ly, n_chains, p.path, tx, ty);
    std::vector<long long> slots(n_img);
    for (int i = 0; i < n_img; ++i)
        slots[i] = slot_bound(g, i, n_gap ? (long long)n_gap[i] : (long long)Lx[i] * Ly[i]);
    size_t sub = 0;
    if (with_sub) MPR_TRY(sub_workspace_size(p, o, n_img, Lx, Ly, &sub));
    *bytes = make_layout(g, slots, sub, staging).total;
    return MPR_OK;
}

mpr_status sub_workspace_size(const mpr_params& p, const mpr_T_opts& o, int n_img, const int* Lx,
                              const int* Ly, size_t* bytes) {
    std::vector<int> L(n_img);
    for (int i = 0; i < n_img; ++i) L[i] = default_T_side(Lx[i], Ly[i], o);
    mpr_params sp = p;
    sp.literal_or = 0;
    sp.path = MPR_PATH_TILED;
    sp.tile_x = sp.tile_y = 0;
    sp.chain_group = 0;
    return workspace_size_impl(n_img, L.data(), L.data(), nullptr, o.chains, sp, o, false, false,
                               bytes);
}

mpr_status validate_shapes(int n_img, const int* Lx, const int* Ly, int n_chains) {
    if (n_img < 1 || !Lx || !Ly) return fail(MPR_ERR_INVALID_ARG, "need n_img >= 1 and sizes");
    if (n_chains < 1 || n_chains > 65535) return fail(MPR_ERR_INVALID_ARG, "n_chains out of range");
    if ((long long)n_img * n_chains > 65535)
        return fail(MPR_ERR_INVALID_ARG, "n_img * n_chains must not exceed 65535");
    for (int i = 0; i < n_img; ++i)
        if (Lx[i] < 2 || Ly[i] < 2 || Lx[i] > 65535 || Ly[i] > 65535)
            return fail(MPR_ERR_INVALID_ARG, "image sides must lie in [2, 65535]");
    return MPR_OK;
}

// Builds a context over `ws`.  unconditional: every site free, no inputs.
mpr_status init_impl(mpr_ctx* c, int n_img, const int* Lx, const int* Ly, int n_chains,
                     const float* z, const uint8_t* gap, mpr_mem where, void* ws, size_t ws_bytes,
                     bool unconditional, cudaStream_t s) {
    if (!ws || (reinterpret_cast<uintptr_t>(ws) % kAlign) != 0)
        return fail(MPR_ERR_WORKSPACE, "workspace must be non-NULL and 256-byte aligned");
    int tx, ty;
    pick_tiles(c->p, n_img, Lx, Ly, n_chains, tx, ty);
    if (c->p.path == MPR_PATH_TILED && !tiled_config_supported(tx, ty))
        return fail(MPR_ERR_INVALID_ARG, "unsupported tile shape");
    c->unconditional = unconditional;
    c->img_tag = unconditional ? (1u << 30) : 0u;
    make_geometry(c->g, n_img, Lx, Ly, n_chains, c->p.path, tx, ty);
    Geometry& g = c->g;
    const bool tiled = g.path == MPR_PATH_TILED;
    const bool staging = !unconditional;
    size_t sub_bytes = 0;
    if (!unconditional) MPR_TRY(sub_workspace_size(c->p, c->topt, n_img, Lx, Ly, &sub_bytes));

    // provisional layout (worst case) to place the regions that do not depend on gap counts
    std::vector<long long> worst(n_img);
    for (int i = 0; i < n_img; ++i) worst[i] = 0;
    c->ws = static_cast<unsigned char*>(ws);
    c->L = make_layout(g, worst, 0, staging);
    if (c->L.scratch + align_up(sizeof(double) * 4 * n_img) > ws_bytes)
        return fail(MPR_ERR_WORKSPACE, "workspace too small");
    bind_views(c);

    c->h_img.assign(n_img, ImgDev{});
    for (int i = 0; i < n_img; ++i) {
        ImgDev& I = c->h_img[i];
        I.Lx = Lx[i];
        I.Ly = Ly[i];
        I.site_off = g.site_off[i];
        I.tile0 = g.tile0[i];
        I.ntiles = g.ntiles[i];
        I.n_bonds = (double)Lx[i] * (Ly[i] - 1) + (double)Ly[i] * (Lx[i] - 1);
        I.T = 1.0;
        I.invT = 1.0f;
    }
    MPR_CUDA(cudaMemcpyAsync(c->d_img, c->h_img.data(), sizeof(ImgDev) * n_img,
                             cudaMemcpyHostToDevice, s));
    const size_t N = (size_t)g.n_sites;
    const float* d_z = nullptr;
    const uint8_t* d_gap = c->d_gst;
    if (unconditional) {
        MPR_CUDA(cudaMemsetAsync(c->d_gst, 1, N, s));
    } else {
        const cudaMemcpyKind k = where == MPR_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
        MPR_CUDA(cudaMemcpyAsync(c->d_zst, z, sizeof(float) * N, k, s));
        MPR_CUDA(cudaMemcpyAsync(c->d_gst, gap, N, k, s));
        d_z = c->d_zst;
    }

    // tile descriptors
    std::vector<TileDesc> tiles;
    if (tiled) {
        tiles.reserve(g.n_tiles);
        for (int i = 0; i < n_img; ++i)
            for (int y0 = 0; y0 < Ly[i]; y0 += ty)
                for (int x0 = 0; x0 < Lx[i]; x0 += tx) {
                    TileDesc t{};
                    t.img = i;
                    t.x0 = x0;
                    t.y0 = y0;
                    tiles.push_back(t);
                }
        MPR_CUDA(cudaMemcpyAsync(c->d_tiles, tiles.data(), sizeof(TileDesc) * g.n_tiles,
                                 cudaMemcpyHostToDevice, s));
    }

    // extremes and gap counts
    double* scratch = at<double>(c->ws, c->L.scratch);
    uint32_t* mm = reinterpret_cast<uint32_t*>(scratch);                         // [2 n_img]
    unsigned long long* ngap = reinterpret_cast<unsigned long long*>(scratch + n_img);  // [n_img]
    std::vector<uint32_t> h_mm(2 * n_img);
    for (int i = 0; i < n_img; ++i) { h_mm[2 * i] = 0xFFFFFFFFu; h_mm[2 * i + 1] = 0u; }
    MPR_CUDA(cudaMemcpyAsync(mm, h_mm.data(), sizeof(uint32_t) * 2 * n_img, cudaMemcpyHostToDevice, s));
    MPR_CUDA(cudaMemsetAsync(ngap, 0, sizeof(unsigned long long) * n_img, s));
    std::vector<unsigned long long> h_ngap(n_img, 0);
    if (!unconditional) {
        long long maxn = 0;
        for (int i = 0; i < n_img; ++i) maxn = std::max(maxn, (long long)Lx[i] * Ly[i]);
        minmax_kernel<<<dim3(grid_for(maxn, 256, 1024), n_img), 256, 0, s>>>(c->d_img, d_z, d_gap, mm, ngap);
        MPR_CUDA(cudaGetLastError());
    }
    std::vector<int> h_counts;
    if (tiled) {
        int* counts = at<int>(c->ws, c->L.counts);
        MPR_CUDA(cudaMemsetAsync(counts, 0, sizeof(int) * 2 * g.n_tiles, s));
        MPR_CUDA(launch_tile_count(c->d_img, c->d_tiles, g.n_tiles, d_gap, tx, ty, counts, s));
        h_counts.resize(2 * g.n_tiles);
        MPR_CUDA(cudaMemcpyAsync(h_counts.data(), counts, sizeof(int) * 2 * g.n_tiles,
                                 cudaMemcpyDeviceToHost, s));
    }
    if (!unconditional) {
        MPR_CUDA(cudaMemcpyAsync(h_mm.data(), mm, sizeof(uint32_t) * 2 * n_img, cudaMemcpyDeviceToHost, s));
        MPR_CUDA(cudaMemcpyAsync(h_ngap.data(), ngap, sizeof(unsigned long long) * n_img,
                                 cudaMemcpyDeviceToHost, s));
    }
    MPR_CUDA(cudaStreamSynchronize(s));

    // per image: range, gap count, slot space
    c->slots.assign(n_img, 0);
    for (int i = 0; i < n_img; ++i) {
        ImgDev& I = c->h_img[i];
        if (unconditional) {
            I.zmin = 0.0f;
            I.zmax = 1.0f;
            I.n_gap = (long long)Lx[i] * Ly[i];
        } else {
            auto dec = [](uint32_t u) {
                uint32_t b = (u & 0x80000000u) ? (u & 0x7FFFFFFFu) : ~u;
                float f;
                std::memcpy(&f, &b, 4);
                return f;
            };
            if (h_mm[2 * i] == 0xFFFFFFFFu)
                return fail(MPR_ERR_DEGENERATE_RANGE, "image " + std::to_string(i) + " has no samples");
            I.zmin = dec(h_mm[2 * i]);
            I.zmax = dec(h_mm[2 * i + 1]);
            if (!(I.zmax > I.zmin))
                return fail(MPR_ERR_DEGENERATE_RANGE,
                            "image " + std::to_string(i) + ": z_max == z_min over the samples");
            if (!std::isfinite(I.zmin) || !std::isfinite(I.zmax))
                return fail(MPR_ERR_INVALID_ARG, "non-finite sample value in image " + std::to_string(i));
            I.n_gap = (long long)h_ngap[i];
            if (I.n_gap == 0)
                return fail(MPR_ERR_INVALID_ARG, "image " + std::to_string(i) + " has no gaps");
        }
        if (tiled) {
            long long off = 0;
            for (int t = g.tile0[i]; t < g.tile0[i] + g.ntiles[i]; ++t) {
                for (int col = 0; col < 2; ++col) {
                    const int n = h_counts[2 * t + col];
                    tiles[t].off[col] = (int)off;
                    tiles[t].cnt[col] = n;
                    off += (n + 3) & ~3;
                }
            }
            c->slots[i] = off;
        } else {
            c->slots[i] = (long long)Lx[i] * Ly[i];
        }
    }
    c->L = make_layout(g, c->slots, sub_bytes, staging);
    if (c->L.total > ws_bytes)
        return fail(MPR_ERR_WORKSPACE, "workspace too small: need " + std::to_string(c->L.total) +
                                           " bytes, have " + std::to_string(ws_bytes));
    bind_views(c);
    long long slot_off = 0, state_off = 0;
    for (int i = 0; i < n_img; ++i) {
        ImgDev& I = c->h_img[i];
        I.slot_off = slot_off;
        I.state_off = state_off;
        // tiled: slot-major, chains interleaved; plain: one dense plane per chain
        I.stride = tiled ? 1 : c->slots[i];
        I.sstride = tiled ? state_chains(g) : 1;
        slot_off += c->slots[i];
        state_off += c->slots[i] * state_chains(g);
    }
    MPR_CUDA(cudaMemcpyAsync(c->d_img, c->h_img.data(), sizeof(ImgDev) * n_img,
                             cudaMemcpyHostToDevice, s));
    if (tiled) {
        for (TileDesc& t : tiles) {
            const ImgDev& I = c->h_img[t.img];
            t.cp = (int)I.sstride;
            t.state_off = I.state_off;
            t.slot_off = I.slot_off;
        }
        MPR_CUDA(cudaMemcpyAsync(c->d_tiles, tiles.data(), sizeof(TileDesc) * g.n_tiles,
                                 cudaMemcpyHostToDevice, s));
        MPR_CUDA(cudaMemsetAsync(c->d_slot_pos, 0xFF, sizeof(uint32_t) * c->L.n_slots, s));
        MPR_CUDA(launch_tile_fill(c->d_img, c->d_tiles, g.n_tiles, d_gap, tx, ty, c->d_slot_pos,
                                  c->d_slot_map, c->d_halo, g.halo_cap, s));
        // table entries of every tile and pass from the ring lists just built
        MPR_CUDA(cudaMemcpyAsync(tiles.data(), c->d_tiles, sizeof(TileDesc) * g.n_tiles,
                                 cudaMemcpyDeviceToHost, s));
        MPR_CUDA(cudaStreamSynchronize(s));
        MPR_TRY(split_tiles(c, tiles, s));
        ChainRange cr[2];
        const bool extra = c->n_light[0] < g.n_tiles || c->n_light[1] < g.n_tiles ||
                           chain_ranges(c, cr) > 1;
        if (extra && !c->side) {
            MPR_CUDA(cudaStreamCreateWithFlags(&c->side, cudaStreamNonBlocking));
            MPR_CUDA(cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming));
            MPR_CUDA(cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming));
        }
    }
    long long maxn = 0;
    for (int i = 0; i < n_img; ++i) maxn = std::max(maxn, (long long)Lx[i] * Ly[i]);
    map_kernel<<<dim3(grid_for(maxn, 256, 2048), n_img), 256, 0, s>>>(c->d_img, d_z, d_gap, c->d_samp,
                                                                      unconditional ? 1 : 0);
    MPR_CUDA(cudaGetLastError());
    if (tiled)
        MPR_CUDA(launch_tile_const(c->d_img, c->d_tiles, g.n_tiles, tx, ty, c->d_slot_pos,
                                   c->d_halo, g.halo_cap, c->d_samp, (float)c->p.q,
                                   c->p.model == MPR_MODEL_GMRF ? 1 : 0, c->d_slot_ref,
                                   c->d_slot_cs, s));
    const uint2 key = make_uint2((uint32_t)c->p.seed, (uint32_t)(c->p.seed >> 32));
    for (int i = 0; i < n_img; ++i) {
        if (tiled) {
            // the temperature lattices start cold (see mpr_estimate_T), images hot
            hot_start_tiled_kernel<<<grid_for(c->slots[i] * state_chains(g) / 2), 256, 0, s>>>(
                c->d_img, c->d_slot_pos, c->d_state, c->slots[i], i, n_chains, key, c->img_tag,
                unconditional ? 1 : 0);
        } else {
            init_plain_kernel<<<grid_for((long long)Lx[i] * Ly[i] * n_chains), 256, 0, s>>>(
                c->d_img, c->d_samp, c->d_state, i, n_chains, key, c->img_tag);
        }
        MPR_CUDA(cudaGetLastError());
    }
    const int nc = n_img * n_chains;
    init_chains_kernel<<<grid_for(nc), 256, 0, s>>>(c->ch, nc);
    MPR_CUDA(cudaGetLastError());
    MPR_CUDA(cudaMemsetAsync(c->d_ctl, 0, sizeof(Control), s));
    MPR_CUDA(cudaMemsetAsync(c->d_acc1, 0, sizeof(double) * c->L.n_slots, s));
    MPR_CUDA(cudaMemsetAsync(c->d_acc2, 0, sizeof(double) * c->L.n_slots, s));

    // sample specific energy
    if (!unconditional) {
        double* sums = scratch + 2 * n_img;
        unsigned long long* npairs = reinterpret_cast<unsigned long long*>(scratch + 3 * n_img);
        MPR_CUDA(cudaMemsetAsync(sums, 0, sizeof(double) * 2 * n_img, s));
        sample_energy_kernel<<<dim3(grid_for(maxn, 256, 1024), n_img), 256, 0, s>>>(
            c->d_img, c->d_samp, c->p.q, c->p.J, c->p.model == MPR_MODEL_GMRF ? 1 : 0, sums, npairs);
        MPR_CUDA(cudaGetLastError());
        std::vector<double> h_sums(n_img);
        std::vector<unsigned long long> h_np(n_img);
        MPR_CUDA(cudaMemcpyAsync(h_sums.data(), sums, sizeof(double) * n_img, cudaMemcpyDeviceToHost, s));
        MPR_CUDA(cudaMemcpyAsync(h_np.data(), npairs, sizeof(unsigned long long) * n_img,
                                 cudaMemcpyDeviceToHost, s));
        MPR_CUDA(cudaStreamSynchronize(s));
        for (int i = 0; i < n_img; ++i) {
            ImgDev& I = c->h_img[i];
            I.n_sp = (long long)h_np[i];
            I.E_ss = h_sums[i];
            I.e_s = I.n_sp > 0 ? h_sums[i] / (double)I.n_sp : std::nan("");
        }
        MPR_CUDA(cudaMemcpyAsync(c->d_img, c->h_img.data(), sizeof(ImgDev) * n_img,
                                 cudaMemcpyHostToDevice, s));
    }
    c->sweep = 0;
    c->equil_index = 0;
    c->n_meas_done = 0;
    return MPR_OK;
}

mpr_status launch_sweeps(mpr_ctx* c, int n, int phase, int flags, bool stats, bool accumulate,
                         cudaStream_t s) {
    const bool equil = phase == MPR_EQUIL;
    const bool record = (flags & MPR_RECORD_ENERGY) != 0;
    SweepArgs a{};
    a.img = c->d_img;
    a.tiles = c->d_tiles;
    a.slot_pos = c->d_slot_pos;
    a.slot_ref = c->d_slot_ref;
    a.slot_cs = c->d_slot_cs;
    a.halo = c->d_halo;
    a.samp = c->d_samp;
    a.state = c->d_state;
    a.acc1 = c->d_acc1;
    a.acc2 = c->d_acc2;
    a.ch = c->ch;
    a.ctl = c->d_ctl;
    a.key = make_uint2((uint32_t)c->p.seed, (uint32_t)(c->p.seed >> 32));
    for (int i = 0; i < 10; ++i) {
        a.rk[2 * i] = a.key.x + (uint32_t)i * 0x9E3779B9u;
        a.rk[2 * i + 1] = a.key.y + (uint32_t)i * 0xBB67AE85u;
    }
    a.q = (float)c->p.q;
    a.inv_q = (float)(1.0 / c->p.q);
    a.two_pi_q = (float)(2.0 * kPiD * c->p.q);
    a.J = (float)c->p.J;
    a.n_chains = c->g.n_chains;
    a.chain_group = pick_chain_group(c);
    a.chain0 = 0;
    a.chain_end = c->g.n_chains;
    ChainRange cr[2];
    const int n_cr = chain_ranges(c, cr);
    a.halo_cap = c->g.halo_cap;
    a.n_img = c->g.n_img;
    a.img_tag = c->img_tag;
    int base = 0;
    if (!equil && accumulate) base |= kAccumulate | kAccumulate2;
    if (!equil && !c->p.freeze_a_in_measure) base |= kAlphaOne;
    base |= model_flags(c->p);
    const bool tiled = c->g.path == MPR_PATH_TILED;
    for (int k = 0; k < n; ++k) {
        for (int colour = 0; colour < 2; ++colour) {
            a.colour = colour;
            a.flags = base | ((record && colour == 1) ? kEnergy : 0);
            cudaError_t e = cudaSuccess;
            if (!tiled) {
                e = launch_plain_pass(a, c->g.max_Lx, c->g.max_Ly, s);
            } else {
                const int nt = c->g.n_tiles, nl = c->n_light[colour];
                // the heavy tiles and the remaining chains go to the side stream
                // when there is a main launch for them to run beside
                const bool extra = nl < nt || n_cr > 1;
                const bool fork = extra && nl > 0 && c->side;
                cudaStream_t s2 = fork ? c->side : s;
                if (fork) {
                    e = cudaEventRecord(c->ev_fork, s);
                    if (e == cudaSuccess) e = cudaStreamWaitEvent(c->side, c->ev_fork, 0);
                }
                // whole chain groups: light tiles, then heavy ones
                a.chain0 = cr[0].chain0;
                a.chain_end = cr[0].chain_end;
                a.chain_group = cr[0].group;
                a.tile_list = nl < nt ? c->d_tile_list + (size_t)colour * nt : nullptr;
                if (e == cudaSuccess && nl > 0) {  // the light tiles (all of them without a heavy launch)
                    a.tile_base = 0;
                    a.n_list = nl;
                    a.gt = nl < nt ? c->gt_light[colour] : c->gt[colour];
                    e = launch_tiled_pass(a, c->g.tx, c->g.ty, s);
                }
                if (e == cudaSuccess && nl < nt) {
                    a.tile_base = nl;
                    a.n_list = nt - nl;
                    a.gt = c->gt[colour];
                    e = launch_tiled_pass(a, c->g.tx, c->g.ty, s2);
                }
                if (e == cudaSuccess && n_cr > 1) {  // the remaining chains, every tile
                    a.chain0 = cr[1].chain0;
                    a.chain_end = cr[1].chain_end;
                    a.chain_group = cr[1].group;
                    a.tile_list = nullptr;
                    a.tile_base = 0;
                    a.n_list = nt;
                    a.gt = c->gt[colour];
                    e = launch_tiled_pass(a, c->g.tx, c->g.ty, s2);
                }
                if (fork && e == cudaSuccess) {
                    e = cudaEventRecord(c->ev_join, c->side);
                    if (e == cudaSuccess) e = cudaStreamWaitEvent(s, c->ev_join, 0);
                }
            }
            if (e != cudaSuccess) return fail(MPR_ERR_CUDA, std::string("sweep launch: ") + cudaGetErrorString(e));
        }
        // one warp per chain, 8 chains per block
        const int nc = c->g.n_img * c->g.n_chains;
        end_sweep_kernel<<<std::min((nc + 7) / 8, 1024), 256, 0, s>>>(
            c->d_img, c->ch, c->d_ctl, c->g.n_img, c->g.n_chains, equil ? 1 : 0, record ? 1 : 0,
            stats ? 1 : 0, tiled ? 1 : 0, c->p.A_targ, c->p.k_a);
        MPR_CUDA(cudaGetLastError());
    }
    return MPR_OK;
}

// Kernel launches of one sweep, as launch_sweeps issues them: per colour the
// light tiles (when any), the heavy tiles (when any) and the remaining chains
// (when the chain count is not a multiple of the group), then the bookkeeping.
int sweep_launch_count(const mpr_ctx* c) {
    if (c->g.path != MPR_PATH_TILED) return 3;
    ChainRange cr[2];
    const int n_cr = chain_ranges(c, cr);
    int n = 1;
    for (int colour = 0; colour < 2; ++colour) {
        const int nt = c->g.n_tiles, nl = c->n_light[colour];
        n += (nl > 0 ? 1 : 0) + (nl < nt ? 1 : 0) + (n_cr > 1 ? 1 : 0);
    }
    return n;
}

// Launch settings that may not change during a stream capture (the colour
// passes' shared-memory attributes) are applied before one begins.
mpr_status prepare_capture(mpr_ctx* c, cudaStream_t s) {
    if (c->g.path != MPR_PATH_TILED) return MPR_OK;
    SweepArgs a{};
    a.n_chains = c->g.n_chains;
    a.flags = model_flags(c->p);
    ChainRange cr[2];
    const int n_cr = chain_ranges(c, cr);
    for (int r = 0; r < n_cr; ++r) {
        a.chain0 = cr[r].chain0;
        a.chain_end = cr[r].chain_end;
        a.chain_group = cr[r].group;
        MPR_CUDA(launch_tiled_pass(a, c->g.tx, c->g.ty, s, true));
    }
    return MPR_OK;
}

// Whether runs of sweeps on stream s may go through CUDA graphs: graphs are
// enabled, the stream is not the legacy one and nobody is capturing it.
bool graphs_usable(const mpr_ctx* c, cudaStream_t s) {
    if (!c->p.use_graphs || s == nullptr || s == cudaStreamLegacy) return false;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    return cudaStreamIsCapturing(s, &cs) == cudaSuccess && cs == cudaStreamCaptureStatusNone;
}

// n sweeps: launched directly, or (sequences of at least 4 sweeps on a stream
// that may be captured) through a CUDA graph captured once per context and
// replayed.  Every argument of the launches is fixed for the context's life
// (temperatures, a, the sweep counter live in device memory), so a graph
// stays valid.
mpr_status run_sweeps(mpr_ctx* c, int n, int phase, int flags, bool stats, bool accumulate,
                      cudaStream_t s) {
    // (a caller that is capturing gets the launches in its own capture)
    const bool graph = n >= 4 && graphs_usable(c, s);
    if (!graph) {
        MPR_TRY(launch_sweeps(c, n, phase, flags, stats, accumulate, s));
    } else {
        const long long key = ((long long)n << 8) | (phase << 4) | ((flags & 1) << 3) |
                              ((stats ? 1 : 0) << 2) | ((accumulate ? 1 : 0) << 1);
        cudaGraphExec_t exec = nullptr;
        for (auto& g : c->graphs)
            if (g.first == key) exec = g.second;
        if (!exec) {
            MPR_TRY(prepare_capture(c, s));
            MPR_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
            const mpr_status st = launch_sweeps(c, n, phase, flags, stats, accumulate, s);
            cudaGraph_t g = nullptr;
            const cudaError_t e = cudaStreamEndCapture(s, &g);
            if (st != MPR_OK) {
                if (g) cudaGraphDestroy(g);
                return st;
            }
            if (e != cudaSuccess) return fail(MPR_ERR_CUDA, std::string("capture: ") + cudaGetErrorString(e));
            const cudaError_t ei = cudaGraphInstantiate(&exec, g, 0);
            cudaGraphDestroy(g);
            if (ei != cudaSuccess) return fail(MPR_ERR_CUDA, std::string("instantiate: ") + cudaGetErrorString(ei));
            c->graphs.emplace_back(key, exec);
        }
        MPR_CUDA(cudaGraphLaunch(exec, s));
    }
    c->sweep += (uint32_t)n;
    if (phase == MPR_EQUIL) c->equil_index += (uint32_t)n;
    if (phase != MPR_EQUIL && accumulate) c->n_meas_done += n;
    return MPR_OK;
}

// Device-side error bits (a bounded wait that gave up); blocking.
mpr_status check_device_status(mpr_ctx* c, cudaStream_t s) {
    uint32_t st[2] = {0u, 0u};
    MPR_CUDA(cudaMemcpyAsync(&st[0], &c->d_ctl->status, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
    if (c->sub) MPR_CUDA(cudaMemcpyAsync(&st[1], &c->sub->d_ctl->status, sizeof(uint32_t),
                                         cudaMemcpyDeviceToHost, s));
    MPR_CUDA(cudaStreamSynchronize(s));
    if (st[0] | st[1])
        return fail(MPR_ERR_DEVICE, "a kernel gave up waiting for an asynchronous copy (status " +
                                        std::to_string(st[0] | st[1]) + ")");
    return MPR_OK;
}

}  // namespace

// ================================================================= ABI

extern "C" {

const char* mpr_version(void) { return "mpr-gb300 0.1 (sm_103a)"; }
const char* mpr_last_error(void) { return g_last_error.c_str(); }

const char* mpr_status_string(mpr_status s) {
    switch (s) {
        case MPR_OK: return "ok";
        case MPR_ERR_INVALID_ARG: return "invalid argument";
        case MPR_ERR_CUDA: return "CUDA error";
        case MPR_ERR_DEGENERATE_RANGE: return "degenerate sample range";
        case MPR_ERR_NO_SAMPLE_PAIRS: return "no sample pairs";
        case MPR_ERR_T_OUT_OF_RANGE: return "temperature out of range";
        case MPR_ERR_WORKSPACE: return "workspace error";
        case MPR_ERR_STATE: return "invalid state";
        case MPR_ERR_DEVICE: return "device-side error";
        default: return "unknown status";
    }
}

mpr_status mpr_default_params(mpr_params* p) {
    if (!p) return fail(MPR_ERR_INVALID_ARG, "NULL");
    std::memset(p, 0, sizeof(*p));
    p->q = 0.5;
    p->J = 1.0;
    p->A_targ = 0.3;
    p->k_a = 3.0;
    p->seed = 0x2545F4914F6CDD1DULL;
    p->freeze_a_in_measure = 1;
    p->path = MPR_PATH_TILED;
    p->use_graphs = 1;
    p->model = MPR_MODEL_MPR;
    return MPR_OK;
}

mpr_status mpr_default_T_opts(mpr_T_opts* o) {
    if (!o) return fail(MPR_ERR_INVALID_ARG, "NULL");
    o->L = 0;
    o->chains = 16;
    o->n_equil = 40;
    o->n_meas = 40;
    o->iters = 4;
    o->T_lo = 1e-5;
    o->T_hi = 20.0;
    return MPR_OK;
}

mpr_status mpr_workspace_size(int n_img, const int* Lx, const int* Ly, const int64_t* n_gap,
                              int n_chains, const mpr_params* p, const mpr_T_opts* T_opts,
                              size_t* bytes) {
    if (!bytes) return fail(MPR_ERR_INVALID_ARG, "bytes is NULL");
    MPR_TRY(validate_shapes(n_img, Lx, Ly, n_chains));
    MPR_TRY(check_params(p));
    mpr_T_opts o;
    mpr_default_T_opts(&o);
    if (T_opts) o = *T_opts;
    if (o.chains < 1) return fail(MPR_ERR_INVALID_ARG, "T_opts.chains < 1");
    return workspace_size_impl(n_img, Lx, Ly, n_gap, n_chains, *p, o, true, true, bytes);
}

mpr_status mpr_init_grid(mpr_ctx** out, int n_img, const int* Lx, const int* Ly, int n_chains,
                         const mpr_params* p, const mpr_T_opts* T_opts, const float* z,
                         const uint8_t* gap, mpr_mem where, void* workspace, size_t ws_bytes,
                         mpr_stream stream) {
    if (!out) return fail(MPR_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    MPR_TRY(validate_shapes(n_img, Lx, Ly, n_chains));
    MPR_TRY(check_params(p));
    if (!z || !gap) return fail(MPR_ERR_INVALID_ARG, "z and gap are required");
    if (where != MPR_HOST && where != MPR_DEVICE) return fail(MPR_ERR_INVALID_ARG, "bad mpr_mem");
    mpr_ctx* c = new (std::nothrow) mpr_ctx();
    if (!c) return fail(MPR_ERR_INVALID_ARG, "out of host memory");
    c->p = *p;
    if (p->chain_group > 0 && (p->chain_group & 3) && p->chain_group < n_chains) {
        delete c;
        return fail(MPR_ERR_INVALID_ARG, "chain_group must be a multiple of 4 or cover every "
                                         "chain (pairs share random numbers; rows are 16-byte "
                                         "aligned)");
    }
    mpr_default_T_opts(&c->topt);
    if (T_opts) c->topt = *T_opts;
    if (c->topt.chains < 1 || c->topt.n_meas < 1 || c->topt.iters < 0 || c->topt.n_equil < 0 ||
        !(c->topt.T_lo > 0.0 && c->topt.T_hi > c->topt.T_lo)) {
        delete c;
        return fail(MPR_ERR_INVALID_ARG, "bad temperature-estimate options");
    }
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    mpr_status st = init_impl(c, n_img, Lx, Ly, n_chains, z, gap, where, workspace, ws_bytes, false, s);
    if (st != MPR_OK) { delete c; return st; }
    // unconditional lattices of the temperature estimate
    c->sub = new (std::nothrow) mpr_ctx();
    if (!c->sub) { delete c; return fail(MPR_ERR_INVALID_ARG, "out of host memory"); }
    c->sub->p = c->p;
    c->sub->p.literal_or = 0;
    c->sub->p.path = MPR_PATH_TILED;
    c->sub->p.tile_x = c->sub->p.tile_y = 0;
    c->sub->p.chain_group = 0;
    c->sub->topt = c->topt;
    std::vector<int> LT(n_img);
    for (int i = 0; i < n_img; ++i) LT[i] = default_T_side(Lx[i], Ly[i], c->topt);
    size_t sub_bytes;
    st = sub_workspace_size(c->p, c->topt, n_img, Lx, Ly, &sub_bytes);
    if (st == MPR_OK)
        st = init_impl(c->sub, n_img, LT.data(), LT.data(), c->topt.chains, nullptr, nullptr,
                       MPR_DEVICE, c->ws + c->L.sub, sub_bytes, true, s);
    if (st == MPR_OK) {
        cudaError_t e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) st = fail(MPR_ERR_CUDA, cudaGetErrorString(e));
    }
    if (st != MPR_OK) { delete c; return st; }
    *out = c;
    return MPR_OK;
}

mpr_status mpr_get_image_info(const mpr_ctx* c, double* e_s, int64_t* n_sp, int64_t* n_gap,
                              float* z_min, float* z_max) {
    if (!c) return fail(MPR_ERR_INVALID_ARG, "ctx is NULL");
    for (int i = 0; i < c->g.n_img; ++i) {
        const ImgDev& I = c->h_img[i];
        if (e_s) e_s[i] = I.e_s;
        if (n_sp) n_sp[i] = I.n_sp;
        if (n_gap) n_gap[i] = I.n_gap;
        if (z_min) z_min[i] = I.zmin;
        if (z_max) z_max[i] = I.zmax;
    }
    return MPR_OK;
}

mpr_status mpr_set_T(mpr_ctx* c, const double* T, mpr_stream stream) {
    if (!c || !T) return fail(MPR_ERR_INVALID_ARG, "NULL argument");
    for (int i = 0; i < c->g.n_img; ++i)
        if (!(T[i] > 0.0) || !std::isfinite(T[i])) return fail(MPR_ERR_INVALID_ARG, "T must be positive");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    double* tmp = c->d_newton;  // 4 doubles per image of room
    MPR_CUDA(cudaMemcpyAsync(tmp, T, sizeof(double) * c->g.n_img, cudaMemcpyHostToDevice, s));
    set_T_kernel<<<grid_for(c->g.n_img), 256, 0, s>>>(c->d_img, tmp, c->g.n_img);
    MPR_CUDA(cudaGetLastError());
    MPR_CUDA(cudaStreamSynchronize(s));
    for (int i = 0; i < c->g.n_img; ++i) { c->h_img[i].T = T[i]; c->h_img[i].invT = (float)(1.0 / T[i]); }
    c->T_set = true;
    return MPR_OK;
}

mpr_status mpr_get_T(mpr_ctx* c, double* T, mpr_stream stream) {
    if (!c || !T) return fail(MPR_ERR_INVALID_ARG, "NULL argument");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    std::vector<ImgDev> h(c->g.n_img);
    MPR_CUDA(cudaMemcpyAsync(h.data(), c->d_img, sizeof(ImgDev) * c->g.n_img, cudaMemcpyDeviceToHost, s));
    MPR_CUDA(cudaStreamSynchronize(s));
    for (int i = 0; i < c->g.n_img; ++i) T[i] = h[i].T;
    return check_device_status(c, s);
}

mpr_status mpr_estimate_T(mpr_ctx* c, double* T_out, mpr_stream stream) {
    if (!c || !c->sub) return fail(MPR_ERR_INVALID_ARG, "ctx is NULL");
    const double J = c->p.J;
    for (int i = 0; i < c->g.n_img; ++i) {
        const ImgDev& I = c->h_img[i];
        if (I.n_sp == 0) return fail(MPR_ERR_NO_SAMPLE_PAIRS, "image " + std::to_string(i) + " has no sample pairs");
        // e(T) runs from -J (T = 0) to the independent-angle value: for the MPR
        // bond -J <cos(q dphi)> = -J (sin(pi q) / (pi q))^2 (-4J/pi^2 at q = 1/2),
        // for the GMRF bond J (<dphi^2> / (2 pi^2) - 1) = -2J/3
        const double sq = std::sin(kPiD * c->p.q) / (kPiD * c->p.q);
        const double e_inf = c->p.model == MPR_MODEL_GMRF ? -2.0 * J / 3.0 : -J * sq * sq;
        if (!(I.e_s > -J && I.e_s < e_inf))
            return fail(MPR_ERR_T_OUT_OF_RANGE, "image " + std::to_string(i) +
                                                    ": e_s outside the range of e(T)");
    }
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    mpr_ctx* u = c->sub;
    const int n_img = c->g.n_img;
    const int K = u->g.n_chains;
    newton_init_kernel<<<grid_for(n_img), 256, 0, s>>>(u->d_img, c->d_img, c->d_newton, n_img,
                                                      c->topt.T_lo, c->topt.T_hi, J);
    MPR_CUDA(cudaGetLastError());
    for (int it = 0; it < c->topt.iters; ++it) {
        const int neq = it == 0 ? 2 * c->topt.n_equil : c->topt.n_equil;
        MPR_TRY(run_sweeps(u, neq, MPR_EQUIL, 0, false, false, s));
        MPR_TRY(run_sweeps(u, c->topt.n_meas, MPR_MEASURE, MPR_RECORD_ENERGY, true, false, s));
        newton_kernel<<<grid_for(n_img), 256, 0, s>>>(u->d_img, c->d_img, u->ch, c->d_newton, n_img,
                                                     K, c->topt.n_meas);
        MPR_CUDA(cudaGetLastError());
    }
    c->T_set = true;
    if (T_out) MPR_TRY(mpr_get_T(c, T_out, stream));
    return MPR_OK;
}

mpr_status mpr_sweep(mpr_ctx* c, int n_sweeps, int phase, int flags, mpr_stream stream) {
    if (!c) return fail(MPR_ERR_INVALID_ARG, "ctx is NULL");
    if (n_sweeps < 0) return fail(MPR_ERR_INVALID_ARG, "n_sweeps < 0");
    if (phase != MPR_EQUIL && phase != MPR_MEASURE) return fail(MPR_ERR_INVALID_ARG, "bad phase");
    if (!c->T_set) return fail(MPR_ERR_STATE, "temperature not set: call mpr_estimate_T or mpr_set_T");
    return run_sweeps(c, n_sweeps, phase, flags, false, true, reinterpret_cast<cudaStream_t>(stream));
}

mpr_status mpr_autotune(int n_img, const int* Lx, const int* Ly, int n_chains, mpr_params* p,
                        const float* z, const uint8_t* gap, mpr_mem where, void* workspace,
                        size_t ws_bytes, int sweeps, double* timings, mpr_stream stream) {
    MPR_TRY(validate_shapes(n_img, Lx, Ly, n_chains));
    MPR_TRY(check_params(p));
    if (p->path != MPR_PATH_TILED) return fail(MPR_ERR_INVALID_ARG, "the autotuner serves the tiled path");
    if (!z || !gap || sweeps < 1) return fail(MPR_ERR_INVALID_ARG, "bad arguments");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    static const int tiles[3][2] = {{32, 16}, {16, 16}, {32, 32}};
    const int groups[3] = {0, 16, 8};
    double best = 1e300;
    int bt = -1, bg = 0;
    for (int ti = 0; ti < 3; ++ti) {
        for (int gi = 0; gi < 3; ++gi) {
            double* slot = timings ? timings + ti * 3 + gi : nullptr;
            if (slot) *slot = -1.0;
            int cg = groups[gi];
            if (cg > 0 && cg >= n_chains) continue;  // same as covering every chain
            if (!tiled_model_supported(tiles[ti][0], tiles[ti][1], model_flags(*p))) continue;
            mpr_ctx c;
            c.p = *p;
            c.p.tile_x = tiles[ti][0];
            c.p.tile_y = tiles[ti][1];
            c.p.chain_group = cg;
            c.p.use_graphs = 0;
            mpr_default_T_opts(&c.topt);
            // the candidate must fit the workspace and the tile's per-lane limit
            if (init_impl(&c, n_img, Lx, Ly, n_chains, z, gap, where, workspace, ws_bytes, false,
                          s) != MPR_OK)
                continue;
            std::vector<double> T(n_img);
            for (int i = 0; i < n_img; ++i) {
                const double e_s = std::isfinite(c.h_img[i].e_s) ? c.h_img[i].e_s : -0.9;
                T[i] = std::min(10.0, std::max(1e-4, 4.0 * (e_s + p->J)));
            }
            MPR_TRY(mpr_set_T(&c, T.data(), stream));
            // a candidate whose buffers do not fit the device is skipped
            if (run_sweeps(&c, 1, MPR_EQUIL, 0, false, false, s) != MPR_OK) continue;
            cudaEvent_t e0, e1;
            MPR_CUDA(cudaEventCreate(&e0));
            MPR_CUDA(cudaEventCreate(&e1));
            MPR_CUDA(cudaEventRecord(e0, s));
            const mpr_status st = run_sweeps(&c, sweeps, MPR_EQUIL, 0, false, false, s);
            MPR_CUDA(cudaEventRecord(e1, s));
            MPR_CUDA(cudaEventSynchronize(e1));
            float ms = 0.0f;
            cudaEventElapsedTime(&ms, e0, e1);
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            if (st != MPR_OK) return st;
            MPR_TRY(check_device_status(&c, s));
            const double per = ms / sweeps;
            if (slot) *slot = per;
            if (per < best) { best = per; bt = ti; bg = cg; }
        }
    }
    if (bt < 0) return fail(MPR_ERR_WORKSPACE, "no tile shape fits the workspace");
    p->tile_x = tiles[bt][0];
    p->tile_y = tiles[bt][1];
    p->chain_group = bg;
    return MPR_OK;
}

mpr_status mpr_eT_table_workspace_size(int L, int n_T, int chains, size_t* bytes) {
    if (!bytes || L < 2 || L > 65535 || n_T < 1 || chains < 1 || (long long)n_T * chains > 65535)
        return fail(MPR_ERR_INVALID_ARG, "need 2 <= L <= 65535, n_T >= 1, chains >= 1");
    mpr_params p;
    mpr_default_params(&p);
    mpr_T_opts o;
    mpr_default_T_opts(&o);
    std::vector<int> Ls(n_T, L);
    return workspace_size_impl(n_T, Ls.data(), Ls.data(), nullptr, chains, p, o, false, false, bytes);
}

mpr_status mpr_eT_table(int L, int n_T, const double* T, int chains, int n_equil, int n_meas,
                        const mpr_params* p, void* workspace, size_t ws_bytes, double* e_out,
                        double* var_out, mpr_stream stream) {
    if (!T || !e_out || n_equil < 0 || n_meas < 1) return fail(MPR_ERR_INVALID_ARG, "bad arguments");
    MPR_TRY(check_params(p));
    size_t need = 0;
    MPR_TRY(mpr_eT_table_workspace_size(L, n_T, chains, &need));
    if (ws_bytes < need) return fail(MPR_ERR_WORKSPACE, "workspace too small for the e(T) table");
    for (int k = 0; k < n_T; ++k)
        if (!(T[k] > 0.0) || !std::isfinite(T[k])) return fail(MPR_ERR_INVALID_ARG, "T must be positive");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    mpr_ctx u;
    u.p = *p;
    u.p.path = MPR_PATH_TILED;
    u.p.literal_or = 0;
    u.p.tile_x = u.p.tile_y = 0;
    u.p.chain_group = 0;
    mpr_default_T_opts(&u.topt);
    std::vector<int> Ls(n_T, L);
    MPR_TRY(init_impl(&u, n_T, Ls.data(), Ls.data(), chains, nullptr, nullptr, MPR_DEVICE, workspace,
                      ws_bytes, true, s));
    u.img_tag = 1u << 29;  // a stream of its own
    MPR_CUDA(cudaMemcpyAsync(u.d_newton, T, sizeof(double) * n_T, cudaMemcpyHostToDevice, s));
    set_T_kernel<<<grid_for(n_T), 256, 0, s>>>(u.d_img, u.d_newton, n_T);
    MPR_CUDA(cudaGetLastError());
    MPR_TRY(run_sweeps(&u, n_equil, MPR_EQUIL, 0, false, false, s));
    MPR_TRY(run_sweeps(&u, n_meas, MPR_MEASURE, MPR_RECORD_ENERGY, true, false, s));
    const int nc = n_T * chains;
    std::vector<double> s1(nc), s2(nc);
    MPR_CUDA(cudaMemcpyAsync(s1.data(), u.ch.e_sum, sizeof(double) * nc, cudaMemcpyDeviceToHost, s));
    MPR_CUDA(cudaMemcpyAsync(s2.data(), u.ch.e_sum2, sizeof(double) * nc, cudaMemcpyDeviceToHost, s));
    MPR_CUDA(cudaStreamSynchronize(s));
    MPR_TRY(check_device_status(&u, s));
    for (int k = 0; k < n_T; ++k) {
        double a = 0.0, b = 0.0;
        for (int j = 0; j < chains; ++j) { a += s1[k * chains + j]; b += s2[k * chains + j]; }
        const double n = (double)chains * n_meas;
        e_out[k] = a / n;
        if (var_out) var_out[k] = std::max(b / n - (a / n) * (a / n), 0.0);
    }
    return MPR_OK;
}

mpr_status mpr_set_T_from_table(mpr_ctx* c, int n_T, const double* T, const double* e,
                                double* T_out, mpr_stream stream) {
    if (!c || !T || !e || n_T < 2) return fail(MPR_ERR_INVALID_ARG, "need a table of >= 2 points");
    for (int k = 1; k < n_T; ++k)
        if (!(T[k] > T[k - 1]) || !(e[k] > e[k - 1]))
            return fail(MPR_ERR_INVALID_ARG, "the table must increase in T and in e");
    std::vector<double> out(c->g.n_img);
    for (int i = 0; i < c->g.n_img; ++i) {
        const double es = c->h_img[i].e_s;
        if (c->h_img[i].n_sp == 0) return fail(MPR_ERR_NO_SAMPLE_PAIRS, "image without sample pairs");
        if (!(es >= e[0] && es <= e[n_T - 1]))
            return fail(MPR_ERR_T_OUT_OF_RANGE, "e_s of image " + std::to_string(i) +
                                                    " lies outside the table");
        int k = 0;
        while (k + 2 < n_T && e[k + 1] < es) ++k;
        // linear in (e, log T) between the bracketing points
        const double w = (es - e[k]) / (e[k + 1] - e[k]);
        out[i] = std::exp(std::log(T[k]) + w * (std::log(T[k + 1]) - std::log(T[k])));
    }
    MPR_TRY(mpr_set_T(c, out.data(), stream));
    if (T_out) std::copy(out.begin(), out.end(), T_out);
    return MPR_OK;
}

mpr_status mpr_equilibrate(mpr_ctx* c, int n_f, int n_fit, int i_max, int* n_done,
                           mpr_stream stream) {
    if (!c) return fail(MPR_ERR_INVALID_ARG, "ctx is NULL");
    if (n_f < 1 || n_fit < 2 || n_fit > kHist || i_max < 1)
        return fail(MPR_ERR_INVALID_ARG, "need n_f >= 1, 2 <= n_fit <= 512, i_max >= 1");
    if (!c->T_set) return fail(MPR_ERR_STATE, "temperature not set: call mpr_estimate_T or mpr_set_T");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const int n_img = c->g.n_img;
    MPR_CUDA(cudaMemsetAsync(c->d_sg, 0, sizeof(int) * (n_img + 3), s));
    int done = 0;
    if (graphs_usable(c, s)) {
        // the whole run as one graph: a while node whose body is one sweep and the
        // stop rule, which sets the loop's condition on the device (no host round
        // trip per check)
        const long long key = ((long long)n_f << 42) | ((long long)n_fit << 32) | (long long)i_max;
        if (!c->eq_exec || c->eq_key != key) {
            if (c->eq_exec) cudaGraphExecDestroy(c->eq_exec);
            c->eq_exec = nullptr;
            MPR_TRY(prepare_capture(c, s));
            cudaGraph_t g = nullptr;
            MPR_CUDA(cudaGraphCreate(&g, 0));
            cudaGraphConditionalHandle h;
            cudaGraphNode_t node;
            cudaGraphNodeParams np{};
            np.type = cudaGraphNodeTypeConditional;
            cudaError_t e = cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault);
            if (e == cudaSuccess) {
                np.conditional.handle = h;
                np.conditional.type = cudaGraphCondTypeWhile;
                np.conditional.size = 1;
                e = cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &np);
            }
            mpr_status st = MPR_OK;
            if (e == cudaSuccess)
                e = cudaStreamBeginCaptureToGraph(s, np.conditional.phGraph_out[0], nullptr, nullptr,
                                                  0, cudaStreamCaptureModeThreadLocal);
            if (e == cudaSuccess) {
                st = launch_sweeps(c, 1, MPR_EQUIL, MPR_RECORD_ENERGY, false, true, s);
                if (st == MPR_OK) {
                    sg_step_kernel<<<1, 256, 0, s>>>(c->ch, c->d_hist, c->d_sg, n_img, c->g.n_chains,
                                                     n_fit, n_f, i_max, h, 1);
                    e = cudaGetLastError();
                }
                cudaGraph_t body = nullptr;
                const cudaError_t ee = cudaStreamEndCapture(s, &body);
                if (e == cudaSuccess) e = ee;
            }
            if (st == MPR_OK && e == cudaSuccess) e = cudaGraphInstantiate(&c->eq_exec, g, 0);
            cudaGraphDestroy(g);
            if (st != MPR_OK) return st;
            if (e != cudaSuccess)
                return fail(MPR_ERR_CUDA, std::string("equilibration graph: ") + cudaGetErrorString(e));
            c->eq_key = key;
        }
        MPR_CUDA(cudaGraphLaunch(c->eq_exec, s));
        MPR_CUDA(cudaMemcpyAsync(&done, c->d_sg + n_img + 1, sizeof(int), cudaMemcpyDeviceToHost, s));
        MPR_CUDA(cudaStreamSynchronize(s));
        c->sweep += (uint32_t)done;
        c->equil_index += (uint32_t)done;
    } else {
        for (int i = 0; i <= i_max; ++i) {
            // sweep i of this equilibration (Alg. 2 step 4.1-4.3), energies recorded
            MPR_TRY(run_sweeps(c, 1, MPR_EQUIL, MPR_RECORD_ENERGY, false, true, s));
            sg_step_kernel<<<1, 256, 0, s>>>(c->ch, c->d_hist, c->d_sg, n_img, c->g.n_chains, n_fit,
                                             n_f, i_max, cudaGraphConditionalHandle{}, 0);
            MPR_CUDA(cudaGetLastError());
            done = i + 1;
            if (i >= n_fit && i % n_f == 0) {
                int stop = 0;
                MPR_CUDA(cudaMemcpyAsync(&stop, c->d_sg + n_img + 2, sizeof(int), cudaMemcpyDeviceToHost, s));
                MPR_CUDA(cudaStreamSynchronize(s));
                if (stop) break;
            }
        }
    }
    if (n_done) *n_done = done;
    return check_device_status(c, s);
}

mpr_status mpr_sweep_launches(const mpr_ctx* c, int* per_sweep, int* per_T_sweep) {
    if (!c || !per_sweep) return fail(MPR_ERR_INVALID_ARG, "NULL argument");
    *per_sweep = sweep_launch_count(c);
    if (per_T_sweep) *per_T_sweep = c->sub ? sweep_launch_count(c->sub) : 0;
    return MPR_OK;
}

mpr_status mpr_get_energy_history(mpr_ctx* c, double* out, mpr_stream stream) {
    static_assert(kHist == MPR_HISTORY, "history length");
    if (!c || !out) return fail(MPR_ERR_INVALID_ARG, "NULL argument");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    MPR_CUDA(cudaMemcpyAsync(out, c->d_hist, sizeof(double) * kHist * c->g.n_img,
                             cudaMemcpyDeviceToHost, s));
    MPR_CUDA(cudaStreamSynchronize(s));
    return MPR_OK;
}

mpr_status mpr_energy(mpr_ctx* c, double* e_out, mpr_mem where, mpr_stream stream) {
    if (!c || !e_out) return fail(MPR_ERR_INVALID_ARG, "NULL argument");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const int nc = c->g.n_img * c->g.n_chains;
    double* d_out = where == MPR_DEVICE ? e_out : c->d_eout;
    MPR_CUDA(cudaMemsetAsync(d_out, 0, sizeof(double) * nc, s));
    long long maxn = 0;
    for (int i = 0; i < c->g.n_img; ++i) maxn = std::max(maxn, (long long)c->g.Lx[i] * c->g.Ly[i]);
    energy_kernel<<<dim3(grid_for(maxn, 256, 512), nc), 256, 0, s>>>(
        c->d_img, c->d_state, c->d_samp, c->d_slot_map, c->g.path == MPR_PATH_TILED ? 1 : 0,
        c->g.n_chains, (float)c->p.q, (float)c->p.J, c->p.model == MPR_MODEL_GMRF ? 1 : 0, d_out);
    MPR_CUDA(cudaGetLastError());
    energy_finish_kernel<<<grid_for(nc), 256, 0, s>>>(c->d_img, d_out, c->g.n_chains, nc);
    MPR_CUDA(cudaGetLastError());
    if (where == MPR_HOST) {
        MPR_CUDA(cudaMemcpyAsync(e_out, d_out, sizeof(double) * nc, cudaMemcpyDeviceToHost, s));
        MPR_CUDA(cudaStreamSynchronize(s));
    }
    return MPR_OK;
}

mpr_status mpr_predict(mpr_ctx* c, float* z_hat, float* z_std, mpr_mem where, mpr_stream stream) {
    if (!c || !z_hat) return fail(MPR_ERR_INVALID_ARG, "NULL argument");
    if (c->n_meas_done == 0) return fail(MPR_ERR_STATE, "no measurement sweep has run");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const size_t N = (size_t)c->g.n_sites;
    float* dh = where == MPR_DEVICE ? z_hat : c->d_out;
    float* ds = where == MPR_DEVICE ? z_std : (z_std ? c->d_out + N : nullptr);
    long long maxn = 0;
    for (int i = 0; i < c->g.n_img; ++i) maxn = std::max(maxn, (long long)c->g.Lx[i] * c->g.Ly[i]);
    predict_kernel<<<dim3(grid_for(maxn, 256, 2048), c->g.n_img), 256, 0, s>>>(
        c->d_img, c->d_acc1, c->d_acc2, c->d_zst, c->d_slot_map, c->d_samp,
        c->g.path == MPR_PATH_TILED ? 1 : 0, (double)c->n_meas_done * c->g.n_chains, dh, ds);
    MPR_CUDA(cudaGetLastError());
    if (where == MPR_HOST) {
        MPR_CUDA(cudaMemcpyAsync(z_hat, dh, sizeof(float) * N, cudaMemcpyDeviceToHost, s));
        if (z_std) MPR_CUDA(cudaMemcpyAsync(z_std, ds, sizeof(float) * N, cudaMemcpyDeviceToHost, s));
        MPR_CUDA(cudaStreamSynchronize(s));
        return check_device_status(c, s);
    }
    return MPR_OK;
}

mpr_status mpr_reset_accumulators(mpr_ctx* c, mpr_stream stream) {
    if (!c) return fail(MPR_ERR_INVALID_ARG, "ctx is NULL");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    MPR_CUDA(cudaMemsetAsync(c->d_acc1, 0, sizeof(double) * c->L.n_slots, s));
    MPR_CUDA(cudaMemsetAsync(c->d_acc2, 0, sizeof(double) * c->L.n_slots, s));
    c->n_meas_done = 0;
    return MPR_OK;
}

// One accumulator array <-> a dense [sum Lx*Ly] double array (host buffers
// go through the output staging area, 8 bytes per pixel).
static mpr_status acc_copy(mpr_ctx* c, double* acc, double* dense, mpr_mem where, int dir,
                           cudaStream_t s) {
    const size_t N = (size_t)c->g.n_sites;
    double* d = where == MPR_DEVICE ? dense : reinterpret_cast<double*>(c->d_out);
    if (where == MPR_HOST && dir == 1)
        MPR_CUDA(cudaMemcpyAsync(d, dense, sizeof(double) * N, cudaMemcpyHostToDevice, s));
    long long maxn = 0;
    for (int i = 0; i < c->g.n_img; ++i) maxn = std::max(maxn, (long long)c->g.Lx[i] * c->g.Ly[i]);
    acc_dense_kernel<<<dim3(grid_for(maxn, 256, 1024), c->g.n_img), 256, 0, s>>>(
        c->d_img, acc, c->d_slot_map, c->d_samp, c->g.path == MPR_PATH_TILED ? 1 : 0, d, dir);
    MPR_CUDA(cudaGetLastError());
    if (where == MPR_HOST) {
        if (dir == 0) MPR_CUDA(cudaMemcpyAsync(dense, d, sizeof(double) * N, cudaMemcpyDeviceToHost, s));
        MPR_CUDA(cudaStreamSynchronize(s));
    }
    return MPR_OK;
}

mpr_status mpr_get_accumulators(mpr_ctx* c, double* sum, double* sum2, int64_t* n_terms,
                                mpr_mem where, mpr_stream stream) {
    if (!c) return fail(MPR_ERR_INVALID_ARG, "ctx is NULL");
    if (where != MPR_HOST && where != MPR_DEVICE) return fail(MPR_ERR_INVALID_ARG, "bad mpr_mem");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if (sum) MPR_TRY(acc_copy(c, c->d_acc1, sum, where, 0, s));
    if (sum2) MPR_TRY(acc_copy(c, c->d_acc2, sum2, where, 0, s));
    if (n_terms) *n_terms = (int64_t)c->n_meas_done * c->g.n_chains;
    return MPR_OK;
}

mpr_status mpr_set_accumulators(mpr_ctx* c, const double* sum, const double* sum2,
                                int64_t n_terms, mpr_mem where, mpr_stream stream) {
    if (!c || !sum) return fail(MPR_ERR_INVALID_ARG, "NULL argument");
    if (where != MPR_HOST && where != MPR_DEVICE) return fail(MPR_ERR_INVALID_ARG, "bad mpr_mem");
    if (n_terms < 0 || n_terms % c->g.n_chains != 0)
        return fail(MPR_ERR_INVALID_ARG, "n_terms must be a multiple of the chain count");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    MPR_CUDA(cudaMemsetAsync(c->d_acc1, 0, sizeof(double) * c->L.n_slots, s));
    MPR_CUDA(cudaMemsetAsync(c->d_acc2, 0, sizeof(double) * c->L.n_slots, s));
    MPR_TRY(acc_copy(c, c->d_acc1, const_cast<double*>(sum), where, 1, s));
    if (sum2) MPR_TRY(acc_copy(c, c->d_acc2, const_cast<double*>(sum2), where, 1, s));
    c->n_meas_done = n_terms / c->g.n_chains;
    return MPR_OK;
}

static mpr_status state_copy(mpr_ctx* c, float* phi, mpr_mem where, int dir, cudaStream_t s) {
    const int tiled = c->g.path == MPR_PATH_TILED ? 1 : 0;
    const int nc = c->g.n_img * c->g.n_chains;
    if (where == MPR_DEVICE) {
        long long maxn = 0;
        for (int i = 0; i < c->g.n_img; ++i) maxn = std::max(maxn, (long long)c->g.Lx[i] * c->g.Ly[i]);
        state_copy_kernel<<<dim3(grid_for(maxn, 256, 1024), nc), 256, 0, s>>>(
            c->d_img, c->d_state, c->d_samp, c->d_slot_map, tiled, c->g.n_chains, phi, dir, 0,
            nullptr);
        MPR_CUDA(cudaGetLastError());
        return MPR_OK;
    }
    // host buffers: one (image, chain) plane at a time through the output staging area
    float* stage = c->d_out;
    for (int ic = 0; ic < nc; ++ic) {
        const int im = ic / c->g.n_chains, chain = ic - im * c->g.n_chains;
        const long long n = (long long)c->g.Lx[im] * c->g.Ly[im];
        float* h = phi + c->g.site_off[im] * c->g.n_chains + (long long)chain * n;
        if (dir == 1) MPR_CUDA(cudaMemcpyAsync(stage, h, sizeof(float) * n, cudaMemcpyHostToDevice, s));
        state_copy_kernel<<<dim3(grid_for(n, 256, 1024), 1), 256, 0, s>>>(
            c->d_img, c->d_state, c->d_samp, c->d_slot_map, tiled, c->g.n_chains, nullptr, dir, ic,
            stage);
        MPR_CUDA(cudaGetLastError());
        if (dir == 0) MPR_CUDA(cudaMemcpyAsync(h, stage, sizeof(float) * n, cudaMemcpyDeviceToHost, s));
    }
    MPR_CUDA(cudaStreamSynchronize(s));
    return MPR_OK;
}

mpr_status mpr_get_state(mpr_ctx* c, float* phi, mpr_mem where, mpr_stream stream) {
    if (!c || !phi) return fail(MPR_ERR_INVALID_ARG, "NULL argument");
    return state_copy(c, phi, where, 0, reinterpret_cast<cudaStream_t>(stream));
}

mpr_status mpr_set_state(mpr_ctx* c, const float* phi, mpr_mem where, mpr_stream stream) {
    if (!c || !phi) return fail(MPR_ERR_INVALID_ARG, "NULL argument");
    return state_copy(c, const_cast<float*>(phi), where, 1, reinterpret_cast<cudaStream_t>(stream));
}

mpr_status mpr_get_chain_info(mpr_ctx* c, float* a, uint32_t* accepted, double* e_last,
                              mpr_stream stream) {
    if (!c) return fail(MPR_ERR_INVALID_ARG, "ctx is NULL");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const int nc = c->g.n_img * c->g.n_chains;
    if (a) MPR_CUDA(cudaMemcpyAsync(a, c->ch.a, sizeof(float) * nc, cudaMemcpyDeviceToHost, s));
    if (accepted) MPR_CUDA(cudaMemcpyAsync(accepted, c->ch.acc_last, sizeof(uint32_t) * nc, cudaMemcpyDeviceToHost, s));
    if (e_last) MPR_CUDA(cudaMemcpyAsync(e_last, c->ch.e_last, sizeof(double) * nc, cudaMemcpyDeviceToHost, s));
    MPR_CUDA(cudaStreamSynchronize(s));
    return check_device_status(c, s);
}

mpr_status mpr_set_chain_a(mpr_ctx* c, const float* a, mpr_stream stream) {
    if (!c || !a) return fail(MPR_ERR_INVALID_ARG, "NULL argument");
    const int nc = c->g.n_img * c->g.n_chains;
    for (int i = 0; i < nc; ++i)
        if (!(a[i] >= 1.0f) || !std::isfinite(a[i])) return fail(MPR_ERR_INVALID_ARG, "a must be >= 1");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    MPR_CUDA(cudaMemcpyAsync(c->ch.a, a, sizeof(float) * nc, cudaMemcpyHostToDevice, s));
    set_alpha_kernel<<<grid_for(nc), 256, 0, s>>>(c->ch, nc);
    MPR_CUDA(cudaGetLastError());
    MPR_CUDA(cudaStreamSynchronize(s));
    return MPR_OK;
}

mpr_status mpr_get_sweep_index(const mpr_ctx* c, uint32_t* sweep, uint32_t* equil_index) {
    if (!c) return fail(MPR_ERR_INVALID_ARG, "ctx is NULL");
    if (sweep) *sweep = c->sweep;
    if (equil_index) *equil_index = c->equil_index;
    return MPR_OK;
}

mpr_status mpr_set_sweep_index(mpr_ctx* c, uint32_t sweep, uint32_t equil_index, mpr_stream stream) {
    if (!c) return fail(MPR_ERR_INVALID_ARG, "ctx is NULL");
    Control h{sweep, equil_index, 0u, 0u};
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    MPR_CUDA(cudaMemcpyAsync(c->d_ctl, &h, sizeof(Control), cudaMemcpyHostToDevice, s));
    MPR_CUDA(cudaStreamSynchronize(s));
    c->sweep = sweep;
    c->equil_index = equil_index;
    return MPR_OK;
}

void mpr_destroy(mpr_ctx* c) { delete c; }

}  // extern "C"
