/*
 * mpr.h -- C ABI of the GB300 library for gap filling with the modified
 * planar rotator (MPR) Gibbs Markov random field (Zukovic & Hristopulos,
 * arXiv:1710.03038).
 *
 * Conventions (all entry points):
 *  - Every function returns an mpr_status (MPR_OK = 0) and never throws.
 *    mpr_last_error() returns a static, thread-local description of the last
 *    failure in the calling thread.
 *  - Device buffers are owned by the caller.  The library allocates no
 *    device memory: the caller queries mpr_workspace_size(), allocates one
 *    device workspace and passes it to mpr_init_grid(); the context keeps
 *    pointers into it and only a small host-side descriptor of its own.
 *  - Functions taking an mpr_stream enqueue their work on that stream and
 *    return without waiting unless stated otherwise ("blocking").  Outputs
 *    written to device memory are valid once the stream has reached that
 *    point.  Host outputs are written before the function returns.
 *  - Image data are passed as the row-major images concatenated in order:
 *    image i starts at element sum_{k<i} Lx[k] * Ly[k].
 *  - Angles are single precision radians; energies and temperatures are
 *    double precision.
 *  - An mpr_ctx is not thread safe; distinct contexts are independent.
 */
#ifndef MPR_H
#define MPR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int mpr_status;
#define MPR_OK                   0
#define MPR_ERR_INVALID_ARG      1  /* null pointer, bad size or flag            */
#define MPR_ERR_CUDA             2  /* a CUDA runtime call failed                */
#define MPR_ERR_DEGENERATE_RANGE 3  /* an image has z_max == z_min over samples  */
#define MPR_ERR_NO_SAMPLE_PAIRS  4  /* no sample-sample bond: e_s undefined      */
#define MPR_ERR_T_OUT_OF_RANGE   5  /* e_s outside the range of e(T)              */
#define MPR_ERR_WORKSPACE        6  /* workspace missing, misaligned or too small */
#define MPR_ERR_STATE            7  /* call not valid in the context's state      */
#define MPR_ERR_DEVICE           8  /* a kernel reported an error (status word)   */

/* A CUDA stream (binary compatible with cudaStream_t); NULL = legacy stream. */
typedef struct CUstream_st* mpr_stream;

typedef struct mpr_ctx mpr_ctx;

/* Where a user buffer lives. */
typedef enum { MPR_DEVICE = 0, MPR_HOST = 1 } mpr_mem;

/* Kernel family used by a context. */
typedef enum {
    MPR_PATH_TILED = 0,  /* batched: compact gap state, tile-major, chain-inner loop */
    MPR_PATH_PLAIN = 1   /* dense per-chain planes, one thread per site, two passes  */
} mpr_path;

/* Pair interaction: the MPR bond -J cos(q dphi) (Eq. Hamiltonian_mod) or the
 * GMRF bond J (dphi^2 / (2 pi^2) - 1) of Sec. 4.3. */
typedef enum { MPR_MODEL_MPR = 0, MPR_MODEL_GMRF = 1 } mpr_model;

/* Sweep phases of Alg. 2: equilibration (step 4, a adapted) and sampling
 * (step 5, a frozen, realisations accumulated). */
typedef enum { MPR_EQUIL = 0, MPR_MEASURE = 1 } mpr_phase;

/* Flags of mpr_sweep. */
#define MPR_RECORD_ENERGY 1  /* reduce H / N_GP of every chain after every sweep (Alg. 2 step 4.3) */

/* Model and simulation parameters (Sec. 2.2, 2.5).  mpr_default_params()
 * fills the paper's values. */
typedef struct {
    double q;                /* modification factor of Eq. Hamiltonian_mod, 0 < q <= 1/2; 0.5 */
    double J;                /* exchange interaction J > 0; 1                                  */
    double A_targ;           /* target acceptance ratio of Alg. 2 step 4.2; 0.3                */
    double k_a;              /* rate of the perturbation control factor a; 3                   */
    uint64_t seed;           /* Philox key (64 bits)                                           */
    int freeze_a_in_measure; /* 1: keep the last equilibration a while sampling; 0: a = 1
                                as printed in Alg. 2 step 5.2                                   */
    int path;                /* mpr_path                                                       */
    int tile_x, tile_y;      /* tiled path tile shape (16x16, 32x16 or 32x32); 0 = 16x16
                                (mpr_autotune times all three)                                 */
    int chain_group;         /* tiled path: chains per thread block, a multiple of 4 or
                                >= n_chains; values above 32 act as 32; 0 = automatic          */
    int literal_or;          /* 1: over-relaxation as printed in Eq. over-relax (q = 1 field,
                                always applied), for comparison; tiled path: 16x16 tiles; 0    */
    int use_graphs;          /* 1: runs of 4 or more sweeps on a non-default stream are captured
                                once into a CUDA graph and replayed; 1                         */
    int model;               /* mpr_model (MPR_MODEL_GMRF: the over-relaxation reflects about
                                the neighbour mean; tiled path: 16x16 tiles); MPR              */
} mpr_params;

/* Options of the specific-energy-matching temperature estimate (Sec. 2.3). */
typedef struct {
    int L;                 /* side of the unconditional lattice for e(T); 0: min(256, image side) */
    int chains;            /* independent unconditional chains per image; 16                     */
    int n_equil;           /* sweeps after each temperature change (twice that from the hot
                              start); 40                                                         */
    int n_meas;            /* sweeps averaged for <e> and Var(e) per iteration; 40               */
    int iters;             /* Newton iterations; 4                                               */
    double T_lo, T_hi;     /* safeguarding bracket; 1e-5, 20                                      */
} mpr_T_opts;

const char* mpr_version(void);
const char* mpr_last_error(void);
const char* mpr_status_string(mpr_status s);

mpr_status mpr_default_params(mpr_params* p);
mpr_status mpr_default_T_opts(mpr_T_opts* o);

/* Bytes of device workspace a context needs (Sec. 2.5 state: angles of every
 * realisation, accumulators, tile tables, the unconditional lattices of the
 * temperature estimate and input/output staging).
 *  n_img       number of images, >= 1
 *  Lx, Ly      host [n_img] image sizes, 2 <= Lx <= 65535, 2 <= Ly <= 65535
 *  n_gap       host [n_img] number of missing pixels per image, or NULL to
 *              size for the worst case (every pixel missing)
 *  n_chains    realisations per image, >= 1
 *  p, T_opts   the parameters the context will use (T_opts may be NULL for
 *              the defaults)
 *  bytes       out: required size; the workspace must be 256-byte aligned. */
mpr_status mpr_workspace_size(int n_img, const int* Lx, const int* Ly, const int64_t* n_gap,
                              int n_chains, const mpr_params* p, const mpr_T_opts* T_opts,
                              size_t* bytes);

/* Alg. 2 steps 1-2 and 3.1 for a batch of images: maps the sample values to
 * angles with Eq. map (extremes over sample sites), builds the gap layout,
 * draws the hot start of every realisation (gap angles ~ U(0, 2 pi), step
 * 1.8), sets a = 1, and computes the sample specific energy e_s of
 * Eq. mpr-sse (mean over unordered sample-sample bonds; FP32 bond terms
 * summed in FP64).
 *  z       [sum Lx*Ly] float values; entries at gap pixels are ignored
 *  gap     [sum Lx*Ly] uint8, nonzero = missing
 *  where   whether z and gap are host or device pointers
 *  workspace, ws_bytes  caller-owned device memory of mpr_workspace_size() bytes
 * Blocking.  Errors: INVALID_ARG, WORKSPACE (too small for the actual gap
 * counts), DEGENERATE_RANGE (fewer than two distinct sample values).
 * On success *out owns no device memory; release it with mpr_destroy(). */
mpr_status mpr_init_grid(mpr_ctx** out, int n_img, const int* Lx, const int* Ly, int n_chains,
                         const mpr_params* p, const mpr_T_opts* T_opts,
                         const float* z, const uint8_t* gap, mpr_mem where,
                         void* workspace, size_t ws_bytes, mpr_stream stream);

/* Autotuner of the tiled path: times `sweeps` equilibration sweeps of the
 * given batch (after one warm-up sweep, temperature from the harmonic guess
 * 4 (e_s + J)) for each candidate tile shape (32x16, 16x16, 32x32) and chain
 * group (automatic, 16, 8) that fits `workspace`, and writes the fastest into
 * p->tile_x, tile_y, chain_group.  The chain group also sets the sites per
 * thread: a lane takes one chain pair of a site, so a warp step covers
 * 64 / group sites and a thread updates about (own-colour gap sites of the
 * tile) x group / (2 x threads per block) sites per launch (6.4, 3.2 and 1.6
 * for groups of 32, 16 and 8 on 16x16 tiles with 40% gaps).  timings (nullable, host [9]) receives
 * milliseconds per sweep, tile-major, -1 for skipped candidates.  The
 * workspace is scratch here (size it with mpr_workspace_size for 16x16
 * tiles, the largest layout).  Blocking; the batch itself is not changed. */
mpr_status mpr_autotune(int n_img, const int* Lx, const int* Ly, int n_chains, mpr_params* p,
                        const float* z, const uint8_t* gap, mpr_mem where, void* workspace,
                        size_t ws_bytes, int sweeps, double* timings, mpr_stream stream);

/* Host copy of what init computed per image: e_s (nan when N_SP = 0), N_SP,
 * P (gap count), z_min, z_max.  Any pointer may be NULL. */
mpr_status mpr_get_image_info(const mpr_ctx* ctx, double* e_s, int64_t* n_sp, int64_t* n_gap,
                              float* z_min, float* z_max);

/* Specific energy matching (Sec. 2.3, Alg. 2 step 3): for every image finds
 * T with e(T, L_T) = e_s, where e(T, L_T) = <H>/N_GP of an unconditional
 * simulation on an L_T x L_T lattice started cold (every angle pi; Sec. 2.5
 * names this start among those tested).  Newton iterations on the device use
 * the fluctuation relation d<e>/dT = N_GP Var(e) / T^2, safeguarded by a
 * bracket; every iteration re-equilibrates the lattices (warm start) and
 * averages n_meas sweeps over all chains.  The result becomes the context's
 * temperature.  T_out: host [n_img] (blocking) or NULL (asynchronous).
 * Errors: NO_SAMPLE_PAIRS, T_OUT_OF_RANGE (e_s <= -J, or e_s at or above the
 * infinite-temperature value: -J (sin(pi q) / (pi q))^2 for the MPR bond,
 * -4J/pi^2 at q = 1/2; -2J/3 for the GMRF bond). */
mpr_status mpr_estimate_T(mpr_ctx* ctx, double* T_out, mpr_stream stream);

/* The equilibrium specific energy e(T, L) of Eq. ene as a table (Sec. 2.3:
 * computed once, then inverted for every sample): one unconditional L x L
 * lattice per temperature T[k] (host [n_T], positive), `chains` chains each,
 * cold start, n_equil sweeps with the a-adaptation, then the mean (e_out,
 * host [n_T]) and variance (var_out, nullable) of H/N_GP over n_meas sweeps
 * and all chains.  The lattices live in a caller workspace of
 * mpr_eT_table_workspace_size() bytes.  Blocking. */
mpr_status mpr_eT_table_workspace_size(int L, int n_T, int chains, size_t* bytes);
mpr_status mpr_eT_table(int L, int n_T, const double* T, int chains, int n_equil, int n_meas,
                        const mpr_params* p, void* workspace, size_t ws_bytes, double* e_out,
                        double* var_out, mpr_stream stream);

/* T_hat = e^-1(e_s | L) from a table (T, e) increasing in both (host [n_T]):
 * linear interpolation in (e, log T) at every image's e_s, which becomes the
 * context's temperature (T_out host [n_img], nullable).  Errors:
 * T_OUT_OF_RANGE when e_s lies outside the table, NO_SAMPLE_PAIRS. */
mpr_status mpr_set_T_from_table(mpr_ctx* ctx, int n_T, const double* T, const double* e,
                                double* T_out, mpr_stream stream);

/* Cross-validated choice of the modification factor q for one Lx x Ly image.
 * The conclusions name choosing q in (0, 1/2] by cross-validation, instead of
 * fixing q = 1/2, as an extension of the method; the procedure here follows the
 * paper's validation design (Sec. 3: a set-aside portion of the samples is the
 * validation set, the absolute error averaged over it scores a prediction).
 * For each candidate q[k] (host [n_q], each in (0, 1/2]):
 *   1. the samples flagged in `holdout` become gaps next to the image's own
 *      gaps (flags on gap pixels are ignored); the angle map uses the extremes
 *      of the remaining samples;
 *   2. the gap fill of Alg. 2 at q[k] with the parameters p (seed included, the
 *      same for every candidate): sample specific energy of the remaining
 *      samples, SEM temperature (mpr_estimate_T with T_opts), n_equil
 *      equilibration and n_meas sampling sweeps of n_chains realisations,
 *      prediction;
 *   3. scores[k] = mean over validation points of |z_hat - z| (FP64 sum).
 * A candidate with no SEM temperature (e_s outside the range of e(T) at that q)
 * scores +inf and gets T_out[k] = nan.  *q_best (nullable) receives the first
 * candidate with the smallest score; T_out (nullable, host [n_q]) the SEM
 * temperatures.
 *  z, gap, holdout  [Lx*Ly] float / uint8 / uint8 (nonzero = validation
 *                   point), host or device as `where` says
 *  p                p->model must be MPR_MODEL_MPR and p->literal_or 0
 *  workspace        caller-owned device memory of
 *                   mpr_select_q_workspace_size() bytes, 256-byte aligned; it
 *                   holds one context at a time and the staged inputs
 * Blocking.  Errors: INVALID_ARG (bad sizes, q outside (0, 1/2], no validation
 * point), WORKSPACE, DEGENERATE_RANGE / NO_SAMPLE_PAIRS from the init of the
 * reduced sample set, T_OUT_OF_RANGE when no candidate has a SEM temperature. */
mpr_status mpr_select_q_workspace_size(int Lx, int Ly, int n_chains, const mpr_params* p,
                                       const mpr_T_opts* T_opts, size_t* bytes);
mpr_status mpr_select_q(int Lx, int Ly, const float* z, const uint8_t* gap, const uint8_t* holdout,
                        mpr_mem where, int n_q, const double* q, int n_chains, int n_equil,
                        int n_meas, const mpr_params* p, const mpr_T_opts* T_opts, void* workspace,
                        size_t ws_bytes, double* scores, double* T_out, double* q_best,
                        mpr_stream stream);

/* Kernel launches one sweep of the context issues (per_sweep) and one sweep of
 * its temperature lattices (per_T_sweep, nullable; 0 without lattices): per
 * colour pass one launch for the tiles whose tables fit the blocks per SM the
 * threads allow, one for the rest when there are any, one for the chains left
 * over by the chain groups when there are any, and one bookkeeping launch per
 * sweep (the plain path: two passes and the bookkeeping).  A graph replay of n
 * sweeps runs n times that many kernels.  Host only. */
mpr_status mpr_sweep_launches(const mpr_ctx* ctx, int* per_sweep, int* per_T_sweep);

/* Sets / reads the reduced temperature of every image (host [n_img]). */
mpr_status mpr_set_T(mpr_ctx* ctx, const double* T, mpr_stream stream);
mpr_status mpr_get_T(mpr_ctx* ctx, double* T, mpr_stream stream);

/* n_sweeps hybrid sweeps (Alg. 1) of every realisation on the red/black
 * checkerboard (red = (x + y) even first).  Each gap site gets the
 * over-relaxation reflection (Eq. over-relax, q-consistent), then the
 * restricted Metropolis proposal phi'' = (phi' + 2 pi (u - 1/2)/a) mod 2 pi
 * accepted with probability min(1, exp(-dH/T)).  phase MPR_EQUIL applies
 * Alg. 2 step 4.2 after every sweep (a <- 1 + (i+1)/k_a when the chain's
 * acceptance ratio is below A_targ, i the equilibration sweep index);
 * MPR_MEASURE keeps a and adds every sweep's angles to the realisation
 * accumulators (Alg. 2 step 5).  flags: MPR_RECORD_ENERGY.  Asynchronous. */
mpr_status mpr_sweep(mpr_ctx* ctx, int n_sweeps, int phase, int flags, mpr_stream stream);

/* Equilibration with the automatic stop of Alg. 2 step 4 (Sec. 2.4-2.5):
 * equilibration sweeps i = 0, 1, ... with energies recorded; once i >= n_fit,
 * every n_f sweeps (i mod n_f == 0) the slope of the least-squares line
 * (a Savitzky-Golay fit of degree 1) through the last n_fit chain-averaged
 * specific energies of each image is taken; the run stops after the first
 * check at which no image has a negative slope, or after sweep i_max.
 * Paper defaults n_f = 5, n_fit = 20.  Blocking (one 4-byte read per check).
 * n_done (nullable) receives the number of sweeps run.  2 <= n_fit <= 512. */
mpr_status mpr_equilibrate(mpr_ctx* ctx, int n_f, int n_fit, int i_max, int* n_done,
                           mpr_stream stream);

/* The chain-averaged specific energies recorded by the last mpr_equilibrate:
 * out host [n_img * MPR_HISTORY], image-major, entry (i mod MPR_HISTORY) for
 * sweep i.  Blocking. */
#define MPR_HISTORY 512
mpr_status mpr_get_energy_history(mpr_ctx* ctx, double* out, mpr_stream stream);

/* Specific energy H/N_GP (Eq. ene, FP64) of every realisation in its current
 * state, e_out [n_img * n_chains] (image-major) on the host (blocking) or the
 * device (asynchronous). */
mpr_status mpr_energy(mpr_ctx* ctx, double* e_out, mpr_mem where, mpr_stream stream);

/* Prediction = conditional mean over realisations (Sec. 3; Alg. 2 steps
 * 5.3 and 6): for gap pixels z_min + (z_max - z_min) * mean(phi) / (2 pi),
 * the mean over every chain and every measurement sweep; sample pixels
 * return their value.  z_std (nullable) receives the standard deviation of
 * the back-transformed realisations (0 at samples).  Both [sum Lx*Ly] on
 * the host (blocking) or the device.  Error STATE if no measurement sweep ran. */
mpr_status mpr_predict(mpr_ctx* ctx, float* z_hat, float* z_std, mpr_mem where,
                       mpr_stream stream);

/* Clears the realisation accumulators (keeps the chains' states). */
mpr_status mpr_reset_accumulators(mpr_ctx* ctx, mpr_stream stream);

/* The realisation sums behind mpr_predict (Alg. 2 step 5): for every gap
 * pixel the sum, over every chain and every measurement sweep so far, of phi
 * and of phi^2; 0 at sample pixels.  sum, sum2 (nullable): [sum Lx*Ly]
 * doubles, image-major, row-major, on the host (blocking) or the device
 * (asynchronous).  n_terms (host, nullable) receives the number of terms of
 * each sum (measurement sweeps x chains).  mpr_set_accumulators restores
 * them, e.g. to resume a checkpointed sampling run (sum2 may be NULL: the
 * squares restart at 0); n_terms must be a multiple of the chain count. */
mpr_status mpr_get_accumulators(mpr_ctx* ctx, double* sum, double* sum2, int64_t* n_terms,
                                mpr_mem where, mpr_stream stream);
mpr_status mpr_set_accumulators(mpr_ctx* ctx, const double* sum, const double* sum2,
                                int64_t n_terms, mpr_mem where, mpr_stream stream);

/* Checkpoint / parity access to the full simulation state.
 * phi: [sum over images of n_chains * Lx * Ly] floats, image-major then
 * chain-major, row-major; get writes sample pixels with their fixed angles,
 * set reads only gap pixels.  Device or host (blocking). */
mpr_status mpr_get_state(mpr_ctx* ctx, float* phi, mpr_mem where, mpr_stream stream);
mpr_status mpr_set_state(mpr_ctx* ctx, const float* phi, mpr_mem where, mpr_stream stream);

/* Per realisation (image-major, [n_img * n_chains], host, blocking): the
 * perturbation control factor a, the accepted proposals of the last sweep
 * and the specific energy recorded after the last sweep (nan if the last
 * sweep did not record it).  Any pointer may be NULL. */
mpr_status mpr_get_chain_info(mpr_ctx* ctx, float* a, uint32_t* accepted, double* e_last,
                              mpr_stream stream);
/* Overwrites a per realisation (host [n_img * n_chains]). */
mpr_status mpr_set_chain_a(mpr_ctx* ctx, const float* a, mpr_stream stream);

/* Sweep counter that keys the random stream (sweep field of the Philox
 * counter) and the equilibration index i of Alg. 2 step 4.2. */
mpr_status mpr_get_sweep_index(const mpr_ctx* ctx, uint32_t* sweep, uint32_t* equil_index);
mpr_status mpr_set_sweep_index(mpr_ctx* ctx, uint32_t sweep, uint32_t equil_index,
                               mpr_stream stream);

/* Releases the host descriptor.  The workspace stays the caller's. */
void mpr_destroy(mpr_ctx* ctx);

/* ---- context-free kernels ---------------------------------------------- */

/* Energy of Eq. Hamiltonian_mod on n dense angle grids (device, row-major,
 * grid k at offset sum_{j<k} Lx[j]*Ly[j]; open boundaries): H_out device
 * [n] FP64.  Lx, Ly host [n].  Asynchronous. */
mpr_status mpr_lattice_energy(int n, const int* Lx, const int* Ly, const float* phi,
                              double q, double J, double* H_out, mpr_stream stream);

/* Gradient of the same energy with respect to the angles: grad_i = g_k * J q
 * sum_j sin(q (phi_i - phi_j)) for site i of grid k (the torque, the local
 * field of the sweep), with g device [n] FP64 upstream weights (dL/dH_k).
 * grad device, same layout as phi.  Asynchronous. */
mpr_status mpr_lattice_torque(int n, const int* Lx, const int* Ly, const float* phi,
                              double q, double J, const double* g, float* grad,
                              mpr_stream stream);

/* Both gradients of L = sum_k g_k H_k in one pass (the backward of the energy
 * as a differentiable function of the angles and of J): grad_phi as
 * mpr_lattice_torque (nullable), and grad_J device [1] FP64 (nullable)
 * = sum_k g_k dH_k/dJ = -sum_k g_k sum_<ij> cos(q (phi_i - phi_j)) (= H/J,
 * Eq. Hamiltonian_mod being linear in J).  Asynchronous. */
mpr_status mpr_lattice_grad(int n, const int* Lx, const int* Ly, const float* phi, double q,
                            double J, const double* g, float* grad_phi, double* grad_J,
                            mpr_stream stream);

/* Philox4x32-10 blocks of the library's random stream for n counters
 * (device uint32 [4n] in, [4n] out; key host [2]).  reference != 0 runs the
 * CUDA toolkit's own Philox4x32-10 device routine instead, for
 * cross-checking.  Asynchronous. */
mpr_status mpr_philox(int n, const uint32_t* ctr, const uint32_t* key, uint32_t* out,
                      int reference, mpr_stream stream);

/* Evaluates one of the library's own single-precision approximations, or the
 * CUDA math routine it stands in for, on n inputs (device float arrays), so
 * that tests can bound their error: fn 0 = the atan2 used by the
 * over-relaxation step, atan2(a, b); 1 = CUDA atan2f(a, b); 2 = the series
 * sine used for half proposal steps, sin(a) for |a| <= pi/2; 3 = CUDA sinf(a).
 * b may be NULL for fn 2-3.  Asynchronous. */
mpr_status mpr_math_probe(int fn, int n, const float* a, const float* b, float* out,
                          mpr_stream stream);

/* ---- allocation-free entry point ------------------------------------------
 *
 * The sample specific energy (the mean of -J cos(q dphi) over the nearest-
 * neighbour bonds whose both ends are samples, with the angles of the linear
 * map of the sample values onto [0, 2 pi]), with the sample extremes and the
 * number of such bonds, for callers that may not allocate device memory at
 * all: code running where every byte of device memory belongs to another
 * allocator (a plugin inside a framework with its own memory pool),
 * real-time pipelines that forbid allocation once running, or hosts where an
 * allocation would synchronise the device.  The paper has no counterpart of
 * this entry point; for the MPR model it computes what mpr_init_grid()
 * reports through mpr_get_image_info() (a GMRF context reports its own bond
 * instead), for up to MPR_NOALLOC_MAX_IMAGES images per call.
 *
 * Inputs and outputs are the caller's: z, gap as for mpr_init_grid (device,
 * concatenated); e_s device [n_img] (nan when an image has fewer than two
 * distinct sample values, no sample pair, or a non-finite sample value);
 * n_sp, z_min, z_max device [n_img] or NULL.  Its temporary results go to a
 * fixed array of about 0.5 MB that this library reserves in every GPU's
 * memory when it is loaded (held until the process exits).  It calls no
 * allocator.
 *  - The first call on a device looks the array's device address up (a
 *    cudaGetSymbolAddress); make that first call before any stream capture.
 *  - Every call on a device uses the same array: calls that may overlap on
 *    the GPU (different streams, graph branches) race and must be ordered
 *    by the caller.
 * Asynchronous.  Errors: INVALID_ARG (n_img outside [1, 64], NULL pointers,
 * bad sizes; the message names the limit), CUDA. */
#define MPR_NOALLOC_MAX_IMAGES 64
mpr_status mpr_sample_energy_noalloc(int n_img, const int* Lx, const int* Ly, const float* z,
                                     const uint8_t* gap, double q, double J, double* e_s,
                                     int64_t* n_sp, float* z_min, float* z_max,
                                     mpr_stream stream);

#ifdef __cplusplus
}
#endif
#endif /* MPR_H */
