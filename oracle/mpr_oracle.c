/*
 * Plain FP64 CPU oracle of MPR conditional simulation (Zukovic & Hristopulos,
 * "Gibbs Markov random fields with continuous values based on the modified
 * planar rotator model").
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may link, load or
 * call this file: only the test suite, the smoke check and the benchmark's
 * CPU-baseline leg use it.  It shares no code, header or constant table with
 * the CUDA library.
 *
 * Everything is written the slow, literal way: double precision, direct sums
 * of cosines over the nearest neighbours, row-major loops, no blocking.
 *
 * Readings of the paper taken here (each listed in the design notes):
 *  - open boundaries; an out-of-grid neighbour does not exist (Sec. 2.2; the
 *    auxiliary mirror nodes of Sec. 2.5 copy the site itself, so their bonds
 *    have zero contrast and constant energy and are dropped);
 *  - over-relaxation is the reflection of theta = q*phi about the local-field
 *    angle of the q-scaled neighbour spins, kept only when the reflected angle
 *    stays inside [0, 2*pi*q) (Eq. over-relax, made consistent with the q of
 *    Eq. Hamiltonian_mod; for q = 1 it is the printed formula exactly).  The
 *    printed q = 1 formula is available as `literal_or`;
 *  - the sample specific energy averages over unordered sample-sample bonds
 *    (Eq. mpr-sse with N_SP the number of such pairs);
 *  - random numbers: Philox4x32-10 (Salmon et al., SC'11) with key = seed and
 *    counter = (row << 16 | x >> 1, sweep, chain >> 1, image | colour << 31),
 *    one call per site and pair of realisations (words 0-1 for the even
 *    realisation, 2-3 for the odd one); uniform = (w >> 8) * 2^-24.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_PI 3.14159265358979323846
#define OR_TWO_PI 6.28318530717958647692
#define OR_EPS_FIELD 1e-6  /* a local field shorter than this vanishes (no reflection) */

/* ---------------------------------------------------------------- Philox */

/* Philox4x32-10: ten rounds of two 32x32->64 multiplies with the Weyl key
 * schedule k_{i+1} = k_i + (0x9E3779B9, 0xBB67AE85) (Salmon et al. 2011, Sec. 4). */
void oracle_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4])
{
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; ++round) {
        uint64_t prod0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
        uint64_t prod1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(prod0 >> 32), lo0 = (uint32_t)prod0;
        uint32_t hi1 = (uint32_t)(prod1 >> 32), lo1 = (uint32_t)prod1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

static double u24(uint32_t w) { return (double)(w >> 8) * (1.0 / 16777216.0); }

/* The two uniforms (u, r) of site (x, y) of colour `colour` in realisation
 * `chain` at a given sweep.  In row y the sites of one colour have packed
 * column k = x >> 1; one Philox call keyed by (row, k) serves that site in the
 * two realisations 2m and 2m + 1: the even one takes words 0-1, the odd one
 * words 2-3. */
static void site_uniforms(uint64_t seed, uint32_t img, uint32_t chain, uint32_t sweep,
                          int x, int y, int colour, double* u, double* r)
{
    uint32_t k = (uint32_t)x >> 1;
    uint32_t ctr[4] = { ((uint32_t)y << 16) | k, sweep, chain >> 1,
                        img | ((uint32_t)colour << 31) };
    uint32_t key[2] = { (uint32_t)seed, (uint32_t)(seed >> 32) };
    uint32_t w[4];
    oracle_philox4x32_10(ctr, key, w);
    if ((chain & 1u) == 0) { *u = u24(w[0]); *r = u24(w[1]); }
    else                   { *u = u24(w[2]); *r = u24(w[3]); }
}

static double mod_two_pi(double t) { return t - OR_TWO_PI * floor(t / OR_TWO_PI); }

/* ------------------------------------------------------------ Sec. 2.1 map */

/* Eq. map: phi = 2 pi (z - z_min) / (z_max - z_min) with the extremes taken
 * over the sample sites only.  Gap sites are left at 0.  Returns 0, or -1 when
 * fewer than one sample exists or z_max == z_min. */
int oracle_map(int Lx, int Ly, const double* z, const uint8_t* gap,
               double* phi, double* zmin_out, double* zmax_out)
{
    long n = (long)Lx * Ly;
    double zmin = INFINITY, zmax = -INFINITY;
    for (long i = 0; i < n; ++i) {
        if (gap[i]) continue;
        if (z[i] < zmin) zmin = z[i];
        if (z[i] > zmax) zmax = z[i];
    }
    if (!(zmax > zmin)) return -1;
    for (long i = 0; i < n; ++i)
        phi[i] = gap[i] ? 0.0 : OR_TWO_PI * (z[i] - zmin) / (zmax - zmin);
    *zmin_out = zmin;
    *zmax_out = zmax;
    return 0;
}

/* Inverse map of Alg. 2 step 5.3: z = z_min + (z_max - z_min) phi / (2 pi). */
double oracle_unmap(double phi, double zmin, double zmax)
{
    return zmin + (zmax - zmin) * phi / OR_TWO_PI;
}

/* Hot start (Alg. 2 step 1.8): every gap angle drawn from U(0, 2 pi) with
 * the first uniform of its site at sweep index 0xFFFFFFFF. */
void oracle_hot_start(int Lx, int Ly, const uint8_t* gap, double* phi,
                      uint64_t seed, uint32_t img, uint32_t chain)
{
    for (int y = 0; y < Ly; ++y)
        for (int x = 0; x < Lx; ++x) {
            long i = (long)y * Lx + x;
            if (!gap[i]) continue;
            double u, r;
            site_uniforms(seed, img, chain, 0xFFFFFFFFu, x, y, (x + y) & 1, &u, &r);
            phi[i] = OR_TWO_PI * u;
        }
}

/* --------------------------------------------------- Sec. 2.2 energies */

/* Eq. mpr-sse: e_s = -(J / N_SP) sum over unordered nearest-neighbour pairs
 * with both ends sampled of cos(q (phi_i - phi_j)).  Returns N_SP; e_s is
 * left untouched when N_SP = 0. */
long oracle_sample_energy(int Lx, int Ly, const double* phi, const uint8_t* gap,
                          double q, double J, double* e_s)
{
    double sum = 0.0;
    long nsp = 0;
    for (int y = 0; y < Ly; ++y)
        for (int x = 0; x < Lx; ++x) {
            long i = (long)y * Lx + x;
            if (gap[i]) continue;
            if (x + 1 < Lx && !gap[i + 1]) { sum += cos(q * (phi[i] - phi[i + 1])); ++nsp; }
            if (y + 1 < Ly && !gap[i + Lx]) { sum += cos(q * (phi[i] - phi[i + Lx])); ++nsp; }
        }
    if (nsp > 0) *e_s = -J * sum / (double)nsp;
    return nsp;
}

/* Eq. Hamiltonian_mod with open boundaries: H = -J sum_<ij> cos(q (phi_i - phi_j)). */
double oracle_energy(int Lx, int Ly, const double* phi, double q, double J)
{
    double sum = 0.0;
    for (int y = 0; y < Ly; ++y)
        for (int x = 0; x < Lx; ++x) {
            long i = (long)y * Lx + x;
            if (x + 1 < Lx) sum += cos(q * (phi[i] - phi[i + 1]));
            if (y + 1 < Ly) sum += cos(q * (phi[i] - phi[i + Lx]));
        }
    return -J * sum;
}

/* N_GP of Eq. ene for an Lx x Ly grid: Lx (Ly - 1) + Ly (Lx - 1). */
long oracle_n_bonds(int Lx, int Ly) { return (long)Lx * (Ly - 1) + (long)Ly * (Lx - 1); }

/* dH/dphi_i = J q sum_j sin(q (phi_i - phi_j)); dH/dJ = H / J. */
void oracle_torque(int Lx, int Ly, const double* phi, double q, double J, double* grad)
{
    for (int y = 0; y < Ly; ++y)
        for (int x = 0; x < Lx; ++x) {
            long i = (long)y * Lx + x;
            double s = 0.0;
            if (x > 0)      s += sin(q * (phi[i] - phi[i - 1]));
            if (x + 1 < Lx) s += sin(q * (phi[i] - phi[i + 1]));
            if (y > 0)      s += sin(q * (phi[i] - phi[i - Lx]));
            if (y + 1 < Ly) s += sin(q * (phi[i] - phi[i + Lx]));
            grad[i] = J * q * s;
        }
}

/* --------------------------------------------------- Sec. 2.4 updates */

static int neighbours(int Lx, int Ly, int x, int y, long nb[4])
{
    int n = 0;
    long i = (long)y * Lx + x;
    if (y > 0)      nb[n++] = i - Lx;
    if (y + 1 < Ly) nb[n++] = i + Lx;
    if (x > 0)      nb[n++] = i - 1;
    if (x + 1 < Lx) nb[n++] = i + 1;
    return n;
}

/* Over-relaxation of one spin (Eq. over-relax).
 * q-consistent reading: Psi = atan2(sum sin(q phi_j), sum cos(q phi_j)),
 * theta' = (2 Psi - q phi) mod 2pi, and phi' = theta'/q when theta' < 2 pi q,
 * otherwise phi' = phi.  literal != 0 applies the printed q = 1 formula
 * phi' = (2 Phi - phi) mod 2pi with Phi = atan2(sum sin phi_j, sum cos phi_j).
 * `slack` (nullable) receives the distance of the reflected angle to the
 * nearest point where the result jumps (a multiple of 2 pi before the modulo,
 * or 2 pi q after it); `field` (nullable) receives the local-field length.
 * atan2 needs a field of nonzero length; one shorter than 1e-6 (a few units
 * of the resolution of a sum of four unit vectors in single precision, and
 * the exact value 0 of antipodal neighbours, e.g. the sample extremes 0 and
 * 2 pi at q = 1/2) counts as vanishing and leaves the spin unreflected. */
double oracle_over_relax(double phi, const double* nbr, int n, double q, int literal,
                         double* slack, double* field)
{
    double C = 0.0, S = 0.0;
    if (literal) {
        for (int j = 0; j < n; ++j) { C += cos(nbr[j]); S += sin(nbr[j]); }
    } else {
        for (int j = 0; j < n; ++j) { C += cos(q * nbr[j]); S += sin(q * nbr[j]); }
    }
    double R = sqrt(C * C + S * S);
    if (field) *field = R;
    /* no reflection is attempted: no range decision to report (the field test is) */
    if (R < OR_EPS_FIELD) { if (slack) *slack = 1e30; return phi; }
    double Psi = atan2(S, C);
    if (literal) {
        double t = 2.0 * Psi - phi;
        double tm = mod_two_pi(t);
        if (slack) { double d = fabs(t - OR_TWO_PI * floor(t / OR_TWO_PI + 0.5)); *slack = d; }
        return tm;
    }
    double t = 2.0 * Psi - q * phi;
    double tm = mod_two_pi(t);
    if (slack) {
        double d_wrap = fabs(t - OR_TWO_PI * floor(t / OR_TWO_PI + 0.5));
        double d_edge = fabs(tm - OR_TWO_PI * q);
        *slack = d_wrap < d_edge ? d_wrap : d_edge;
    }
    return (tm < OR_TWO_PI * q) ? tm / q : phi;
}

/* Site energy of spin value v against its neighbours: -J sum_j cos(q (v - phi_j)). */
static double site_energy(double v, const double* nbr, int n, double q, double J)
{
    double s = 0.0;
    for (int j = 0; j < n; ++j) s += cos(q * (v - nbr[j]));
    return -J * s;
}

/* Per-site diagnostics of one sweep (8 doubles per site; untouched for
 * sample sites): r - AP, AP, dH/T, OR slack, wrap slack, field length,
 * sensitivity of dH/T to a unit angle error, accepted flag. */
enum { D_RMAP = 0, D_AP, D_DHT, D_ORSLACK, D_WRAPSLACK, D_FIELD, D_SENS, D_ACC, D_N };

/* Alg. 1 applied to one gap site (x, y) of colour `colour` whose current
 * angle is phi and whose n existing neighbours hold nbr[0..n-1]: the
 * over-relaxation step, then the restricted Metropolis step
 * phi'' = (phi' + 2 pi (u - 1/2) / a) mod 2 pi, accepted iff
 * r < min(1, exp(-dH / T)) (ties reject).  Returns the new angle; *acc
 * receives 1 if the proposal was accepted; d (nullable) the D_N diagnostics. */
double oracle_site_update(double phi, const double* nbr, int n, double q, double J, double T,
                          double a, uint64_t seed, uint32_t img, uint32_t chain, uint32_t sweep,
                          int x, int y, int colour, int literal_or, int* acc, double* d)
{
    double or_slack, field;
    double p1 = oracle_over_relax(phi, nbr, n, q, literal_or, &or_slack, &field);
    double u, r;
    site_uniforms(seed, img, chain, sweep, x, y, colour, &u, &r);
    double raw = p1 + (OR_TWO_PI / a) * (u - 0.5);
    double p2 = mod_two_pi(raw);
    double dH = site_energy(p2, nbr, n, q, J) - site_energy(p1, nbr, n, q, J);
    double ap = dH <= 0.0 ? 1.0 : exp(-dH / T);
    int ok = r < ap;
    if (d) {
        double sens = 0.0;
        for (int j = 0; j < n; ++j)
            sens += fabs(sin(q * (p2 - nbr[j]))) + fabs(sin(q * (p1 - nbr[j])));
        double w0 = fabs(raw), w1 = fabs(raw - OR_TWO_PI);
        d[D_RMAP] = r - ap;
        d[D_AP] = ap;
        d[D_DHT] = dH / T;
        d[D_ORSLACK] = or_slack;
        d[D_WRAPSLACK] = w0 < w1 ? w0 : w1;
        d[D_FIELD] = field;
        d[D_SENS] = J * q * sens / T;
        d[D_ACC] = ok;
    }
    *acc = ok;
    return ok ? p2 : p1;
}

/* One hybrid sweep (Alg. 1) on the red/black checkerboard: colour 0
 * ((x + y) even) first, then colour 1; within a colour every gap site in
 * row-major order gets oracle_site_update().  Returns the number of accepted
 * proposals. */
long oracle_sweep(int Lx, int Ly, double* phi, const uint8_t* gap,
                  double q, double J, double T, double a,
                  uint64_t seed, uint32_t img, uint32_t chain, uint32_t sweep,
                  int literal_or, double* diag)
{
    long n_acc = 0;
    double nbr[4];
    long nb[4];
    for (int colour = 0; colour < 2; ++colour)
        for (int y = 0; y < Ly; ++y)
            for (int x = 0; x < Lx; ++x) {
                if (((x + y) & 1) != colour) continue;
                long i = (long)y * Lx + x;
                if (!gap[i]) continue;
                int n = neighbours(Lx, Ly, x, y, nb);
                for (int j = 0; j < n; ++j) nbr[j] = phi[nb[j]];
                int acc;
                phi[i] = oracle_site_update(phi[i], nbr, n, q, J, T, a, seed, img, chain, sweep,
                                            x, y, colour, literal_or, &acc,
                                            diag ? diag + (long)D_N * i : NULL);
                n_acc += acc;
            }
    return n_acc;
}

/* Alg. 2 step 4.2: after equilibration sweep i with acceptance ratio A
 * below A_targ, a(i+1) = 1 + (i+1)/k_a; otherwise a is kept. */
double oracle_adapt_a(double a, long n_acc, long n_gap, long i, double A_targ, double k_a)
{
    if ((double)n_acc < A_targ * (double)n_gap) return 1.0 + (double)(i + 1) / k_a;
    return a;
}

/* --------------------------------------------------- Sec. 2.3 SEM */

/* Equilibrium specific energy e(T, L) of Eq. ene by unconditional simulation
 * (empty sample set) of K chains on an L x L lattice: cold start (every angle
 * pi, the "ferromagnetic" start of Sec. 2.5, which reaches the low-temperature
 * equilibrium far sooner than a random start), n_eq sweeps with the
 * a-adaptation of Alg. 2, then n_meas sweeps with a frozen; the specific energy
 * H/N_GP of every measurement sweep of every chain is averaged.  The variance
 * of those values is returned in *var (nullable).  Chain k uses image tag
 * img | 1 << 30 and chain index k. */
double oracle_e_of_T(int L, int K, int n_eq, int n_meas, double q, double J, double T,
                     double A_targ, double k_a, uint64_t seed, uint32_t img, double* var)
{
    long n = (long)L * L;
    double* phi = (double*)malloc(sizeof(double) * n);
    uint8_t* gap = (uint8_t*)malloc(n);
    memset(gap, 1, n);
    double nb = (double)oracle_n_bonds(L, L);
    double sum = 0.0, sum2 = 0.0;
    long cnt = 0;
    uint32_t tag = img | (1u << 30);
    for (int k = 0; k < K; ++k) {
        for (long i = 0; i < n; ++i) phi[i] = OR_PI;
        double a = 1.0;
        for (int s = 0; s < n_eq; ++s) {
            long acc = oracle_sweep(L, L, phi, gap, q, J, T, a, seed, tag, (uint32_t)k,
                                    (uint32_t)s, 0, NULL);
            a = oracle_adapt_a(a, acc, n, s, A_targ, k_a);
        }
        for (int s = 0; s < n_meas; ++s) {
            oracle_sweep(L, L, phi, gap, q, J, T, a, seed, tag, (uint32_t)k,
                         (uint32_t)(n_eq + s), 0, NULL);
            double e = oracle_energy(L, L, phi, q, J) / nb;
            sum += e; sum2 += e * e; ++cnt;
        }
    }
    free(phi);
    free(gap);
    double m = sum / (double)cnt;
    if (var) *var = sum2 / (double)cnt - m * m;
    return m;
}

/* T_hat = e^-1(e_s | L) (Sec. 2.3) by bisection on log T inside
 * [T_lo, T_hi], using that e(T) increases with T.  Every evaluation of
 * e(T) uses the same random stream.  Stops when (T_hi - T_lo)/T_mid < rel_tol
 * or after max_iter halvings.  Returns 0; -1 when e_s lies outside the
 * range of e(T) between T = 0 (aligned spins, -J) and T = infinity
 * (independent uniform angles: <cos(q dphi)> = (sin(pi q) / (pi q))^2, so
 * -J (sin(pi q) / (pi q))^2, which is -4J/pi^2 at q = 1/2). */
int oracle_estimate_T(double e_s, int L, int K, int n_eq, int n_meas, double q, double J,
                      double A_targ, double k_a, uint64_t seed, uint32_t img,
                      double T_lo, double T_hi, double rel_tol, int max_iter, double* T_out)
{
    const double sq = sin(OR_PI * q) / (OR_PI * q);
    if (!(e_s > -J && e_s < -J * sq * sq)) return -1;
    double lo = log(T_lo), hi = log(T_hi);
    for (int it = 0; it < max_iter; ++it) {
        double mid = 0.5 * (lo + hi);
        if (exp(hi) - exp(lo) < rel_tol * exp(mid)) break;
        double e = oracle_e_of_T(L, K, n_eq, n_meas, q, J, exp(mid), A_targ, k_a, seed, img, NULL);
        if (e < e_s) lo = mid; else hi = mid;
    }
    *T_out = exp(0.5 * (lo + hi));
    return 0;
}

/* --------------------------------------------------- Alg. 2 driver */

/* Conditional simulation of one image (Alg. 2 with fixed sweep counts) over
 * R independent chains, at a given temperature T.  Chain c: hot start,
 * n_equil sweeps with the a-adaptation, then n_meas sweeps with a frozen at
 * its last value (freeze_a != 0) or a = 1 as printed in step 5.2.  phi_mean
 * receives the arithmetic mean of phi over all measurement sweeps of all
 * chains; e_hist (nullable) receives H/N_GP after every sweep, chain-major
 * [R][n_equil + n_meas]; a_out (nullable) the final a per chain;
 * acc_hist (nullable) the accepted count per sweep, like e_hist. */
int oracle_simulate(int Lx, int Ly, const double* phi_s, const uint8_t* gap,
                    double q, double J, double T, double A_targ, double k_a,
                    int R, int n_equil, int n_meas, int freeze_a, int literal_or,
                    uint64_t seed, uint32_t img,
                    double* phi_mean, double* e_hist, double* a_out, double* acc_hist)
{
    long n = (long)Lx * Ly;
    long P = 0;
    for (long i = 0; i < n; ++i) P += gap[i] != 0;
    double nb = (double)oracle_n_bonds(Lx, Ly);
    double* phi = (double*)malloc(sizeof(double) * n);
    double* acc = (double*)calloc((size_t)n, sizeof(double));
    int n_sw = n_equil + n_meas;
    for (int c = 0; c < R; ++c) {
        memcpy(phi, phi_s, sizeof(double) * n);
        oracle_hot_start(Lx, Ly, gap, phi, seed, img, (uint32_t)c);
        double a = 1.0;
        for (int s = 0; s < n_sw; ++s) {
            int meas = s >= n_equil;
            double a_use = (meas && !freeze_a) ? 1.0 : a;
            long na = oracle_sweep(Lx, Ly, phi, gap, q, J, T, a_use, seed, img, (uint32_t)c,
                                   (uint32_t)s, literal_or, NULL);
            if (!meas) a = oracle_adapt_a(a, na, P, s, A_targ, k_a);
            if (e_hist) e_hist[(long)c * n_sw + s] = oracle_energy(Lx, Ly, phi, q, J) / nb;
            if (acc_hist) acc_hist[(long)c * n_sw + s] = (double)na;
            if (meas)
                for (long i = 0; i < n; ++i) acc[i] += phi[i];
        }
        if (a_out) a_out[c] = a;
    }
    double denom = (double)R * (double)n_meas;
    for (long i = 0; i < n; ++i) phi_mean[i] = gap[i] ? acc[i] / denom : phi_s[i];
    free(phi);
    free(acc);
    return 0;
}

/* Least-squares slope of y[0..n-1] against 0..n-1 (a Savitzky-Golay fit of
 * degree 1, the reading taken for the unspecified degree of Sec. 2.4). */
double oracle_sg_slope(const double* y, int n)
{
    double xm = 0.5 * (n - 1), ym = 0.0, sxy = 0.0, sxx = 0.0;
    for (int k = 0; k < n; ++k) ym += y[k];
    ym /= n;
    for (int k = 0; k < n; ++k) { sxy += (k - xm) * (y[k] - ym); sxx += (k - xm) * (k - xm); }
    return sxy / sxx;
}

/* Alg. 2 step 4 for R chains stepped together from their hot starts: sweep
 * i, a-adaptation, chain-mean specific energy e(i+1); once i >= n_fit and
 * i mod n_f == 0 the slope k of the last n_fit energies is taken and the
 * loop ends when k >= 0, or after sweep i_max.  phi_out [R][N] receives the
 * states, e_mean [i_max + 1] the chain-mean energies; returns sweeps run. */
int oracle_equilibrate(int Lx, int Ly, const double* phi_s, const uint8_t* gap, double q,
                       double J, double T, double A_targ, double k_a, int R, int n_f, int n_fit,
                       int i_max, uint64_t seed, uint32_t img, double* phi_out, double* e_mean)
{
    long n = (long)Lx * Ly;
    long P = 0;
    for (long i = 0; i < n; ++i) P += gap[i] != 0;
    double nb = (double)oracle_n_bonds(Lx, Ly);
    double* a = (double*)malloc(sizeof(double) * R);
    for (int c = 0; c < R; ++c) {
        memcpy(phi_out + (long)c * n, phi_s, sizeof(double) * n);
        oracle_hot_start(Lx, Ly, gap, phi_out + (long)c * n, seed, img, (uint32_t)c);
        a[c] = 1.0;
    }
    int done = 0;
    for (int i = 0; i <= i_max; ++i) {
        double es = 0.0;
        for (int c = 0; c < R; ++c) {
            double* p = phi_out + (long)c * n;
            long na = oracle_sweep(Lx, Ly, p, gap, q, J, T, a[c], seed, img, (uint32_t)c,
                                   (uint32_t)i, 0, NULL);
            a[c] = oracle_adapt_a(a[c], na, P, i, A_targ, k_a);
            es += oracle_energy(Lx, Ly, p, q, J) / nb;
        }
        e_mean[i] = es / R;
        done = i + 1;
        if (i >= n_fit && i % n_f == 0 && oracle_sg_slope(e_mean + i + 1 - n_fit, n_fit) >= 0.0)
            break;
    }
    free(a);
    return done;
}

/* ------------------------------------------------ Sec. 4.3 GMRF variant */
/* Pair interaction H_ij = -Dphi^2 / (2 pi^2) + 1 and H = -J sum H_ij, i.e.
 * every bond costs J (Dphi^2 / (2 pi^2) - 1).  The site energy is quadratic
 * in phi with its minimum at the mean m of the existing neighbours, so the
 * over-relaxation reflects about m: phi' = 2 m - phi, kept when it stays in
 * [0, 2 pi) (the reading taken; the paper does not spell the GMRF update
 * out).  Everything else (checkerboard, proposal, acceptance, a schedule,
 * random stream) is shared with the MPR sweep. */

static double gmrf_bond(double d) { return d * d / (2.0 * OR_PI * OR_PI) - 1.0; }

static double gmrf_site_energy(double v, const double* nbr, int n, double J)
{
    double s = 0.0;
    for (int j = 0; j < n; ++j) s += gmrf_bond(v - nbr[j]);
    return J * s;
}

double oracle_gmrf_energy(int Lx, int Ly, const double* phi, double J)
{
    double sum = 0.0;
    for (int y = 0; y < Ly; ++y)
        for (int x = 0; x < Lx; ++x) {
            long i = (long)y * Lx + x;
            if (x + 1 < Lx) sum += gmrf_bond(phi[i] - phi[i + 1]);
            if (y + 1 < Ly) sum += gmrf_bond(phi[i] - phi[i + Lx]);
        }
    return J * sum;
}

long oracle_gmrf_sample_energy(int Lx, int Ly, const double* phi, const uint8_t* gap, double J,
                               double* e_s)
{
    double sum = 0.0;
    long nsp = 0;
    for (int y = 0; y < Ly; ++y)
        for (int x = 0; x < Lx; ++x) {
            long i = (long)y * Lx + x;
            if (gap[i]) continue;
            if (x + 1 < Lx && !gap[i + 1]) { sum += gmrf_bond(phi[i] - phi[i + 1]); ++nsp; }
            if (y + 1 < Ly && !gap[i + Lx]) { sum += gmrf_bond(phi[i] - phi[i + Lx]); ++nsp; }
        }
    if (nsp > 0) *e_s = J * sum / (double)nsp;
    return nsp;
}

double oracle_gmrf_site_update(double phi, const double* nbr, int n, double J, double T, double a,
                               uint64_t seed, uint32_t img, uint32_t chain, uint32_t sweep, int x,
                               int y, int colour, int* acc, double* d)
{
    double m = 0.0;
    for (int j = 0; j < n; ++j) m += nbr[j];
    m /= n;
    double t = 2.0 * m - phi;
    double p1 = (t >= 0.0 && t < OR_TWO_PI) ? t : phi;
    double u, r;
    site_uniforms(seed, img, chain, sweep, x, y, colour, &u, &r);
    double raw = p1 + (OR_TWO_PI / a) * (u - 0.5);
    double p2 = mod_two_pi(raw);
    double dH = gmrf_site_energy(p2, nbr, n, J) - gmrf_site_energy(p1, nbr, n, J);
    double ap = dH <= 0.0 ? 1.0 : exp(-dH / T);
    int ok = r < ap;
    if (d) {
        double w0 = fabs(raw), w1 = fabs(raw - OR_TWO_PI);
        double e0 = fabs(t), e1 = fabs(t - OR_TWO_PI);
        double sens = 0.0;
        for (int j = 0; j < n; ++j) sens += fabs(p2 - nbr[j]) + fabs(p1 - nbr[j]);
        d[D_RMAP] = r - ap;
        d[D_AP] = ap;
        d[D_DHT] = dH / T;
        d[D_ORSLACK] = e0 < e1 ? e0 : e1;
        d[D_WRAPSLACK] = w0 < w1 ? w0 : w1;
        d[D_FIELD] = (double)n;
        d[D_SENS] = J * sens / (OR_PI * OR_PI * T);
        d[D_ACC] = ok;
    }
    *acc = ok;
    return ok ? p2 : p1;
}

long oracle_gmrf_sweep(int Lx, int Ly, double* phi, const uint8_t* gap, double J, double T,
                       double a, uint64_t seed, uint32_t img, uint32_t chain, uint32_t sweep,
                       double* diag)
{
    long n_acc = 0;
    double nbr[4];
    long nb[4];
    for (int colour = 0; colour < 2; ++colour)
        for (int y = 0; y < Ly; ++y)
            for (int x = 0; x < Lx; ++x) {
                if (((x + y) & 1) != colour) continue;
                long i = (long)y * Lx + x;
                if (!gap[i]) continue;
                int n = neighbours(Lx, Ly, x, y, nb);
                for (int j = 0; j < n; ++j) nbr[j] = phi[nb[j]];
                int acc;
                phi[i] = oracle_gmrf_site_update(phi[i], nbr, n, J, T, a, seed, img, chain, sweep,
                                                 x, y, colour, &acc,
                                                 diag ? diag + (long)D_N * i : NULL);
                n_acc += acc;
            }
    return n_acc;
}

/* Conditional simulation of one image with the GMRF energy, like oracle_simulate. */
int oracle_gmrf_simulate(int Lx, int Ly, const double* phi_s, const uint8_t* gap, double J,
                         double T, double A_targ, double k_a, int R, int n_equil, int n_meas,
                         uint64_t seed, uint32_t img, double* phi_mean, double* e_mean)
{
    long n = (long)Lx * Ly;
    long P = 0;
    for (long i = 0; i < n; ++i) P += gap[i] != 0;
    double nb = (double)oracle_n_bonds(Lx, Ly);
    double* phi = (double*)malloc(sizeof(double) * n);
    double* acc = (double*)calloc((size_t)n, sizeof(double));
    double esum = 0.0;
    for (int c = 0; c < R; ++c) {
        memcpy(phi, phi_s, sizeof(double) * n);
        oracle_hot_start(Lx, Ly, gap, phi, seed, img, (uint32_t)c);
        double a = 1.0;
        for (int s = 0; s < n_equil + n_meas; ++s) {
            long na = oracle_gmrf_sweep(Lx, Ly, phi, gap, J, T, a, seed, img, (uint32_t)c,
                                        (uint32_t)s, NULL);
            if (s < n_equil) a = oracle_adapt_a(a, na, P, s, A_targ, k_a);
            else {
                for (long i = 0; i < n; ++i) acc[i] += phi[i];
                esum += oracle_gmrf_energy(Lx, Ly, phi, J) / nb;
            }
        }
    }
    for (long i = 0; i < n; ++i) phi_mean[i] = gap[i] ? acc[i] / ((double)R * n_meas) : phi_s[i];
    if (e_mean) *e_mean = esum / ((double)R * n_meas);
    free(phi);
    free(acc);
    return 0;
}
