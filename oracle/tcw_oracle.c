/*
 * tcw_oracle.c -- plain FP64 CPU oracle for the long-transient (tCW) template
 * track statistic of Merou, Tenorio & Sintes, "GPU-Accelerated Searches for
 * Long-Transient Gravitational Waves from Newborn Neutron Stars"
 * (arXiv:2507.07816).
 *
 * THIS IS TEST INFRASTRUCTURE, NOT PART OF THE PRODUCT.  Only the test suite,
 * the smoke check and the CPU-baseline leg of the benchmark may load it.  It
 * shares no code, header, table or constant generator with the CUDA library;
 * the two are compared element by element on the same seeded inputs.
 *
 * Everything here is written to be checked against the paper by eye: plain
 * nested loops, one `pow` per lookup, no tables, no reordering, no blocking.
 *
 *   Eq. 1 (Sec. 1)   f_gw(t) = f0 * ((t - T0)/tau + 1)^(1/(1-n))
 *   Eq. 2 (Sec. 1)   fhat(t) = f_gw(t) * (1 + v(t).nhat / c)
 *   Sec. 2           the track selects one data bin per segment; the weighted
 *                    normalized power is summed over the selected bins
 *   Eq. 4 (Sec. 2)   Psi = (s - <s>) / sigma_s
 *
 * Readings of points the paper leaves open:
 *   - segment time t_j is the caller-supplied segment mid-time;
 *   - segments with t_j < T0 contribute nothing (Eq. 1 starts at T0);
 *   - bin k has centre f_min + k*df and the track takes the nearest centre,
 *     k = floor((fhat - f_min)/df + 1/2) (ties go up);
 *   - lookups outside [0, Nbin) are skipped and their weight is dropped;
 *   - normalized power is Exp(1) under noise, so for s = sum w*rho the mean is
 *     <s> = W1 = sum w and the standard deviation is sigma_s = sqrt(W2),
 *     W2 = sum w^2, both over the lookups actually summed;
 *   - detectors are combined inside one sum;
 *   - Psi = -inf when no lookup is valid (W2 == 0);
 *   - top-k orders by (Psi descending, template index ascending).
 *
 * Number count (Sec. 2, the second statistic of the paper): each lookup
 * contributes nu = 1 when the bin's normalized power exceeds rho_th strictly
 * (compared in double), else 0, so s = sum w*nu.  Under noise rho is Exp(1),
 * so nu is Bernoulli(q) with q = exp(-rho_th): <s> = q*W1 and
 * sigma_s^2 = q(1-q)*W2.  rho_th is a caller parameter.
 *
 * Two-bin tracks (an extension for tracks that fall between bins or move by
 * more than a bin within one SFT, where a signal's power leaks into the
 * neighbouring bin): with track_bins = 2 each lookup takes the two bins whose
 * centres bracket the track, k = floor(x) and k + 1 (x the bin coordinate),
 * valid when both lie in the band; its value is the sum of their powers (or
 * counts).  Bins are independent under noise, so <s> and sigma_s^2 double.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORACLE_C_LIGHT 299792458.0 /* m/s, exact SI value */

/* Eq. 1: GW frequency of the msMagnetar model at detector time t (t >= T0). */
double oracle_track_frequency(double f0, double tau, double n, double T0, double t)
{
    return f0 * pow((t - T0) / tau + 1.0, 1.0 / (1.0 - n));
}

/* Eq. 2: Doppler-modulated frequency for detector velocity v (m/s) and unit
 * sky vector nhat (both in the same frame). */
double oracle_doppler_frequency(double f, const double v[3], const double nhat[3])
{
    double vn = v[0] * nhat[0] + v[1] * nhat[1] + v[2] * nhat[2];
    return f * (1.0 + vn / ORACLE_C_LIGHT);
}

/* Continuous bin coordinate x = (fhat - f_min)/df; bin k has centre f_min + k*df. */
double oracle_bin_coordinate(double fhat, double f_min, double df)
{
    return (fhat - f_min) / df;
}

/* Nearest-centre bin index, ties upward. */
int64_t oracle_bin_index(double fhat, double f_min, double df)
{
    return (int64_t)floor(oracle_bin_coordinate(fhat, f_min, df) + 0.5);
}

/* Eq. 4 with <s> = W1 and sigma_s = sqrt(W2). */
double oracle_critical_ratio(double S, double W1, double W2)
{
    if (W2 <= 0.0) return -INFINITY;
    return (S - W1) / sqrt(W2);
}

/* Eq. 4 for the number count: <s> = q*W1, sigma_s = sqrt(q(1-q)*W2), q = exp(-rho_th). */
double oracle_critical_ratio_count(double S, double W1, double W2, double rho_th)
{
    double q = exp(-rho_th);
    if (W2 <= 0.0) return -INFINITY;
    return (S - q * W1) / sqrt(q * (1.0 - q) * W2);
}

/* Eq. 4 when each lookup sums m independent bins: mean and variance scale by m. */
static double oracle_critical_ratio_bins(double S, double W1, double W2, int number_count,
                                         double rho_th, int m)
{
    if (W2 <= 0.0) return -INFINITY;
    double mean = 1.0, var = 1.0;
    if (number_count) {
        mean = exp(-rho_th);
        var = mean * (1.0 - mean);
    }
    return (S - m * mean * W1) / sqrt(m * var * W2);
}

/*
 * Statistic of one (sky, template) pair: S = sum w*rho, W1 = sum w,
 * W2 = sum w^2 over every detector d and segment j whose track bin lies in
 * the band (Sec. 2, Eq. 1, Eq. 2).
 *
 *   rho      [D][Nseg][Nbin]  normalized power (float, converted to double)
 *   t_mid    [Nseg]           segment mid-times, s (shared by all detectors)
 *   w        [D][Nseg]        per-detector, per-segment weights (NULL = 1)
 *   v        [D][Nseg][3]     detector velocity w.r.t. the SSB, m/s
 *   nhat     [3]              unit vector toward the source
 */
static void oracle_pair_stats(const float *rho, int D, int Nseg, int Nbin,
                              double f_min, double df, const double *t_mid,
                              const float *w, const double *v,
                              const double *nhat, double f0, double tau,
                              double n, double T0, int amp_power,
                              int number_count, double rho_th, int track_bins,
                              double out[3])
{
    double S = 0.0, W1 = 0.0, W2 = 0.0;
    for (int d = 0; d < D; ++d) {
        for (int j = 0; j < Nseg; ++j) {
            double t = t_mid[j];
            if (t < T0) continue;
            double f = oracle_track_frequency(f0, tau, n, T0, t);
            double fh = oracle_doppler_frequency(f, v + ((size_t)d * Nseg + j) * 3, nhat);
            int64_t k;
            if (track_bins == 2) {
                k = (int64_t)floor(oracle_bin_coordinate(fh, f_min, df));
                if (k < 0 || k + 1 >= Nbin) continue;
            } else {
                k = oracle_bin_index(fh, f_min, df);
                if (k < 0 || k >= Nbin) continue;
            }
            double wj = w ? (double)w[(size_t)d * Nseg + j] : 1.0;
            /* optional amplitude weight: the signal power follows h0^2 and
             * h0 grows as f^2 (Eq. 3), so a template's expected excess in
             * segment j scales as (f(t_j)/f0)^4 (amp_power = 4) */
            if (amp_power > 0) wj *= pow(f / f0, (double)amp_power);
            const float *row = rho + ((size_t)d * Nseg + j) * (size_t)Nbin;
            double r = 0.0;
            for (int64_t b = k; b < k + track_bins; ++b) {
                double rb = (double)row[b];
                r += number_count ? (rb > rho_th ? 1.0 : 0.0) : rb;
            }
            S += wj * r;
            W1 += wj;
            W2 += wj * wj;
        }
    }
    out[0] = S;
    out[1] = W1;
    out[2] = W2;
}

/*
 * Statistics for a list of (sky, template) pairs, or for the full grid when
 * pairs == NULL (then P is ignored and the output is [S][B], sky-major).
 * Outputs S_out, W1_out, W2_out, Psi_out (any may be NULL).
 * nthreads <= 0 uses the OpenMP default.
 */
void oracle_search_stats_ext(const float *rho, int D, int Nseg, int Nbin,
                             double f_min, double df, const double *t_mid,
                             const float *w, const double *v,
                             const double *nhat, int n_sky,
                             const double *f0, const double *tau, const double *n,
                             int n_tmpl, double T0, int amp_power,
                             int number_count, double rho_th, int track_bins,
                             const int64_t *pairs, int64_t P,
                             double *S_out, double *W1_out, double *W2_out,
                             double *Psi_out, int nthreads);

void oracle_search_stats(const float *rho, int D, int Nseg, int Nbin,
                         double f_min, double df, const double *t_mid,
                         const float *w, const double *v,
                         const double *nhat, int n_sky,
                         const double *f0, const double *tau, const double *n,
                         int n_tmpl, double T0,
                         const int64_t *pairs, int64_t P,
                         double *S_out, double *W1_out, double *W2_out,
                         double *Psi_out, int nthreads)
{
    oracle_search_stats_ext(rho, D, Nseg, Nbin, f_min, df, t_mid, w, v, nhat, n_sky, f0, tau, n,
                            n_tmpl, T0, 0, 0, 0.0, 1, pairs, P, S_out, W1_out, W2_out, Psi_out,
                            nthreads);
}

/* As oracle_search_stats, with every weight multiplied by (f(t_j)/f0)^amp_power
 * (amp_power = 0: none), with the number count of threshold rho_th in place of
 * the power when number_count != 0, and with two-bin lookups when
 * track_bins == 2 (1: the nearest bin). */
void oracle_search_stats_ext(const float *rho, int D, int Nseg, int Nbin,
                             double f_min, double df, const double *t_mid,
                             const float *w, const double *v,
                             const double *nhat, int n_sky,
                             const double *f0, const double *tau, const double *n,
                             int n_tmpl, double T0, int amp_power,
                             int number_count, double rho_th, int track_bins,
                             const int64_t *pairs, int64_t P,
                             double *S_out, double *W1_out, double *W2_out,
                             double *Psi_out, int nthreads)
{
    int64_t total = pairs ? P : (int64_t)n_sky * n_tmpl;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 16)
#endif
    for (int64_t i = 0; i < total; ++i) {
        int64_t s, b;
        if (pairs) {
            s = pairs[2 * i];
            b = pairs[2 * i + 1];
        } else {
            s = i / n_tmpl;
            b = i % n_tmpl;
        }
        double st[3];
        oracle_pair_stats(rho, D, Nseg, Nbin, f_min, df, t_mid, w, v,
                          nhat + 3 * s, f0[b], tau[b], n[b], T0, amp_power,
                          number_count, rho_th, track_bins, st);
        if (S_out) S_out[i] = st[0];
        if (W1_out) W1_out[i] = st[1];
        if (W2_out) W2_out[i] = st[2];
        if (Psi_out) {
            if (track_bins == 2)
                Psi_out[i] = oracle_critical_ratio_bins(st[0], st[1], st[2], number_count, rho_th, 2);
            else
                Psi_out[i] = number_count ? oracle_critical_ratio_count(st[0], st[1], st[2], rho_th)
                                          : oracle_critical_ratio(st[0], st[1], st[2]);
        }
    }
}

/*
 * Bin coordinate x (before rounding) of every lookup of the given pairs:
 * out[i][d][j] = (fhat - f_min)/df, NaN where t_j < T0.  Used by the tests to
 * find lookups inside the rounding tie band and to compare indices.
 */
void oracle_track_coordinates(int D, int Nseg, double f_min, double df,
                              const double *t_mid, const double *v,
                              const double *nhat, const double *f0,
                              const double *tau, const double *n, double T0,
                              const int64_t *pairs, int64_t P, double *out)
{
    for (int64_t i = 0; i < P; ++i) {
        int64_t s = pairs[2 * i], b = pairs[2 * i + 1];
        for (int d = 0; d < D; ++d) {
            for (int j = 0; j < Nseg; ++j) {
                double *o = out + ((size_t)i * D + d) * Nseg + j;
                if (t_mid[j] < T0) {
                    *o = NAN;
                    continue;
                }
                double f = oracle_track_frequency(f0[b], tau[b], n[b], T0, t_mid[j]);
                double fh = oracle_doppler_frequency(f, v + ((size_t)d * Nseg + j) * 3, nhat + 3 * s);
                *o = oracle_bin_coordinate(fh, f_min, df);
            }
        }
    }
}

/* Top-k of one row of Psi by (Psi descending, index ascending). */
typedef struct {
    double psi;
    int64_t idx;
} oracle_entry;

static int oracle_entry_cmp(const void *a, const void *b)
{
    const oracle_entry *x = (const oracle_entry *)a, *y = (const oracle_entry *)b;
    if (x->psi > y->psi) return -1;
    if (x->psi < y->psi) return 1;
    return (x->idx < y->idx) ? -1 : (x->idx > y->idx);
}

/* psi [rows][B] -> idx_out/val_out [rows][k]; k <= B. */
void oracle_topk(const double *psi, int64_t rows, int64_t B, int64_t k,
                 int64_t *idx_out, double *val_out)
{
    oracle_entry *e = (oracle_entry *)malloc(sizeof(oracle_entry) * (size_t)B);
    if (!e) return;
    for (int64_t r = 0; r < rows; ++r) {
        for (int64_t b = 0; b < B; ++b) {
            e[b].psi = psi[r * B + b];
            e[b].idx = b;
        }
        qsort(e, (size_t)B, sizeof(oracle_entry), oracle_entry_cmp);
        for (int64_t i = 0; i < k; ++i) {
            idx_out[r * k + i] = e[i].idx;
            val_out[r * k + i] = e[i].psi;
        }
    }
    free(e);
}

int oracle_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/*
 * Template banks (Sec. 2: a cubic lattice with equal spacing per axis, or
 * templates drawn uniformly over the parameter box), written out template by
 * template so that any range [first, first + count) of a bank of 1e8-1e9
 * templates can be produced on its own.
 *
 * Lattice of n_f0 x n_tau x n_n points, f0 fastest:
 *   t -> (i0, i1, i2) = (t mod n_f0, (t / n_f0) mod n_tau, t / (n_f0 n_tau));
 *   axis value at i of m points: lo for i = 0 (or m = 1), hi for i = m - 1,
 *   else fma(hi - lo, i / (m - 1), lo).
 * Uniform random: the 4 x 64-bit output of Philox4x64-10 (Salmon, Moraes, Dror
 * and Shaw, "Parallel random numbers: as easy as 1, 2, 3", SC 2011) at counter
 * (t, 0, 0, 0) and key (seed, 0); u_a = (x_a >> 11) 2^-53 for a = 0, 1, 2 and
 * value = fma(hi - lo, u, lo) for f0, tau, n in that order.
 */
static void oracle_mulhilo64(uint64_t a, uint64_t b, uint64_t *hi, uint64_t *lo)
{
    unsigned __int128 p = (unsigned __int128)a * (unsigned __int128)b;
    *hi = (uint64_t)(p >> 64);
    *lo = (uint64_t)p;
}

/* Philox4x64 with 10 rounds: the multipliers and Weyl key increments are the
 * ones the SC 2011 paper gives for the 4 x 64 variant. */
void oracle_philox4x64_10(const uint64_t ctr[4], const uint64_t key[2], uint64_t out[4])
{
    const uint64_t M0 = 0xD2E7470EE14C6C93ULL, M1 = 0xCA5A826395121157ULL;
    const uint64_t W0 = 0x9E3779B97F4A7C15ULL, W1 = 0xBB67AE8584CAA73BULL;
    uint64_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint64_t k0 = key[0], k1 = key[1];
    for (int r = 0; r < 10; ++r) {
        uint64_t hi0, lo0, hi1, lo1;
        oracle_mulhilo64(M0, x0, &hi0, &lo0);
        oracle_mulhilo64(M1, x2, &hi1, &lo1);
        uint64_t y0 = hi1 ^ x1 ^ k0, y1 = lo1, y2 = hi0 ^ x3 ^ k1, y3 = lo0;
        x0 = y0;
        x1 = y1;
        x2 = y2;
        x3 = y3;
        k0 += W0;
        k1 += W1;
    }
    out[0] = x0;
    out[1] = x1;
    out[2] = x2;
    out[3] = x3;
}

static double oracle_lattice_axis(double lo, double hi, int64_t m, int64_t i)
{
    if (m == 1 || i == 0) return lo;
    if (i == m - 1) return hi;
    return fma(hi - lo, (double)i / (double)(m - 1), lo);
}

/* kind 0 = lattice (n_f0, n_tau, n_n), 1 = uniform random (seed);
 * lo/hi = {f0, tau, n} bounds.  Writes templates first .. first + count - 1. */
void oracle_bank_templates(int kind, int64_t n_f0, int64_t n_tau, int64_t n_n,
                           const double lo[3], const double hi[3], uint64_t seed,
                           int64_t first, int64_t count,
                           double *f0, double *tau, double *n)
{
    for (int64_t i = 0; i < count; ++i) {
        int64_t t = first + i;
        double v[3];
        if (kind == 0) {
            int64_t idx[3] = {t % n_f0, (t / n_f0) % n_tau, t / (n_f0 * n_tau)};
            int64_t m[3] = {n_f0, n_tau, n_n};
            for (int a = 0; a < 3; ++a) v[a] = oracle_lattice_axis(lo[a], hi[a], m[a], idx[a]);
        } else {
            uint64_t ctr[4] = {(uint64_t)t, 0, 0, 0}, key[2] = {seed, 0}, x[4];
            oracle_philox4x64_10(ctr, key, x);
            for (int a = 0; a < 3; ++a) {
                double u = (double)(x[a] >> 11) * 0x1p-53;
                v[a] = fma(hi[a] - lo[a], u, lo[a]);
            }
        }
        f0[i] = v[0];
        tau[i] = v[1];
        n[i] = v[2];
    }
}
