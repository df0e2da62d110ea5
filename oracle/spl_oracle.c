/*
 * FP64 CPU oracle for the robust depth estimate and the online spatio-temporal filter of
 * "Robust 3D reconstruction of dynamic scenes from single-photon lidar using Beta-divergences"
 * (Legros et al., arXiv 2004.09211).
 *
 * TEST INFRASTRUCTURE. This file is the plain, slow, obviously correct statement of what the CUDA library
 * computes. It is loaded only by the tests, by the package's smoke check and by the benchmark's CPU-baseline
 * leg; the library itself never calls it. It shares no code, header, table or constant with the CUDA
 * sources. Every function works in double precision on host arrays and follows the paper's definitions in
 * the paper's order, with no blocking, pruning or reordering.
 *
 * Conventions (readings of the paper, each one stated where it is used):
 *   - Time and depth are measured in histogram bins; 2d/c is never formed (Sec. IV gives sigma_RW in bins).
 *   - h[0..L) is the tabulated IRF and `peak` = j_p the index of its maximum. A surface at depth d puts tap j
 *     in bin t = d - peak + j, i.e. the template is s_d[t] = h[t - d + peak], zero outside [0, L).
 *   - The candidate depths are the integers d in [dmin, dmax], inside the full-support range
 *     [peak, T - L + peak]. On that range every template lies inside the histogram, which is what makes the
 *     integral of f0^(1+beta) independent of d (the condition stated after Eq. beta_div2).
 *   - 0^beta = 0 (an IRF tap of zero contributes nothing).
 *
 * Parity pins (all in tests/test_oracle_pins.py): beta = 1 against numpy.correlate (matched filter,
 * Sec. II-B); the photon-list form of Eq. beta_div2 against the histogram form; strict argmax recovery on
 * noiseless templates (Hoelder); invariance of sum s_d^(1+beta) over the domain; a one-photon box-IRF
 * closed form of the posterior moments; posterior = prior on an empty histogram (Gaussian moments);
 * translation equivariance and the dependency cone of the filter; the box-IRF closed form of the intensity
 * MLE and its KKT conditions checked by scipy; the fixed points of Eq. prior_detect; for the detection
 * surrogate, the box-IRF closed form of the two-region Poisson likelihood ratio, the logistic combination with
 * pi0 and its limits; for the sub-bin grid, the reduction to the integer grid at S = 1, the half-bin average
 * at beta = 1 (linear interpolation commutes with the correlation), translation and the empty histogram; for the
 * multispectral product (Appendix), the reduction to the single-band estimate for one band, the photon-list form of
 * Eq. div_MSL, identical bands, strict recovery of noiseless multi-band templates, empty bands and band order.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
    int T;            /* histogram bins N_T                                   */
    int L;            /* IRF taps                                             */
    int peak;         /* index j_p of the IRF maximum                         */
    int dmin, dmax;   /* candidate depth range, inclusive, in bins            */
    double beta;      /* divergence parameter beta > 0                        */
    double sigma_rw2; /* random-walk variance sigma_RW^2 (s^2 in Algorithm 1)  */
    double nu[9];     /* 3x3 mixture weights, row-major, centre nu[4]         */
} orc_params;

/* ---------------------------------------------------------------------------------------------------- */
/* Set-up                                                                                                */
/* ---------------------------------------------------------------------------------------------------- */

int orc_set_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
    return omp_get_max_threads();
#else
    (void)n;
    return 1;
#endif
}

/* 0 when the candidate range lies inside the full-support range [peak, T - L + peak] (the reading of the
 * "shape never changes" condition of Sec. II-B and Sec. III-A); nonzero otherwise. */
int orc_check_domain(const orc_params* q) {
    if (q->T < 1 || q->L < 1 || q->L > q->T) return 1;
    if (q->peak < 0 || q->peak >= q->L) return 2;
    if (q->dmin > q->dmax) return 3;
    if (q->dmin < q->peak || q->dmax > q->T - q->L + q->peak) return 4;
    if (!(q->beta > 0.0)) return 5;
    return 0;
}

/* powered IRF value h^beta with 0^beta = 0 */
static double powb(double h, double beta) { return h > 0.0 ? pow(h, beta) : 0.0; }

/* template value s_d[t] = h[t - d + peak] (zero outside the taps) -- Eq. lik_ideal_poisson */
static double tmpl(const orc_params* q, const double* h, int d, int t) {
    int j = t - d + q->peak;
    return (j >= 0 && j < q->L) ? h[j] : 0.0;
}

/* sum_t s_d[t]^expo over the whole histogram: the integral of f0^(1+beta) that Eq. beta_div2 drops as a
 * constant. Used by the shift-invariance pin. */
double orc_template_power_sum(const orc_params* q, const double* h, int d, double expo) {
    double s = 0.0;
    for (int t = 0; t < q->T; ++t) s += powb(tmpl(q, h, d, t), expo);
    return s;
}

/* ---------------------------------------------------------------------------------------------------- */
/* Robust data term: C(d) = z^T s_d^beta (histogram form of Eq. beta_div2, Sec. II-B)                   */
/* ---------------------------------------------------------------------------------------------------- */

static void cost_one(const orc_params* q, const double* h, const double* z, double* C) {
    const int D = q->dmax - q->dmin + 1;
    for (int k = 0; k < D; ++k) {
        const int d = q->dmin + k;
        double c = 0.0;
        for (int t = d - q->peak; t < d - q->peak + q->L; ++t)   /* support of s_d */
            c += z[t] * powb(tmpl(q, h, d, t), q->beta);
        C[k] = c;
    }
}

/* C[p][k] = C(dmin + k) for each of the P histograms z[p][0..T). */
void orc_cost(const orc_params* q, const double* h, const double* z, long P, double* C) {
    const int D = q->dmax - q->dmin + 1;
#pragma omp parallel for schedule(dynamic, 16)
    for (long p = 0; p < P; ++p) cost_one(q, h, z + p * (long)q->T, C + p * (long)D);
}

/* Photon-list form of Eq. beta_div2 without the 1/K: sum over photons k of f0(y_k | d)^beta, the ToA bins
 * y[0..K). */
void orc_cost_toa(const orc_params* q, const double* h, const int32_t* y, int K, double* C) {
    const int D = q->dmax - q->dmin + 1;
    for (int k = 0; k < D; ++k) {
        const int d = q->dmin + k;
        double c = 0.0;
        for (int i = 0; i < K; ++i) c += powb(tmpl(q, h, d, y[i]), q->beta);
        C[k] = c;
    }
}

/* ---------------------------------------------------------------------------------------------------- */
/* Pseudo-posterior (Eq. approx_post) and its moments (numerical integration on the grid, Sec. II-C)     */
/* ---------------------------------------------------------------------------------------------------- */

/* ell[k] = log pseudo-posterior (up to a constant) at d = dmin + k. Writes the smallest maximiser, the mean
 * and the variance of the normalised weights exp(ell - max). Variance is taken in two passes. */
void orc_posterior(int D, int dmin, const double* ell, int* argmax, double* mu, double* var) {
    int a = 0;
    for (int k = 1; k < D; ++k)
        if (ell[k] > ell[a]) a = k;
    const double m = ell[a];
    double s0 = 0.0, s1 = 0.0;
    for (int k = 0; k < D; ++k) {
        const double w = exp(ell[k] - m);
        s0 += w;
        s1 += w * (double)(dmin + k);
    }
    const double mean = s1 / s0;
    double s2 = 0.0;
    for (int k = 0; k < D; ++k) {
        const double w = exp(ell[k] - m);
        const double e = (double)(dmin + k) - mean;
        s2 += w * e * e;
    }
    *argmax = dmin + a;
    *mu = mean;
    *var = s2 / s0;
}

/* log of the Gaussian mixture sum_c nu_c N(d; m_c, s2_c), by log-sum-exp. */
double orc_log_mixture(int n, const double* nu, const double* m, const double* s2, double d) {
    double lt[9];
    double mx = -INFINITY;
    for (int c = 0; c < n; ++c) {
        const double e = d - m[c];
        lt[c] = log(nu[c]) - 0.5 * log(2.0 * M_PI * s2[c]) - e * e / (2.0 * s2[c]);
        if (lt[c] > mx) mx = lt[c];
    }
    double s = 0.0;
    for (int c = 0; c < n; ++c) s += exp(lt[c] - mx);
    return mx + log(s);
}

/* lambda = (beta + 1) / beta: the factor in K * CE_beta(d) = -lambda * C(d) (Eq. beta_CE). */
static double lambda_of(double beta) { return (beta + 1.0) / beta; }

/* Single-frame estimate. With prior_mu == NULL the prior is uniform on [dmin, dmax], so the argmax is the
 * minimum-divergence estimator of Sec. II-B; otherwise the prior is N(prior_mu[p], prior_var[p]).
 * ell_out (nullable) receives ell[p][k]. */
void orc_estimate(const orc_params* q, const double* h, const double* z, long P, const double* prior_mu,
                  const double* prior_var, int* argmax, double* mu, double* var, double* ell_out) {
    const int D = q->dmax - q->dmin + 1;
    const double lam = lambda_of(q->beta);
#pragma omp parallel
    {
        double* C = (double*)malloc(sizeof(double) * D);
        double* ell = (double*)malloc(sizeof(double) * D);
#pragma omp for schedule(dynamic, 16)
        for (long p = 0; p < P; ++p) {
            cost_one(q, h, z + p * (long)q->T, C);
            for (int k = 0; k < D; ++k) {
                double lp = 0.0;
                if (prior_mu) {
                    const double one = 1.0, m = prior_mu[p], s2 = prior_var[p];
                    lp = orc_log_mixture(1, &one, &m, &s2, (double)(q->dmin + k));
                }
                ell[k] = lam * C[k] + lp;
            }
            orc_posterior(D, q->dmin, ell, argmax + p, mu + p, var + p);
            if (ell_out) memcpy(ell_out + p * (long)D, ell, sizeof(double) * D);
        }
        free(C);
        free(ell);
    }
}

/* ---------------------------------------------------------------------------------------------------- */
/* Multispectral data (Appendix, Eq. div_MSL)                                                           */
/* ---------------------------------------------------------------------------------------------------- */

/* nb bands recorded at once by independent detectors: the ideal model is the product over bands of the band
 * models f_l(y_l | d) = s_l(y_l - 2d/c), and the beta-divergence between the product of the empirical marginals and
 * that model is, up to a constant, -lambda * M(d) with
 *     M(d) = prod_l (1 / K_l) sum_k f_l(y_{l,k} | d)^beta = prod_l C_l(d) / K_l,
 * C_l(d) the histogram form of band l's sum (Eq. beta_div2 with band l's IRF h_l) and K_l its photon count.
 * Readings: a band with K_l = 0 has no empirical distribution and contributes no factor; every band has L taps
 * and the same peak index. The pseudo-posterior (a reading: the paper defines only the minimum-divergence
 * estimator for these data) is f(d) exp(lambda K M(d)), K = sum_l K_l, which for one band is the single-band
 * pseudo-posterior exp(lambda C(d)) of Eq. approx_post. Layouts: h[l][0..L), z[l][p][0..T).
 * Outputs per pixel: argmax (smallest maximiser of ell; with no prior, of M: the minimum-divergence estimate),
 * mean and variance of the pseudo-posterior; M_out[p][k] (nullable) = M(dmin + k); ell_out (nullable). */
void orc_estimate_msl(const orc_params* q, int nb, const double* h, const double* z, long P, const double* prior_mu,
                      const double* prior_var, int* argmax, double* mu, double* var, double* M_out, double* ell_out) {
    const int D = q->dmax - q->dmin + 1;
    const double lam = lambda_of(q->beta);
#pragma omp parallel
    {
        double* C = (double*)malloc(sizeof(double) * D);
        double* M = (double*)malloc(sizeof(double) * D);
        double* ell = (double*)malloc(sizeof(double) * D);
#pragma omp for schedule(dynamic, 16)
        for (long p = 0; p < P; ++p) {
            for (int k = 0; k < D; ++k) M[k] = 1.0;
            double Ktot = 0.0;
            for (int l = 0; l < nb; ++l) {
                const double* zl = z + ((long)l * P + p) * (long)q->T;
                double Kl = 0.0;
                for (int t = 0; t < q->T; ++t) Kl += zl[t];
                if (Kl <= 0.0) continue;
                cost_one(q, h + (long)l * q->L, zl, C);
                for (int k = 0; k < D; ++k) M[k] *= C[k] / Kl;
                Ktot += Kl;
            }
            for (int k = 0; k < D; ++k) {
                double lp = 0.0;
                if (prior_mu) {
                    const double one = 1.0, m = prior_mu[p], s2 = prior_var[p];
                    lp = orc_log_mixture(1, &one, &m, &s2, (double)(q->dmin + k));
                }
                ell[k] = (Ktot > 0.0 ? lam * Ktot * M[k] : 0.0) + lp;
            }
            orc_posterior(D, q->dmin, ell, argmax + p, mu + p, var + p);
            if (M_out) memcpy(M_out + p * (long)D, M, sizeof(double) * D);
            if (ell_out) memcpy(ell_out + p * (long)D, ell, sizeof(double) * D);
        }
        free(C);
        free(M);
        free(ell);
    }
}

/* ---------------------------------------------------------------------------------------------------- */
/* Sub-bin depth: Eq. beta_div2 with a continuous IRF on a fine candidate grid                           */
/* ---------------------------------------------------------------------------------------------------- */

/* Continuous IRF from the taps (a reading: the paper's continuous model, Eq. lik_ideal and Eq. beta_div2 over
 * continuous ToAs, uses the instrument's continuous response, of which the tabulated taps are samples):
 * piecewise-linear interpolation of h[0..L) with h[-1] = h[L] = 0, i.e. support (-1, L). Taps <= 0 (or NaN)
 * count as 0 before the interpolation, as they do on the integer grid. */
static double irf_c(const orc_params* q, const double* h, double x) {
    if (!(x > -1.0) || !(x < (double)q->L)) return 0.0;
    const double fl = floor(x);
    const int j = (int)fl;
    const double w = x - fl;
    const double a = (j >= 0 && h[j] > 0.0) ? h[j] : 0.0;
    const double b = (j + 1 < q->L && h[j + 1] > 0.0) ? h[j + 1] : 0.0;
    return (1.0 - w) * a + w * b;
}

/* Single-frame estimate on the fine grid d_k = dmin + k / S, k = 0 .. (dmax - dmin) S. The binned template of a
 * surface at d is s_d[t] = h_c(t - d + peak) (for whole-bin d the taps themselves); the data term of Eq.
 * beta_div2 is C(d) = sum_t z_t s_d[t]^beta (0^beta = 0). The pseudo-likelihood is exp(-K D_beta) with the
 * beta-divergence between the histogram (normalised by its photon count K) and s_d, whose d-dependent part is
 * lambda C(d) / K - sum_t s_d[t]^(1+beta): Eq. beta_div2 drops the second sum because it is the same for every
 * whole-bin shift (Sec. II-B); at fractional shifts the interpolated template's power changes with the phase,
 * so it is kept here:
 *     ell(d) = lambda C(d) - K sum_t s_d[t]^(1+beta) + log N(d; prior_mu[p], prior_var[p])
 * (uniform without a prior). Outputs the smallest maximising index k, and the mean and variance of the
 * normalised weights on the fine grid (two passes). With S = 1 the kept sum is one constant and this is
 * orc_estimate. ell_out / cost_out (nullable) receive ell[p][k] and C[p][k]. */
void orc_estimate_fine(const orc_params* q, int S, const double* h, const double* z, long P,
                       const double* prior_mu, const double* prior_var, int* argmax_k, double* mu, double* var,
                       double* ell_out, double* cost_out) {
    const int Kf = (q->dmax - q->dmin) * S + 1;
    const double lam = lambda_of(q->beta);
#pragma omp parallel
    {
        double* ell = (double*)malloc(sizeof(double) * Kf);
#pragma omp for schedule(dynamic, 16)
        for (long p = 0; p < P; ++p) {
            const double* zp = z + p * (long)q->T;
            double K = 0.0;
            for (int t = 0; t < q->T; ++t) K += zp[t];
            for (int k = 0; k < Kf; ++k) {
                const double d = q->dmin + (double)k / S;
                double c = 0.0, pw = 0.0;
                for (int t = 0; t < q->T; ++t) {
                    const double x = t - d + q->peak;
                    if (!(x > -1.0 && x < (double)q->L)) continue;
                    const double sv = irf_c(q, h, x);
                    if (zp[t] != 0.0) c += zp[t] * powb(sv, q->beta);
                    pw += powb(sv, 1.0 + q->beta);
                }
                double lp = 0.0;
                if (prior_mu) {
                    const double one = 1.0, m = prior_mu[p], s2 = prior_var[p];
                    lp = orc_log_mixture(1, &one, &m, &s2, d);
                }
                ell[k] = lam * c - K * pw + lp;
                if (cost_out) cost_out[p * (long)Kf + k] = c;
            }
            int a = 0;
            for (int k = 1; k < Kf; ++k)
                if (ell[k] > ell[a]) a = k;
            double s0 = 0.0, s1 = 0.0;
            for (int k = 0; k < Kf; ++k) {
                const double w = exp(ell[k] - ell[a]);
                s0 += w;
                s1 += w * (q->dmin + (double)k / S);
            }
            const double mean = s1 / s0;
            double s2 = 0.0;
            for (int k = 0; k < Kf; ++k) {
                const double w = exp(ell[k] - ell[a]);
                const double e = q->dmin + (double)k / S - mean;
                s2 += w * e * e;
            }
            argmax_k[p] = a;
            mu[p] = mean;
            var[p] = s2 / s0;
            if (ell_out) memcpy(ell_out + p * (long)Kf, ell, sizeof(double) * Kf);
        }
        free(ell);
    }
}

/* ---------------------------------------------------------------------------------------------------- */
/* Spatio-temporal prior (Eq. predict with the ADF Gaussians of Eq. KL_div) and one filter step           */
/* ---------------------------------------------------------------------------------------------------- */

/* Components of the prior of pixel (y, x): one per stencil entry with nu > 0. A neighbour that is inside
 * the image, present (its detection at the previous frame) and not faulty contributes N(mu, var + s^2):
 * its Gaussian q convolved with the random walk. Any other entry contributes the weakly informative
 * N((dmin+dmax)/2, (dmax-dmin)^2/12 + s^2) (Sec. III-A: absent pixels and pixels outside the field of
 * view; the random walk is applied to it as to every q). Weights are used as given. Returns the count. */
static int prior_components(const orc_params* q, int H, int W, int y, int x, const double* mu_in,
                            const double* var_in, const uint8_t* present_in, const uint8_t* faulty,
                            double* nu, double* m, double* s2) {
    const double flat_m = 0.5 * (q->dmin + q->dmax);
    const double flat_v = (double)(q->dmax - q->dmin) * (double)(q->dmax - q->dmin) / 12.0;
    int n = 0;
    for (int k = 0; k < 9; ++k) {
        if (!(q->nu[k] > 0.0)) continue;
        const int yy = y + k / 3 - 1, xx = x + k % 3 - 1;
        int informative = 0;
        long i = 0;
        if (yy >= 0 && yy < H && xx >= 0 && xx < W) {
            i = (long)yy * W + xx;
            informative = (present_in ? present_in[i] != 0 : 1) && !(faulty && faulty[i]);
        }
        nu[n] = q->nu[k];
        m[n] = informative ? mu_in[i] : flat_m;
        s2[n] = (informative ? var_in[i] : flat_v) + q->sigma_rw2;
        ++n;
    }
    return n;
}

/* One outer iteration of Algorithm 1 for the whole frame: prior from the previous frame's Gaussians,
 * pseudo-posterior with this frame's histograms, moment matching. A faulty pixel has no data: its
 * pseudo-posterior is its prior (Sec. III-B). present_in / faulty may be NULL (all present / none faulty).
 * ell_out (nullable) receives ell[p][k]. */
void orc_filter_step(const orc_params* q, int H, int W, const double* h, const double* z,
                     const uint8_t* faulty, const double* mu_in, const double* var_in,
                     const uint8_t* present_in, int* argmax, double* mu_out, double* var_out,
                     double* ell_out) {
    const int D = q->dmax - q->dmin + 1;
    const double lam = lambda_of(q->beta);
    const long P = (long)H * W;
#pragma omp parallel
    {
        double* C = (double*)malloc(sizeof(double) * D);
        double* ell = (double*)malloc(sizeof(double) * D);
#pragma omp for schedule(dynamic, 16)
        for (long p = 0; p < P; ++p) {
            const int y = (int)(p / W), x = (int)(p % W);
            double nu[9], m[9], s2[9];
            const int nc = prior_components(q, H, W, y, x, mu_in, var_in, present_in, faulty, nu, m, s2);
            const int has_data = !(faulty && faulty[p]);
            if (has_data) cost_one(q, h, z + p * (long)q->T, C);
            for (int k = 0; k < D; ++k)
                ell[k] = (has_data ? lam * C[k] : 0.0) +
                         orc_log_mixture(nc, nu, m, s2, (double)(q->dmin + k));
            orc_posterior(D, q->dmin, ell, argmax + p, mu_out + p, var_out + p);
            if (ell_out) memcpy(ell_out + p * (long)D, ell, sizeof(double) * D);
        }
        free(C);
        free(ell);
    }
}

/* ---------------------------------------------------------------------------------------------------- */
/* Background and reflectivity (Sec. II-E)                                                              */
/* ---------------------------------------------------------------------------------------------------- */

/* Maximum-likelihood (r, b) of Eq. lik_bg_poisson, z_t ~ P(r h[t - dr + peak] + b), with the template at
 * the integer position dr. The log-likelihood is concave in (r, b) and its maximiser satisfies
 * r * sum(h) + b * T = K (sum of the two stationarity conditions, and also true on the boundaries r = 0,
 * b = 0), so the MLE is the maximiser of the concave restriction phi(r) on r in [0, K / sum(h)]. phi' is
 * decreasing; the root is found by bisection to full double precision. */
void orc_intensity_mle(const orc_params* q, const double* h, const double* z, int dr, double* r_out,
                       double* b_out) {
    const int T = q->T, L = q->L, t0 = dr - q->peak;
    if (t0 < 0 || t0 > T - L) {          /* template must lie inside the histogram */
        *r_out = NAN;
        *b_out = NAN;
        return;
    }
    double K = 0.0, Kin = 0.0, Hs = 0.0;
    for (int t = 0; t < T; ++t) K += z[t];
    for (int j = 0; j < L; ++j) {
        Kin += z[t0 + j];
        Hs += h[j];
    }
    const double Kout = K - Kin;
    if (K <= 0.0 || Hs <= 0.0) {
        *r_out = 0.0;
        *b_out = K / T;
        return;
    }
    const double rmax = K / Hs;
    /* phi'(r) = sum_W z_t (h_t - Hs/T) / (r h_t + b) - (Hs/T) Kout / b, b = (K - r Hs) / T; valid for
     * r < rmax where b > 0. */
#define DPHI(r, out)                                                         \
    do {                                                                     \
        const double b_ = (K - (r) * Hs) / T;                                \
        double g_ = -(Hs / T) * Kout / b_;                                   \
        for (int j = 0; j < L; ++j)                                          \
            if (z[t0 + j] != 0.0) g_ += z[t0 + j] * (h[j] - Hs / T) / ((r) * h[j] + b_); \
        (out) = g_;                                                          \
    } while (0)
    double g0;
    DPHI(0.0, g0);
    double r;
    if (g0 <= 0.0) {
        r = 0.0;
    } else {
        double lo = 0.0, hi = rmax;
        for (int it = 0; it < 400 && hi - lo > 1e-16 * rmax; ++it) {
            const double mid = 0.5 * (lo + hi);
            if (!(mid < rmax)) break;
            double g;
            DPHI(mid, g);
            if (g > 0.0) lo = mid; else hi = mid;
        }
        r = 0.5 * (lo + hi);
    }
#undef DPHI
    double b = (K - r * Hs) / T;
    if (b < 0.0) b = 0.0;
    *r_out = r;
    *b_out = b;
}

/* Per pixel: absent -> b = K / T, r = 0; present -> the MLE above with the template at round(mu) (round half
 * to even, the depth point estimate being the posterior mean). dr (nullable) overrides the template
 * position per pixel. Faulty pixels have no data: r = b = 0. */
void orc_intensity(const orc_params* q, const double* h, const double* z, long P, const double* mu,
                   const int32_t* dr, const uint8_t* present, const uint8_t* faulty, double* refl,
                   double* bg) {
#pragma omp parallel for schedule(dynamic, 64)
    for (long p = 0; p < P; ++p) {
        const double* zp = z + p * (long)q->T;
        if (faulty && faulty[p]) {
            refl[p] = 0.0;
            bg[p] = 0.0;
            continue;
        }
        if (present && !present[p]) {
            double K = 0.0;
            for (int t = 0; t < q->T; ++t) K += zp[t];
            refl[p] = 0.0;
            bg[p] = K / q->T;
            continue;
        }
        const int d = dr ? dr[p] : (int)rint(mu[p]);
        orc_intensity_mle(q, h, zp, d, refl + p, bg + p);
    }
}

/* ---------------------------------------------------------------------------------------------------- */
/* Presence probability: a detection surrogate                                                          */
/* ---------------------------------------------------------------------------------------------------- */

/* Log-likelihood ratio of Eq. lik_bg_poisson between (r, b) with the template at the integer position dr and
 * the background-only model (r = 0, b = K / T), summed over every bin t of the histogram:
 *     sum_t z_t log(lambda_t / lambda0) - sum_t (lambda_t - lambda0),
 *     lambda_t = r h[t - dr + peak] + b,  lambda0 = K / T  (the log z_t! terms cancel).
 * A bin with z_t > 0 and lambda_t = 0 makes the ratio -infinity. */
double orc_log_lik_ratio(const orc_params* q, const double* h, const double* z, int dr, double r, double b) {
    const int T = q->T;
    double K = 0.0;
    for (int t = 0; t < T; ++t) K += z[t];
    if (K <= 0.0) return 0.0;
    const double l0 = K / T;
    double s = 0.0;
    for (int t = 0; t < T; ++t) {
        const double lam = r * tmpl(q, h, dr, t) + b;
        if (z[t] > 0.0) s += (lam > 0.0) ? z[t] * log(lam / l0) : -INFINITY;
        s -= lam - l0;
    }
    return s;
}

/* Detection surrogate. The paper decides presence with the Bayesian test of [TachellaSPIE2019] (Sec. II-E,
 * Algorithm 1 step "Estimate pi", Sec. III-B), which it cites but does not define; that test marginalises the
 * depth with the pseudo-posterior as its prior (Sec. III-B, empirical Bayes). This surrogate keeps the test's
 * inputs and output -- the likelihood Eq. lik_bg_poisson, the pseudo-posterior, the prior probability of
 * presence pi0 of Eq. prior_detect, and the posterior probability pi of r > 0 -- and replaces the
 * marginalisations by their maximum-point (Laplace / Bayesian-information-criterion) approximations:
 *   - depth: Laplace's method for the integral of the likelihood ratio against the pseudo-posterior (variance
 *     var) at its mode dmap; the likelihood ratio's width in depth is taken as the template's, sigma_h^2 =
 *     sum_j a_j (j - mean)^2 with a = max(h, 0) / sum(max(h, 0)), and a pseudo-posterior narrower than that
 *     costs nothing: the Occam term is max(0, (1/2) log(var / sigma_h^2));
 *   - (r, b): their maximum likelihood, one extra parameter (r) over about K photons: (1/2) log max(K, 1).
 *     log BF = LLR(dmap; r_hat, b_hat) - (1/2) log max(K, 1) - max(0, (1/2) log(var / sigma_h^2)),
 *     pi = sigmoid(logit(pi0) + log BF),
 * with (r_hat, b_hat) from orc_intensity_mle at dmap and LLR from orc_log_lik_ratio. pi0 (nullable: 0.5
 * everywhere) is limited to [1e-7, 1 - 1e-7] as in Eq. prior_detect. Faulty pixels: pi = 0.5, r = b = 0
 * (Sec. III-B). Then Algorithm 1's branch with the intensity rule of Sec. II-E: present = pi > 0.5 gives the
 * MLE (r, b) with the template at the depth point estimate round-half-even(mu); absent gives r = 0, b = K / T.
 * dmap nullable: round-half-even(mu); var nullable: no Occam term. llr (nullable) receives LLR (0 for faulty
 * pixels). */
void orc_detect(const orc_params* q, const double* h, const double* z, long P, const double* mu, const int32_t* dmap,
                const double* var, const double* pi0, const uint8_t* faulty, double* pi, double* llr,
                uint8_t* present, double* refl, double* bg) {
    double hs = 0.0, hm = 0.0, hv = 0.0;
    for (int j = 0; j < q->L; ++j) {
        const double a = h[j] > 0.0 ? h[j] : 0.0;
        hs += a;
        hm += a * j;
    }
    if (hs > 0.0) {
        hm /= hs;
        for (int j = 0; j < q->L; ++j) {
            const double a = h[j] > 0.0 ? h[j] : 0.0;
            hv += a / hs * (j - hm) * (j - hm);
        }
    }
#pragma omp parallel for schedule(dynamic, 64)
    for (long p = 0; p < P; ++p) {
        const double* zp = z + p * (long)q->T;
        if (faulty && faulty[p]) {
            pi[p] = 0.5;
            if (llr) llr[p] = 0.0;
            present[p] = 0;
            refl[p] = 0.0;
            bg[p] = 0.0;
            continue;
        }
        double K = 0.0;
        for (int t = 0; t < q->T; ++t) K += zp[t];
        const int d = (int)rint(mu[p]), dm = dmap ? dmap[p] : d;
        double r, b, rm, bm;
        orc_intensity_mle(q, h, zp, d, &r, &b);
        orc_intensity_mle(q, h, zp, dm, &rm, &bm);
        const double l = orc_log_lik_ratio(q, h, zp, dm, rm, bm);
        const double lmax = log(1e7 - 1.0);
        const double v = pi0 ? pi0[p] : 0.5;
        double lg = log(v) - log1p(-v);
        if (!(lg > -lmax)) lg = -lmax;
        if (!(lg < lmax)) lg = lmax;
        double occam = 0.0;
        if (var && hv > 0.0 && var[p] > hv) occam = 0.5 * log(var[p] / hv);
        const double x = lg + l - 0.5 * log(K > 1.0 ? K : 1.0) - occam;
        pi[p] = 1.0 / (1.0 + exp(-x));
        if (llr) llr[p] = l;
        present[p] = pi[p] > 0.5;
        if (present[p]) {
            refl[p] = r;
            bg[p] = b;
        } else {
            refl[p] = 0.0;
            bg[p] = K / q->T;
        }
    }
}

/* ---------------------------------------------------------------------------------------------------- */
/* Prior probability of presence (Eq. prior_detect)                                                     */
/* ---------------------------------------------------------------------------------------------------- */

/* pi0[p] = sigmoid(sum_k nu_k logit(pi[p + k])). Readings: a neighbour outside the image enters with
 * pi = 0.5 (logit 0, no information); a faulty pixel has pi = 0.5 (Sec. III-B), both as input and as
 * output; pi is limited to [1e-7, 1 - 1e-7] before the logit, applied as the equivalent clamp of the logit
 * to +-log(1e7 - 1) (logit is monotone), so that a single-precision implementation clamps at the same
 * value. */
void orc_pi_propagate(int H, int W, const double* nu, const double* pi_in, const uint8_t* faulty,
                      double* pi_out) {
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
            const long p = (long)y * W + x;
            if (faulty && faulty[p]) {
                pi_out[p] = 0.5;
                continue;
            }
            double a = 0.0;
            for (int k = 0; k < 9; ++k) {
                const int yy = y + k / 3 - 1, xx = x + k % 3 - 1;
                double v = 0.5;
                if (yy >= 0 && yy < H && xx >= 0 && xx < W) {
                    const long i = (long)yy * W + xx;
                    v = (faulty && faulty[i]) ? 0.5 : pi_in[i];
                }
                const double lmax = log(1e7 - 1.0);
                double lg = log(v) - log1p(-v);
                if (!(lg > -lmax)) lg = -lmax;
                if (!(lg < lmax)) lg = lmax;
                a += nu[k] * lg;
            }
            pi_out[p] = 1.0 / (1.0 + exp(-a));
        }
}
