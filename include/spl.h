/*
 * spl.h -- C ABI of libspl, the CUDA (sm_103a) hot path of the online robust depth reconstruction method of
 * "Robust 3D reconstruction of dynamic scenes from single-photon lidar using Beta-divergences"
 * (Legros et al., arXiv 2004.09211).
 *
 * General conventions
 *   - Every array argument is a DEVICE pointer to memory the caller allocated and owns, unless the comment
 *     says "host". The library keeps no pointer after a call returns.
 *   - Calls are asynchronous: they validate their arguments on the host, enqueue kernels on `stream`
 *     (a cudaStream_t passed as void*; NULL = the legacy default stream) and return. No call synchronises the
 *     device, allocates device memory or copies device data to the host.
 *   - Argument errors are reported before anything is launched: the call returns SPL_EINVAL and
 *     spl_last_error() (a per-thread message) says which argument is wrong. A failed launch returns SPL_ECUDA.
 *   - Depth and time are measured in histogram bins. h[0..L) is the tabulated instrument response (IRF) and
 *     `peak` the index j_p of its maximum; a surface at depth d puts tap j in bin t = d - peak + j, i.e. the
 *     template is s_d[t] = h[t - d + peak] (Eq. lik_ideal_poisson, Sec. II-D: the surface sits at the IRF
 *     maximum).
 *   - Candidate depths are the integers dmin..dmax (D = dmax - dmin + 1 of them). They must lie in the
 *     full-support range [peak, T - L + peak], on which every template lies inside the histogram; that is the
 *     condition under which the integral of f0^(1+beta) does not depend on d (Sec. II-B, below Eq. beta_div2,
 *     and Sec. III-A on choosing T).
 *   - IRF taps that are <= 0 or NaN count as zero (0^beta = 0). The IRF is used as given, never renormalised.
 *   - Per-pixel maps are [H][W] row-major. Histograms are [P][pitch] with P = H*W; see spl_hist.
 */
#ifndef SPL_H
#define SPL_H

#include <stdint.h>

#if defined(__GNUC__)
#define SPL_API __attribute__((visibility("default")))
#else
#define SPL_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    SPL_OK = 0,
    SPL_EINVAL = 1,       /* invalid argument (checked on the host, nothing launched) */
    SPL_ENOMEM = 2,       /* the call needed memory it could not get */
    SPL_ECUDA = 3,        /* a CUDA launch or runtime call failed; spl_last_error() has the CUDA message */
    SPL_ETIMEOUT = 4,     /* a bounded device-side wait ran out */
    SPL_EUNSUPPORTED = 5  /* valid request outside what the library supports (e.g. L above SPL_MAX_TAPS) */
} spl_status;

/* Storage of the photon-count histograms z. Counts are non-negative integers in every format. */
typedef enum {
    SPL_HIST_U16 = 0,     /* uint16 counts                                      */
    SPL_HIST_F16 = 1,     /* IEEE half counts (integers up to 2048 are exact)   */
    SPL_HIST_F32 = 2      /* float counts                                       */
} spl_hist_format;

/* Largest IRF length and histogram length the library supports. */
#define SPL_MAX_TAPS 128
#define SPL_MAX_BINS 8192

/* Histogram cube of one frame: pixel p's counts z_p[0..T) start at element p * pitch of `data`. pitch >= T,
 * and pitch * element size must be a multiple of 16 bytes with `data` 16-byte aligned, so every row can be
 * read with 16-byte loads. Elements T..pitch-1 are ignored. */
typedef struct {
    spl_hist_format fmt;
    const void* data;     /* device */
    int64_t pitch;        /* elements between consecutive pixels */
} spl_hist;

/* Fixed inputs of one frame (Algorithm 1's fixed parameters plus the problem geometry). */
typedef struct {
    int32_t H, W;         /* pixels per frame (P = H*W)                                         */
    int32_t T;            /* histogram bins N_T (Eq. lik_ideal_poisson)                         */
    int32_t L, peak;      /* IRF taps and the index of the IRF maximum                          */
    int32_t dmin, dmax;   /* candidate depths, inclusive; see the conventions above             */
    float beta;           /* beta-divergence parameter, > 0 (Eq. beta_div)                      */
    float sigma_rw2;      /* random-walk variance sigma_RW^2 = s^2 of Algorithm 1, > 0          */
    float nu[9];          /* 3x3 mixture weights of Eq. predict, row-major, nu[4] = centre;
                             the paper's M = 5 choice is nu0 at the centre and (1 - nu0)/4 on the
                             four edge neighbours. Each >= 0, finite, sum > 0.                  */
} spl_params;

/* Version string of the library. */
SPL_API const char* spl_version(void);

/* Message of the last failed call on this thread ("" if none). Valid until the next call on the thread. */
SPL_API const char* spl_last_error(void);

/*
 * spl_depth_cost -- robust data term for every candidate depth (Sec. II-B).
 *   C(d) = sum_t z_t h[t - d + peak]^beta, the histogram form of Eq. beta_div2: minimising the
 *   beta-divergence between the empirical ToA distribution and f0(.|d) maximises z^T s_d^beta.
 *   cost   : [P][D] float, cost[p][k] = C(dmin + k). May be NULL if only argmax is wanted.
 *   argmax : [P] int32 (nullable) = the smallest d maximising C(d): the minimum-divergence estimator.
 *   h      : [L] float IRF (device).
 *   Uses H, W, T, L, peak, dmin, dmax, beta of prm.
 */
SPL_API spl_status spl_depth_cost(const spl_params* prm, const spl_hist* z, const float* h, float* cost,
                          int32_t* argmax, void* stream);

/*
 * spl_depth_cost_tc -- the robust data term of spl_depth_cost on the tensor cores (mixed precision).
 *   Same outputs as spl_depth_cost (cost [P][D] = C(dmin + k), argmax nullable), from FP16 histograms
 *   (SPL_HIST_F16; integer counts up to 2048 are exact in FP16). C is computed as a banded-Toeplitz matrix
 *   product (128 pixels x 64 candidates per tile) with FP16 operands and FP32 accumulation: the powered IRF
 *   g = h^beta is scaled by 2^15 and split into an FP16 high part and an FP16 low part whose products both
 *   accumulate, so each tap carries about 22 significant bits (relative cost error ~1e-6 against FP64).
 *   Requires L <= SPL_MAX_TAPS. A bounded internal wait that runs out sets flag 1 of spl_tc_status.
 */
SPL_API spl_status spl_depth_cost_tc(const spl_params* prm, const spl_hist* z, const float* h, float* cost,
                                     int32_t* argmax, void* stream);

/* Reads and clears the tensor-core kernels' device condition flags (synchronous). */
SPL_API spl_status spl_tc_status(uint32_t* flags);

/*
 * spl_depth_estimate -- single-frame pseudo-Bayesian depth estimate (Sec. II-C, Eq. approx_post).
 *   log pseudo-posterior ell(d) = lambda C(d) + log f(d), lambda = (beta + 1) / beta (Eq. beta_CE), on the
 *   integer grid dmin..dmax. f(d) = N(d; prior_mu[p], prior_var[p]) when prior_mu != NULL, else uniform
 *   (then the argmax is the minimum-divergence estimator).
 *   Outputs per pixel (all [P]): argmax (smallest maximiser of ell), mu and var = mean and variance of the
 *   normalised pseudo-posterior on the grid (the depth estimate and its uncertainty).
 *   refl, bg (nullable, both or neither): reflectivity r and background b per Sec. II-E. A pixel with
 *   present[p] == 0 gets b = K/T, r = 0 (K = total photon count); otherwise (r, b) is the maximum-likelihood
 *   estimate under Eq. lik_bg_poisson with the template at round-half-even(mu). present may be NULL
 *   (every pixel present).
 *   prior_var must be > 0 where given.
 *   Arithmetic as spl_filter_step: uint16 frames of at least 128 pixels per SM on the tensor cores (counts
 *   converted to FP16 on chip, exact below 1024; a 128-pixel block with a larger count, or a pixel whose data term
 *   exceeds 1024 bits, goes to the FP32 kernel), other frames on the FP32 kernel; a bounded wait of the
 *   tensor-core kernel that runs out sets flag 1 of spl_tc_status.
 */
SPL_API spl_status spl_depth_estimate(const spl_params* prm, const spl_hist* z, const float* h, const float* prior_mu,
                              const float* prior_var, const uint8_t* present, int32_t* argmax, float* mu,
                              float* var, float* refl, float* bg, void* stream);

/*
 * spl_depth_estimate_fine -- spl_depth_estimate on a sub-bin candidate grid (the continuous form of the data
 *   term, Eq. beta_div2 over continuous times of arrival). Candidates d_k = dmin + k / S, k = 0 .. (dmax - dmin) S.
 *   The IRF is made continuous by piecewise-linear interpolation of its taps, with h[-1] = h[L] = 0 (support
 *   (-1, L)); a surface at d has the binned template s_d[t] = h_c(t - d + peak) and C(d) = sum_t z_t s_d[t]^beta.
 *   The pseudo-likelihood is exp(-K D_beta) with the whole beta-divergence: the template-power term
 *   -K sum_t s_d[t]^(1+beta), which Eq. beta_div2 drops because it is the same for every whole-bin shift, changes
 *   with the phase of an interpolated template and is kept (K = the photon count):
 *     ell(d) = lambda C(d) - K sum_t s_d[t]^(1+beta) + log N(d; prior_mu[p], prior_var[p])
 *   (uniform prior when prior_mu is NULL). Outputs per pixel: argmax_fine (nullable) = the smallest maximising
 *   index k (depth dmin + k / S), mu and var = mean and variance of the normalised pseudo-posterior on the fine
 *   grid. Every candidate is evaluated (no pruning). S in 1..16 and (dmax - dmin) S + 1 <= 16384, else
 *   SPL_EUNSUPPORTED. S = 1 gives the results of spl_depth_estimate (the kept term is then one constant).
 */
SPL_API spl_status spl_depth_estimate_fine(const spl_params* prm, int S, const spl_hist* z, const float* h,
                                           const float* prior_mu, const float* prior_var, int32_t* argmax_fine,
                                           float* mu, float* var, void* stream);

/* Most spectral bands spl_depth_estimate_msl accepts. */
#define SPL_MAX_BANDS 8

/*
 * spl_depth_estimate_msl -- depth from multispectral data (Appendix, Eq. div_MSL): nbands wavelengths recorded at
 *   once by independent detectors, band l with its own IRF h + l * L (all bands have L taps and their maximum at
 *   tap `peak`, and share beta). The beta-divergence between the product of the bands' empirical ToA distributions
 *   and the product model is, up to a constant, -lambda M(d) with
 *     M(d) = prod_l C_l(d) / K_l,   C_l(d) = sum_t z_l[t] h_l[t - d + peak]^beta,   K_l = photons of band l
 *   (a product over bands of normalised sums). A band without photons contributes no factor.
 *   Pseudo-posterior (a reading: the paper defines the minimum-divergence estimator for these data, not the scale
 *   of a pseudo-likelihood): f(d) exp(lambda K M(d)) with K = sum_l K_l, which for one band is the pseudo-posterior
 *   of spl_depth_estimate. f = N(prior_mu[p], prior_var[p]) or uniform (prior_mu NULL); without a prior the argmax
 *   is the minimum-divergence estimate.
 *   z: histograms of every band, band l's row of pixel p at element (l * P + p) * pitch of z->data (same layout
 *   rules as spl_hist). h: [nbands][L] device. nbands in 1..SPL_MAX_BANDS.
 *   Outputs: argmax [P] (nullable: smallest maximiser of the log pseudo-posterior), mu, var [P] (its mean and
 *   variance), cost [P][D] (nullable: M(dmin + k)).
 */
SPL_API spl_status spl_depth_estimate_msl(const spl_params* prm, int nbands, const spl_hist* z, const float* h,
                                          const float* prior_mu, const float* prior_var, int32_t* argmax, float* mu,
                                          float* var, float* cost, void* stream);

/*
 * spl_filter_step -- one frame of the online filter (one outer iteration of Algorithm 1).
 *   Prior (Eq. predict): for each pixel p, a Gaussian mixture over the 3x3 stencil with weights nu. Stencil
 *   entry p' contributes N(mu_in[p'], var_in[p'] + sigma_rw2) if p' is inside the frame, present_in[p'] != 0
 *   and faulty[p'] == 0; otherwise the weakly informative N((dmin+dmax)/2, (dmax-dmin)^2/12 + sigma_rw2)
 *   (Sec. III-A: absent and out-of-view neighbours). Entries with nu = 0 are skipped.
 *   Pseudo-posterior as in spl_depth_estimate with that prior; a faulty pixel has no data (C = 0), so its
 *   pseudo-posterior is its prior (Sec. III-B).
 *   ADF (Eq. KL_div): mu_out, var_out = mean and variance of the pseudo-posterior (the Gaussian q_{p,n}).
 *   mu_in/var_in/present_in describe frame n-1; present_now (frame n detections) selects the intensity rule
 *   as in spl_depth_estimate. present_in, faulty, present_now may be NULL (all present / none faulty).
 *   argmax, refl, bg are nullable (refl and bg both or neither). Faulty pixels get refl = bg = 0.
 *   mu_out/var_out must not alias mu_in/var_in (neighbours read the previous frame); use two buffers.
 *   Arithmetic. uint16 histograms (SPL_HIST_U16) of at least 128 pixels per SM (19456 on a 152-SM GPU) go
 *   through the tensor cores as in spl_filter_step_tc: each landed tile of counts is converted to FP16 on chip
 *   (exact: counts below 1024), the taps h^beta are split into high and low FP16 parts (about 22 significant
 *   bits) and the products are accumulated in FP32; the rest is FP32. A 128-pixel block holding a count of 1024
 *   or more, and a pixel whose data term lambda log2(e) max C exceeds 1024 bits (beyond it the tensor cores'
 *   rounding bound on ell passes 1e-3 bits), are computed instead by the FP32 kernel of spl_filter_step_fp32, in
 *   a second launch that reads the same inputs. A bounded internal wait of the tensor-core kernel that runs out
 *   sets flag 1 of spl_tc_status (the outputs are then incomplete). Smaller frames, and FP16 and FP32
 *   histograms, go through the FP32 kernel. The results meet the same tolerances against the FP64 definition
 *   either way (1e-4 relative on mu, var, refl, bg).
 */
SPL_API spl_status spl_filter_step(const spl_params* prm, const spl_hist* z, const float* h, const float* mu_in,
                           const float* var_in, const uint8_t* present_in, const uint8_t* faulty,
                           const uint8_t* present_now, float* mu_out, float* var_out, int32_t* argmax,
                           float* refl, float* bg, void* stream);

/*
 * spl_filter_step_fp32 -- spl_filter_step with every format on the FP32 CUDA-core kernel (the data term as FP32
 *   products and sums, warp per pixel): the plain path that the tensor-core route of uint16 histograms is
 *   measured against. Same arguments, outputs and rules as spl_filter_step.
 */
SPL_API spl_status spl_filter_step_fp32(const spl_params* prm, const spl_hist* z, const float* h, const float* mu_in,
                                        const float* var_in, const uint8_t* present_in, const uint8_t* faulty,
                                        const uint8_t* present_now, float* mu_out, float* var_out, int32_t* argmax,
                                        float* refl, float* bg, void* stream);

/*
 * spl_filter_step_detect -- spl_filter_step with the presence decision of Algorithm 1 made on the device
 *   ("Estimate pi", then "if target present, i.e. pi > 0.5"). The detector the paper uses ([TachellaSPIE2019],
 *   Sec. II-E, Sec. III-B) is cited but not defined there; this call implements a SURROGATE with the same
 *   inputs and output, and takes its marginalisations at their maximum points (Laplace / Bayesian-information-
 *   criterion approximation): the depth at the pseudo-posterior's mode (argmax, the cited test's depth prior
 *   being the pseudo-posterior), (r, b) at their maximum likelihood under Eq. lik_bg_poisson. With K the
 *   pixel's photon count and (r, b) the MLE with the template at argmax,
 *     LLR     = log L(r, b) - log L(0, K/T)            (maximised log-likelihood ratio, >= 0)
 *     log BF  = LLR - log(max(K, 1)) / 2               (one extra parameter over about K photons)
 *               - max(0, log(var_out / sigma_h^2) / 2) (Laplace over the depth: a pseudo-posterior wider
 *                                                       than the template, sigma_h^2 = its variance in bins^2)
 *     pi      = sigmoid(logit(pi0) + log BF)            (posterior probability of presence)
 *   pi0[p] is the prior probability of presence (Eq. prior_detect, e.g. spl_pi_propagate of the previous
 *   frame's pi; NULL = 0.5 everywhere), limited to [1e-7, 1 - 1e-7]. present = pi > 0.5 then selects the
 *   intensity rule (present: the MLE (r, b) with the template at the depth point estimate
 *   round-half-even(mu_out), as in spl_depth_estimate; absent: r = 0, b = K/T). Faulty pixels get pi = 0.5,
 *   absent, refl = bg = 0 (Sec. III-B).
 *   Arguments as spl_filter_step, with present_now replaced by pi0; outputs argmax (required here), pi [P]
 *   float (required), present_out [P] uint8 (nullable: 1 where pi > 0.5, usable as the next frame's
 *   present_in), refl and bg (required). pi must not alias pi0. The depth step's arithmetic is that of
 *   spl_filter_step (large uint16 frames on the tensor cores, other frames on the FP32 kernel); the presence
 *   decision is made in the intensity launch that follows either.
 */
SPL_API spl_status spl_filter_step_detect(const spl_params* prm, const spl_hist* z, const float* h,
                                          const float* mu_in, const float* var_in, const uint8_t* present_in,
                                          const uint8_t* faulty, const float* pi0, float* mu_out, float* var_out,
                                          int32_t* argmax, float* pi, uint8_t* present_out, float* refl, float* bg,
                                          void* stream);

/*
 * spl_state_init -- initial Gaussians of Algorithm 1 (n = 0): the weakly informative Gaussian of Sec. III-A,
 *   mu = (dmin + dmax)/2 and var = (dmax - dmin)^2/12, for every pixel. mu, var: [P] float.
 */
SPL_API spl_status spl_state_init(const spl_params* prm, float* mu, float* var, void* stream);

/*
 * spl_pi_propagate -- prior probability of presence for the next frame (Eq. prior_detect):
 *   pi0[p] = sigmoid(sum_k nu_k logit(pi[p + k])) over the 3x3 stencil of prm->nu. A neighbour outside the
 *   frame enters with pi = 0.5 (no information); faulty pixels have pi = 0.5 as input and output
 *   (Sec. III-B); pi is clamped to [1e-7, 1 - 1e-7] before the logit. pi_in, pi_out: [P] float, must not
 *   alias. faulty nullable.
 */
SPL_API spl_status spl_pi_propagate(const spl_params* prm, const float* pi_in, const uint8_t* faulty, float* pi_out,
                            void* stream);

/*
 * spl_filter_step_tc -- spl_filter_step (one outer iteration of Algorithm 1) with the data term on the tensor
 *   cores at any frame size, for FP16 histograms (SPL_HIST_F16; integer counts up to 2048 are exact) or uint16
 *   histograms (the conversion, redo and accuracy rule of spl_filter_step's uint16 route). Same arguments, outputs and
 *   rules as spl_filter_step. C(d) (Eq. beta_div2) is formed as in spl_depth_cost_tc (FP16 operands, the taps
 *   h^beta scaled by 2^15 and split into high and low FP16 parts, FP32 accumulation: about 22 significant bits
 *   per tap) and consumed on chip: no per-candidate value is written to memory. The photon count K of each
 *   pixel is accumulated by the tensor cores from the same tiles. Candidates whose pseudo-posterior weight is
 *   provably below 2^-64 of the largest are skipped, as in spl_filter_step. A bounded internal wait that runs
 *   out sets flag 1 of spl_tc_status (the outputs of that launch are then incomplete).
 */
SPL_API spl_status spl_filter_step_tc(const spl_params* prm, const spl_hist* z, const float* h, const float* mu_in,
                                      const float* var_in, const uint8_t* present_in, const uint8_t* faulty,
                                      const uint8_t* present_now, float* mu_out, float* var_out, int32_t* argmax,
                                      float* refl, float* bg, void* stream);

/*
 * spl_toa_histogram -- the histograms of one frame from its photon time-of-arrival lists (Sec. II-A: the ToAs
 *   y_{p,n} of pixel p, binned on the N_T = T bins of Eq. lik_ideal_poisson; z_p[t] = number of photons in bin t,
 *   the histogram on which the histogram form of Eq. beta_div2 and Eq. lik_bg_poisson are written). The result
 *   is a SPL_HIST_U16 cube for spl_filter_step, spl_depth_estimate and the other histogram calls; built on the
 *   device, it lets a caller move a frame's photon lists to the GPU instead of its histograms.
 *   offsets  : [P + 1] int32 (device); pixel p's photons are bins[offsets[p] .. offsets[p + 1]).
 *   bins     : [nphotons] uint16 (device) bin indices, in any order within a pixel; may be NULL when nphotons = 0.
 *   out      : [P][pitch] uint16 (device), 16-byte aligned, pitch >= T and a multiple of 8; every element of every
 *              row is written (elements T..pitch-1 as 0).
 *   Uses H, W, T of prm (T <= SPL_MAX_BINS). Counts are exact: the same histogram for every order of the
 *   photons. Device-detected conditions, read and cleared by spl_toa_status:
 *     SPL_TOA_BAD_BIN (1)     a photon with bin >= T was dropped;
 *     SPL_TOA_SATURATED (2)   a bin held more than 65535 photons and was written as 65535;
 *     SPL_TOA_BAD_OFFSETS (4) a pixel's offsets were not 0 <= offsets[p] <= offsets[p + 1] <= nphotons: its row is
 *                             written as zeros and none of its photons is read.
 *   Host checks (nothing launched on failure): prm, offsets and out non-NULL, bins non-NULL unless nphotons = 0,
 *   0 <= nphotons < 2^31, out 16-byte aligned, pitch >= T and a multiple of 8 -> SPL_EINVAL; T > SPL_MAX_BINS ->
 *   SPL_EUNSUPPORTED.
 */
#define SPL_TOA_BAD_BIN 1
#define SPL_TOA_SATURATED 2
#define SPL_TOA_BAD_OFFSETS 4
SPL_API spl_status spl_toa_histogram(const spl_params* prm, const int32_t* offsets, const uint16_t* bins,
                                     int64_t nphotons, uint16_t* out, int64_t pitch, void* stream);
SPL_API spl_status spl_toa_status(uint32_t* flags);

/* ------------------------------------------------------------------------------------------------------------
 * Batched filtering of many independent sequences from photon time-of-arrival lists
 *
 * The photon data of one pixel and frame is its set of ToAs y_k (Sec. II-A, Eq. lik_ideal) as integer bins in
 * [0, T), stored in CSR form: the photons of pixel p are bins[offsets[p] .. offsets[p+1]). With photon lists
 * the data term is C(d) = sum_k h[y_k - d + peak]^beta, the photon-sum form of Eq. beta_div2 (repeated bins
 * count once per photon), which equals the histogram form on the histogram of the list. Everything else is
 * spl_filter_step. Sequences may differ in every spl_params field (H, W, T, L, peak, dmin, dmax, beta,
 * sigma_rw2, nu) and in their IRF.
 *
 * A batch plan owns a small device work queue and per-frame descriptor tables ("slots"). Typical use:
 *   spl_batch_create(prms, nseq, nslots, &b);              allocates device tables
 *   spl_batch_set(b, slot, frames) for each slot;          uploads pointers (synchronous, outside capture)
 *   spl_batch_tune(b, slot, stream);                       optional: times tile sizes on real data
 *   spl_batch_step(b, slot, stream) for frame after frame; one persistent launch per size class each;
 *                                                          capturable in a CUDA graph (a memset and one or
 *                                                          two kernel launches)
 *   spl_batch_status(b, &flags); spl_batch_destroy(b);
 * The plan splits its sequences into two size classes when that raises the resident warps of the shorter ones:
 * those with more than half the longest sequence's candidate count, and the rest, each class with shared-memory
 * slices sized for its own longest sequence.
 * ------------------------------------------------------------------------------------------------------------ */

/* Device pointers of one sequence for one frame (all [P] of that sequence unless stated). */
typedef struct {
    const float* h;            /* [L] IRF of the sequence                                              */
    const int32_t* offsets;    /* [P + 1] CSR offsets into bins, non-decreasing, offsets[0] = 0          */
    const int32_t* bins;       /* photon ToA bins in [0, T)                                              */
    const float* mu_in;        /* previous-frame Gaussians (as spl_filter_step)                          */
    const float* var_in;
    const uint8_t* present_in; /* nullable                                                               */
    const uint8_t* faulty;     /* nullable                                                               */
    const uint8_t* present_now;/* nullable                                                               */
    float* mu_out;             /* must not alias mu_in / var_in                                          */
    float* var_out;
    int32_t* argmax;           /* nullable                                                               */
    float* refl;               /* nullable (refl and bg both or neither)                                 */
    float* bg;
} spl_seq_frame;

typedef struct spl_batch spl_batch;

/* Device-side conditions recorded by spl_batch_step (read with spl_batch_status). */
#define SPL_BATCH_BAD_BIN 1u       /* a photon bin outside [0, T): the photon was ignored              */
#define SPL_BATCH_TOO_MANY 2u      /* a pixel had more than SPL_MAX_PHOTONS photons: outputs set to NaN */
#define SPL_BATCH_DESC_MISMATCH 4u /* spl_batch_step_noalloc: a device descriptor's candidate count or IRF length
                                      is outside what its host copy allowed: that unit's outputs set to NaN */
#define SPL_MAX_PHOTONS 1024

/* Creates a plan for nseq sequences (prms: host array, validated like spl_filter_step) with nslots
 * descriptor tables, on the current device. Allocates device memory (SPL_ENOMEM if it cannot). */
SPL_API spl_status spl_batch_create(const spl_params* prms, int nseq, int nslots, spl_batch** out);

/* Frees the plan's device memory. Must not be called while a step of the plan is in flight. */
SPL_API void spl_batch_destroy(spl_batch* b);

/* Uploads the per-sequence pointers of one frame (frames: host array of nseq) into table `slot`.
 * Synchronous (a host-to-device copy); call it outside stream capture. */
SPL_API spl_status spl_batch_set(spl_batch* b, int slot, const spl_seq_frame* frames);

/* Runs one frame of every sequence (one outer iteration of Algorithm 1 each) from table `slot` on `stream`:
 * a reset of the slot's work-queue head and one persistent kernel whose warps take (sequence, pixel-tile)
 * units largest-first. Asynchronous, allocation-free; may be captured in a CUDA graph. Steps of the same
 * slot must not run concurrently. */
SPL_API spl_status spl_batch_step(spl_batch* b, int slot, void* stream);

/* Times every candidate tile size (pixels per work unit) on table `slot` and keeps the fastest (the outputs
 * of that slot are written several times with the same values). Synchronises the stream. */
SPL_API spl_status spl_batch_tune(spl_batch* b, int slot, void* stream);

/* Reports the plan's launch configuration (any pointer may be NULL): tile size, work units of both classes, and the
 * CTAs and warps per CTA of the launch of the longer sequences' class. */
SPL_API spl_status spl_batch_info(const spl_batch* b, int* tile, int* units, int* ctas, int* warps_per_cta);

/* Reports size class cls (0 = the longer sequences; 0 <= cls < *nclass) of the plan: the class count (1 or 2), the
 * class's work units, CTAs, warps per CTA and longest candidate grid (dmax - dmin + 1). Any output pointer may be
 * NULL; SPL_EINVAL for a NULL plan or a class the plan does not have. */
SPL_API spl_status spl_batch_class_info(const spl_batch* b, int cls, int* nclass, int* units, int* ctas,
                                        int* warps_per_cta, int* max_candidates);

/* Reads and clears the device-side condition flags (SPL_BATCH_*) accumulated since the last call.
 * Synchronous. */
SPL_API spl_status spl_batch_status(spl_batch* b, uint32_t* flags);

/* ------------------------------------------------------------------------------------------------------------
 * Differentiable filter: soft-argmax readout, loss to reference depths, gradients for calibration
 *
 * Over nframes frames of one sequence (all pixels present, none faulty) the forward pass runs the filter of
 * spl_filter_step with every candidate evaluated exactly (no pruning) and, per pixel and frame, the soft-argmax
 * readout s = sum_d d softmax(ell / tau)(d) (tau = 1 gives the pseudo-posterior mean of Sec. II-C). The loss is
 * the mean over frames and pixels of (s - d_ref)^2. The backward pass gives d loss / d h (IRF taps), d beta and
 * d nu (the 3x3 weights of Eq. predict) by a reverse sweep over the frames that recomputes each frame from the
 * checkpointed states (mu_states, var_states) of the forward pass. Reductions have a fixed order: results are
 * bitwise reproducible. Histograms: uint16, frame n of nframes at element n * P * pitch of z->data, pitch a
 * multiple of 8. mu_states, var_states: [(nframes + 1)][P]; row 0 must hold the initial state (spl_state_init);
 * the forward pass fills rows 1..nframes. scratch: device memory of spl_diff_scratch_size bytes owned by the
 * caller (about 88 bytes per pixel plus a few hundred KB), used by both passes.
 * ------------------------------------------------------------------------------------------------------------ */

/* Bytes of scratch that spl_diff_forward / spl_diff_backward need for this frame size on the current device. */
SPL_API spl_status spl_diff_scratch_size(const spl_params* prm, size_t* bytes);

/* Forward pass. dsoft ([nframes][P], nullable) receives the readouts; loss (one float, nullable) the loss, which
 * needs d_ref ([nframes][P]). tau > 0. */
SPL_API spl_status spl_diff_forward(const spl_params* prm, int nframes, const spl_hist* z, const float* h, float tau,
                                    const float* d_ref, float* mu_states, float* var_states, float* dsoft,
                                    float* loss, void* scratch, size_t scratch_bytes, void* stream);

/* Backward pass from the forward checkpoints: grad_h [L], grad_beta [1], grad_nu [9] (device). */
SPL_API spl_status spl_diff_backward(const spl_params* prm, int nframes, const spl_hist* z, const float* h,
                                     float tau, const float* d_ref, const float* mu_states, const float* var_states,
                                     float* grad_h, float* grad_beta, float* grad_nu, void* scratch,
                                     size_t scratch_bytes, void* stream);

/* ------------------------------------------------------------------------------------------------------------
 * Allocation-free batched step
 *
 * The paper has no counterpart to this call; it exists for callers that cannot allocate device memory
 * themselves through CUDA -- for example a host application whose device memory is entirely handed out by
 * another framework's pool allocator, or a real-time loop that must never enter cudaMalloc. Such callers
 * cannot create a spl_batch plan (its tables are allocated), so this entry point takes everything from the
 * caller's own memory and keeps its working memory in a fixed-size array compiled into the library.
 * ------------------------------------------------------------------------------------------------------------ */

/* One sequence for spl_batch_step_noalloc: its parameters and this frame's device pointers. */
typedef struct {
    spl_params prm;
    spl_seq_frame f;
} spl_seq_desc;

/* Most sequences one spl_batch_step_noalloc call accepts (the capacity of its fixed working array). */
#define SPL_NOALLOC_MAX_SEQ 4096

/*
 * spl_batch_step_noalloc -- one frame of every sequence, like spl_batch_step, without allocating anything.
 *   descs_host : host array of nseq descriptors (validated on the host, as spl_batch_create and
 *                spl_batch_set validate theirs).
 *   descs_dev  : the same nseq descriptors in device memory the caller owns (for example copied there with
 *                cudaMemcpy into memory the caller's pool provides). The kernels read only this copy; the host copy
 *                sizes the shared-memory slices. Where the two differ, a device descriptor whose candidate count
 *                exceeds the host copies' largest (or whose IRF length is invalid) is refused on the device: its
 *                outputs are set to NaN and SPL_BATCH_DESC_MISMATCH is raised in status; any other difference
 *                gives results for the device copy's parameters.
 *   tile       : pixels per work unit, 1..4096 (spl_batch_tune's choice of a plan is a good value; 32 is a
 *                reasonable default). Units are processed in sequence order.
 *   status     : nullable device uint32; SPL_BATCH_* condition flags are OR-ed into it.
 * Results equal those of spl_batch_step on the same data.
 * Working memory: a file-scope device array of (2 + SPL_NOALLOC_MAX_SEQ) 32-bit words (about 16 KB) that every
 * GPU which loads the library keeps until the process exits; nseq above SPL_NOALLOC_MAX_SEQ is rejected with
 * SPL_EINVAL. The call allocates no device or pinned memory (no cudaMalloc, no cudaFree, no allocating
 * library routine): it launches a small set-up kernel that resets the array's work-queue head and writes its
 * unit table, then the batch kernel, both on `stream`.
 * The first call on each device looks up the array's device address (cudaGetSymbolAddress, with that device
 * current) and caches it; make that first call before any stream capture on the device.
 * All calls on a device share the one array, and it keeps the last call's contents: calls whose kernels may
 * overlap on the GPU (other streams, other host threads) race on it and must be serialised by the caller,
 * for example by issuing them on one stream.
 */
SPL_API spl_status spl_batch_step_noalloc(const spl_seq_desc* descs_host, const spl_seq_desc* descs_dev, int nseq,
                                          int tile, uint32_t* status, void* stream);

/* ------------------------------------------------------------------------------------------------------------
 * Throughput probes (no counterpart in the paper)
 *
 * The depth kernels are bound by arithmetic issue rather than by HBM on most workloads; their ALU rooflines are
 * quoted against these measured rates instead of nominal ones.
 * ------------------------------------------------------------------------------------------------------------ */

#define SPL_PROBE_FFMA 0   /* fma.rn.f32 (FFMA)                              */
#define SPL_PROBE_FFMA2 1  /* fma.rn.f32x2 (two FP32 FMAs per instruction)   */
#define SPL_PROBE_EX2 2    /* ex2.approx.ftz.f32 (the special-function unit) */

/*
 * spl_probe_throughput -- runs one arithmetic-throughput microkernel on every SM of the current device.
 *   blocks_per_sm (1..8) blocks of 256 threads per SM; each thread executes iters * 128 operations of `kind` in
 *   8 independent chains (an f32x2 instruction counts as two operations).
 *   blocks (host out): number of blocks; ops_per_thread (host out): operations per thread.
 *   sink  : device float [blocks * 256] (one result per thread, so the work is live).
 *   cycles: device uint64 [blocks], SM clocks each block spent (clock64 difference).
 *   With sink or cycles NULL the call only fills blocks and ops_per_thread (size query) and launches nothing.
 *   Asynchronous on `stream`; time it with events on that stream.
 */
SPL_API spl_status spl_probe_throughput(int kind, int blocks_per_sm, int iters, float* sink,
                                        unsigned long long* cycles, int* blocks, long long* ops_per_thread,
                                        void* stream);

#ifdef __cplusplus
}
#endif

#endif /* SPL_H */
