// Internal declarations shared by the translation units of libspl (never installed, never part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "spl.h"

namespace spl {

enum PriorMode : int {
    PRIOR_UNIFORM = 0,  // log f(d) = 0 on the grid
    PRIOR_GAUSS = 1,    // one Gaussian per pixel, N(pmu[p], pvar[p])
    PRIOR_STENCIL = 2   // Eq. predict: 3x3 Gaussian mixture from the previous frame's state
};

// Everything one launch of the fused per-pixel kernel needs. Plain device pointers and scalars.
struct EstimateArgs {
    // observations
    const void* z;          // [P][pitch] counts
    long long pitch;        // elements
    int fmt;                // spl_hist_format
    const float* h;         // [L] IRF
    int H, W, T, L, peak, dmin, D;
    float beta;
    float lam2;             // lambda * log2(e), lambda = (beta + 1) / beta
    // prior
    int prior_mode;
    const float* pmu;       // PRIOR_GAUSS: prior mean;  PRIOR_STENCIL: previous-frame mean
    const float* pvar;      // PRIOR_GAUSS: prior var;   PRIOR_STENCIL: previous-frame variance
    const uint8_t* present_in;
    const uint8_t* faulty;
    float sigma_rw2, flat_m, flat_v;
    float nu[9];
    // outputs
    float* cost;            // [P][D] (cost-only launches)
    int* argmax;
    float* mu;
    float* var;
    float* refl;
    float* bg;
    const uint8_t* present_now;
    // detection surrogate (intensity launch only): present_now is then ignored
    int detect;
    const float* pi0;       // prior probability of presence (nullable: 0.5)
    float* pi_out;          // posterior probability of presence
    uint8_t* present_out;   // pi_out > 0.5 (nullable)
};

// One launch of the multispectral estimate (msl.cu): band l's row of pixel p is row l * P + p of z.
struct MslArgs {
    const void* z;
    long long pitch;
    int fmt;
    const float* h;  // [nbands][L]
    int nbands;
    int H, W, T, L, peak, dmin, D;
    float beta;
    float lam2;      // lambda * log2(e)
    const float* pmu;
    const float* pvar;
    int* argmax;
    float* mu;
    float* var;
    float* cost;     // [P][D] M(d), nullable
};

// Launch geometry chosen on the host for one launch.
struct Geometry {
    int warps_per_cta;
    int ctas;
    size_t smem_bytes;
};

// Records a formatted message as this thread's last error.
void set_error(const char* fmt, ...);

// Host-side validation of one frame's parameters (need_filter adds sigma_rw2 and nu); sets the error message.
spl_status check_params(const spl_params* q, bool need_filter);

// Kernel launchers (estimate.cu / aux.cu). They return cudaSuccess or the launch error.
cudaError_t launch_estimate(const EstimateArgs& a, bool cost_only, cudaStream_t s);
// Sub-bin grid (fine.cu): S steps per bin; argmax_k receives fine indices. Shared memory per warp: fine_warp_bytes.
cudaError_t launch_estimate_fine(const EstimateArgs& a, int S, int* argmax_k, cudaStream_t s);
size_t fine_warp_bytes(int T, int D, int S);
cudaError_t launch_estimate_msl(const MslArgs& a, cudaStream_t s);
size_t msl_warp_bytes(int T, int D);
cudaError_t launch_state_init(int P, float m, float v, float* mu, float* var, cudaStream_t s);
cudaError_t launch_pi_propagate(int H, int W, const float* nu, const float* pi_in, const uint8_t* faulty,
                                float* pi_out, cudaStream_t s);

// Tensor-core correlation (tc.cu).
cudaError_t launch_cost_tc(const spl_params* q, const void* z, long long pitch, const float* h, float* cost,
                           int* argmax, unsigned* status, cudaStream_t s);
// Intensity step of Sec. II-E after a depth kernel that left each pixel's photon count in a.bg (intensity.cu).
cudaError_t launch_intensity(const EstimateArgs& a, cudaStream_t s);
// Filter step with the data term on the tensor cores (tcfilter.cu); a.z holds FP16 or uint16 histograms (then
// followed by launch_estimate_redo). Returns cudaErrorInvalidConfiguration, before launching anything, when the
// shape does not fit the kernel's shared memory.
cudaError_t launch_filter_tc(const EstimateArgs& a, unsigned* status, cudaStream_t s);
// The FP32 filter step on the pixels that the uint16 tensor-core step marked with mu = NaN (estimate.cu).
cudaError_t launch_estimate_redo(const EstimateArgs& a, cudaStream_t s);
unsigned* tc_status_ptr();
cudaError_t tc_status_read(unsigned* out);
// uint16 histograms [P][pitch] from CSR photon lists (toa.cu); its condition flags are read by toa_status_read.
cudaError_t launch_toa_hist(const int32_t* offsets, const uint16_t* bins, long long nph, int T, long long pitch,
                            long long P, uint16_t* out, cudaStream_t s);
cudaError_t toa_status_read(unsigned* out);

}  // namespace spl
