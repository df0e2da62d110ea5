// Host side of the C ABI declared in include/spl.h: argument validation, launch configuration, error
// reporting. No call allocates, synchronises or copies device data.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include "spl_internal.h"

namespace spl {
namespace {
thread_local char g_err[512] = "";
}

void set_error(const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}

namespace {

#define SPL_REQUIRE(cond, ...)              \
    do {                                    \
        if (!(cond)) {                      \
            set_error(__VA_ARGS__);         \
            return SPL_EINVAL;              \
        }                                   \
    } while (0)

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

size_t elem_size(int fmt) { return fmt == SPL_HIST_F32 ? 4 : 2; }

}  // namespace

// Geometry, domain and parameter checks shared by the depth calls (the domain reading is stated in spl.h).
spl_status check_params(const spl_params* q, bool need_filter) {
    SPL_REQUIRE(q != nullptr, "prm is NULL");
    SPL_REQUIRE(q->H >= 1 && q->W >= 1, "H and W must be >= 1 (got %d x %d)", q->H, q->W);
    SPL_REQUIRE(static_cast<long long>(q->H) * q->W <= (1LL << 31) - 1, "H*W exceeds 2^31-1");
    SPL_REQUIRE(q->L >= 1, "L must be >= 1 (got %d)", q->L);
    SPL_REQUIRE(q->T >= q->L, "T (%d) must be >= L (%d)", q->T, q->L);
    SPL_REQUIRE(q->peak >= 0 && q->peak < q->L, "peak (%d) must be in [0, L)", q->peak);
    SPL_REQUIRE(q->dmin <= q->dmax, "dmin (%d) > dmax (%d)", q->dmin, q->dmax);
    SPL_REQUIRE(q->dmin >= q->peak && q->dmax <= q->T - q->L + q->peak,
                "candidate depths [%d, %d] leave the full-support range [%d, %d]", q->dmin, q->dmax, q->peak,
                q->T - q->L + q->peak);
    SPL_REQUIRE(q->beta > 0.f && isfinite(q->beta), "beta must be finite and > 0 (got %g)", q->beta);
    if (q->L > SPL_MAX_TAPS || q->T > SPL_MAX_BINS) {
        set_error("L (%d) above %d or T (%d) above %d is not supported by the library", q->L, SPL_MAX_TAPS, q->T,
                  SPL_MAX_BINS);
        return SPL_EUNSUPPORTED;
    }
    if (need_filter) {
        SPL_REQUIRE(q->sigma_rw2 > 0.f && isfinite(q->sigma_rw2), "sigma_rw2 must be finite and > 0 (got %g)",
                    q->sigma_rw2);
        float s = 0.f;
        for (int k = 0; k < 9; ++k) {
            SPL_REQUIRE(q->nu[k] >= 0.f && isfinite(q->nu[k]), "nu[%d] must be finite and >= 0 (got %g)", k,
                        q->nu[k]);
            s += q->nu[k];
        }
        SPL_REQUIRE(s > 0.f, "the mixture weights nu sum to 0");
    }
    return SPL_OK;
}

namespace {

spl_status check_hist(const spl_params* q, const spl_hist* z) {
    SPL_REQUIRE(z != nullptr && z->data != nullptr, "histogram z (or z->data) is NULL");
    SPL_REQUIRE(z->fmt == SPL_HIST_U16 || z->fmt == SPL_HIST_F16 || z->fmt == SPL_HIST_F32,
                "unknown histogram format %d", static_cast<int>(z->fmt));
    SPL_REQUIRE(z->pitch >= q->T, "pitch (%lld) < T (%d)", static_cast<long long>(z->pitch), q->T);
    SPL_REQUIRE((z->pitch * static_cast<int64_t>(elem_size(z->fmt))) % 16 == 0,
                "pitch * element size must be a multiple of 16 bytes (pitch %lld)",
                static_cast<long long>(z->pitch));
    SPL_REQUIRE(aligned16(z->data), "z->data must be 16-byte aligned");
    return SPL_OK;
}

spl_status cuda_status(cudaError_t e, const char* what) {
    if (e == cudaSuccess) return SPL_OK;
    set_error("%s: %s", what, cudaGetErrorString(e));
    return SPL_ECUDA;
}

EstimateArgs base_args(const spl_params* q, const spl_hist* z, const float* h) {
    EstimateArgs a;
    memset(&a, 0, sizeof(a));
    a.z = z->data;
    a.pitch = z->pitch;
    a.fmt = z->fmt;
    a.h = h;
    a.H = q->H;
    a.W = q->W;
    a.T = q->T;
    a.L = q->L;
    a.peak = q->peak;
    a.dmin = q->dmin;
    a.D = q->dmax - q->dmin + 1;
    a.beta = q->beta;
    a.lam2 = static_cast<float>((static_cast<double>(q->beta) + 1.0) / q->beta * 1.4426950408889634);
    a.sigma_rw2 = q->sigma_rw2;
    a.flat_m = 0.5f * static_cast<float>(q->dmin + q->dmax);
    const double span = static_cast<double>(q->dmax - q->dmin);
    a.flat_v = static_cast<float>(span * span / 12.0);
    for (int k = 0; k < 9; ++k) a.nu[k] = q->nu[k];
    return a;
}

}  // namespace
}  // namespace spl

namespace spl {
namespace {

// Pixels from which the automatic entries take uint16 frames to the tensor cores: one 128-pixel block per SM. A
// smaller frame leaves most SMs idle in the block-per-CTA tensor-core kernel, where the warp-per-pixel FP32 kernel
// still spreads it (a 32x32 frame: 29 us against 59 us, measured).
long long tc_min_pixels() {
    int dev = 0, nsm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) !=
                                                  cudaSuccess)
        return 1LL << 62;
    return 128LL * nsm;
}

// Launches one step of spl_filter_step, spl_filter_step_detect or spl_depth_estimate: uint16 frames of at least
// tc_min_pixels() through the tensor-core kernel when tc is set (its redo and intensity launches follow), falling
// back to the FP32 kernel only for a shape the tensor-core kernel cannot hold (nothing is launched then); every
// other frame through the FP32 kernel.
spl_status launch_step(const EstimateArgs& a, cudaStream_t s, bool tc, const char* what) {
    if (tc && a.fmt == SPL_HIST_U16 && static_cast<long long>(a.H) * a.W >= tc_min_pixels()) {
        unsigned* status = tc_status_ptr();
        SPL_REQUIRE(status != nullptr, "no device status word (no CUDA device?)");
        const cudaError_t e = launch_filter_tc(a, status, s);
        if (e != cudaErrorInvalidConfiguration) return cuda_status(e, what);
        cudaGetLastError();  // nothing was launched: clear the configuration error, take the FP32 kernel
    }
    return cuda_status(launch_estimate(a, false, s), what);
}

// The filter step of spl_filter_step / spl_filter_step_fp32: uint16 histograms on the tensor cores when tc is set
// (falling back to the FP32 kernel only for a shape the tensor-core kernel cannot hold), else the FP32 kernel.
spl_status filter_step(const spl_params* prm, const spl_hist* z, const float* h, const float* mu_in,
                       const float* var_in, const uint8_t* present_in, const uint8_t* faulty,
                       const uint8_t* present_now, float* mu_out, float* var_out, int32_t* argmax, float* refl,
                       float* bg, void* stream, bool tc) {
    g_err[0] = 0;
    spl_status st = check_params(prm, true);
    if (st != SPL_OK) return st;
    if ((st = check_hist(prm, z)) != SPL_OK) return st;
    SPL_REQUIRE(h != nullptr, "h is NULL");
    SPL_REQUIRE(mu_in && var_in && mu_out && var_out, "mu_in, var_in, mu_out and var_out are required");
    SPL_REQUIRE(mu_out != mu_in && var_out != var_in && mu_out != var_in && var_out != mu_in,
                "outputs must not alias the previous-frame state");
    SPL_REQUIRE((refl == nullptr) == (bg == nullptr), "give both refl and bg or neither");
    EstimateArgs a = base_args(prm, z, h);
    a.prior_mode = PRIOR_STENCIL;
    a.pmu = mu_in;
    a.pvar = var_in;
    a.present_in = present_in;
    a.faulty = faulty;
    a.present_now = present_now;
    a.argmax = argmax;
    a.mu = mu_out;
    a.var = var_out;
    a.refl = refl;
    a.bg = bg;
    return launch_step(a, static_cast<cudaStream_t>(stream), tc, "spl_filter_step launch");
}

}  // namespace
}  // namespace spl

using namespace spl;

extern "C" {

const char* spl_version(void) { return "libspl 0.1 (sm_103a)"; }

const char* spl_last_error(void) { return g_err; }

spl_status spl_depth_cost(const spl_params* prm, const spl_hist* z, const float* h, float* cost, int32_t* argmax,
                          void* stream) {
    g_err[0] = 0;
    spl_status st = check_params(prm, false);
    if (st != SPL_OK) return st;
    if ((st = check_hist(prm, z)) != SPL_OK) return st;
    SPL_REQUIRE(h != nullptr, "h is NULL");
    SPL_REQUIRE(cost != nullptr || argmax != nullptr, "both cost and argmax are NULL: nothing to compute");
    EstimateArgs a = base_args(prm, z, h);
    a.cost = cost;
    a.argmax = argmax;
    return cuda_status(launch_estimate(a, true, static_cast<cudaStream_t>(stream)), "spl_depth_cost launch");
}

spl_status spl_depth_cost_tc(const spl_params* prm, const spl_hist* z, const float* h, float* cost,
                             int32_t* argmax, void* stream) {
    g_err[0] = 0;
    spl_status st = check_params(prm, false);
    if (st != SPL_OK) return st;
    if ((st = check_hist(prm, z)) != SPL_OK) return st;
    SPL_REQUIRE(z->fmt == SPL_HIST_F16, "spl_depth_cost_tc takes FP16 histograms (SPL_HIST_F16)");
    SPL_REQUIRE(h != nullptr, "h is NULL");
    SPL_REQUIRE(cost != nullptr || argmax != nullptr, "both cost and argmax are NULL: nothing to compute");
    unsigned* status = tc_status_ptr();
    SPL_REQUIRE(status != nullptr, "no device status word (no CUDA device?)");
    return cuda_status(launch_cost_tc(prm, z->data, z->pitch, h, cost, argmax, status,
                                      static_cast<cudaStream_t>(stream)),
                       "spl_depth_cost_tc launch");
}

spl_status spl_tc_status(uint32_t* flags) {
    g_err[0] = 0;
    SPL_REQUIRE(flags != nullptr, "flags is NULL");
    unsigned v = 0;
    spl_status st = cuda_status(tc_status_read(&v), "spl_tc_status");
    if (st == SPL_OK) *flags = v;
    return st;
}

spl_status spl_depth_estimate(const spl_params* prm, const spl_hist* z, const float* h, const float* prior_mu,
                              const float* prior_var, const uint8_t* present, int32_t* argmax, float* mu,
                              float* var, float* refl, float* bg, void* stream) {
    g_err[0] = 0;
    spl_status st = check_params(prm, false);
    if (st != SPL_OK) return st;
    if ((st = check_hist(prm, z)) != SPL_OK) return st;
    SPL_REQUIRE(h != nullptr, "h is NULL");
    SPL_REQUIRE(mu != nullptr && var != nullptr, "mu and var outputs are required");
    SPL_REQUIRE((prior_mu == nullptr) == (prior_var == nullptr), "give both prior_mu and prior_var or neither");
    SPL_REQUIRE((refl == nullptr) == (bg == nullptr), "give both refl and bg or neither");
    EstimateArgs a = base_args(prm, z, h);
    a.prior_mode = prior_mu ? PRIOR_GAUSS : PRIOR_UNIFORM;
    a.pmu = prior_mu;
    a.pvar = prior_var;
    a.argmax = argmax;
    a.mu = mu;
    a.var = var;
    a.refl = refl;
    a.bg = bg;
    a.present_now = present;
    return launch_step(a, static_cast<cudaStream_t>(stream), true, "spl_depth_estimate launch");
}

spl_status spl_depth_estimate_msl(const spl_params* prm, int nbands, const spl_hist* z, const float* h,
                                  const float* prior_mu, const float* prior_var, int32_t* argmax, float* mu, float* var,
                                  float* cost, void* stream) {
    g_err[0] = 0;
    spl_status st = check_params(prm, false);
    if (st != SPL_OK) return st;
    if ((st = check_hist(prm, z)) != SPL_OK) return st;
    SPL_REQUIRE(nbands >= 1 && nbands <= SPL_MAX_BANDS, "nbands must be in 1..%d (got %d)", SPL_MAX_BANDS, nbands);
    SPL_REQUIRE(h != nullptr, "h is NULL");
    SPL_REQUIRE(mu != nullptr && var != nullptr, "mu and var outputs are required");
    SPL_REQUIRE((prior_mu == nullptr) == (prior_var == nullptr), "give both prior_mu and prior_var or neither");
    MslArgs a;
    memset(&a, 0, sizeof(a));
    a.z = z->data;
    a.pitch = z->pitch;
    a.fmt = z->fmt;
    a.h = h;
    a.nbands = nbands;
    a.H = prm->H;
    a.W = prm->W;
    a.T = prm->T;
    a.L = prm->L;
    a.peak = prm->peak;
    a.dmin = prm->dmin;
    a.D = prm->dmax - prm->dmin + 1;
    a.beta = prm->beta;
    a.lam2 = static_cast<float>((static_cast<double>(prm->beta) + 1.0) / prm->beta * 1.4426950408889634);
    a.pmu = prior_mu;
    a.pvar = prior_var;
    a.argmax = argmax;
    a.mu = mu;
    a.var = var;
    a.cost = cost;
    return cuda_status(launch_estimate_msl(a, static_cast<cudaStream_t>(stream)), "spl_depth_estimate_msl launch");
}

spl_status spl_depth_estimate_fine(const spl_params* prm, int S, const spl_hist* z, const float* h,
                                   const float* prior_mu, const float* prior_var, int32_t* argmax_fine, float* mu,
                                   float* var, void* stream) {
    g_err[0] = 0;
    spl_status st = check_params(prm, false);
    if (st != SPL_OK) return st;
    if ((st = check_hist(prm, z)) != SPL_OK) return st;
    SPL_REQUIRE(h != nullptr, "h is NULL");
    SPL_REQUIRE(S >= 1 && S <= 16, "S must be in 1..16 (got %d)", S);
    SPL_REQUIRE(mu != nullptr && var != nullptr, "mu and var outputs are required");
    SPL_REQUIRE((prior_mu == nullptr) == (prior_var == nullptr), "give both prior_mu and prior_var or neither");
    const long long Kf = static_cast<long long>(prm->dmax - prm->dmin) * S + 1;
    if (Kf > 16384 || fine_warp_bytes(prm->T, prm->dmax - prm->dmin + 1, S) > 200 * 1024) {
        set_error("fine grid of %lld candidates (S = %d) exceeds the 16384 a warp holds in shared memory", Kf, S);
        return SPL_EUNSUPPORTED;
    }
    EstimateArgs a = base_args(prm, z, h);
    a.prior_mode = prior_mu ? PRIOR_GAUSS : PRIOR_UNIFORM;
    a.pmu = prior_mu;
    a.pvar = prior_var;
    a.mu = mu;
    a.var = var;
    return cuda_status(launch_estimate_fine(a, S, argmax_fine, static_cast<cudaStream_t>(stream)),
                       "spl_depth_estimate_fine launch");
}

spl_status spl_filter_step(const spl_params* prm, const spl_hist* z, const float* h, const float* mu_in,
                           const float* var_in, const uint8_t* present_in, const uint8_t* faulty,
                           const uint8_t* present_now, float* mu_out, float* var_out, int32_t* argmax,
                           float* refl, float* bg, void* stream) {
    return filter_step(prm, z, h, mu_in, var_in, present_in, faulty, present_now, mu_out, var_out, argmax, refl, bg,
                       stream, true);
}

spl_status spl_filter_step_fp32(const spl_params* prm, const spl_hist* z, const float* h, const float* mu_in,
                                const float* var_in, const uint8_t* present_in, const uint8_t* faulty,
                                const uint8_t* present_now, float* mu_out, float* var_out, int32_t* argmax,
                                float* refl, float* bg, void* stream) {
    return filter_step(prm, z, h, mu_in, var_in, present_in, faulty, present_now, mu_out, var_out, argmax, refl, bg,
                       stream, false);
}

spl_status spl_filter_step_detect(const spl_params* prm, const spl_hist* z, const float* h, const float* mu_in,
                                  const float* var_in, const uint8_t* present_in, const uint8_t* faulty,
                                  const float* pi0, float* mu_out, float* var_out, int32_t* argmax, float* pi,
                                  uint8_t* present_out, float* refl, float* bg, void* stream) {
    g_err[0] = 0;
    spl_status st = check_params(prm, true);
    if (st != SPL_OK) return st;
    if ((st = check_hist(prm, z)) != SPL_OK) return st;
    SPL_REQUIRE(h != nullptr, "h is NULL");
    SPL_REQUIRE(mu_in && var_in && mu_out && var_out, "mu_in, var_in, mu_out and var_out are required");
    SPL_REQUIRE(mu_out != mu_in && var_out != var_in && mu_out != var_in && var_out != mu_in,
                "outputs must not alias the previous-frame state");
    SPL_REQUIRE(argmax != nullptr && pi != nullptr && refl != nullptr && bg != nullptr,
                "argmax, pi, refl and bg are required");
    SPL_REQUIRE(pi0 == nullptr || pi0 != pi, "pi must not alias pi0");
    EstimateArgs a = base_args(prm, z, h);
    a.prior_mode = PRIOR_STENCIL;
    a.pmu = mu_in;
    a.pvar = var_in;
    a.present_in = present_in;
    a.faulty = faulty;
    a.argmax = argmax;
    a.mu = mu_out;
    a.var = var_out;
    a.refl = refl;
    a.bg = bg;
    a.detect = 1;
    a.pi0 = pi0;
    a.pi_out = pi;
    a.present_out = present_out;
    return launch_step(a, static_cast<cudaStream_t>(stream), true, "spl_filter_step_detect launch");
}

spl_status spl_filter_step_tc(const spl_params* prm, const spl_hist* z, const float* h, const float* mu_in,
                              const float* var_in, const uint8_t* present_in, const uint8_t* faulty,
                              const uint8_t* present_now, float* mu_out, float* var_out, int32_t* argmax,
                              float* refl, float* bg, void* stream) {
    g_err[0] = 0;
    spl_status st = check_params(prm, true);
    if (st != SPL_OK) return st;
    if ((st = check_hist(prm, z)) != SPL_OK) return st;
    SPL_REQUIRE(z->fmt == SPL_HIST_F16 || z->fmt == SPL_HIST_U16,
                "spl_filter_step_tc takes FP16 or uint16 histograms (SPL_HIST_F16, SPL_HIST_U16)");
    SPL_REQUIRE(h != nullptr, "h is NULL");
    SPL_REQUIRE(mu_in && var_in && mu_out && var_out, "mu_in, var_in, mu_out and var_out are required");
    SPL_REQUIRE(mu_out != mu_in && var_out != var_in && mu_out != var_in && var_out != mu_in,
                "outputs must not alias the previous-frame state");
    SPL_REQUIRE((refl == nullptr) == (bg == nullptr), "give both refl and bg or neither");
    unsigned* status = tc_status_ptr();
    SPL_REQUIRE(status != nullptr, "no device status word (no CUDA device?)");
    EstimateArgs a = base_args(prm, z, h);
    a.prior_mode = PRIOR_STENCIL;
    a.pmu = mu_in;
    a.pvar = var_in;
    a.present_in = present_in;
    a.faulty = faulty;
    a.present_now = present_now;
    a.argmax = argmax;
    a.mu = mu_out;
    a.var = var_out;
    a.refl = refl;
    a.bg = bg;
    return cuda_status(launch_filter_tc(a, status, static_cast<cudaStream_t>(stream)), "spl_filter_step_tc launch");
}

spl_status spl_state_init(const spl_params* prm, float* mu, float* var, void* stream) {
    g_err[0] = 0;
    SPL_REQUIRE(prm != nullptr, "prm is NULL");
    SPL_REQUIRE(prm->H >= 1 && prm->W >= 1, "H and W must be >= 1");
    SPL_REQUIRE(prm->dmin <= prm->dmax, "dmin > dmax");
    SPL_REQUIRE(mu != nullptr && var != nullptr, "mu and var are required");
    const double span = static_cast<double>(prm->dmax - prm->dmin);
    return cuda_status(launch_state_init(prm->H * prm->W, 0.5f * static_cast<float>(prm->dmin + prm->dmax),
                                         static_cast<float>(span * span / 12.0), mu, var,
                                         static_cast<cudaStream_t>(stream)),
                       "spl_state_init launch");
}

spl_status spl_pi_propagate(const spl_params* prm, const float* pi_in, const uint8_t* faulty, float* pi_out,
                            void* stream) {
    g_err[0] = 0;
    SPL_REQUIRE(prm != nullptr, "prm is NULL");
    SPL_REQUIRE(prm->H >= 1 && prm->W >= 1, "H and W must be >= 1");
    SPL_REQUIRE(pi_in != nullptr && pi_out != nullptr, "pi_in and pi_out are required");
    SPL_REQUIRE(pi_in != pi_out, "pi_out must not alias pi_in");
    for (int k = 0; k < 9; ++k)
        SPL_REQUIRE(isfinite(prm->nu[k]), "nu[%d] is not finite", k);
    return cuda_status(launch_pi_propagate(prm->H, prm->W, prm->nu, pi_in, faulty, pi_out,
                                           static_cast<cudaStream_t>(stream)),
                       "spl_pi_propagate launch");
}

spl_status spl_toa_histogram(const spl_params* prm, const int32_t* offsets, const uint16_t* bins, int64_t nphotons,
                             uint16_t* out, int64_t pitch, void* stream) {
    g_err[0] = 0;
    SPL_REQUIRE(prm != nullptr, "prm is NULL");
    SPL_REQUIRE(prm->H >= 1 && prm->W >= 1, "H and W must be >= 1 (got %d x %d)", prm->H, prm->W);
    SPL_REQUIRE(static_cast<long long>(prm->H) * prm->W <= (1LL << 31) - 1, "H*W exceeds 2^31-1");
    SPL_REQUIRE(prm->T >= 1, "T must be >= 1 (got %d)", prm->T);
    if (prm->T > SPL_MAX_BINS) {
        set_error("T (%d) above %d is not supported by the library", prm->T, SPL_MAX_BINS);
        return SPL_EUNSUPPORTED;
    }
    SPL_REQUIRE(offsets != nullptr, "offsets is NULL");
    SPL_REQUIRE(nphotons >= 0 && nphotons <= (1LL << 31) - 1, "nphotons (%lld) must be in [0, 2^31-1]",
                static_cast<long long>(nphotons));
    SPL_REQUIRE(bins != nullptr || nphotons == 0, "bins is NULL with nphotons > 0");
    SPL_REQUIRE(out != nullptr, "out is NULL");
    SPL_REQUIRE(aligned16(out), "out must be 16-byte aligned");
    SPL_REQUIRE(pitch >= prm->T && pitch % 8 == 0, "pitch (%lld) must be >= T (%d) and a multiple of 8",
                static_cast<long long>(pitch), prm->T);
    return cuda_status(launch_toa_hist(offsets, bins, nphotons, prm->T, pitch,
                                       static_cast<long long>(prm->H) * prm->W, out,
                                       static_cast<cudaStream_t>(stream)),
                       "spl_toa_histogram launch");
}

spl_status spl_toa_status(uint32_t* flags) {
    g_err[0] = 0;
    SPL_REQUIRE(flags != nullptr, "flags is NULL");
    unsigned v = 0;
    spl_status st = cuda_status(toa_status_read(&v), "spl_toa_status");
    if (st == SPL_OK) *flags = v;
    return st;
}

}  // extern "C"
