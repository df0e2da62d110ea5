// Intensity step of Sec. II-E as its own launch, after the depth kernels (k_estimate, k_filter_tc): per pixel,
// b = K / T and r = 0 when the pixel is not present (K = its photon count), r = b = 0 when it is faulty, else the
// maximum-likelihood (r, b) under Eq. lik_bg_poisson with the template at round-half-even(mu), the depth the
// depth kernel wrote. The depth kernel leaves K in bg; these kernels replace it with b and write refl.
//
// The solve: with u = 1/T and the template a normalised to unit sum on the window W of L bins at the pixel's depth,
// psi(f) = sum_W z (a - u) / (u + f (a - u)) - Kout / (1 - f) is decreasing on [0, 1) in the signal fraction f;
// safeguarded Newton on psi keeps a bracket [lo, hi] around its root; then r = f K / sum(h), b = (1 - f) K / T.
//
// Kept out of the depth kernels: there a solve holds the pixel's warp (or the 128-pixel block of the tensor-core
// pipeline) until its slowest pixel converges; here every resident warp hides the others' latency, and with
// templates of at most 64 taps a warp solves four pixels at once, one per group of 8 lanes.
//
// Detection mode (a.detect): the presence decision of Algorithm 1 comes from a surrogate of the cited detector,
// its marginalisations taken at their maximum points: the template at the pseudo-posterior's mode (argmax),
// (r, b) at the solve's maximum there, and
//   log BF = LLR - log(max(K, 1)) / 2 - max(0, log(var / sigma_h^2) / 2),
//   LLR = sum_{t in W, z_t > 0} z_t log(1 - f + T f a_t) + K_out log(1 - f)
// (the maximised log-likelihood ratio against b = K / T alone; sum_t lambda_t = K at the maximum; the last
// term is Laplace's method over the depth for a pseudo-posterior of variance var wider than the template,
// sigma_h^2 = the template's variance), then pi = sigmoid(logit(pi0) + log BF) with pi0 limited to
// [1e-7, 1 - 1e-7] as in Eq. prior_detect, and present = pi > 0.5 selects the intensity rule (at round(mu),
// the depth point estimate) in place of present_now. Faulty pixels: pi = 0.5.
#include <cuda_fp16.h>
#include <math.h>
#include <stdint.h>

#include "pixel.cuh"
#include "spl_internal.h"

namespace spl {
namespace {

// pi = sigmoid(logit(pi0) + llr - log(max(K, 1)) / 2 - occam), pi0 limited to [1e-7, 1 - 1e-7] (through its
// logit); occam = max(0, log(var / sigma_h^2) / 2) for a pseudo-posterior of variance var.
__device__ __forceinline__ float presence(float pi0, float llr, float K, float var, float hvar) {
    const float lmax = 16.118095f;  // log(1e7 - 1)
    float lg = logf(pi0) - log1pf(-pi0);
    if (!(lg > -lmax)) lg = -lmax;
    if (!(lg < lmax)) lg = lmax;
    const float occam = hvar > 0.f && var > hvar ? 0.5f * logf(var / hvar) : 0.f;
    const float x = lg + llr - 0.5f * logf(fmaxf(K, 1.f)) - occam;
    return 1.f / (1.f + expf(-x));
}

// Count in bin t of pixel p's row (u16, f16 or f32 storage).
template <int FMT>
__device__ __forceinline__ float hist_value(const void* z, long long pitch, long long p, int t) {
    const long long i = p * pitch + t;
    if (FMT == SPL_HIST_F32) return static_cast<const float*>(z)[i];
    if (FMT == SPL_HIST_F16) return __half2float(static_cast<const __half*>(z)[i]);
    return static_cast<float>(static_cast<const unsigned short*>(z)[i]);
}

// Normalised template h / sum(h) (taps <= 0 count as 0) into as[0 .. SPL_MAX_TAPS); returns sum(h), and the
// template's variance in bins^2 (sum_j a_j (j - mean)^2) in *s_hvar. Block-wide.
__device__ __forceinline__ float template_table(const EstimateArgs& a, float* as, float* s_hsum, float* s_hvar) {
    for (int j = threadIdx.x; j < SPL_MAX_TAPS; j += blockDim.x) {
        const float hj = j < a.L ? a.h[j] : 0.f;
        as[j] = hj > 0.f ? hj : 0.f;
    }
    __syncthreads();
    if (threadIdx.x < 32) {
        float sum = 0.f;
        for (int j = threadIdx.x; j < a.L; j += 32) sum += as[j];
        sum = px::warp_sum(sum);
        if (threadIdx.x == 0) *s_hsum = sum;
    }
    __syncthreads();
    const float hsum = *s_hsum;
    if (hsum > 0.f)
        for (int j = threadIdx.x; j < a.L; j += blockDim.x) as[j] /= hsum;
    __syncthreads();
    if (threadIdx.x < 32) {
        float m = 0.f;
        for (int j = threadIdx.x; j < a.L; j += 32) m = fmaf(as[j], static_cast<float>(j), m);
        m = px::warp_sum(m);
        float v = 0.f;
        for (int j = threadIdx.x; j < a.L; j += 32) {
            const float e = static_cast<float>(j) - m;
            v = fmaf(as[j] * e, e, v);
        }
        v = px::warp_sum(v);
        if (threadIdx.x == 0) *s_hvar = v;
    }
    __syncthreads();
    return hsum;
}

// Template position of a pixel: round-half-even(mu) - peak, kept inside the histogram.
__device__ __forceinline__ int window_start(const EstimateArgs& a, float mu) {
    const int rm = __float2int_rn(fminf(fmaxf(mu, 0.f), static_cast<float>(a.T)));
    return min(max(rm - a.peak, 0), a.T - a.L);
}

// Sum over the 8 lanes of this lane's group (lanes 8 g .. 8 g + 7).
__device__ __forceinline__ float group8_sum(float v) {
#pragma unroll
    for (int o = 4; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Packs the group's bins with photons (z > 0) to the front: lane s of the group then holds packed entries s + 8 q
// (zeros past the group's count). Every sum of the solve runs over bins with photons only, so afterwards it needs
// ceil(n / 8) entries per lane instead of 8; the count is returned as the largest over the warp's four groups
// (warp-uniform). buf: 128 floats of shared memory per group.
__device__ __forceinline__ int pack_group8(float* zj, float* aj, float* buf, int sl) {
    int cnt = 0;
#pragma unroll
    for (int q = 0; q < 8; ++q) cnt += zj[q] > 0.f ? 1 : 0;
    int inc = cnt;  // inclusive prefix over the group's lanes
#pragma unroll
    for (int o = 1; o < 8; o <<= 1) {
        const int v = __shfl_up_sync(0xffffffffu, inc, o, 8);
        if (sl >= o) inc += v;
    }
    const int total = __shfl_sync(0xffffffffu, inc, 7, 8);
    int k = inc - cnt;
#pragma unroll
    for (int q = 0; q < 8; ++q)
        if (zj[q] > 0.f) {
            buf[2 * k] = zj[q];
            buf[2 * k + 1] = aj[q];
            ++k;
        }
    __syncwarp();
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        const int e = sl + 8 * q;
        const bool in = e < total;
        zj[q] = in ? buf[2 * e] : 0.f;
        aj[q] = in ? buf[2 * e + 1] : 0.f;
    }
    __syncwarp();
    return static_cast<int>(__reduce_max_sync(0xffffffffu, static_cast<unsigned>((total + 7) >> 3)));
}

// The solve for four pixels per warp, one per group of 8 lanes (lane s of a group holds its bins with photons, as
// packed by pack_group8, in entries q < nq). The groups iterate together (the shuffles are warp-wide) until every
// group has converged; a converged group keeps its f. need == false: the group only takes part (f = 0). Returns
// the signal fraction f.
__device__ __forceinline__ float fraction_g8(const float* zj, const float* aj, int nq, float K, int L, int T,
                                             bool need) {
    const float u = 1.f / static_cast<float>(T);
    float kin = 0.f, za = 0.f, p1 = 0.f;
    bool zero_tap = false;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        if (q >= nq) break;
        kin += zj[q];
        za = fmaf(zj[q], aj[q], za);
        if (zj[q] > 0.f) {
            if (aj[q] > 0.f) p1 += zj[q] * __fdividef(aj[q] - u, aj[q]);
            else zero_tap = true;
        }
    }
    kin = group8_sum(kin);
    za = group8_sum(za);
    p1 = group8_sum(p1);
    const unsigned zt = __ballot_sync(0xffffffffu, zero_tap);
    zero_tap = ((zt >> (threadIdx.x & 24)) & 0xffu) != 0;
    const float kout = fmaxf(K - kin, 0.f);
    const float psi0 = static_cast<float>(T) * za - K;
    float f = 0.f, lo = 0.f, hi = 1.f;
    bool active = false;
    if (!need || !(psi0 > 0.f)) {
        f = 0.f;
    } else if (!(kout > 0.f) && !zero_tap && p1 >= 0.f) {
        f = 1.f;
    } else {
        // start from the box-template estimate (window excess over the flat background)
        const float fr = static_cast<float>(L) * u;
        f = fr < 1.f ? (kin - K * fr) / (K * (1.f - fr)) : 0.5f;
        f = fminf(fmaxf(f, 0.02f), 0.98f);
        active = true;
    }
    for (int it = 0; it < 64; ++it) {
        if (!__any_sync(0xffffffffu, active)) break;
        float gs = 0.f, gp = 0.f;
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            if (q >= nq) break;
            if (zj[q] > 0.f) {
                const float e = __fdividef(aj[q] - u, fmaf(f, aj[q] - u, u));
                gs = fmaf(zj[q], e, gs);
                gp = fmaf(zj[q] * e, e, gp);
            }
        }
        gs = group8_sum(gs);
        gp = group8_sum(gp);
        if (active) {
            const float rom = __fdividef(1.f, 1.f - f);
            gs = fmaf(-kout, rom, gs);
            gp = fmaf(kout * rom, rom, gp);
            const float step = __fdividef(gs, gp);  // Newton step on psi (psi' = -gp)
            if (fabsf(step) <= px::kNewtonTol * f) {  // converged (tested before the bracket update)
                f += step;
                active = false;
            } else {
                if (gs > 0.f) lo = f; else hi = f;
                float fn = f + step;
                if (!(fn > lo && fn < hi)) fn = 0.5f * (lo + hi);
                if (hi - lo <= 1e-7f * hi) active = false;
                f = fn;
            }
        }
    }
    return f;
}

// Maximised log-likelihood ratio of the group's window at signal fraction f (0 when need == false):
// sum_{z_t > 0} z_t log(1 - f + T f a_t) + K_out log(1 - f), over the packed entries q < nq. Warp-collective.
__device__ __forceinline__ float llr_g8(const float* zj, const float* aj, int nq, float f, float K, int T,
                                        bool need) {
    const float tf = static_cast<float>(T) * f, of = 1.f - f;
    float s = 0.f, kin = 0.f;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        if (q >= nq) break;
        kin += zj[q];
        if (zj[q] > 0.f) s = fmaf(zj[q], logf(fmaf(tf, aj[q], of)), s);
    }
    s = group8_sum(s);
    kin = group8_sum(kin);
    const float kout = fmaxf(K - kin, 0.f);
    return need ? s + (kout > 0.f ? kout * log1pf(-f) : 0.f) : 0.f;
}

// Writes pixel p's outputs from its solve: the intensity rule of Sec. II-E with the presence decision of the
// detection surrogate (detect) or of present_now.
template <bool DETECT>
__device__ __forceinline__ void write_pixel(const EstimateArgs& a, long long p, bool faulty, bool present_now,
                                            float K, float hsum, float hvar, float r, float b, float llr) {
    bool present = present_now;
    if (DETECT) {
        const float pi = faulty ? 0.5f : presence(a.pi0 ? a.pi0[p] : 0.5f, llr, K, a.var[p], hvar);
        present = !faulty && pi > 0.5f;
        a.pi_out[p] = pi;
        if (a.present_out) a.present_out[p] = present ? 1 : 0;
    }
    if (faulty) {
        r = b = 0.f;
    } else if (!present || !(K > 0.f) || !(hsum > 0.f)) {
        r = 0.f;
        b = K / static_cast<float>(a.T);
    }
    a.refl[p] = r;
    a.bg[p] = b;
}

// Four pixels per warp (templates of at most 64 taps).
template <int FMT, bool DETECT>
__global__ void __launch_bounds__(256) k_intensity4(const EstimateArgs a) {
    __shared__ float as[SPL_MAX_TAPS];
    __shared__ float s_hsum, s_hvar;
    __shared__ float s_pack[8][4][128];  // per warp and group: the packed (z, a) pairs
    const float hsum = template_table(a, as, &s_hsum, &s_hvar);
    const float hvar = s_hvar;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, grp = lane >> 3, sl = lane & 7;
    float* pbuf = s_pack[warp][grp];
    const long long P = static_cast<long long>(a.H) * a.W;
    const long long stride = 4LL * gridDim.x * (blockDim.x >> 5);
    for (long long p0 = 4LL * (static_cast<long long>(blockIdx.x) * (blockDim.x >> 5) + warp); p0 < P; p0 += stride) {
        const long long p = p0 + grp;
        const bool valid = p < P;
        const float K = valid ? a.bg[p] : 0.f;
        const bool faulty = valid && a.faulty ? a.faulty[p] != 0 : false;
        const bool present = valid && (DETECT || (a.present_now ? a.present_now[p] != 0 : true));
        const bool need = valid && !faulty && present && K > 0.f && hsum > 0.f;
        const int t0 = need ? window_start(a, a.mu[p]) : 0;
        float zj[8], aj[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int j = sl + 8 * q;
            zj[q] = need && j < a.L ? hist_value<FMT>(a.z, a.pitch, p, t0 + j) : 0.f;
            aj[q] = j < a.L ? as[j] : 0.f;
        }
        int nq = pack_group8(zj, aj, pbuf, sl);
        const float f = fraction_g8(zj, aj, nq, K, a.L, a.T, need);
        const float r = f * K / hsum, b = (1.f - f) * K * (1.f / static_cast<float>(a.T));
        float llr = 0.f;
        if (DETECT) {  // the evidence with the template at the pseudo-posterior mode
            const int t1 = need ? window_start(a, static_cast<float>(a.argmax[p])) : t0;
            float fm = f;
            if (__any_sync(0xffffffffu, t1 != t0)) {  // some group's mode differs from round(mu): solve there
                const bool again = need && t1 != t0;
                if (again) {
#pragma unroll
                    for (int q = 0; q < 8; ++q) {
                        const int j = sl + 8 * q;
                        zj[q] = j < a.L ? hist_value<FMT>(a.z, a.pitch, p, t1 + j) : 0.f;
                        aj[q] = j < a.L ? as[j] : 0.f;
                    }
                }
                const int nq1 = pack_group8(zj, aj, pbuf, sl);  // every group repacks (warp-collective)
                nq = nq1;
                const float f1 = fraction_g8(zj, aj, nq, K, a.L, a.T, again);
                if (again) fm = f1;
            }
            llr = llr_g8(zj, aj, nq, fm, K, a.T, need);
        }
        if (valid && sl == 0) write_pixel<DETECT>(a, p, faulty, present, K, hsum, hvar, r, b, llr);
        __syncwarp();
    }
}

// One pixel per warp (any template length up to SPL_MAX_TAPS): the warp-cooperative solve of pixel.cuh.
template <int FMT, bool DETECT>
__global__ void __launch_bounds__(256) k_intensity1(const EstimateArgs a) {
    __shared__ float as[SPL_MAX_TAPS];
    __shared__ float s_hsum, s_hvar;
    const float hsum = template_table(a, as, &s_hsum, &s_hvar);
    const float hvar = s_hvar;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const long long P = static_cast<long long>(a.H) * a.W;
    const long long stride = static_cast<long long>(gridDim.x) * (blockDim.x >> 5);
    for (long long p = static_cast<long long>(blockIdx.x) * (blockDim.x >> 5) + warp; p < P; p += stride) {
        const float K = a.bg[p];
        const bool faulty = a.faulty ? a.faulty[p] != 0 : false;
        const bool present = DETECT || (a.present_now ? a.present_now[p] != 0 : true);
        float r = 0.f, b = 0.f, llr = 0.f;
        if (!faulty && present && K > 0.f && hsum > 0.f) {  // warp-uniform
            constexpr int NQ = SPL_MAX_TAPS / 32;
            const int t0 = window_start(a, a.mu[p]);
            float zj[NQ], aj[NQ];
#pragma unroll
            for (int q = 0; q < NQ; ++q) {
                const int j = lane + 32 * q;
                zj[q] = j < a.L ? hist_value<FMT>(a.z, a.pitch, p, t0 + j) : 0.f;
                aj[q] = j < a.L ? as[j] : 0.f;
            }
            const float f0 = px::intensity_fraction<NQ>(zj, aj, K, a.L, a.T);
            r = f0 * K / hsum;
            b = (1.f - f0) * K * (1.f / static_cast<float>(a.T));
            if (DETECT) {  // the evidence with the template at the pseudo-posterior mode
                const int t1 = window_start(a, static_cast<float>(a.argmax[p]));
                float f = f0;
                if (t1 != t0) {  // warp-uniform
#pragma unroll
                    for (int q = 0; q < NQ; ++q) {
                        const int j = lane + 32 * q;
                        zj[q] = j < a.L ? hist_value<FMT>(a.z, a.pitch, p, t1 + j) : 0.f;
                    }
                    f = px::intensity_fraction<NQ>(zj, aj, K, a.L, a.T);
                }
                const float tf = static_cast<float>(a.T) * f, of = 1.f - f;
                float s = 0.f, kin = 0.f;
#pragma unroll
                for (int q = 0; q < NQ; ++q) {
                    kin += zj[q];
                    if (zj[q] > 0.f) s = fmaf(zj[q], logf(fmaf(tf, aj[q], of)), s);
                }
                s = px::warp_sum(s);
                kin = px::warp_sum(kin);
                const float kout = fmaxf(K - kin, 0.f);
                llr = s + (kout > 0.f ? kout * log1pf(-f) : 0.f);
            }
        }
        if (lane == 0) write_pixel<DETECT>(a, p, faulty, present, K, hsum, hvar, r, b, llr);
        __syncwarp();
    }
}

template <int FMT>
cudaError_t launch_fmt(const EstimateArgs& a, int nsm, cudaStream_t s) {
    const long long P = static_cast<long long>(a.H) * a.W;
    const long long px_per_block = a.L <= 64 ? 32 : 8;  // 8 warps of 4 pixels, or of one pixel
    const long long blocks = (P + px_per_block - 1) / px_per_block;
    const long long cap = static_cast<long long>(nsm) * 8;  // at most 8 resident blocks of 256 threads per SM
    const unsigned nb = static_cast<unsigned>(blocks < cap ? blocks : cap);
    if (a.detect) {  // the detection surrogate's kernels (kept apart: their extra state costs the plain ones)
        if (a.L <= 64) k_intensity4<FMT, true><<<nb, 256, 0, s>>>(a);
        else k_intensity1<FMT, true><<<nb, 256, 0, s>>>(a);
    } else {
        if (a.L <= 64) k_intensity4<FMT, false><<<nb, 256, 0, s>>>(a);
        else k_intensity1<FMT, false><<<nb, 256, 0, s>>>(a);
    }
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_intensity(const EstimateArgs& a, cudaStream_t s) {
    int dev = 0, nsm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    switch (a.fmt) {
        case SPL_HIST_U16: return launch_fmt<SPL_HIST_U16>(a, nsm, s);
        case SPL_HIST_F16: return launch_fmt<SPL_HIST_F16>(a, nsm, s);
        case SPL_HIST_F32: return launch_fmt<SPL_HIST_F32>(a, nsm, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace spl
