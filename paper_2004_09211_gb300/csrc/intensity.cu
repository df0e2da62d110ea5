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
#include <cuda_fp16.h>
#include <math.h>
#include <stdint.h>

#include "pixel.cuh"
#include "spl_internal.h"

namespace spl {
namespace {

// Count in bin t of pixel p's row (u16, f16 or f32 storage).
template <int FMT>
__device__ __forceinline__ float hist_value(const void* z, long long pitch, long long p, int t) {
    const long long i = p * pitch + t;
    if (FMT == SPL_HIST_F32) return static_cast<const float*>(z)[i];
    if (FMT == SPL_HIST_F16) return __half2float(static_cast<const __half*>(z)[i]);
    return static_cast<float>(static_cast<const unsigned short*>(z)[i]);
}

// Normalised template h / sum(h) (taps <= 0 count as 0) into as[0 .. SPL_MAX_TAPS); returns sum(h). Block-wide.
__device__ __forceinline__ float template_table(const EstimateArgs& a, float* as, float* s_hsum) {
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

// The solve for four pixels per warp, one per group of 8 lanes (lane s of a group holds bins s + 8 q, q < 8, so
// L <= 64). The groups iterate together (the shuffles are warp-wide) until every group has converged; a
// converged group keeps its f. need == false: the group only takes part.
__device__ __forceinline__ void intensity_mle_g8(const float* zj, const float* aj, float K, int L, int T, float hsum,
                                                 bool need, float& r, float& b) {
    const float u = 1.f / static_cast<float>(T);
    float kin = 0.f, za = 0.f, p1 = 0.f;
    bool zero_tap = false;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
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
    r = f * K / hsum;
    b = (1.f - f) * K * u;
}

// Four pixels per warp (templates of at most 64 taps).
template <int FMT>
__global__ void __launch_bounds__(256) k_intensity4(const EstimateArgs a) {
    __shared__ float as[SPL_MAX_TAPS];
    __shared__ float s_hsum;
    const float hsum = template_table(a, as, &s_hsum);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, grp = lane >> 3, sl = lane & 7;
    const long long P = static_cast<long long>(a.H) * a.W;
    const long long stride = 4LL * gridDim.x * (blockDim.x >> 5);
    for (long long p0 = 4LL * (static_cast<long long>(blockIdx.x) * (blockDim.x >> 5) + warp); p0 < P; p0 += stride) {
        const long long p = p0 + grp;
        const bool valid = p < P;
        const float K = valid ? a.bg[p] : 0.f;
        const bool faulty = valid && a.faulty ? a.faulty[p] != 0 : false;
        const bool present = valid && (a.present_now ? a.present_now[p] != 0 : true);
        const bool need = valid && !faulty && present && K > 0.f && hsum > 0.f;
        const int t0 = need ? window_start(a, a.mu[p]) : 0;
        float zj[8], aj[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int j = sl + 8 * q;
            zj[q] = need && j < a.L ? hist_value<FMT>(a.z, a.pitch, p, t0 + j) : 0.f;
            aj[q] = j < a.L ? as[j] : 0.f;
        }
        float r = 0.f, b = 0.f;
        intensity_mle_g8(zj, aj, K, a.L, a.T, hsum, need, r, b);
        if (valid && sl == 0) {
            if (faulty) {
                r = b = 0.f;
            } else if (!need) {
                r = 0.f;
                b = K / static_cast<float>(a.T);
            }
            a.refl[p] = r;
            a.bg[p] = b;
        }
        __syncwarp();
    }
}

// One pixel per warp (any template length up to SPL_MAX_TAPS): the warp-cooperative solve of pixel.cuh.
template <int FMT>
__global__ void __launch_bounds__(256) k_intensity1(const EstimateArgs a) {
    __shared__ float as[SPL_MAX_TAPS];
    __shared__ float s_hsum;
    const float hsum = template_table(a, as, &s_hsum);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const long long P = static_cast<long long>(a.H) * a.W;
    const long long stride = static_cast<long long>(gridDim.x) * (blockDim.x >> 5);
    for (long long p = static_cast<long long>(blockIdx.x) * (blockDim.x >> 5) + warp; p < P; p += stride) {
        const float K = a.bg[p];
        const bool faulty = a.faulty ? a.faulty[p] != 0 : false;
        const bool present = a.present_now ? a.present_now[p] != 0 : true;
        float r = 0.f, b = 0.f;
        if (faulty) {
            r = b = 0.f;
        } else if (!present || !(K > 0.f) || !(hsum > 0.f)) {
            r = 0.f;
            b = K / static_cast<float>(a.T);
        } else {
            const int t0 = window_start(a, a.mu[p]);
            float zj[SPL_MAX_TAPS / 32], aj[SPL_MAX_TAPS / 32];
#pragma unroll
            for (int q = 0; q < SPL_MAX_TAPS / 32; ++q) {
                const int j = lane + 32 * q;
                zj[q] = j < a.L ? hist_value<FMT>(a.z, a.pitch, p, t0 + j) : 0.f;
                aj[q] = j < a.L ? as[j] : 0.f;
            }
            px::intensity_mle<SPL_MAX_TAPS / 32>(zj, aj, K, a.L, a.T, hsum, r, b);
        }
        if (lane == 0) {
            a.refl[p] = r;
            a.bg[p] = b;
        }
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
    if (a.L <= 64) k_intensity4<FMT><<<nb, 256, 0, s>>>(a);
    else k_intensity1<FMT><<<nb, 256, 0, s>>>(a);
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
