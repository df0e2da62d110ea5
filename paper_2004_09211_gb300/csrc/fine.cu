// Sub-bin depth: the single-frame pseudo-Bayesian estimate (Eq. approx_post) on a fine candidate grid
// d_k = dmin + k / S, k = 0 .. (dmax - dmin) S, with the data term of Eq. beta_div2 taken at fractional shifts of
// a continuous IRF. The continuous IRF is the piecewise-linear interpolation of the taps with h[-1] = h[L] = 0
// (support (-1, L)); the histogram's photons sit at their bin positions t, so
//     C(d) = sum_t z_t h_c(t - d + peak)^beta.
// A candidate d = d0 + phi / S (d0 integer, 0 <= phi < S) reads bins d0 - peak + j, j = 0 .. L, against the tap
// table g_phi[j] = h_c(j - phi / S)^beta: S interleaved integer-grid correlations. The pseudo-likelihood is
// exp(-K D_beta) with the whole beta-divergence between the histogram and the binned template s_d: besides
// lambda C(d) it keeps -K sum_j s_d[j]^(1+beta), which Eq. beta_div2 drops because it is the same for every
// whole-bin shift but which changes with the phase of an interpolated template (K = the photon count):
//     ell(d) = lambda C(d) - K pw_phi + log N(d; prior),  pw_phi = sum_j h_c(j - phi / S)^(1+beta).
//
// Mapping: one warp per pixel (persistent grid). The row is converted to floats in the warp's shared slice
// (zero past T); each phase's correlation is register-blocked (8 candidates per lane, taps in groups of 4);
// C of every fine candidate goes to shared memory, then two passes give the smallest maximiser of
// ell = lambda log2(e) C + log2 N(d; prior) and the argmax-centred moments, and a third pass takes the moments
// again about the rounded mean when it lies more than two standard deviations from the maximiser. No pruning:
// every candidate is evaluated exactly in the log domain.
#include <cuda_fp16.h>
#include <math.h>

#include <atomic>

#include "pixel.cuh"
#include "spl_internal.h"

namespace spl {
namespace {

using namespace px;

constexpr int kFineMaxS = 16;
constexpr int kTapPad = ((SPL_MAX_TAPS + 1 + 3) / 4) * 4;  // L + 1 taps per phase, padded to groups of 4
constexpr int kRowPad = kTapPad + 16;                       // zero floats after the row (window overreach)

struct FineArgs {
    const void* z;
    long long pitch;
    int fmt;
    const float* h;
    int H, W, T, L, peak, dmin, D, S, Kf;
    float beta, lam2;
    const float* pmu;
    const float* pvar;
    int* argmax;
    float* mu;
    float* var;
};

__host__ __device__ __forceinline__ int row_words(int T) { return ((T + kRowPad + 3) / 4) * 4; }
__host__ __device__ __forceinline__ int fine_words(const FineArgs& a) {
    return row_words(a.T) + ((a.Kf + 3) / 4) * 4;
}

template <int FMT>
__device__ __forceinline__ float count_at(const void* z, long long i) {
    if (FMT == SPL_HIST_F32) return static_cast<const float*>(z)[i];
    if (FMT == SPL_HIST_F16) return __half2float(static_cast<const __half*>(z)[i]);
    return static_cast<float>(static_cast<const unsigned short*>(z)[i]);
}

template <int FMT>
__global__ void __launch_bounds__(256) k_estimate_fine(const FineArgs a) {
    extern __shared__ __align__(16) float dyn[];
    __shared__ __align__(16) float gt[kFineMaxS * kTapPad];  // g_phi[j], phase-major
    __shared__ float hp[kFineMaxS * kTapPad];                 // h_c(j - phi / S)^(1 + beta)
    __shared__ float pw[kFineMaxS];                           // sum_j of the above, per phase (log2 units)
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const int S = a.S, L = a.L, T = a.T, D = a.D, Kf = a.Kf;
    for (int i = threadIdx.x; i < S * kTapPad; i += blockDim.x) {
        const int phi = i / kTapPad, j = i - phi * kTapPad;
        float v = 0.f;
        if (j <= L) {
            // h_c(x), x = j - phi / S in (-1, L]: interpolation between taps fl and fl + 1 (zero outside 0..L-1)
            const float x = static_cast<float>(j) - static_cast<float>(phi) / static_cast<float>(S);
            const float fl = floorf(x);
            const int jl = static_cast<int>(fl);
            const float w = x - fl;
            const float ha = jl >= 0 && jl < L ? a.h[jl] : 0.f;
            const float hb = jl + 1 >= 0 && jl + 1 < L ? a.h[jl + 1] : 0.f;
            const float hc = (1.f - w) * fmaxf(ha, 0.f) + w * fmaxf(hb, 0.f);
            v = hc > 0.f ? powf(hc, a.beta) : 0.f;
            hp[i] = v * hc;
        } else {
            hp[i] = 0.f;
        }
        gt[i] = v;
    }
    __syncthreads();
    for (int ph = warp; ph < S; ph += nwarps) {  // one warp per phase
        float sp = 0.f;
        for (int j = lane; j < kTapPad; j += 32) sp += hp[ph * kTapPad + j];
        sp = warp_sum(sp);
        if (lane == 0) pw[ph] = sp * kLog2e;
    }
    __syncthreads();

    float* row = dyn + static_cast<size_t>(warp) * fine_words(a);
    float* cs = row + row_words(T);
    const int rw = row_words(T);
    const long long P = static_cast<long long>(a.H) * a.W;
    const int u0 = a.dmin - a.peak;
    for (long long p = static_cast<long long>(blockIdx.x) * nwarps + warp; p < P;
         p += static_cast<long long>(gridDim.x) * nwarps) {
        // the row as floats, zero past T (unrolled: several loads in flight per lane), and the photon count K
        float K = 0.f;
#pragma unroll 8
        for (int t = lane; t < rw; t += 32) {
            const float v = t < T ? count_at<FMT>(a.z, p * a.pitch + t) : 0.f;
            row[t] = v;
            K += v;
        }
        K = warp_sum(K);
        __syncwarp();
        // C for every fine candidate: phase phi, integer offsets c (d0 = dmin + c), fine index k = c S + phi
        for (int phi = 0; phi < S; ++phi) {
            const float4* g4 = reinterpret_cast<const float4*>(gt + phi * kTapPad);
            const int Dphi = phi == 0 ? D : D - 1;  // the grid ends at dmax
            for (int cb = -(u0 & 3); cb < Dphi; cb += 256) {
                const int cl = cb + 8 * lane;
                if (cl < Dphi && cl + 7 >= 0) {
                    const int t0 = u0 + cl;  // a multiple of 4
                    const float4* r4 = reinterpret_cast<const float4*>(row + t0);
                    float acc[8];
#pragma unroll
                    for (int r = 0; r < 8; ++r) acc[r] = 0.f;
                    float4 c0 = r4[0], c1 = r4[1];
                    for (int jg = 0; jg <= L; jg += 4) {
                        const float4 nx = r4[jg / 4 + 2];
                        const float4 g = g4[jg / 4];
                        const float w[12] = {c0.x, c0.y, c0.z, c0.w, c1.x, c1.y, c1.z, c1.w, nx.x, nx.y, nx.z, nx.w};
#pragma unroll
                        for (int r = 0; r < 8; ++r) {
                            acc[r] = fmaf(g.x, w[r], acc[r]);
                            acc[r] = fmaf(g.y, w[r + 1], acc[r]);
                            acc[r] = fmaf(g.z, w[r + 2], acc[r]);
                            acc[r] = fmaf(g.w, w[r + 3], acc[r]);
                        }
                        c0 = c1;
                        c1 = nx;
                    }
#pragma unroll
                    for (int r = 0; r < 8; ++r) {
                        const int c = cl + r;
                        if (c >= 0 && c < Dphi) cs[c * S + phi] = acc[r];
                    }
                }
            }
        }
        __syncwarp();
        // pass 1: ell (log2 units) and the smallest maximiser
        const bool has_prior = a.pmu != nullptr;
        const float pm = has_prior ? a.pmu[p] : 0.f;
        const float pk = has_prior ? kLog2e / (2.f * a.pvar[p]) : 0.f;
        const float invS = 1.f / static_cast<float>(S);
        float best = -INFINITY;
        int bk = 0x7fffffff;
        for (int k = lane; k < Kf; k += 32) {
            const float d = static_cast<float>(a.dmin) + static_cast<float>(k) * invS;
            const float e = d - pm;
            const int phi = k - (k / S) * S;
            const float l = fmaf(a.lam2, cs[k], fmaf(-pk * e, e, -K * pw[phi]));
            cs[k] = l;
            if (l > best) {
                best = l;
                bk = k;
            }
        }
        warp_argmax(best, bk);
        if (bk >= Kf) bk = 0;  // every ell was NaN (invalid inputs): keep the index in range
        __syncwarp();
        // pass 2: moments about the maximiser, in fine-index units
        float s0 = 0.f, s1 = 0.f, s2 = 0.f;
        for (int k = lane; k < Kf; k += 32) {
            const float w = ex2(cs[k] - best);
            const float dd = static_cast<float>(k - bk);
            s0 += w;
            s1 = fmaf(w, dd, s1);
            s2 = fmaf(w * dd, dd, s2);
        }
        s0 = warp_sum(s0);
        s1 = warp_sum(s1);
        s2 = warp_sum(s2);
        int ctr = bk;
        float m1 = s1 / s0;
        float var = s2 / s0 - m1 * m1;
        if (m1 * m1 > 4.f * var + 1.f) {
            // pass 3: the maximiser lies more than two standard deviations from the mean (a broad or bimodal
            // posterior), where S2/S0 and the squared offset would cancel: the moments again about the rounded
            // mean
            ctr = __float2int_rn(static_cast<float>(bk) + m1);
            s0 = s1 = s2 = 0.f;
            for (int k = lane; k < Kf; k += 32) {
                const float w = ex2(cs[k] - best);
                const float dd = static_cast<float>(k - ctr);
                s0 += w;
                s1 = fmaf(w, dd, s1);
                s2 = fmaf(w * dd, dd, s2);
            }
            s0 = warp_sum(s0);
            s1 = warp_sum(s1);
            s2 = warp_sum(s2);
            m1 = s1 / s0;
            var = s2 / s0 - m1 * m1;
        }
        if (lane == 0) {
            if (a.argmax) a.argmax[p] = bk;
            a.mu[p] = static_cast<float>(a.dmin) + (static_cast<float>(ctr) + m1) * invS;
            a.var[p] = fmaxf(var, 0.f) * invS * invS;
        }
        __syncwarp();
    }
}

template <int FMT>
cudaError_t launch_fmt(const FineArgs& a, cudaStream_t s) {
    auto kern = k_estimate_fine<FMT>;
    const size_t per_warp = sizeof(float) * static_cast<size_t>(fine_words(a));
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    static std::atomic<int> configured[64];
    if (dev >= 64 || !configured[dev].load(std::memory_order_acquire)) {
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        if (e != cudaSuccess) return e;
        if (dev < 64) configured[dev].store(1, std::memory_order_release);
    }
    int nsm = 0;
    e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    int best_wpc = 0, best_ctas = 0, best_warps = 0;
    for (int wpc = 8; wpc >= 1; --wpc) {
        const size_t smem = per_warp * wpc;
        if (smem > 200 * 1024) continue;
        int per_sm = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, wpc * 32, smem);
        if (e != cudaSuccess) return e;
        if (per_sm * wpc > best_warps) {
            best_warps = per_sm * wpc;
            best_wpc = wpc;
            best_ctas = per_sm;
        }
    }
    if (best_wpc == 0) return cudaErrorInvalidConfiguration;
    const long long P = static_cast<long long>(a.H) * a.W;
    long long ctas = (P + best_wpc - 1) / best_wpc;
    const long long cap = static_cast<long long>(nsm) * best_ctas;
    if (ctas > cap) ctas = cap;
    if (ctas < 1) ctas = 1;
    kern<<<static_cast<unsigned>(ctas), best_wpc * 32, per_warp * best_wpc, s>>>(a);
    return cudaGetLastError();
}

}  // namespace

size_t fine_warp_bytes(int T, int D, int S) {
    const long long Kf = static_cast<long long>(D - 1) * S + 1;
    return sizeof(float) * static_cast<size_t>(row_words(T) + ((Kf + 3) / 4) * 4);
}

cudaError_t launch_estimate_fine(const EstimateArgs& e, int S, int* argmax_k, cudaStream_t s) {
    FineArgs a;
    a.z = e.z;
    a.pitch = e.pitch;
    a.fmt = e.fmt;
    a.h = e.h;
    a.H = e.H;
    a.W = e.W;
    a.T = e.T;
    a.L = e.L;
    a.peak = e.peak;
    a.dmin = e.dmin;
    a.D = e.D;
    a.S = S;
    a.Kf = (e.D - 1) * S + 1;
    a.beta = e.beta;
    a.lam2 = e.lam2;
    a.pmu = e.prior_mode == PRIOR_GAUSS ? e.pmu : nullptr;
    a.pvar = e.prior_mode == PRIOR_GAUSS ? e.pvar : nullptr;
    a.argmax = argmax_k;
    a.mu = e.mu;
    a.var = e.var;
    switch (a.fmt) {
        case SPL_HIST_U16: return launch_fmt<SPL_HIST_U16>(a, s);
        case SPL_HIST_F16: return launch_fmt<SPL_HIST_F16>(a, s);
        case SPL_HIST_F32: return launch_fmt<SPL_HIST_F32>(a, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace spl
