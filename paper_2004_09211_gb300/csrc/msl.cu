// Multispectral depth estimate (Appendix, Eq. div_MSL): nb bands recorded at once by independent detectors, each
// with its own IRF h_l. The beta-divergence between the product of the bands' empirical ToA distributions and the
// product model is, up to a constant, -lambda M(d) with
//     M(d) = prod_l C_l(d) / K_l,   C_l(d) = sum_t z_l[t] h_l[t - d + peak]^beta,   K_l = photons of band l,
// a product over bands of normalised sums (where a maximum-likelihood fit would add log-likelihoods). Bands without
// photons contribute no factor. The pseudo-posterior is f(d) exp(lambda K M(d)) with K = sum_l K_l (for one band it
// is the single-band pseudo-posterior of Eq. approx_post); without a prior its maximiser is the minimum-divergence
// estimate of Eq. div_MSL.
//
// Mapping. One warp per pixel (persistent grid-stride loop). For each band in turn the row is read with 16-byte
// loads, converted to floats in the warp's shared slice, and correlated by a register-blocked direct sum (8
// candidates per lane, taps in groups of 4, the same tap-ordered chain per candidate as the single-band kernel);
// each candidate's running product M is multiplied by C_l / K_l in place. The pseudo-posterior moments then come
// from posterior.cuh with the data term lambda K M(d).
#include <cuda_fp16.h>
#include <math.h>

#include <atomic>

#include "pixel.cuh"
#include "posterior.cuh"
#include "spl_internal.h"

namespace spl {
namespace {

using namespace px;

// Shared slice of one warp (words): the band's row as floats (T rounded up to 4, plus 16 zero words that the
// register-blocked windows read past the row), M per candidate (NB * 32), per-block bounds (NB).
struct MSlice {
    int zf, cs, ubs, words;
};

__host__ __device__ __forceinline__ MSlice make_mslice(int T, int D) {
    MSlice s;
    const int nb = (D + 31) / 32;
    s.zf = 0;
    s.cs = ((T + 3) & ~3) + 16;
    s.ubs = s.cs + nb * 32;
    s.words = s.ubs + ((nb + 3) & ~3);
    return s;
}

// Row p of band l as floats into zf (bins >= T and the padding are zero); returns the band's photon count
// (warp-uniform).
template <int FMT>
__device__ __forceinline__ float load_row(const MslArgs& a, long long row, float* zf, int lane) {
    constexpr int CB = FMT == SPL_HIST_F32 ? 4 : 8;
    constexpr int ESZ = FMT == SPL_HIST_F32 ? 4 : 2;
    const int T = a.T;
    const int nch = (T + CB - 1) / CB;
    const uint4* src = reinterpret_cast<const uint4*>(static_cast<const char*>(a.z) + row * a.pitch * ESZ);
    float ks = 0.f;
    for (int i = lane; i < nch; i += 32) {
        const uint4 v = __ldcs(src + i);
        float f[CB];
        if (FMT == SPL_HIST_F32) {
            f[0] = __uint_as_float(v.x);
            f[1] = __uint_as_float(v.y);
            f[2] = __uint_as_float(v.z);
            f[3] = __uint_as_float(v.w);
        } else {
            const unsigned w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                if (FMT == SPL_HIST_U16) {
                    f[2 * k] = __int_as_float(0x4B000000 | (w[k] & 0xffffu)) - 8388608.f;
                    f[2 * k + 1] = __int_as_float(0x4B000000 | (w[k] >> 16)) - 8388608.f;
                } else {
                    f[2 * k] = __half2float(__ushort_as_half(static_cast<unsigned short>(w[k] & 0xffffu)));
                    f[2 * k + 1] = __half2float(__ushort_as_half(static_cast<unsigned short>(w[k] >> 16)));
                }
            }
        }
#pragma unroll
        for (int k = 0; k < CB; ++k) {
            if (i * CB + k >= T) f[k] = 0.f;  // elements T..pitch-1 are not data
            ks += f[k];
        }
        // 4 or 8 floats of bins i*CB.. (T is padded to a multiple of 4 in the slice; writes past it land in the
        // zero padding, which is rewritten below)
        reinterpret_cast<float4*>(zf)[i * (CB / 4)] = make_float4(f[0], f[1], f[2], f[3]);
        if (CB == 8) reinterpret_cast<float4*>(zf)[i * 2 + 1] = make_float4(f[4], f[5], f[6], f[7]);
    }
    __syncwarp();
    const int tp = (T + 3) & ~3;
    if (lane < 4) reinterpret_cast<float4*>(zf + tp)[lane] = make_float4(0.f, 0.f, 0.f, 0.f);
    __syncwarp();
    return warp_sum(ks);
}

// M(c) *= C_l(c) / K_l for every candidate c (register-blocked direct sum from the float row; windows start on
// 4-bin boundaries and may read up to 11 bins past the row, which are zero).
__device__ __forceinline__ void multiply_band(const float* __restrict__ gs, const float* zf, float* cs, int D, int L,
                                              int u0, float inv_k, int lane) {
    for (int cb = -(u0 & 3); cb < D; cb += 256) {
        const int cl = cb + 8 * lane;
        if (cl < D && cl + 7 >= 0) {
            const float4* r4 = reinterpret_cast<const float4*>(zf + u0 + cl);
            const float4* g4 = reinterpret_cast<const float4*>(gs);
            float acc[8];
#pragma unroll
            for (int r = 0; r < 8; ++r) acc[r] = 0.f;
            float4 c0 = r4[0], c1 = r4[1];
            for (int jg = 0; jg < L; jg += 4) {
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
            for (int r = 0; r < 8; ++r)
                if (cl + r >= 0 && cl + r < D) cs[cl + r] *= acc[r] * inv_k;
        }
    }
    __syncwarp();
}

template <int FMT>
__global__ void __launch_bounds__(256) k_estimate_msl(const MslArgs a) {
    extern __shared__ __align__(16) float dyn[];
    __shared__ __align__(16) float gsb[SPL_MAX_BANDS][SPL_MAX_TAPS + 4];  // g = h^beta per band (0 past L)
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const int nb = a.nbands, L = a.L, D = a.D, T = a.T, u0 = a.dmin - a.peak, NB = (D + 31) >> 5;
    for (int i = threadIdx.x; i < SPL_MAX_BANDS * (SPL_MAX_TAPS + 4); i += blockDim.x) {
        const int l = i / (SPL_MAX_TAPS + 4), j = i - l * (SPL_MAX_TAPS + 4);
        const float hj = (l < nb && j < L) ? a.h[l * L + j] : 0.f;
        gsb[l][j] = hj > 0.f ? powf(hj, a.beta) : 0.f;
    }
    __syncthreads();

    const MSlice sl = make_mslice(T, D);
    float* base = dyn + static_cast<size_t>(warp) * sl.words;
    float* zf = base + sl.zf;
    float* cs = base + sl.cs;
    float* ubs = base + sl.ubs;
    const long long P = static_cast<long long>(a.H) * a.W;
    const long long stride = static_cast<long long>(gridDim.x) * nwarps;

    for (long long p = static_cast<long long>(blockIdx.x) * nwarps + warp; p < P; p += stride) {
        for (int c = lane; c < NB * 32; c += 32) cs[c] = 1.f;  // the empty product
        __syncwarp();
        float ktot = 0.f;
        for (int l = 0; l < nb; ++l) {
            const float kl = load_row<FMT>(a, static_cast<long long>(l) * P + p, zf, lane);
            if (!(kl > 0.f)) continue;  // no photons in this band: no factor
            multiply_band(gsb[l], zf, cs, D, L, u0, 1.f / kl, lane);
            ktot += kl;
        }
        float mmax = 0.f;
        for (int c = lane; c < D; c += 32) mmax = fmaxf(mmax, cs[c]);
        mmax = warp_max(mmax);
        if (a.cost) {
            for (int c = lane; c < D; c += 32) __stcs(a.cost + p * D + c, cs[c]);
        }

        Prior pr;
        {
            float w = 0.f, m = 0.f, v = 1.f;
            if (a.pmu && lane == 0) {
                w = 1.f;
                m = a.pmu[p];
                v = a.pvar[p];
            }
            build_prior(w, m, v, lane, pr);
        }
        Grid grid;
        grid.D = D;
        grid.NB = NB;
        grid.dmin = a.dmin;
        grid.u0 = u0;
        grid.L = L;
        grid.lam2 = a.lam2 * ktot;  // ell in log2 units: lambda K M(d) log2(e) + log2 f(d)
        grid.gmax = 0.f;
        const float dub = grid.lam2 * mmax * 1.0001f;  // every block's data term is at most lambda K max M
        const int ub_b = block_bounds(grid, pr, ubs, [&](int) { return dub; }, lane);
        int bidx;
        float mu, var;
        posterior_eval(
            grid, pr, mmax, cs, ubs, ub_b,
            [&]() {  // rare fallback: M again on every candidate
                for (int c = lane; c < NB * 32; c += 32) cs[c] = 1.f;
                __syncwarp();
                for (int l = 0; l < nb; ++l) {
                    const float kl = load_row<FMT>(a, static_cast<long long>(l) * P + p, zf, lane);
                    if (kl > 0.f) multiply_band(gsb[l], zf, cs, D, L, u0, 1.f / kl, lane);
                }
            },
            lane, bidx, mu, var);
        if (lane == 0) {
            if (a.argmax) a.argmax[p] = a.dmin + bidx;
            a.mu[p] = mu;
            a.var[p] = var;
        }
        __syncwarp();
    }
}

template <int FMT>
cudaError_t launch_t(const MslArgs& a, cudaStream_t s) {
    auto kern = k_estimate_msl<FMT>;
    const size_t per_warp = sizeof(float) * static_cast<size_t>(make_mslice(a.T, a.D).words);
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

size_t msl_warp_bytes(int T, int D) { return sizeof(float) * static_cast<size_t>(make_mslice(T, D).words); }

cudaError_t launch_estimate_msl(const MslArgs& a, cudaStream_t s) {
    switch (a.fmt) {
        case SPL_HIST_U16: return launch_t<SPL_HIST_U16>(a, s);
        case SPL_HIST_F16: return launch_t<SPL_HIST_F16>(a, s);
        case SPL_HIST_F32: return launch_t<SPL_HIST_F32>(a, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace spl
