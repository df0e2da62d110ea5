// Fused per-pixel kernel: robust data term (Eq. beta_div2), pseudo-posterior on the depth grid
// (Eq. approx_post) with the spatio-temporal Gaussian-mixture prior (Eq. predict), moment matching
// (Eq. KL_div), and the background/reflectivity estimate (Sec. II-E).
//
// Mapping: one warp owns one pixel at a time (persistent grid-stride loop over pixels). The warp streams the
// pixel's histogram row from HBM once with 16-byte loads into its shared-memory slice, evaluates C(d) for all
// candidates, then the log pseudo-posterior, its argmax and its argmax-centred moments, and finally the
// intensity MLE on the IRF window it already holds. Nothing but the per-pixel outputs goes back to HBM.
#include <cuda_fp16.h>
#include <math.h>

#include "spl_internal.h"

namespace spl {
namespace {

constexpr float kLog2e = 1.4426950408889634f;
constexpr float kLog2TwoPi = 2.6514961294723187f;  // log2(2 pi)
constexpr int kMaxComp = 10;                        // 9 stencil entries + 1 merged weakly informative one

__device__ __forceinline__ float ex2(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float lg2(float x) {
    float y;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Butterfly arg-max: every lane ends with the same (value, index); ties go to the smaller index.
__device__ __forceinline__ void warp_argmax(float& v, int& i) {
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        const float ov = __shfl_xor_sync(0xffffffffu, v, o);
        const int oi = __shfl_xor_sync(0xffffffffu, i, o);
        if (ov > v || (ov == v && oi < i)) {
            v = ov;
            i = oi;
        }
    }
}

// Loads pixel p's counts z[0..T) into zs (float), zero past T. Returns this lane's partial photon count.
template <int FMT>
__device__ __forceinline__ float load_row(const EstimateArgs& a, long long p, float* zs, int lane) {
    float K = 0.f;
    if (FMT == SPL_HIST_F32) {
        const float4* row = reinterpret_cast<const float4*>(static_cast<const float*>(a.z) + p * a.pitch);
        const int nch = (a.T + 3) >> 2;
        for (int i = lane; i < nch; i += 32) {
            float4 v = __ldcs(row + i);
            const int b = i * 4;
            if (b + 3 >= a.T) {
                if (b + 1 >= a.T) v.y = 0.f;
                if (b + 2 >= a.T) v.z = 0.f;
                if (b + 3 >= a.T) v.w = 0.f;
            }
            K += (v.x + v.y) + (v.z + v.w);
            reinterpret_cast<float4*>(zs)[i] = v;
        }
    } else {
        const uint4* row = reinterpret_cast<const uint4*>(static_cast<const uint16_t*>(a.z) + p * a.pitch);
        const int nch = (a.T + 7) >> 3;
        for (int i = lane; i < nch; i += 32) {
            const uint4 v = __ldcs(row + i);
            const unsigned w[4] = {v.x, v.y, v.z, v.w};
            float f[8];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                if (FMT == SPL_HIST_U16) {
                    f[2 * k] = static_cast<float>(w[k] & 0xffffu);
                    f[2 * k + 1] = static_cast<float>(w[k] >> 16);
                } else {
                    f[2 * k] = __half2float(__ushort_as_half(static_cast<unsigned short>(w[k] & 0xffffu)));
                    f[2 * k + 1] = __half2float(__ushort_as_half(static_cast<unsigned short>(w[k] >> 16)));
                }
            }
            const int b = i * 8;
#pragma unroll
            for (int k = 0; k < 8; ++k)
                if (b + k >= a.T) f[k] = 0.f;
            K += ((f[0] + f[1]) + (f[2] + f[3])) + ((f[4] + f[5]) + (f[6] + f[7]));
            reinterpret_cast<float4*>(zs)[2 * i] = make_float4(f[0], f[1], f[2], f[3]);
            reinterpret_cast<float4*>(zs)[2 * i + 1] = make_float4(f[4], f[5], f[6], f[7]);
        }
    }
    return K;
}

// Mixture prior in log2 units: component c contributes 2^(ca[c] - ck[c] (d - cm[c])^2).
struct Prior {
    float ca[kMaxComp], ck[kMaxComp], cm[kMaxComp];
    int n;
};

__device__ __forceinline__ void prior_add(Prior& pr, float w, float m, float v) {
    const float ca = lg2(w) - 0.5f * (kLog2TwoPi + lg2(v));
    const float ck = kLog2e / (2.f * v);
#pragma unroll
    for (int i = 0; i < kMaxComp; ++i)
        if (i == pr.n) {
            pr.ca[i] = ca;
            pr.ck[i] = ck;
            pr.cm[i] = m;
        }
    ++pr.n;
}

__device__ __forceinline__ void build_prior(const EstimateArgs& a, long long p, Prior& pr) {
    pr.n = 0;
    if (a.prior_mode == PRIOR_GAUSS) {
        prior_add(pr, 1.f, a.pmu[p], a.pvar[p]);
    } else if (a.prior_mode == PRIOR_STENCIL) {
        const int y = static_cast<int>(p / a.W), x = static_cast<int>(p - static_cast<long long>(y) * a.W);
        float flat_w = 0.f;
#pragma unroll
        for (int k = 0; k < 9; ++k) {
            const float w = a.nu[k];
            if (!(w > 0.f)) continue;
            const int yy = y + k / 3 - 1, xx = x + k % 3 - 1;
            bool informative = false;
            long long i = 0;
            if (yy >= 0 && yy < a.H && xx >= 0 && xx < a.W) {
                i = static_cast<long long>(yy) * a.W + xx;
                informative = (a.present_in ? a.present_in[i] != 0 : true) && !(a.faulty && a.faulty[i]);
            }
            if (informative)
                prior_add(pr, w, a.pmu[i], a.pvar[i] + a.sigma_rw2);
            else
                flat_w += w;  // every weakly informative entry is the same Gaussian: merge them
        }
        if (flat_w > 0.f) prior_add(pr, flat_w, a.flat_m, a.flat_v + a.sigma_rw2);
    }
}

// log2 of the prior density at depth d (up to the constant shared by all d).
__device__ __forceinline__ float log2_prior(const Prior& pr, float d) {
    if (pr.n == 0) return 0.f;
    if (pr.n == 1) {
        const float e = d - pr.cm[0];
        return pr.ca[0] - pr.ck[0] * e * e;
    }
    float t[kMaxComp];
    float mx = -INFINITY;
#pragma unroll
    for (int i = 0; i < kMaxComp; ++i) {
        if (i >= pr.n) break;
        const float e = d - pr.cm[i];
        t[i] = pr.ca[i] - pr.ck[i] * e * e;
        mx = fmaxf(mx, t[i]);
    }
    float s = 0.f;
#pragma unroll
    for (int i = 0; i < kMaxComp; ++i) {
        if (i >= pr.n) break;
        s += ex2(t[i] - mx);
    }
    return mx + lg2(s);
}

template <int FMT, bool COST_ONLY>
__global__ void __launch_bounds__(256) k_estimate(const EstimateArgs a) {
    extern __shared__ __align__(16) float dyn[];
    __shared__ float gs[SPL_MAX_TAPS];   // g_j = h_j^beta (0 for taps <= 0)
    __shared__ float as[SPL_MAX_TAPS];   // h_j / sum(h): the normalised template of the intensity model
    __shared__ float s_hsum;

    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    for (int j = threadIdx.x; j < a.L; j += blockDim.x) {
        const float hj = a.h[j];
        gs[j] = hj > 0.f ? powf(hj, a.beta) : 0.f;
        as[j] = hj > 0.f ? hj : 0.f;
    }
    __syncthreads();
    if (warp == 0) {
        float s = 0.f;
        for (int j = lane; j < a.L; j += 32) s += as[j];
        s = warp_sum(s);
        if (lane == 0) s_hsum = s;
    }
    __syncthreads();
    const float hsum = s_hsum;
    if (hsum > 0.f)
        for (int j = threadIdx.x; j < a.L; j += blockDim.x) as[j] /= hsum;
    __syncthreads();

    const int T = a.T, L = a.L, D = a.D, u0 = a.dmin - a.peak;
    const int Tz = (T + 7) & ~7, Dz = (D + 3) & ~3;
    float* zs = dyn + static_cast<size_t>(warp) * (Tz + Dz);
    float* cs = zs + Tz;
    const long long P = static_cast<long long>(a.H) * a.W;

    for (long long p = static_cast<long long>(blockIdx.x) * nwarps + warp; p < P;
         p += static_cast<long long>(gridDim.x) * nwarps) {
        const bool faulty = !COST_ONLY && a.faulty && a.faulty[p];
        float K = 0.f;
        if (!faulty) K = warp_sum(load_row<FMT>(a, p, zs, lane));
        __syncwarp();

        // ---- robust data term C(d) = sum_j g_j z[d - peak + j] for every candidate ----
        float best = -INFINITY;
        int bidx = 0x7fffffff;
        for (int c = lane; c < D; c += 32) {
            float acc = 0.f;
            if (!faulty) {
                const float* zz = zs + u0 + c;
                for (int j = 0; j < L; ++j) acc = fmaf(gs[j], zz[j], acc);
            }
            if (COST_ONLY) {
                if (a.cost) __stcs(a.cost + p * D + c, acc);
                if (acc > best) {
                    best = acc;
                    bidx = c;
                }
            } else {
                cs[c] = acc;
            }
        }
        if (COST_ONLY) {
            if (a.argmax) {
                warp_argmax(best, bidx);
                if (lane == 0) a.argmax[p] = a.dmin + bidx;
            }
            __syncwarp();
            continue;
        }

        // ---- log2 pseudo-posterior ell(d) = lambda log2(e) C(d) + log2 f(d), its argmax ----
        Prior pr;
        build_prior(a, p, pr);
        for (int c = lane; c < D; c += 32) {
            const float l = fmaf(a.lam2, cs[c], log2_prior(pr, static_cast<float>(a.dmin + c)));
            cs[c] = l;
            if (l > best) {
                best = l;
                bidx = c;
            }
        }
        warp_argmax(best, bidx);
        if (bidx == 0x7fffffff) bidx = 0;  // every ell was NaN (invalid inputs): keep indices in range

        // ---- moments of the normalised weights 2^(ell - max), centred on the argmax ----
        float s0 = 0.f, s1 = 0.f, s2 = 0.f;
        for (int c = lane; c < D; c += 32) {
            const float w = ex2(cs[c] - best);
            const float dd = static_cast<float>(c - bidx);
            s0 += w;
            s1 = fmaf(w, dd, s1);
            s2 = fmaf(w * dd, dd, s2);
        }
        s0 = warp_sum(s0);
        s1 = warp_sum(s1);
        s2 = warp_sum(s2);
        const float m1 = s1 / s0;
        const float mu = static_cast<float>(a.dmin + bidx) + m1;
        const float var = fmaxf(s2 / s0 - m1 * m1, 0.f);
        if (lane == 0) {
            a.mu[p] = mu;
            a.var[p] = var;
            if (a.argmax) a.argmax[p] = a.dmin + bidx;
        }

        // ---- background b and reflectivity r (Sec. II-E) ----
        if (a.refl) {
            float r = 0.f, b = 0.f;
            const bool present = a.present_now ? a.present_now[p] != 0 : true;
            if (faulty) {
                r = b = 0.f;
            } else if (!present || !(K > 0.f) || !(hsum > 0.f)) {
                r = 0.f;
                b = K / static_cast<float>(T);
            } else {
                // MLE of the signal fraction f of the two-component model "template a_t, uniform 1/T"
                // (Eq. lik_bg with the template at round(mu)); then r = f K / sum(h), b = (1 - f) K / T.
                // psi(f) = sum_W z (a - u) / (u + f (a - u)) - Kout / (1 - f) is decreasing on [0, 1).
                int t0 = __float2int_rn(mu) - a.peak;
                t0 = min(max(t0, 0), T - L);
                const float u = 1.f / static_cast<float>(T);
                float zj[SPL_MAX_TAPS / 32], aj[SPL_MAX_TAPS / 32];
                float kin = 0.f, za = 0.f, p1 = 0.f;
                bool zero_tap = false;
#pragma unroll
                for (int q = 0; q < SPL_MAX_TAPS / 32; ++q) {
                    const int j = lane + 32 * q;
                    zj[q] = j < L ? zs[t0 + j] : 0.f;
                    aj[q] = j < L ? as[j] : 0.f;
                    kin += zj[q];
                    za = fmaf(zj[q], aj[q], za);
                    if (zj[q] > 0.f) {
                        if (aj[q] > 0.f) p1 += zj[q] * (aj[q] - u) / aj[q];
                        else zero_tap = true;
                    }
                }
                kin = warp_sum(kin);
                za = warp_sum(za);
                p1 = warp_sum(p1);
                zero_tap = __any_sync(0xffffffffu, zero_tap);
                const float kout = fmaxf(K - kin, 0.f);
                const float psi0 = static_cast<float>(T) * za - K;
                float f;
                if (!(psi0 > 0.f)) {
                    f = 0.f;
                } else if (!(kout > 0.f) && !zero_tap && p1 >= 0.f) {
                    f = 1.f;
                } else {
                    float lo = 0.f, hi = 1.f;
                    f = 0.5f;
                    for (int it = 0; it < 64; ++it) {
                        float g = 0.f, gp = 0.f;
#pragma unroll
                        for (int q = 0; q < SPL_MAX_TAPS / 32; ++q) {
                            if (zj[q] > 0.f) {
                                const float e = (aj[q] - u) / fmaf(f, aj[q] - u, u);
                                g = fmaf(zj[q], e, g);
                                gp = fmaf(zj[q] * e, e, gp);
                            }
                        }
                        g = warp_sum(g);
                        gp = warp_sum(gp);
                        const float om = 1.f - f;
                        g -= kout / om;
                        gp += kout / (om * om);
                        if (g > 0.f) lo = f; else hi = f;
                        float fn = f + g / gp;  // Newton step on psi (psi' = -gp)
                        if (!(fn > lo && fn < hi)) fn = 0.5f * (lo + hi);
                        const bool done = fabsf(fn - f) <= 1e-7f * fn || hi - lo <= 1e-7f * hi;
                        f = fn;
                        if (done) break;
                    }
                }
                r = f * K / hsum;
                b = (1.f - f) * K * u;
            }
            if (lane == 0) {
                a.refl[p] = r;
                a.bg[p] = b;
            }
        }
        __syncwarp();
    }
}

template <int FMT, bool COST_ONLY>
cudaError_t launch_t(const EstimateArgs& a, cudaStream_t s) {
    auto kern = k_estimate<FMT, COST_ONLY>;
    const size_t per_warp = sizeof(float) * (((a.T + 7) & ~7) + ((a.D + 3) & ~3));
    const size_t budget = 200 * 1024;
    int wpc = static_cast<int>(budget / per_warp);
    if (wpc > 8) wpc = 8;
    if (wpc < 1) return cudaErrorInvalidConfiguration;
    const size_t smem = per_warp * wpc;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    static int configured[64] = {0};
    if (dev < 64 && !configured[dev]) {
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024);
        if (e != cudaSuccess) return e;
        configured[dev] = 1;
    }
    int nsm = 0, per_sm = 0;
    e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, wpc * 32, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
    const long long P = static_cast<long long>(a.H) * a.W;
    long long ctas = (P + wpc - 1) / wpc;
    const long long cap = static_cast<long long>(nsm) * per_sm;
    if (ctas > cap) ctas = cap;
    if (ctas < 1) ctas = 1;
    kern<<<static_cast<unsigned>(ctas), wpc * 32, smem, s>>>(a);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_estimate(const EstimateArgs& a, bool cost_only, cudaStream_t s) {
    switch (a.fmt) {
        case SPL_HIST_U16:
            return cost_only ? launch_t<SPL_HIST_U16, true>(a, s) : launch_t<SPL_HIST_U16, false>(a, s);
        case SPL_HIST_F16:
            return cost_only ? launch_t<SPL_HIST_F16, true>(a, s) : launch_t<SPL_HIST_F16, false>(a, s);
        case SPL_HIST_F32:
            return cost_only ? launch_t<SPL_HIST_F32, true>(a, s) : launch_t<SPL_HIST_F32, false>(a, s);
        default:
            return cudaErrorInvalidValue;
    }
}

}  // namespace spl
