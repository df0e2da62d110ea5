// Per-pixel device code shared by the depth kernels (histograms: estimate.cu; photon lists: batch.cu,
// noalloc.cu; the tensor-core filter, the differentiable filter and the intensity launch): one warp per pixel.
//
//   build_prior     Eq. predict: the Gaussian-mixture prior of one pixel (lanes 0-8 own the 3x3 entries).
//   log2_prior      the prior on the depth grid (log-sum-exp), and an upper bound of it over a range of depths.
//   intensity_mle   Sec. II-E: background and reflectivity by maximum likelihood under Eq. lik_bg_poisson.
//
// The pseudo-posterior moments on the integer grid (pruning and the linear-domain epilogue) are in posterior.cuh.
#pragma once

#include <math.h>
#include <stdint.h>

namespace spl {
namespace px {

constexpr float kLog2e = 1.4426950408889634f;
constexpr float kLog2TwoPi = 2.6514961294723187f;  // log2(2 pi)
constexpr int kMaxComp = 9;                         // at most 9 distinct components (3x3 stencil)
constexpr float kPrune2 = 64.f;                     // log2 margin below the best value for dropping a block
// Newton on the signal fraction stops once its step is below this fraction of f: the error after that step is of
// the order of the step squared, below FP32 resolution. The test comes before the bracket update: at the root,
// psi's rounding noise can put the next iterate on the bracket's end, and a bisection from there would throw away
// a converged f.
constexpr float kNewtonTol = 1e-5f;

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
__device__ __forceinline__ float warp_max(float v) {
#pragma unroll
    for (int o = 16; o; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
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

__device__ __forceinline__ void zero_words(float* x, int n4, int lane) {
    for (int i = lane; i < n4; i += 32) reinterpret_cast<float4*>(x)[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    __syncwarp();
}

// ------------------------------------------------------------------------------------------------------------
// Prior (Eq. predict) in log2 units: component c contributes 2^(ca[c] - ck[c] (d - cm[c])^2)
// ------------------------------------------------------------------------------------------------------------

struct Prior {
    float ca[kMaxComp], ck[kMaxComp], cm[kMaxComp];
    float minv;  // smallest component variance
    int n;
};

// Lane k (< 9) passes stencil entry k as (weight w, mean m, variance v); w = 0 marks an unused entry. Entries
// with identical Gaussians (every weakly informative one, and equal neighbour states) are merged by matching
// their (mean, variance) bits and summing their weights; the distinct components are then broadcast to every
// lane in lane order.
__device__ __forceinline__ void build_prior(float w, float m, float v, int lane, Prior& pr) {
    const bool act = w > 0.f;
    if (!act) v = 1.f;
    const unsigned long long key =
        act ? (static_cast<unsigned long long>(__float_as_uint(m)) << 32) | __float_as_uint(v)
            : 0xFFFFFFFF00000000ull | static_cast<unsigned>(lane);
    const unsigned peers = __match_any_sync(0xffffffffu, key);
    float wsum = 0.f;
#pragma unroll
    for (int k = 0; k < 9; ++k) {
        const float wk = __shfl_sync(0xffffffffu, w, k);
        if ((peers >> k) & 1u) wsum += wk;
    }
    const bool leader = act && lane == __ffs(peers) - 1;
    unsigned lead = __ballot_sync(0xffffffffu, leader);
    pr.n = __popc(lead);
    const float ca_l = lg2(wsum) - 0.5f * (kLog2TwoPi + lg2(v));
    const float ck_l = kLog2e / (2.f * v);
    pr.minv = INFINITY;
#pragma unroll
    for (int i = 0; i < kMaxComp; ++i) {
        if (i < pr.n) {  // warp-uniform: only the distinct components are broadcast
            const int src = __ffs(lead) - 1;
            lead &= lead - 1;
            pr.ca[i] = __shfl_sync(0xffffffffu, ca_l, src);
            pr.ck[i] = __shfl_sync(0xffffffffu, ck_l, src);
            pr.cm[i] = __shfl_sync(0xffffffffu, m, src);
            pr.minv = fminf(pr.minv, __shfl_sync(0xffffffffu, v, src));
        } else {
            pr.ca[i] = pr.ck[i] = pr.cm[i] = 0.f;
        }
    }
}

// log2 of the prior density at depth d (up to the constant shared by all d), by log-sum-exp.
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

// Upper bound of log2_prior over depths [lo, hi].
__device__ __forceinline__ float log2_prior_bound(const Prior& pr, float lo, float hi) {
    if (pr.n == 0) return 0.f;
    float mx = -INFINITY;
#pragma unroll
    for (int i = 0; i < kMaxComp; ++i) {
        if (i >= pr.n) break;
        const float e = fmaxf(fmaxf(lo - pr.cm[i], pr.cm[i] - hi), 0.f);
        mx = fmaxf(mx, pr.ca[i] - pr.ck[i] * e * e);
    }
    return pr.n > 1 ? mx + lg2(static_cast<float>(pr.n)) + 1e-3f : mx + 1e-3f;
}

// ------------------------------------------------------------------------------------------------------------
// Background and reflectivity (Sec. II-E)
// ------------------------------------------------------------------------------------------------------------

// MLE of the signal fraction f of the two-component model "template a_t, uniform 1/T" (Eq. lik_bg with the
// template placed on the window W); intensity_mle then gives r = f K / sum(h) and b = (1 - f) K / T. Lane items: zj[q] = photons
// in a window bin whose normalised template value is aj[q] (items of all lanes together cover W once).
// psi(f) = sum_W z (a - u) / (u + f (a - u)) - Kout / (1 - f), u = 1/T, is decreasing on [0, 1): safeguarded
// Newton on psi with the bracket [lo, hi] kept around its root.
template <int NQ>
__device__ __forceinline__ float intensity_fraction(const float* zj, const float* aj, float K, int L, int T) {
    const float u = 1.f / static_cast<float>(T);
    float kin = 0.f, za = 0.f, p1 = 0.f;
    bool zero_tap = false;
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
        kin += zj[q];
        za = fmaf(zj[q], aj[q], za);
        if (zj[q] > 0.f) {
            if (aj[q] > 0.f) p1 += zj[q] * __fdividef(aj[q] - u, aj[q]);
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
        // start from the box-template estimate (window excess over the flat background)
        const float fr = static_cast<float>(L) * u;
        f = fr < 1.f ? (kin - K * fr) / (K * (1.f - fr)) : 0.5f;
        f = fminf(fmaxf(f, 0.02f), 0.98f);
        for (int it = 0; it < 64; ++it) {
            float gs = 0.f, gp = 0.f;
#pragma unroll
            for (int q = 0; q < NQ; ++q) {
                if (zj[q] > 0.f) {
                    const float e = __fdividef(aj[q] - u, fmaf(f, aj[q] - u, u));
                    gs = fmaf(zj[q], e, gs);
                    gp = fmaf(zj[q] * e, e, gp);
                }
            }
            gs = warp_sum(gs);
            gp = warp_sum(gp);
            const float rom = __fdividef(1.f, 1.f - f);
            gs = fmaf(-kout, rom, gs);
            gp = fmaf(kout * rom, rom, gp);
            const float step = __fdividef(gs, gp);  // Newton step on psi (psi' = -gp)
            if (fabsf(step) <= kNewtonTol * f) {  // converged (tested before the bracket: see kNewtonTol)
                f += step;
                break;
            }
            if (gs > 0.f) lo = f; else hi = f;
            float fn = f + step;
            if (!(fn > lo && fn < hi)) fn = 0.5f * (lo + hi);
            const bool conv = hi - lo <= 1e-7f * hi;
            f = fn;
            if (conv) break;
        }
    }
    return f;
}

// (r, b) from the signal fraction above: r = f K / sum(h), b = (1 - f) K / T.
template <int NQ>
__device__ __forceinline__ void intensity_mle(const float* zj, const float* aj, float K, int L, int T, float hsum,
                                              float& r, float& b) {
    const float f = intensity_fraction<NQ>(zj, aj, K, L, T);
    r = f * K / hsum;
    b = (1.f - f) * K * (1.f / static_cast<float>(T));
}

}  // namespace px
}  // namespace spl
