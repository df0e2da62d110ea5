// One frame of the online filter (Algorithm 1) with the data term on the tensor cores: FP16 or uint16 histograms
// in, the same outputs as the FP32 filter step out, nothing per candidate written to memory.
//
// Data term. C(d) = sum_j g_j z[d - peak + j] (Eq. beta_div2) for 128 pixels x 64 candidates per tile, as the
// banded-Toeplitz product of tc.cu: C[p, 64 t + n] = sum_k Z[p, a0 + 64 t + k] G[k, n] with G[k, n] =
// g[k - n - delta] * 2^15 split into FP16 high and low parts, accumulated in FP32 in tensor memory.
// The photon count K of every pixel (Sec. II-E) comes from the same slabs: one extra N = 16 MMA per 64-bin slab
// against a column of ones, accumulated over all slabs that cover [0, T) (exact in FP32 below 2^24 photons).
//
// Pipeline (persistent CTAs, 6 warps each, one or two CTAs per SM):
//   warp 4  TMA producer: the 64-bin slabs of a 128-pixel block, origin x0 <= 0 so that every bin of [0, T) and
//           every candidate window is covered, into a ring of R slabs (128-byte swizzled; zero fill outside).
//   warp 5  MMA issuer: per slab the count MMA; once a tile's last slab has landed, the tile's MMAs into one of
//           two accumulators; each slab goes back to the producer as soon as no later tile reads it. With uint16
//           histograms the whole warp first converts each landed slab to FP16 in place (convert_slab: exact for
//           counts below 1024) and notes whether the block holds a larger count.
//   warps 0-3 epilogue, thread = pixel = TMEM lane:
//     prior   Eq. predict from the 3x3 neighbour states, equal Gaussians merged (as the warp kernel does);
//     tiles   ell(d) = lambda log2(e) C(d) + log2 f(d) in log2 units. A lower bound of max ell is the prior at its
//             mode (C >= 0). A tile, then each 16-candidate chunk of it, is evaluated only if its upper bound
//             lambda log2(e) max C + max log2 f reaches the running maximum minus 64: a dropped chunk weighs less
//             than 2^-64 of the maximum. Evaluated chunks update the argmax (smallest maximiser) and are merged
//             into running (weight, mean, second central moment) with a shared exponent reference, the chunk's
//             own moments taken about its best candidate (the pairwise update of Chan, Golub and LeVeque), so
//             no step subtracts large nearly equal numbers.
//     output  mu = mean, var = second moment / weight (Eq. KL_div), argmax; the photon count K goes to bg. With
//             uint16 input a block holding a count of 1024 or more (FP16 would not carry it exactly), and a pixel
//             whose data term exceeds kTcMaxBits, get mu = NaN instead, and the FP32 kernel computes them again
//             (k_estimate_redo, estimate.cu).
// A second launch (intensity.cu) then runs the intensity MLE of Sec. II-E on the template at round-half-even(mu)
// with that K and writes refl and bg.
// All mbarrier waits are bounded (status bit 0 on time-out; the roles then stop, in-flight copies and MMAs are
// waited for, tensor memory is released).
#include <math.h>
#include <stdint.h>

#include <mutex>

#include "f32x2.cuh"
#include "pixel.cuh"
#include "spl_internal.h"
#include "tc_common.cuh"

namespace spl {
namespace {

using namespace tc;
using px::ex2;
using px::lg2;
using px::Prior;

constexpr int kM = 128;                          // pixels per block
constexpr int kN = 64;                           // candidates per tile
constexpr int kSlab = 64;                        // bins per slab
constexpr int kMaxRing = 8;
constexpr int kThreads = 192;
constexpr unsigned kTmemCols = 256;              // acc 0 | acc 1 | count 0 | count 1 (64 + 64 + 16 + 16 used)
constexpr unsigned kCntCol = 128;
constexpr float kScale = 32768.f;
constexpr unsigned kSlabBytes = kM * kSlab * 2;  // 16 KB
constexpr unsigned kBSlabBytes = kN * kSlab * 2; // 8 KB
constexpr unsigned kOnesBytes = 16 * kSlab * 2;  // 2 KB
constexpr uint32_t kIdescTile = idesc_f16(kM, kN);
constexpr uint32_t kIdescCnt = idesc_f16(kM, 16);
constexpr float kPrune = px::kPrune2;            // log2 margin below the running maximum
// uint16 input: largest data term lambda log2(e) max C (bits) a pixel keeps on the tensor cores. C here carries the
// taps' 2^-23 relative residual and FP32 accumulation over at most 16 rounded steps, |dC| <= 2^-19.8 max C, so ell
// stays within 1e-3 bits of its exact value below this; a brighter pixel is computed by the FP32 kernel.
constexpr float kTcMaxBits = 1024.f;

struct TcGeom {
    int a0, delta, kw, ntiles, nslab, mlead, S, npt, ring, nbs;
    float lam2s;  // lambda log2(e) 2^-15 (the accumulators hold C * 2^15)
};

// The prior of one pixel, one thread. The filter step (PRIOR_STENCIL), Eq. predict: stencil entry k contributes
// N(mu_in, var_in + sigma_rw2) when the neighbour is inside the frame, present and not faulty, else the weakly
// informative Gaussian; entries with nu_k = 0 are unused. Entries with bitwise equal (mean, variance) are merged by
// adding their weights in stencil order, then the used ones are packed to the front in stencil order. A single
// frame: one Gaussian N(pmu[p], pvar[p]) (PRIOR_GAUSS), or the flat prior (PRIOR_UNIFORM) as one component with
// k = 0, whose value 2^0 is the same at every depth (its recurrence ratios are 1).
__device__ __forceinline__ void prior_thread(const EstimateArgs& a, long long p, Prior& pr, bool& faulty) {
    if (a.prior_mode != PRIOR_STENCIL) {
        const bool gauss = a.prior_mode == PRIOR_GAUSS;
        const float v = gauss ? a.pvar[p] : 1.f;
        pr.n = 1;
        pr.ca[0] = gauss ? -0.5f * (px::kLog2TwoPi + lg2(v)) : 0.f;
        pr.ck[0] = gauss ? px::kLog2e / (2.f * v) : 0.f;
        pr.cm[0] = gauss ? a.pmu[p] : 0.f;
        pr.minv = gauss ? v : INFINITY;
#pragma unroll
        for (int i = 1; i < px::kMaxComp; ++i) {
            pr.ca[i] = -INFINITY;
            pr.ck[i] = pr.cm[i] = 0.f;
        }
        faulty = a.faulty ? a.faulty[p] != 0 : false;
        return;
    }
    const int y = static_cast<int>(p / a.W), x = static_cast<int>(p - static_cast<long long>(y) * a.W);
    float w[9], m[9], v[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) {
        const int yy = y + k / 3 - 1, xx = x + k % 3 - 1;
        bool info = false;
        float mk = 0.f, vk = 0.f;
        if (yy >= 0 && yy < a.H && xx >= 0 && xx < a.W) {
            const long long i = static_cast<long long>(yy) * a.W + xx;
            mk = a.pmu[i];
            vk = a.pvar[i];
            const int pres = a.present_in ? a.present_in[i] : 1;
            const int fl = a.faulty ? a.faulty[i] : 0;
            info = pres != 0 && fl == 0;
        }
        w[k] = a.nu[k];
        m[k] = info ? mk : a.flat_m;
        v[k] = (info ? vk : a.flat_v) + a.sigma_rw2;
    }
    faulty = a.faulty ? a.faulty[p] != 0 : false;
    // an entry equal to an earlier used one joins it (the earlier one is then the only used entry with that
    // Gaussian, so the first match is the representative)
#pragma unroll
    for (int k = 1; k < 9; ++k) {
#pragma unroll
        for (int i = 0; i < k; ++i) {
            const bool same = w[i] > 0.f && w[k] > 0.f && __float_as_uint(m[i]) == __float_as_uint(m[k]) &&
                              __float_as_uint(v[i]) == __float_as_uint(v[k]);
            w[i] = same ? w[i] + w[k] : w[i];
            w[k] = same ? 0.f : w[k];
        }
    }
    // pack the used entries to the front, keeping their order (adjacent exchanges)
#pragma unroll
    for (int pass = 0; pass < 8; ++pass) {
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const bool sw = !(w[j] > 0.f) && w[j + 1] > 0.f;
            const float tw = w[j], tm = m[j], tv = v[j];
            w[j] = sw ? w[j + 1] : w[j];
            m[j] = sw ? m[j + 1] : m[j];
            v[j] = sw ? v[j + 1] : v[j];
            w[j + 1] = sw ? tw : w[j + 1];
            m[j + 1] = sw ? tm : m[j + 1];
            v[j + 1] = sw ? tv : v[j + 1];
        }
    }
    pr.n = 0;
    pr.minv = INFINITY;
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        const bool act = w[i] > 0.f;
        pr.n += act ? 1 : 0;
        const float vi = act ? v[i] : 1.f;
        pr.ca[i] = act ? lg2(w[i]) - 0.5f * (px::kLog2TwoPi + lg2(vi)) : -INFINITY;
        pr.ck[i] = px::kLog2e / (2.f * vi);
        pr.cm[i] = act ? m[i] : 0.f;
        if (act) pr.minv = fminf(pr.minv, vi);
    }
}

// log2 of the prior density at d (up to a constant) over the first NC component slots; slots past the pixel's
// own count have ca = -inf and contribute nothing. NC is the largest component count in the warp, so the loops
// have fixed trip counts instead of per-lane predication over all 9 slots.
template <int NC>
__device__ __forceinline__ float lp_n(const Prior& pr, float d) {
    if (NC == 1) {
        const float e = d - pr.cm[0];
        return pr.ca[0] - pr.ck[0] * e * e;
    }
    float t[NC];
    float mx = -INFINITY;
#pragma unroll
    for (int k = 0; k < NC; ++k) {
        const float e = d - pr.cm[k];
        t[k] = pr.ca[k] - pr.ck[k] * e * e;
        mx = fmaxf(mx, t[k]);
    }
    float sum = 0.f;
#pragma unroll
    for (int k = 0; k < NC; ++k) sum += ex2(t[k] - mx);
    return mx + lg2(sum);
}

// Upper bound of lp_n over depths [lo, hi] (the largest component's maximum there, plus log2 of the count).
template <int NC>
__device__ __forceinline__ float lpb_n(const Prior& pr, float lo, float hi) {
    float mx = -INFINITY;
#pragma unroll
    for (int k = 0; k < NC; ++k) {
        const float e = fmaxf(fmaxf(lo - pr.cm[k], pr.cm[k] - hi), 0.f);
        mx = fmaxf(mx, pr.ca[k] - pr.ck[k] * e * e);
    }
    return NC > 1 && pr.n > 1 ? mx + lg2(static_cast<float>(pr.n)) + 1e-3f : mx + 1e-3f;
}

// Running pseudo-posterior summary of one pixel. Weights are 2^(ell - ref) with the reference kept as a pair,
// ref = l2s cref + pref (l2s = lambda log2(e) 2^-15, cref a raw accumulator value, pref a log2 prior value), so
// every exponent is formed as l2s (c - c') + (p - p'): differences of nearby numbers and one FMA, never the
// difference of two large log values. The reference is any value that keeps the weights in range (it may lie
// above the maximum); the pruning threshold uses `top`, a value of ell actually reached (or the lower bound
// from the prior's mode).
struct Moments {
    float cref, pref;
    float W;      // sum of weights
    float mu;     // weighted mean, candidate index units
    float M2;     // sum of w (d - mu)^2
    float top;    // max(lower bound, largest ell evaluated), absolute log2 units
    float best;   // largest ell evaluated
    int bidx;     // its candidate index (smallest on ties)
    float amax;   // largest raw accumulator seen on any tile
};

// Merges one chunk's sums (s0 = sum u, s1 = sum u x, s2 = sum u x^2 with x = candidate - ctr, weights u
// relative to the chunk reference (cr, pr_)) into the running summary: the pairwise update of Chan, Golub and
// LeVeque after bringing both to the larger reference.
__device__ __forceinline__ void merge(Moments& s, float l2s, float cr, float pr_, float s0, float s1, float s2,
                                      float ctr) {
    const float r0 = 1.f / s0;
    const float cmu = ctr + s1 * r0;
    float cm2 = fmaxf(fmaf(-s1 * r0, s1, s2), 0.f);
    if (!(s.W > 0.f)) {
        s.cref = cr;
        s.pref = pr_;
        s.W = s0;
        s.mu = cmu;
        s.M2 = cm2;
        return;
    }
    const float diff = fmaf(l2s, cr - s.cref, pr_ - s.pref);  // chunk reference - running reference (bits)
    if (diff > 0.f) {
        const float sc = ex2(-diff);
        s.W *= sc;
        s.M2 *= sc;
        s.cref = cr;
        s.pref = pr_;
    } else {
        const float sc = ex2(diff);
        s0 *= sc;
        cm2 *= sc;
    }
    const float Wn = s.W + s0;
    const float dl = cmu - s.mu;
    const float f = s0 / Wn;
    s.mu = fmaf(dl, f, s.mu);
    s.M2 += cm2 + dl * dl * s.W * f;
    s.W = Wn;
}

// As merge, for a chunk whose weight s0, mean cmu (candidate index) and second central moment cm2 are known.
__device__ __forceinline__ void merge_centred(Moments& s, float l2s, float cr, float pr_, float s0, float cmu,
                                              float cm2) {
    if (!(s.W > 0.f)) {
        s.cref = cr;
        s.pref = pr_;
        s.W = s0;
        s.mu = cmu;
        s.M2 = cm2;
        return;
    }
    const float diff = fmaf(l2s, cr - s.cref, pr_ - s.pref);  // chunk reference - running reference (bits)
    if (diff > 0.f) {
        const float sc = ex2(-diff);
        s.W *= sc;
        s.M2 *= sc;
        s.cref = cr;
        s.pref = pr_;
    } else {
        const float sc = ex2(diff);
        s0 *= sc;
        cm2 *= sc;
    }
    const float Wn = s.W + s0;
    const float dl = cmu - s.mu;
    const float f = s0 / Wn;
    s.mu = fmaf(dl, f, s.mu);
    s.M2 += cm2 + dl * dl * s.W * f;
    s.W = Wn;
}

// Exact log-domain chunk: raw accumulators c[0..15] of candidates c0 .. c0 + 15 (those >= D excluded).
template <int NC>
__device__ __forceinline__ void chunk_log(const float* c, int c0, int D, int dmin, float l2s, const Prior& pr,
                                          Moments& s) {
    float lp[16], l[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) {
        const bool in = c0 + i < D;
        lp[i] = in ? lp_n<NC>(pr, static_cast<float>(dmin + c0 + i)) : -INFINITY;
        l[i] = in ? fmaf(l2s, c[i], lp[i]) : -INFINITY;
    }
    float lm = l[0];
#pragma unroll
    for (int i = 1; i < 16; ++i) lm = fmaxf(lm, l[i]);
    int ib = 0;
    float cb = c[0], pb = lp[0];
#pragma unroll
    for (int i = 15; i >= 0; --i) {
        const bool hit = l[i] == lm;
        ib = hit ? i : ib;
        cb = hit ? c[i] : cb;
        pb = hit ? lp[i] : pb;
    }
    if (lm > s.best) {
        s.best = lm;
        s.bidx = c0 + ib;
    }
    s.top = fmaxf(s.top, lm);
    if (!(lm >= s.top - kPrune)) return;
    float s0 = 0.f, s1 = 0.f, s2 = 0.f;
#pragma unroll
    for (int i = 0; i < 16; ++i) {
        const float w = ex2(fmaf(l2s, c[i] - cb, lp[i] - pb));
        const float x = static_cast<float>(i - ib);
        s0 += w;
        s1 = fmaf(w, x, s1);
        s2 = fmaf(w * x, x, s2);
    }
    merge(s, l2s, cb, pb, s0, s1, s2, static_cast<float>(c0 + ib));
}

// Linear-domain chunk. The weight of candidate i relative to the reference (cq = the chunk's largest
// accumulator, pref = an upper bound of the prior on the chunk) is 2^(l2s (c_i - cq)) *
// sum_k 2^(ca_k - ck_k (d_i - m_k)^2 - pref): one exp2 for the data factor and, per mixture component, the exact
// two-multiply recurrence of a Gaussian on a unit grid (value ratio, then ratio of ratios) started from exact
// exponentials at the chunk's first candidate. No value exceeds n; a component that underflows on the chunk is
// below 2^-126 of the reference. Returns false (nothing merged, nothing updated) when the chunk's largest
// weight is below 2^-60 of the reference; the caller then bounds the chunk exactly and, if it can matter, runs
// the exact log-domain chunk. Requires component variances >= 1.5 bins^2, so that 15 steps from the start cannot
// take a component from below the float range up to its peak. FULL: all 16 candidates are < D.
// The chunk's moments are formed in two passes (sum u and sum u i, then sum u (i - mean)^2), so the chunk
// variance is not a difference of large numbers and a mean at the chunk's first candidate keeps its relative
// precision.
template <int NC, bool FULL>
__device__ __forceinline__ bool chunk_lin(const float* c, int c0, int D, int dmin, float l2s, const Prior& pr,
                                         float cq, float pref, Moments& s) {
    float v[NC], q[NC], rho[NC];
    const float d0 = static_cast<float>(dmin + c0);
#pragma unroll
    for (int k = 0; k < NC; ++k) {
        const float e = d0 - pr.cm[k];
        v[k] = ex2(pr.ca[k] - pr.ck[k] * e * e - pref);
        q[k] = ex2(fminf(-pr.ck[k] * (2.f * e + 1.f), 100.f));
        rho[k] = ex2(-2.f * pr.ck[k]);
    }
    float u[16];
    float um = 0.f, s0 = 0.f, s1 = 0.f;
#pragma unroll
    for (int i = 0; i < 16; ++i) {
        float pv = 0.f;
#pragma unroll
        for (int k = 0; k < NC; ++k) {
            pv += v[k];
            v[k] *= q[k];
            q[k] *= rho[k];
        }
        u[i] = ex2(l2s * (c[i] - cq)) * pv;
        if (!FULL) u[i] = c0 + i < D ? u[i] : 0.f;
        um = fmaxf(um, u[i]);
        s0 += u[i];
        s1 = fmaf(u[i], static_cast<float>(i), s1);
    }
    if (!(um >= 0x1p-60f)) return false;
    const float lm = fmaf(l2s, cq, pref) + lg2(um);
    if (lm > s.best) {  // new best: its (smallest) index in the chunk
        int ib = 0;
#pragma unroll
        for (int i = 15; i >= 0; --i) ib = u[i] == um ? i : ib;
        s.best = lm;
        s.bidx = c0 + ib;
    }
    s.top = fmaxf(s.top, lm);
    if (!(lm >= s.top - kPrune)) return true;
    const float m1 = s1 / s0;
    float s2 = 0.f;
#pragma unroll
    for (int i = 0; i < 16; ++i) {
        const float x = static_cast<float>(i) - m1;
        s2 = fmaf(u[i] * x, x, s2);
    }
    merge_centred(s, l2s, cq, pref, s0, static_cast<float>(c0) + m1, s2);
    return true;
}

// chunk_lin with the candidates taken in adjacent pairs (2j, 2j + 1), one packed f32x2 instruction per pair for
// every add, multiply and FMA. Each component then follows two interleaved Gaussians on the even and the odd
// candidates: values V = (v(2j), v(2j + 1)), started from exact exponentials at candidates 0 and 1, step ratios
// v(i + 2) / v(i) = 2^(-k (4 (d_i - m) + 4)), and the ratio of those ratios 2^(-8 k) for both. Same contract and
// the same data factor, bit for bit, as chunk_lin; the prior values and the moment sums differ from it by
// rounding only (eight recurrence steps per value instead of fifteen, sums split into even and odd halves).
template <int NC, bool FULL>
__device__ __forceinline__ bool chunk_lin2(const float* c, int c0, int D, int dmin, float l2s, const Prior& pr,
                                          float cq, float pref, Moments& s) {
    using px::f2;
    f2 V[NC], Q[NC], R[NC];
    const float d0 = static_cast<float>(dmin + c0);
#pragma unroll
    for (int k = 0; k < NC; ++k) {
        const float e = d0 - pr.cm[k], ck = pr.ck[k], b = pr.ca[k] - pref;
        const float e1 = e + 1.f;
        V[k] = px::f2_make(ex2(b - ck * e * e), ex2(b - ck * e1 * e1));
        Q[k] = px::f2_make(ex2(fminf(-ck * fmaf(4.f, e, 4.f), 100.f)), ex2(fminf(-ck * fmaf(4.f, e, 8.f), 100.f)));
        const float r = ex2(-8.f * ck);
        R[k] = px::f2_make(r, r);
    }
    const f2 ncq = px::f2_make(-cq, -cq), sl = px::f2_make(l2s, l2s);
    f2 U[8];
    f2 S0 = px::f2_make(0.f, 0.f), S1 = S0;
    float um = 0.f;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        f2 pv = V[0];
        V[0] = px::f2_mul(V[0], Q[0]);
        Q[0] = px::f2_mul(Q[0], R[0]);
#pragma unroll
        for (int k = 1; k < NC; ++k) {
            pv = px::f2_add(pv, V[k]);
            V[k] = px::f2_mul(V[k], Q[k]);
            Q[k] = px::f2_mul(Q[k], R[k]);
        }
        const f2 t = px::f2_mul(px::f2_add(px::f2_make(c[2 * j], c[2 * j + 1]), ncq), sl);
        f2 u = px::f2_mul(px::f2_make(ex2(px::f2_lo(t)), ex2(px::f2_hi(t))), pv);
        if (!FULL)
            u = px::f2_make(c0 + 2 * j < D ? px::f2_lo(u) : 0.f, c0 + 2 * j + 1 < D ? px::f2_hi(u) : 0.f);
        U[j] = u;
        um = fmaxf(um, fmaxf(px::f2_lo(u), px::f2_hi(u)));
        S0 = px::f2_add(S0, u);
        S1 = px::f2_fma(u, px::f2_make(static_cast<float>(2 * j), static_cast<float>(2 * j + 1)), S1);
    }
    if (!(um >= 0x1p-60f)) return false;
    const float lm = fmaf(l2s, cq, pref) + lg2(um);
    if (lm > s.best) {  // new best: its (smallest) index in the chunk
        int ib = 0;
#pragma unroll
        for (int j = 7; j >= 0; --j) {
            ib = px::f2_hi(U[j]) == um ? 2 * j + 1 : ib;
            ib = px::f2_lo(U[j]) == um ? 2 * j : ib;
        }
        s.best = lm;
        s.bidx = c0 + ib;
    }
    s.top = fmaxf(s.top, lm);
    if (!(lm >= s.top - kPrune)) return true;
    const float s0 = px::f2_lo(S0) + px::f2_hi(S0);
    const float m1 = (px::f2_lo(S1) + px::f2_hi(S1)) / s0;
    const f2 nm = px::f2_make(-m1, -m1);
    f2 S2 = px::f2_make(0.f, 0.f);
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const f2 x = px::f2_add(px::f2_make(static_cast<float>(2 * j), static_cast<float>(2 * j + 1)), nm);
        S2 = px::f2_fma(px::f2_mul(U[j], x), x, S2);
    }
    merge_centred(s, l2s, cq, pref, s0, static_cast<float>(c0) + m1, px::f2_lo(S2) + px::f2_hi(S2));
    return true;
}

// One candidate tile of one pixel (this lane). A tile whose prior bound alone reaches the pruning threshold is
// kept without looking at the data (C >= 0); otherwise its largest accumulator decides. Kept tiles are evaluated
// chunk by chunk with the tile's prior bound as the reference. The tensor-memory loads are warp-collective:
// every lane issues them; the decisions are per lane.
template <int NC>
__device__ __forceinline__ void tile_work(uint32_t tacc, int c0t, int D, int dmin, float l2s, const Prior& pr,
                                          bool valid, bool lin_ok, Moments& st) {
    const int nval = min(kN, D - c0t);
    const float lpt = lpb_n<NC>(pr, static_cast<float>(dmin + c0t), static_cast<float>(dmin + c0t + nval - 1));
    bool alive = valid && lpt >= st.top - kPrune;
    if (__any_sync(0xffffffffu, valid && !alive)) {
        float cm = 0.f;
#pragma unroll
        for (int q = 0; q < kN / 16; ++q) {
            float c[16];
            tmem_ld16(tacc + 16 * q, c);
            tmem_wait_ld();
#pragma unroll
            for (int i = 0; i < 16; ++i) cm = fmaxf(cm, c[i]);
        }
        st.amax = fmaxf(st.amax, cm);
        alive = valid && fmaf(l2s, cm, lpt) >= st.top - kPrune;
    }
    if (!__any_sync(0xffffffffu, alive)) return;
#pragma unroll 1
    for (int q = 0; q < kN / 16 && c0t + 16 * q < D; ++q) {
        const int cq0 = c0t + 16 * q;
        float c[16];
        tmem_ld16(tacc + 16 * q, c);
        tmem_wait_ld();
        if (alive) {
            float cq = c[0];
#pragma unroll
            for (int i = 1; i < 16; ++i) cq = fmaxf(cq, c[i]);
            st.amax = fmaxf(st.amax, cq);
            if (fmaf(l2s, cq, lpt) >= st.top - kPrune) {
                bool done = false;
                if (lin_ok) {
                    if (NC <= 5)  // packed pairs; the nine-component case keeps the scalar form (registers)
                        done = cq0 + 16 <= D ? chunk_lin2<NC, true>(c, cq0, D, dmin, l2s, pr, cq, lpt, st)
                                             : chunk_lin2<NC, false>(c, cq0, D, dmin, l2s, pr, cq, lpt, st);
                    else
                        done = cq0 + 16 <= D ? chunk_lin<NC, true>(c, cq0, D, dmin, l2s, pr, cq, lpt, st)
                                             : chunk_lin<NC, false>(c, cq0, D, dmin, l2s, pr, cq, lpt, st);
                }
                if (!done) {
                    const float lpq = lpb_n<NC>(pr, static_cast<float>(dmin + cq0),
                                                static_cast<float>(dmin + min(cq0 + 15, D - 1)));
                    if (fmaf(l2s, cq, lpq) >= st.top - kPrune) chunk_log<NC>(c, cq0, D, dmin, l2s, pr, st);
                }
            }
        }
        __syncwarp();
    }
}

// One landed slab of uint16 counts (kSlabBytes, any swizzle: elements convert in place) to FP16, by the whole warp.
// For u < 1024 the FP16 number with bits 0x6400 | u is exactly 1024 + u, so one OR and one packed FP16 subtraction
// of 1024 give u exactly, two bins at a time. Returns nonzero (on the lanes that saw one) when a count is 1024 or
// more: bits 10-15 of its 16-bit half are set.
__device__ __forceinline__ unsigned convert_slab(unsigned char* slab, int lane) {
    uint4* v = reinterpret_cast<uint4*>(slab);
    unsigned big = 0;
#pragma unroll 4
    for (int i = lane; i < static_cast<int>(kSlabBytes / 16); i += 32) {
        uint4 w = v[i];
        big |= (w.x | w.y | w.z | w.w) & 0xFC00FC00u;
        unsigned r[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
        for (int k = 0; k < 4; ++k)
            asm("sub.rn.f16x2 %0, %1, %2;" : "=r"(r[k]) : "r"(r[k] | 0x64006400u), "r"(0x64006400u));
        v[i] = make_uint4(r[0], r[1], r[2], r[3]);
    }
    return big;
}

template <bool U16>
__global__ void __launch_bounds__(kThreads, 2)
    k_filter_tc(const __grid_constant__ CUtensorMap zmap, const EstimateArgs a, const TcGeom g, unsigned* status) {
    extern __shared__ unsigned char smem_raw[];
    __shared__ __align__(8) unsigned long long bar[2 * kMaxRing + 11];
    __shared__ int s_ovf[2];  // uint16 input: the block (by parity) holds a count >= 1024
    __shared__ uint32_t tmem_base;
    __shared__ int abort_flag;
    __shared__ float s_g[SPL_MAX_TAPS];

    const unsigned base = (smem_u32(smem_raw) + 1023u) & ~1023u;
    unsigned char* gbase = smem_raw + (base - smem_u32(smem_raw));
    const unsigned ring = static_cast<unsigned>(g.ring);
    const unsigned ringA = base;
    const unsigned Bhi = base + ring * kSlabBytes;
    const unsigned Blo = Bhi + g.nbs * kBSlabBytes;
    const unsigned Bone = Blo + g.nbs * kBSlabBytes;
    const unsigned full0 = smem_u32(&bar[0]), empty0 = smem_u32(&bar[kMaxRing]);
    const unsigned accf0 = smem_u32(&bar[2 * kMaxRing]), acce0 = smem_u32(&bar[2 * kMaxRing + 2]);
    const unsigned cntf0 = smem_u32(&bar[2 * kMaxRing + 4]), cnte0 = smem_u32(&bar[2 * kMaxRing + 6]);
    const unsigned drain = smem_u32(&bar[2 * kMaxRing + 8]);
    const unsigned ovf0 = smem_u32(&bar[2 * kMaxRing + 9]);  // s_ovf of a block written (uint16 input)
    volatile int* stop = &abort_flag;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    // ---- set-up ----
    if (warp == 5) tmem_alloc(smem_u32(&tmem_base), kTmemCols);
    for (int j = tid; j < SPL_MAX_TAPS; j += kThreads) {
        const float hj = j < a.L ? a.h[j] : 0.f;
        s_g[j] = hj > 0.f ? powf(hj, a.beta) : 0.f;
    }
    if (tid == 0) {
        for (unsigned i = 0; i < ring; ++i) {
            mbar_init(full0 + 8 * i, 1);
            mbar_init(empty0 + 8 * i, 1);
        }
        for (int i = 0; i < 2; ++i) {
            mbar_init(accf0 + 8 * i, 1);
            mbar_init(acce0 + 8 * i, 4);
            mbar_init(cntf0 + 8 * i, 1);
            mbar_init(cnte0 + 8 * i, 4);
        }
        mbar_init(drain, 1);
        mbar_init(ovf0, 1);
        mbar_init(ovf0 + 8, 1);
        s_ovf[0] = s_ovf[1] = 0;
        abort_flag = 0;
    }
    __syncthreads();
    for (int e = tid; e < g.nbs * kSlab * kN; e += kThreads) {  // Toeplitz operand, high and low parts
        const int k = e / kN, n = e - k * kN;
        const int j = k - n - g.delta;
        const float gv = (k < g.kw && j >= 0 && j < a.L) ? s_g[j] * kScale : 0.f;
        const __half hi = __float2half_rn(gv);
        const __half lo = __float2half_rn(gv - __half2float(hi));
        const unsigned off = (k / kSlab) * kBSlabBytes + swz_offset(n, k % kSlab);
        *reinterpret_cast<__half*>(gbase + (Bhi - base) + off) = hi;
        *reinterpret_cast<__half*>(gbase + (Blo - base) + off) = lo;
    }
    for (int e = tid; e < 16 * kSlab; e += kThreads)  // ones operand of the count MMA
        *reinterpret_cast<__half*>(gbase + (Bone - base) + swz_offset(e / kSlab, e % kSlab)) = __float2half_rn(1.f);
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = tmem_base;

    if (warp == 4) {
        // ================= TMA producer =================
        if (lane == 0) {
            const int x0 = g.a0 - kSlab * g.mlead;
            unsigned cnt = 0, slot = 0, phase = 0;
            bool ok = true;
            for (int pt = blockIdx.x; pt < g.npt && ok && !*stop; pt += gridDim.x) {
                for (int s = 0; s < g.S; ++s) {
                    if (cnt >= ring && !(ok = wait_bounded(empty0 + 8 * slot, phase ^ 1u, stop, status))) break;
                    mbar_expect_tx(full0 + 8 * slot, kSlabBytes);
                    tma_load_2d(ringA + slot * kSlabBytes, &zmap, x0 + kSlab * s, pt * kM, full0 + 8 * slot);
                    ++cnt;
                    if (++slot == ring) {
                        slot = 0;
                        phase ^= 1u;
                    }
                }
            }
            for (unsigned i = cnt > ring ? cnt - ring : 0; i < cnt; ++i) wait_quiet(full0 + 8 * (i % ring), (i / ring) & 1u);
        }
    } else if (warp == 5) {
        // ================= MMA issuer (lane 0); with uint16 input the warp converts each slab first =================
        unsigned gs = 0, rel = 0, tcount = 0, blk = 0;
        bool ok = true;
        for (int pt = blockIdx.x; pt < g.npt && ok; pt += gridDim.x, ++blk) {
            const unsigned base_s = gs;
            const uint32_t dcnt = tmem + kCntCol + 16u * (blk & 1u);
            if (blk >= 2) {
                if (lane == 0) ok = wait_bounded(cnte0 + 8 * (blk & 1u), ((blk >> 1) - 1) & 1u, stop, status);
                if (!__shfl_sync(0xffffffffu, ok, 0)) {
                    ok = false;
                    break;
                }
            }
            fence_after();
            unsigned big = 0;
            for (int s = 0; s < g.S; ++s, ++gs) {
                if (lane == 0) ok = wait_bounded(full0 + 8 * (gs % ring), (gs / ring) & 1u, stop, status);
                if (!__shfl_sync(0xffffffffu, ok, 0)) {
                    ok = false;
                    break;
                }
                fence_after();
                const unsigned aslab = ringA + (gs % ring) * kSlabBytes;
                if (U16) {  // in place, then made visible to the tensor cores (async proxy) before lane 0 issues
                    big |= convert_slab(gbase + (aslab - base), lane);
                    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
                    __syncwarp();
                }
                if (lane == 0) {
#pragma unroll
                    for (int kk = 0; kk < kSlab; kk += 16)
                        mma_f16<kIdescCnt>(dcnt, desc_sw128(aslab + 2 * kk), desc_sw128(Bone + 2 * kk),
                                           (s > 0 || kk > 0) ? 1u : 0u);
                    const int t = s - g.mlead - g.nslab + 1;
                    if (t >= 0 && t < g.ntiles) {
                        const unsigned acc = tcount & 1u, use = tcount >> 1;
                        if (use > 0) ok = wait_bounded(acce0 + 8 * acc, (use - 1) & 1u, stop, status);
                        if (ok) {
                            fence_after();
                            const uint32_t d = tmem + acc * kN;
                            for (int j = 0; j < g.nslab; ++j) {
                                const unsigned sj = base_s + g.mlead + t + j;
                                const unsigned sl = ringA + (sj % ring) * kSlabBytes;
                                const int k_end = min(kSlab * (j + 1), g.kw);
                                for (int k = kSlab * j; k < k_end; k += 16) {
                                    const unsigned koff = (k - kSlab * j) * 2;
                                    const uint64_t ad = desc_sw128(sl + koff);
                                    mma_f16<kIdescTile>(d, ad, desc_sw128(Bhi + j * kBSlabBytes + koff),
                                                        k > 0 ? 1u : 0u);
                                    mma_f16<kIdescTile>(d, ad, desc_sw128(Blo + j * kBSlabBytes + koff), 1u);
                                }
                            }
                            mma_commit(accf0 + 8 * acc);
                            ++tcount;
                        }
                    }
                    if (ok) {  // slabs that no later tile of the block reads go back to the producer
                        const int tn = max(0, s - g.mlead - g.nslab + 2);
                        const unsigned need = tn < g.ntiles ? base_s + g.mlead + tn : gs + 1;
                        const unsigned lim = min(need, gs + 1);
                        for (; rel < lim; ++rel) mma_commit(empty0 + 8 * (rel % ring));
                    }
                }
                if (!__shfl_sync(0xffffffffu, ok, 0)) {
                    ok = false;
                    break;
                }
            }
            if (!ok) break;
            if (U16) {  // the block's flag, published by the barrier the epilogue waits on before reading it
                const unsigned any = __any_sync(0xffffffffu, big != 0);
                if (lane == 0) {
                    s_ovf[blk & 1u] = any ? 1 : 0;
                    mbar_arrive(ovf0 + 8 * (blk & 1u));
                }
            }
            if (lane == 0) mma_commit(cntf0 + 8 * (blk & 1u));
        }
        if (lane == 0) {
            mma_commit(drain);
            wait_quiet(drain, 0);
        }
    } else {
        // ================= epilogue: thread = pixel = TMEM lane =================
        const long long P = static_cast<long long>(a.H) * a.W;
        const int D = a.D, dmin = a.dmin;
        const uint32_t lane_base = tmem + (static_cast<uint32_t>(warp * 32) << 16);
        unsigned tcount = 0, blk = 0;
        bool ok = true;
        for (int pt = blockIdx.x; pt < g.npt && ok; pt += gridDim.x, ++blk) {
            const long long p = static_cast<long long>(pt) * kM + tid;
            const bool valid = p < P;
            Prior pr;
            bool faulty = false;
            if (valid) {
                prior_thread(a, p, pr, faulty);
            } else {  // padding lane: one flat component, results discarded
                pr.n = 1;
                pr.minv = 1.f;
#pragma unroll
                for (int i = 0; i < px::kMaxComp; ++i) {
                    pr.ca[i] = i == 0 ? 0.f : -INFINITY;
                    pr.ck[i] = 0.f;
                    pr.cm[i] = 0.f;
                }
            }
            const int nw = static_cast<int>(__reduce_max_sync(0xffffffffu, static_cast<unsigned>(pr.n)));
            const float l2s = faulty ? 0.f : g.lam2s;
            Moments st;
            {  // lower bound of max ell: the prior at the mode of its tallest component (C >= 0)
                float top = -INFINITY, tm = 0.f;
#pragma unroll
                for (int i = 0; i < px::kMaxComp; ++i)
                    if (i < pr.n && pr.ca[i] > top) {
                        top = pr.ca[i];
                        tm = pr.cm[i];
                    }
                const float d0 = fminf(fmaxf(rintf(tm), static_cast<float>(dmin)), static_cast<float>(dmin + D - 1));
                st.top = px::log2_prior(pr, d0);
            }
            st.cref = st.pref = 0.f;
            st.W = st.mu = st.M2 = 0.f;
            st.best = -INFINITY;
            st.bidx = 0;
            st.amax = 0.f;
            const bool lin_ok = !(pr.minv < 1.5f);
            for (int t = 0; t < g.ntiles; ++t, ++tcount) {
                const unsigned acc = tcount & 1u, use = tcount >> 1;
                ok = __all_sync(0xffffffffu, wait_bounded(accf0 + 8 * acc, use & 1u, stop, status));
                if (!ok) break;
                fence_after();
                const uint32_t tacc = lane_base + acc * kN;
                const int c0t = kN * t;
                switch (nw) {  // warp-uniform
                    case 1: tile_work<1>(tacc, c0t, D, dmin, l2s, pr, valid, lin_ok, st); break;
                    case 2: tile_work<2>(tacc, c0t, D, dmin, l2s, pr, valid, lin_ok, st); break;
                    case 3: tile_work<3>(tacc, c0t, D, dmin, l2s, pr, valid, lin_ok, st); break;
                    case 4:
                    case 5: tile_work<5>(tacc, c0t, D, dmin, l2s, pr, valid, lin_ok, st); break;
                    default: tile_work<9>(tacc, c0t, D, dmin, l2s, pr, valid, lin_ok, st); break;
                }
                fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(acce0 + 8 * acc);
            }
            if (!ok) break;
            // photon count of the block's pixels
            ok = __all_sync(0xffffffffu,
                            wait_bounded(cntf0 + 8 * (blk & 1u), (blk >> 1) & 1u, stop, status));
            if (!ok) break;
            fence_after();
            const float K = tmem_ld1(lane_base + kCntCol + 16u * (blk & 1u));
            tmem_wait_ld();
            int redo = 0;
            if (U16) {  // read before the count accumulator is released (the issuer then rewrites the flag)
                ok = __all_sync(0xffffffffu, wait_bounded(ovf0 + 8 * (blk & 1u), (blk >> 1) & 1u, stop, status));
                if (!ok) break;
                redo = *reinterpret_cast<volatile int*>(&s_ovf[blk & 1u]);
            }
            fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(cnte0 + 8 * (blk & 1u));
            // outputs; the photon count goes to bg, where the intensity launch reads it
            if (U16 && l2s * st.amax > kTcMaxBits) redo = 1;  // beyond the tensor cores' accuracy bound
            if (valid) {
                if (redo) {
                    a.mu[p] = NAN;  // k_estimate_redo computes this pixel again
                } else {
                    a.mu[p] = static_cast<float>(dmin) + st.mu;
                    a.var[p] = st.M2 / st.W;
                    if (a.argmax) a.argmax[p] = dmin + st.bidx;
                    if (a.refl) a.bg[p] = K;
                }
            }
        }
    }
    fence_before();
    __syncthreads();
    if (warp == 5) {
        fence_after();
        tmem_dealloc(tmem, kTmemCols);
    }
}

}  // namespace

namespace {

struct DevInfo {
    int nsm, smem_sm, smem_blk;
};

constexpr int kMaxDevices = 64;
std::mutex g_mu;
DevInfo g_info[kMaxDevices];
bool g_have_info[kMaxDevices];
size_t g_smem_set[kMaxDevices][2];  // dynamic shared memory last configured per kernel variant (0 = never)

cudaError_t device_info(int dev, DevInfo& out) {
    std::lock_guard<std::mutex> lock(g_mu);
    if (dev >= 0 && dev < kMaxDevices && g_have_info[dev]) {
        out = g_info[dev];
        return cudaSuccess;
    }
    DevInfo d;
    cudaError_t e = cudaDeviceGetAttribute(&d.nsm, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&d.smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&d.smem_blk, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e != cudaSuccess) return e;
    if (dev >= 0 && dev < kMaxDevices) {
        g_info[dev] = d;
        g_have_info[dev] = true;
    }
    out = d;
    return cudaSuccess;
}

// Sets the kernel's shared-memory attributes when the configuration changes and checks that one CTA fits.
cudaError_t prepare_kernel(int dev, int variant, const void* kern, size_t smem) {
    std::lock_guard<std::mutex> lock(g_mu);
    if (dev >= 0 && dev < kMaxDevices && g_smem_set[dev][variant] == smem) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
    if (e == cudaSuccess) e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    int fits = 0;
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&fits, kern, kThreads, smem);
    if (e != cudaSuccess) return e;
    if (fits < 1) return cudaErrorInvalidConfiguration;
    if (dev >= 0 && dev < kMaxDevices) g_smem_set[dev][variant] = smem;
    return cudaSuccess;
}

}  // namespace

cudaError_t launch_filter_tc(const EstimateArgs& a, unsigned* status, cudaStream_t s) {
    TcGeom g;
    const long long P = static_cast<long long>(a.H) * a.W;
    const int u0 = a.dmin - a.peak;  // >= 0 (checked on the host)
    g.a0 = u0 & ~7;
    g.delta = u0 - g.a0;
    g.kw = ((kN + a.L - 1 + g.delta) + 15) & ~15;
    g.ntiles = (a.D + kN - 1) / kN;
    g.nslab = (g.kw + kSlab - 1) / kSlab;
    g.nbs = g.nslab;
    g.mlead = (g.a0 + kSlab - 1) / kSlab;
    const int x0 = g.a0 - kSlab * g.mlead;
    g.S = max(g.mlead + g.ntiles + g.nslab - 1, (a.T - x0 + kSlab - 1) / kSlab);
    g.npt = static_cast<int>((P + kM - 1) / kM);
    g.lam2s = a.lam2 / kScale;

    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    DevInfo info;
    if ((e = device_info(dev, info)) != cudaSuccess) return e;
    const int nsm = info.nsm, smem_sm = info.smem_sm, smem_blk = info.smem_blk;
    const size_t fixed = 1024 + 2 * static_cast<size_t>(g.nbs) * kBSlabBytes + kOnesBytes;
    const size_t static_bytes = 4096;  // barriers, template tables and the per-CTA reservation, rounded up
    // two CTAs per SM when a ring of at least nslab + 2 slabs still fits, else one CTA with a deeper ring
    long long r2 = (static_cast<long long>(smem_sm) / 2 - static_cast<long long>(static_bytes) -
                    static_cast<long long>(fixed)) / kSlabBytes;
    int ring, per_sm;
    if (r2 >= g.nslab + 2) {
        ring = static_cast<int>(r2 < kMaxRing ? r2 : kMaxRing);
        per_sm = 2;
    } else {
        long long r1 = (static_cast<long long>(smem_blk) - static_cast<long long>(static_bytes) -
                        static_cast<long long>(fixed)) / kSlabBytes;
        ring = static_cast<int>(r1 < kMaxRing ? r1 : kMaxRing);
        per_sm = 1;
    }
    if (ring < g.nslab) return cudaErrorInvalidConfiguration;
    g.ring = ring;
    const size_t smem = fixed + static_cast<size_t>(ring) * kSlabBytes;

    const bool u16 = a.fmt == SPL_HIST_U16;
    CUtensorMap map;
    if ((e = hist_map(&map, a.z, a.pitch, a.T, P, u16)) != cudaSuccess) return e;
    const void* kern = u16 ? reinterpret_cast<const void*>(k_filter_tc<true>)
                           : reinterpret_cast<const void*>(k_filter_tc<false>);
    if ((e = prepare_kernel(dev, u16 ? 1 : 0, kern, smem)) != cudaSuccess) return e;
    const long long want = static_cast<long long>(nsm) * per_sm;
    const int grid = static_cast<int>(g.npt < want ? g.npt : want);
    if (u16) k_filter_tc<true><<<grid, kThreads, smem, s>>>(map, a, g, status);
    else k_filter_tc<false><<<grid, kThreads, smem, s>>>(map, a, g, status);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (u16 && (e = launch_estimate_redo(a, s)) != cudaSuccess) return e;
    if (!a.refl) return cudaSuccess;
    return launch_intensity(a, s);
}

}  // namespace spl
