// Pseudo-posterior moments on the integer depth grid, shared by the histogram kernels (estimate.cu), the photon-list
// kernels (batch.cu, noalloc.cu; their data term is in photons.cuh) and the multispectral kernel (msl.cu):
//
//   block_bounds    per-block upper bounds of the log pseudo-posterior (the data part supplied by the caller).
//   posterior_eval  Eq. approx_post + Eq. KL_div: argmax, mean and variance of the pseudo-posterior on the
//                   integer grid, from C(d) already in shared memory, with bound-based block pruning and the
//                   linear-domain evaluation described below.
//
// Pruning. Candidates are grouped in blocks of 32. Each block gets an upper bound of ell = lambda log2(e) C(d)
// + log2 f(d): an upper bound of the data part (lambda log2(e) max(g) times the photons in the block's window, or
// the largest C of a densely correlated row), plus the prior's largest value on the block. The block with the largest bound is evaluated exactly; its best value LB is a lower bound of
// the maximum, and every block whose bound is below LB - 64 is dropped: its weights are below 2^-64 of the
// maximum, so the moments move by less than 8192^3 * 2^-64 < 3e-8 bins^2. The argmax always lies in a kept
// block.
//
// Linear-domain evaluation. Over the range of kept blocks the weights 2^(ell - ref) are formed directly: each
// lane walks a contiguous run of candidates; the data factor costs one exp2 per candidate and each mixture
// component is advanced by the exact two-multiply recurrence of a Gaussian on a unit grid (value ratio, then
// ratio of ratios), restarted from exact exponentials every 16 candidates. All values are scaled by upper
// bounds so nothing overflows; a value that underflows is below 2^-126 while the largest weight must be at
// least 2^-60 (checked), so the lost mass is below 2^-62 per candidate. Components narrower than 1.5 bins^2
// (where 16 steps could underflow a component near its own peak), a scattered set of kept blocks, or a failed
// check send the pixel through the exact log-domain path instead. The moments are accumulated in the same
// pass about the best candidate of the leading block, and again about the rounded mean when that centre lies
// more than two standard deviations away (so S2/S0 and the squared offset of the mean never cancel badly).
#pragma once

#include "pixel.cuh"

namespace spl {
namespace px {

constexpr int kRestart = 16;  // exact restart interval of the mixture recurrences

struct Grid {
    int D, NB, dmin, u0, L;  // candidates, blocks of 32, first depth, first bin of candidate 0, taps
    float lam2, gmax;        // lambda log2(e), max_j g_j
};

// One lane's run of candidates r0 .. r1 - 1 in the linear domain (see above), with the mixture loops sized to
// NC >= pr.n component slots; slots past pr.n start at 0 and stay 0. Writes the weights into cs and accumulates
// the lane's best weight and moments about cstar.
template <int NC>
__device__ __forceinline__ void lin_run(const Grid& g, const Prior& pr, float* cs, int r0, int r1, float sref,
                                        float xref, int cstar, float& best, int& bidx, float& s0, float& s1,
                                        float& s2) {
    float v[NC > 0 ? NC : 1], q[NC > 0 ? NC : 1], kk[NC > 0 ? NC : 1];
#pragma unroll
    for (int i = 0; i < NC; ++i) {
        v[i] = q[i] = 0.f;
        kk[i] = i < pr.n ? ex2(-2.f * pr.ck[i]) : 0.f;
    }
    float dd = static_cast<float>(r0 - cstar);  // offset of candidate c from cstar (integers below 2^24: exact)
    for (int c0 = r0; c0 < r1; c0 += kRestart) {
        const float d = static_cast<float>(g.dmin + c0);  // exact restart of every component
#pragma unroll
        for (int i = 0; i < NC; ++i) {
            const float e = d - pr.cm[i];
            v[i] = i < pr.n ? ex2(pr.ca[i] - pr.ck[i] * e * e - sref) : 0.f;
            q[i] = i < pr.n ? ex2(fminf(-pr.ck[i] * (2.f * e + 1.f), 100.f)) : 0.f;
        }
        const int c1 = min(c0 + kRestart, r1);
        for (int c = c0; c < c1; ++c) {
            float m = NC == 0 ? 1.f : 0.f;
#pragma unroll
            for (int i = 0; i < NC; ++i) {
                m += v[i];
                v[i] *= q[i];
                q[i] *= kk[i];
            }
            const float w = ex2(fmaf(g.lam2, cs[c], -xref)) * m;
            cs[c] = w;
            if (w > best) {
                best = w;
                bidx = c;
            }
            s0 += w;
            s1 = fmaf(w, dd, s1);
            s2 = fmaf(w * dd, dd, s2);
            dd += 1.f;
        }
    }
}

// Per-block upper bounds of ell = lambda log2(e) C(d) + log2 f(d) into ubs[0 .. NB): dub(b) is an upper bound of
// lambda log2(e) C over block b (evaluated per lane), the prior's part is log2_prior_bound. Returns the block with
// the largest bound (warp-uniform; 0 if every bound is NaN).
template <class DataBound>
__device__ __forceinline__ int block_bounds(const Grid& g, const Prior& pr, float* ubs, DataBound dub, int lane) {
    const int D = g.D, NB = g.NB;
    float ubest = -INFINITY;
    int ub_b = 0x7fffffff;
    for (int b = lane; b < NB; b += 32) {
        const int last = min(32 * b + 31, D - 1);
        const float ub = dub(b) +
                         log2_prior_bound(pr, static_cast<float>(g.dmin + 32 * b), static_cast<float>(g.dmin + last));
        ubs[b] = ub;
        if (ub > ubest) {
            ubest = ub;
            ub_b = b;
        }
    }
    warp_argmax(ubest, ub_b);
    if (ub_b >= NB) ub_b = 0;  // every bound was NaN (invalid inputs): keep the block index in range
    __syncwarp();
    return ub_b;
}

// The pseudo-posterior from the block bounds: cs holds C on every candidate (cmax its largest value). The best
// value of block ub_b is a lower bound LB of the maximum; blocks whose bound is below LB - 64 are dropped.
// restore() writes C back on the kept range (needed only on the rare fallback from the linear path, whose weights
// overwrite cs). Outputs: index of the smallest maximiser, mean depth and variance.
template <class Restore>
__device__ __forceinline__ void posterior_eval(const Grid& g, const Prior& pr, float cmax, float* cs, const float* ubs,
                                               int ub_b, Restore restore, int lane, int& bidx_out,
                                               float& mu_out, float& var_out) {
    const int D = g.D, NB = g.NB;
    const float lam2 = g.lam2;

    // exact best value of the block with the largest bound: a lower bound of the maximum, and its position
    float lb;
    int cstar;
    {
        const int c = 32 * ub_b + lane;
        float l = -INFINITY;
        if (c < D) l = fmaf(lam2, cs[c], log2_prior(pr, static_cast<float>(g.dmin + c)));
        cstar = c < D ? c : 0x7fffffff;
        warp_argmax(l, cstar);
        lb = l;
        if (cstar >= D) cstar = min(32 * ub_b, D - 1);
    }
    const float thr = lb - kPrune2;
    int nsurv = 0, bfirst = NB, blast = -1;
    for (int w0 = 0; w0 < NB; w0 += 32) {
        const unsigned m = __ballot_sync(0xffffffffu, (w0 + lane < NB && ubs[w0 + lane] >= thr) || w0 + lane == ub_b);
        if (m) {
            nsurv += __popc(m);
            bfirst = min(bfirst, w0 + __ffs(m) - 1);
            blast = w0 + 31 - __clz(m);
        }
    }


    // ---- linear-domain weights over the range of kept blocks ----
    if ((blast - bfirst + 1) <= max(8, 2 * nsurv) && !(pr.minv < 1.5f)) {
        float sref = pr.n > 0 ? -INFINITY : 0.f;
#pragma unroll
        for (int i = 0; i < kMaxComp; ++i)
            if (i < pr.n) sref = fmaxf(sref, pr.ca[i]);
        const float xref = lam2 * cmax;  // lambda log2(e) max_d C(d)
        const int c_lo = 32 * bfirst, c_hi = min(32 * blast + 31, D - 1);
        const int run = (c_hi - c_lo + 32) >> 5;
        const int r0 = c_lo + lane * run, r1 = min(r0 + run, c_hi + 1);
        float best = -INFINITY;
        int bidx = 0x7fffffff;
        float s0 = 0.f, s1 = 0.f, s2 = 0.f;
        switch (pr.n) {  // warp-uniform: loops sized to the component count
            case 0: lin_run<0>(g, pr, cs, r0, r1, sref, xref, cstar, best, bidx, s0, s1, s2); break;
            case 1: lin_run<1>(g, pr, cs, r0, r1, sref, xref, cstar, best, bidx, s0, s1, s2); break;
            case 2: lin_run<2>(g, pr, cs, r0, r1, sref, xref, cstar, best, bidx, s0, s1, s2); break;
            case 3: lin_run<3>(g, pr, cs, r0, r1, sref, xref, cstar, best, bidx, s0, s1, s2); break;
            case 4:
            case 5: lin_run<5>(g, pr, cs, r0, r1, sref, xref, cstar, best, bidx, s0, s1, s2); break;
            default: lin_run<kMaxComp>(g, pr, cs, r0, r1, sref, xref, cstar, best, bidx, s0, s1, s2); break;
        }
        warp_argmax(best, bidx);
        __syncwarp();
        if (best >= 0x1p-60f) {
            s0 = warp_sum(s0);
            s1 = warp_sum(s1);
            s2 = warp_sum(s2);
            float ctr = static_cast<float>(cstar);
            float m1 = s1 / s0;
            float var = s2 / s0 - m1 * m1;
            if (m1 * m1 > 4.f * var + 1.f) {  // centre far from the mean: again about the rounded mean
                const int cc = __float2int_rn(ctr + m1);
                s0 = s1 = s2 = 0.f;
                for (int c = r0; c < r1; ++c) {
                    const float w = cs[c];
                    const float dd = static_cast<float>(c - cc);
                    s0 += w;
                    s1 = fmaf(w, dd, s1);
                    s2 = fmaf(w * dd, dd, s2);
                }
                s0 = warp_sum(s0);
                s1 = warp_sum(s1);
                s2 = warp_sum(s2);
                ctr = static_cast<float>(cc);
                m1 = s1 / s0;
                var = s2 / s0 - m1 * m1;
            }
            bidx_out = bidx;
            mu_out = static_cast<float>(g.dmin) + ctr + m1;
            var_out = fmaxf(var, 0.f);
            return;
        }
        restore();  // the weights overwrote C on the kept range
    }

    // ---- exact log-domain ell on the kept blocks ----
    float best = -INFINITY;
    int bidx = 0x7fffffff;
    for (int w0 = 0; w0 < NB; w0 += 32) {
        unsigned m = __ballot_sync(0xffffffffu, (w0 + lane < NB && ubs[w0 + lane] >= thr) || w0 + lane == ub_b);
        while (m) {
            const int b = w0 + __ffs(m) - 1;
            m &= m - 1;
            const int c = 32 * b + lane;
            float l = -INFINITY;
            if (c < D) l = fmaf(lam2, cs[c], log2_prior(pr, static_cast<float>(g.dmin + c)));
            cs[c] = l;
            if (l > best || (l == best && c < bidx)) {
                best = l;
                bidx = c;
            }
        }
    }
    warp_argmax(best, bidx);
    if (bidx == 0x7fffffff) bidx = 0;  // every ell was NaN (invalid inputs): keep indices in range
    __syncwarp();
    float s0 = 0.f, s1 = 0.f, s2 = 0.f;
    for (int w0 = 0; w0 < NB; w0 += 32) {
        unsigned m = __ballot_sync(0xffffffffu, (w0 + lane < NB && ubs[w0 + lane] >= thr) || w0 + lane == ub_b);
        while (m) {
            const int b = w0 + __ffs(m) - 1;
            m &= m - 1;
            const int c = 32 * b + lane;
            const float w = ex2(cs[c] - best);  // 0 for lanes past D (ell = -inf)
            const float dd = static_cast<float>(c - bidx);
            s0 += w;
            s1 = fmaf(w, dd, s1);
            s2 = fmaf(w * dd, dd, s2);
        }
    }
    s0 = warp_sum(s0);
    s1 = warp_sum(s1);
    s2 = warp_sum(s2);
    const float m1 = s1 / s0;
    bidx_out = bidx;
    mu_out = static_cast<float>(g.dmin + bidx) + m1;
    var_out = fmaxf(s2 / s0 - m1 * m1, 0.f);
}

}  // namespace px
}  // namespace spl
