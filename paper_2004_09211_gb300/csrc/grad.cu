// Differentiable online filter: a soft-argmax depth readout per pixel and frame, a mean-squared-error loss to
// reference depths, and the gradient of that loss with respect to the IRF taps h, the divergence parameter beta
// and the 3x3 mixture weights nu, by a hand-written reverse sweep over the frames.
//
// Forward, frame n, pixel p (one warp per pixel, every candidate evaluated exactly in the log domain):
//   C(d) = sum_j g_j z[d - peak + j], g = h^beta                                            (Eq. beta_div2)
//   ell(d) = lambda C(d) + log sum_k nu_k N(d; m_k, s2_k), lambda = (beta+1)/beta      (Eq. predict, approx_post)
//   w = softmax(ell): mu_n = sum w d, var_n = sum w (d - mu_n)^2                            (Eq. KL_div)
//   readout s_n = sum softmax(ell / tau) d; loss = mean over (n, p) of (s_n - d_ref)^2.
// Stencil entry k of pixel p is N(mu_{n-1}, var_{n-1} + sigma_RW^2) of neighbour p + off_k when it is inside the
// frame, else the weakly informative Gaussian (all pixels present, none faulty in this path).
//
// Backward, frames N..1. With w_tau = softmax(ell / tau) and the adjoints mu_bar, var_bar of this frame's state
// (from the next frame) and s_bar = 2 (s - d_ref) / (N P):
//   ell_bar(d) = mu_bar w (d - mu) + var_bar w ((d - mu)^2 - var) + (s_bar / tau) w_tau (d - s)
//   lambda_bar += sum_d ell_bar C;  g_bar_j += sum_d lambda ell_bar(d) z[d - peak + j]
//   with r_k(d) = N_k(d) / sum_i nu_i N_i(d):
//   nu_bar_k += sum_d ell_bar r_k;  m_bar_k = sum_d ell_bar nu_k r_k (d - m_k) / s2_k;
//   s2_bar_k = sum_d ell_bar nu_k r_k ((d - m_k)^2 - s2_k) / (2 s2_k^2)
// m_bar_k and s2_bar_k of informative entries become the previous frame's state adjoints of neighbour p + off_k;
// a gather kernel sums, for every pixel, the contributions of the pixels whose stencils contain it. Finally
// h_bar_j = g_bar_j beta h_j^(beta-1) and beta_bar = sum_j g_bar_j g_j ln h_j - lambda_bar / beta^2.
//
// Every reduction has a fixed order (per-lane accumulation in a fixed pixel order, warps in index order, CTAs in
// index order), so results are bitwise reproducible run to run. The forward states of every frame are the
// checkpoints the backward sweep recomputes each frame from.
#include <math.h>
#include <string.h>

#include "pixel.cuh"
#include "spl_internal.h"

namespace spl {
namespace {

using namespace px;

constexpr int kPartial = SPL_MAX_TAPS + 1 + 9;  // per-CTA partial sums: g_bar[128], lambda_bar, nu_bar[9]

struct DiffArgs {
    const uint16_t* z;  // frame's rows, [P][pitch] counts
    long long pitch;
    const float* h;
    int H, W, T, L, peak, dmin, D, u0;
    float beta, lam, lam2, sigma_rw2, flat_m, flat_v, tau, inv_np;
    float nu[9];
    const float* mu_prev;  // [P] state n-1
    const float* var_prev;
    float* mu_out;         // [P] state n (forward)
    float* var_out;
    float* dsoft;          // [P] readout (forward)
    const float* d_ref;    // [P] (nullable in forward: no loss)
    float* loss_part;      // [grid] forward loss partials (accumulated across frames)
    const float* abar_mu;  // [P] adjoint of state n (backward)
    const float* abar_var;
    float* E;              // [P][9][2] (backward)
    float* part;           // [grid][kPartial] (backward, accumulated across frames)
};

// Shared-memory slice of one warp: the row as floats (zero from T on: the blocked correlation's windows read up
// to 12 bins past the last candidate's), C, ell.
constexpr int kRowPad = 16;
struct DSlice {
    int zs, cs, ls, ent, words;
};
__host__ __device__ __forceinline__ int dslice_row(int T) { return ((T + 3) & ~3) + kRowPad; }
__host__ __device__ __forceinline__ DSlice make_dslice(int T, int D) {
    DSlice s;
    const int Dp = (D + 3) & ~3;
    s.zs = 0;
    s.cs = s.zs + dslice_row(T);
    s.ls = s.cs + Dp;
    s.ent = s.ls + Dp;
    s.words = s.ent + ((T + 3) & ~3);
    return s;
}

// One pixel's forward quantities, every lane holding the warp-uniform results.
struct PixFwd {
    float M2;      // max of ell (log2 units)
    float S0, S0t; // sums of 2^(ell - M2) and 2^((ell - M2) / tau)
    float mu, var, s;
    int nnz;       // non-empty bins (listed in ent)
};

// Loads the row, lists its non-empty bins, computes C into cs and ell (log2) into ls, and the moments.
__device__ __forceinline__ PixFwd pixel_forward(const DiffArgs& a, int p, const float* gs, float* zs, float* cs,
                                                float* ls, int* ent, const Prior& pr, int lane) {
    const int T = a.T, L = a.L, D = a.D, u0 = a.u0;
    const uint16_t* row = a.z + static_cast<long long>(p) * a.pitch;
    for (int t = lane; t < T; t += 32) zs[t] = static_cast<float>(row[t]);
    __syncwarp();
    // non-empty bins, in order (each lane owns a contiguous segment of bins)
    const int seg = (T + 31) >> 5, b0 = min(lane * seg, T), b1 = min(b0 + seg, T);
    int cnt = 0;
    for (int t = b0; t < b1; ++t) cnt += zs[t] != 0.f;
    int incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += v;
    }
    int o = incl - cnt;
    for (int t = b0; t < b1; ++t)
        if (zs[t] != 0.f) ent[o++] = t;
    const int nnz = __shfl_sync(0xffffffffu, incl, 31);
    __syncwarp();
    // C(d): 8 consecutive candidates per lane from a register window of the row, taps in order in groups of 4
    // (each C is the same tap-ordered fmaf chain as a per-candidate loop); windows start on 4-bin boundaries
    const float4* g4 = reinterpret_cast<const float4*>(gs);
    for (int cb = -(u0 & 3); cb < D; cb += 256) {
        const int cl = cb + 8 * lane;
        if (cl < D && cl + 7 >= 0) {
            const float4* r4 = reinterpret_cast<const float4*>(zs + u0 + cl);
            float acc[8];
#pragma unroll
            for (int r = 0; r < 8; ++r) acc[r] = 0.f;
            float4 c0 = r4[0], c1 = r4[1];
            for (int jg = 0; jg < L; jg += 4) {
                const float4 nx = r4[jg / 4 + 2];
                const float4 g = g4[jg / 4];
                const float wv[12] = {c0.x, c0.y, c0.z, c0.w, c1.x, c1.y, c1.z, c1.w, nx.x, nx.y, nx.z, nx.w};
#pragma unroll
                for (int r = 0; r < 8; ++r) {
                    acc[r] = fmaf(g.x, wv[r], acc[r]);
                    acc[r] = fmaf(g.y, wv[r + 1], acc[r]);
                    acc[r] = fmaf(g.z, wv[r + 2], acc[r]);
                    acc[r] = fmaf(g.w, wv[r + 3], acc[r]);
                }
                c0 = c1;
                c1 = nx;
            }
#pragma unroll
            for (int r = 0; r < 8; ++r)
                if (cl + r >= 0 && cl + r < D) cs[cl + r] = acc[r];
        }
    }
    __syncwarp();
    // ell and its maximum (ties to the smallest candidate)
    float best = -INFINITY;
    int bidx = 0x7fffffff;
    for (int c = lane; c < D; c += 32) {
        const float l = fmaf(a.lam2, cs[c], log2_prior(pr, static_cast<float>(a.dmin + c)));
        ls[c] = l;
        if (l > best) {
            best = l;
            bidx = c;
        }
    }
    warp_argmax(best, bidx);
    if (bidx == 0x7fffffff) bidx = 0;
    __syncwarp();
    const float itau = 1.f / a.tau;
    float s0 = 0.f, s1 = 0.f, s2 = 0.f, t0 = 0.f, t1 = 0.f;
    for (int c = lane; c < D; c += 32) {
        const float e = ls[c] - best;
        const float w = ex2(e), wt = ex2(e * itau);
        const float dd = static_cast<float>(c - bidx);
        s0 += w;
        s1 = fmaf(w, dd, s1);
        s2 = fmaf(w * dd, dd, s2);
        t0 += wt;
        t1 = fmaf(wt, dd, t1);
    }
    s0 = warp_sum(s0);
    s1 = warp_sum(s1);
    s2 = warp_sum(s2);
    t0 = warp_sum(t0);
    t1 = warp_sum(t1);
    PixFwd r;
    r.M2 = best;
    r.S0 = s0;
    r.S0t = t0;
    const float m1 = s1 / s0;
    r.mu = static_cast<float>(a.dmin + bidx) + m1;
    r.var = fmaxf(s2 / s0 - m1 * m1, 0.f);
    r.s = static_cast<float>(a.dmin + bidx) + t1 / t0;
    r.nnz = nnz;
    return r;
}

// Stencil entry of this lane (lanes 0-8): weight, mean, variance, and whether it is a neighbour's state.
__device__ __forceinline__ void stencil_entry(const DiffArgs& a, int p, int lane, float& w, float& m, float& v,
                                              bool& info) {
    w = 0.f;
    m = 0.f;
    v = 1.f;
    info = false;
    if (lane < 9) {
        w = a.nu[lane];
        const int y = p / a.W, x = p - y * a.W;
        const int yy = y + lane / 3 - 1, xx = x + lane % 3 - 1;
        if (yy >= 0 && yy < a.H && xx >= 0 && xx < a.W) {
            const int i = yy * a.W + xx;
            m = a.mu_prev[i];
            v = a.var_prev[i] + a.sigma_rw2;
            info = true;
        } else {
            m = a.flat_m;
            v = a.flat_v + a.sigma_rw2;
        }
    }
}

__device__ __forceinline__ void load_irf(const DiffArgs& a, float* gs) {
    for (int j = threadIdx.x; j < SPL_MAX_TAPS; j += blockDim.x) {
        const float hj = j < a.L ? a.h[j] : 0.f;
        gs[j] = hj > 0.f ? powf(hj, a.beta) : 0.f;
    }
    __syncthreads();
}

__global__ void __launch_bounds__(256) k_diff_forward(const DiffArgs a, DSlice sl) {
    extern __shared__ __align__(16) float dyn[];
    __shared__ __align__(16) float gs[SPL_MAX_TAPS];
    __shared__ float wl[8];
    load_irf(a, gs);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    float* base = dyn + static_cast<size_t>(warp) * sl.words;
    float* zs = base + sl.zs;
    for (int t = a.T + lane; t < dslice_row(a.T); t += 32) zs[t] = 0.f;  // the row loads never write past T
    float* cs = base + sl.cs;
    float* ls = base + sl.ls;
    int* ent = reinterpret_cast<int*>(base + sl.ent);
    const int P = a.H * a.W;
    float lacc = 0.f;
    for (int p = blockIdx.x * nwarps + warp; p < P; p += gridDim.x * nwarps) {
        float w, m, v;
        bool info;
        stencil_entry(a, p, lane, w, m, v, info);
        Prior pr;
        build_prior(w, m, v, lane, pr);
        const PixFwd f = pixel_forward(a, p, gs, zs, cs, ls, ent, pr, lane);
        if (lane == 0) {
            a.mu_out[p] = f.mu;
            a.var_out[p] = f.var;
            if (a.dsoft) a.dsoft[p] = f.s;
            if (a.d_ref) {
                const float e = f.s - a.d_ref[p];
                lacc = fmaf(e, e, lacc);
            }
        }
        __syncwarp();
    }
    if (lane == 0) wl[warp] = lacc;
    __syncthreads();
    if (threadIdx.x == 0 && a.loss_part) {
        float s = 0.f;
        for (int i = 0; i < nwarps; ++i) s += wl[i];
        a.loss_part[blockIdx.x] += s;
    }
}

__global__ void __launch_bounds__(256) k_diff_backward(const DiffArgs a, DSlice sl) {
    extern __shared__ __align__(16) float dyn[];
    __shared__ __align__(16) float gs[SPL_MAX_TAPS];
    __shared__ float red[8][kPartial];
    load_irf(a, gs);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    float* base = dyn + static_cast<size_t>(warp) * sl.words;
    float* zs = base + sl.zs;
    for (int t = a.T + lane; t < dslice_row(a.T); t += 32) zs[t] = 0.f;  // the row loads never write past T
    float* cs = base + sl.cs;
    float* ls = base + sl.ls;
    int* ent = reinterpret_cast<int*>(base + sl.ent);
    const int P = a.H * a.W, D = a.D, L = a.L;
    const float itau = 1.f / a.tau;
    float gbar[SPL_MAX_TAPS / 32] = {0.f, 0.f, 0.f, 0.f};  // tap lane + 32 q
    float lbar = 0.f;
    float nubar[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) nubar[k] = 0.f;

    for (int p = blockIdx.x * nwarps + warp; p < P; p += gridDim.x * nwarps) {
        float w, m, v;
        bool info;
        stencil_entry(a, p, lane, w, m, v, info);
        Prior pr;
        build_prior(w, m, v, lane, pr);
        const PixFwd f = pixel_forward(a, p, gs, zs, cs, ls, ent, pr, lane);
        const float mub = a.abar_mu ? a.abar_mu[p] : 0.f;
        const float varb = a.abar_var ? a.abar_var[p] : 0.f;
        const float sb = 2.f * (f.s - a.d_ref[p]) * a.inv_np;
        // the 9 stencil entries (weight, mean, variance, log2 normaliser) in every lane
        float ew[9], em[9], ev[9], ec[9], ek[9];
#pragma unroll
        for (int k = 0; k < 9; ++k) {
            ew[k] = __shfl_sync(0xffffffffu, w, k);
            em[k] = __shfl_sync(0xffffffffu, m, k);
            ev[k] = __shfl_sync(0xffffffffu, v, k);
            ec[k] = -0.5f * (kLog2TwoPi + lg2(ev[k]));
            ek[k] = kLog2e / (2.f * ev[k]);
        }
        float mbar[9], vbar[9];
#pragma unroll
        for (int k = 0; k < 9; ++k) mbar[k] = vbar[k] = 0.f;
        const float i0 = 1.f / f.S0, i0t = 1.f / f.S0t;
        const float l0 = lg2(f.S0), l0t = lg2(f.S0t);
        for (int c = lane; c < D; c += 32) {
            const float d = static_cast<float>(a.dmin + c);
            const float e = ls[c] - f.M2;
            const float wn = ex2(e) * i0, wt = ex2(e * itau) * i0t;
            const float dm = d - f.mu;
            const float ca = mub * dm + varb * (dm * dm - f.var);  // coefficient of w
            const float cb = sb * itau * (d - f.s);                // coefficient of w_tau
            const float lb = ca * wn + cb * wt;
            const float C = cs[c];
            lbar = fmaf(lb, C, lbar);
            cs[c] = a.lam * lb;  // C_bar, for the tap gradient below
            const float lp2 = ls[c] - a.lam2 * C;  // log2 of the prior mixture at d
#pragma unroll
            for (int k = 0; k < 9; ++k) {
                const float de = d - em[k];
                const float lnk = ec[k] - ek[k] * de * de;  // log2 N_k(d)
                if (ew[k] > 0.f) {
                    // r = N_k / sum_i nu_i N_i <= 1 / nu_k: finite
                    const float t = lb * ex2(lnk - lp2);
                    nubar[k] += t;
                    const float tw = t * ew[k];
                    mbar[k] = fmaf(tw, de / ev[k], mbar[k]);
                    vbar[k] = fmaf(tw, (de * de - ev[k]) / (2.f * ev[k] * ev[k]), vbar[k]);
                } else {
                    // zero weight: N_k / sum_i nu_i N_i is unbounded, its product with the weights is not; keep
                    // the ratio inside one exponent
                    nubar[k] += ca * ex2(e - l0 + lnk - lp2) + cb * ex2(e * itau - l0t + lnk - lp2);
                }
            }
        }
        __syncwarp();
        // tap gradient from the non-empty bins: g_bar_j += z_t C_bar(t - u0 - j)
        for (int i = 0; i < f.nnz; ++i) {
            const int t = ent[i];
            const float zt = zs[t];
#pragma unroll
            for (int q = 0; q < SPL_MAX_TAPS / 32; ++q) {
                const int j = lane + 32 * q;
                const int c = t - a.u0 - j;
                if (j < L && c >= 0 && c < D) gbar[q] = fmaf(zt, cs[c], gbar[q]);
            }
        }
        // this pixel's neighbour-state adjoints, entry k -> E[p][k]
#pragma unroll
        for (int k = 0; k < 9; ++k) {
            mbar[k] = warp_sum(mbar[k]);
            vbar[k] = warp_sum(vbar[k]);
        }
        const bool info_k = info;
        if (lane < 9) {
            float om = 0.f, ov = 0.f;
#pragma unroll
            for (int k = 0; k < 9; ++k)
                if (k == lane) {
                    om = mbar[k];
                    ov = vbar[k];
                }
            a.E[(static_cast<long long>(p) * 9 + lane) * 2] = info_k ? om : 0.f;
            a.E[(static_cast<long long>(p) * 9 + lane) * 2 + 1] = info_k ? ov : 0.f;
        }
        __syncwarp();
    }
    // block partials in a fixed order: lanes, then warps
    lbar = warp_sum(lbar);
#pragma unroll
    for (int k = 0; k < 9; ++k) nubar[k] = warp_sum(nubar[k]);
#pragma unroll
    for (int q = 0; q < SPL_MAX_TAPS / 32; ++q) red[warp][lane + 32 * q] = gbar[q];
    if (lane == 0) {
        red[warp][SPL_MAX_TAPS] = lbar;
#pragma unroll
        for (int k = 0; k < 9; ++k) red[warp][SPL_MAX_TAPS + 1 + k] = nubar[k];
    }
    __syncthreads();
    for (int i = threadIdx.x; i < kPartial; i += blockDim.x) {
        float s = 0.f;
        for (int wv = 0; wv < nwarps; ++wv) s += red[wv][i];
        a.part[static_cast<long long>(blockIdx.x) * kPartial + i] += s;
    }
}

// State adjoints of the previous frame: pixel q gathers entry k of pixel q - off_k (fixed order k = 0..8).
__global__ void k_diff_gather(int H, int W, const float* __restrict__ E, float* abar_mu, float* abar_var) {
    const int P = H * W;
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < P; q += gridDim.x * blockDim.x) {
        const int y = q / W, x = q - y * W;
        float sm = 0.f, sv = 0.f;
        for (int k = 0; k < 9; ++k) {
            const int py = y - (k / 3 - 1), px = x - (k % 3 - 1);
            if (py < 0 || py >= H || px < 0 || px >= W) continue;
            const long long i = (static_cast<long long>(py) * W + px) * 9 + k;
            sm += E[2 * i];
            sv += E[2 * i + 1];
        }
        abar_mu[q] = sm;
        abar_var[q] = sv;
    }
}

__global__ void k_diff_loss(const float* part, int n, float scale, float* loss) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        float s = 0.f;
        for (int i = 0; i < n; ++i) s += part[i];
        *loss = s * scale;
    }
}

// Sums the CTA partials (fixed order) and applies the chain rule through g = h^beta and lambda = (beta+1)/beta.
__global__ void k_diff_finalize(const float* part, int n, const float* h, int L, float beta, float* grad_h,
                                float* grad_beta, float* grad_nu) {
    __shared__ float tot[kPartial];
    for (int i = threadIdx.x; i < kPartial; i += blockDim.x) {
        float s = 0.f;
        for (int c = 0; c < n; ++c) s += part[static_cast<long long>(c) * kPartial + i];
        tot[i] = s;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        float gb = 0.f;
        for (int j = 0; j < L; ++j) {
            const float hj = h[j];
            if (hj > 0.f) {
                const float g = powf(hj, beta);
                grad_h[j] = tot[j] * beta * g / hj;
                gb = fmaf(tot[j] * g, logf(hj), gb);
            } else {
                grad_h[j] = 0.f;
            }
        }
        *grad_beta = gb - tot[SPL_MAX_TAPS] / (beta * beta);
        for (int k = 0; k < 9; ++k) grad_nu[k] = tot[SPL_MAX_TAPS + 1 + k];
    }
}

// Scratch layout (in floats): abar_mu[2][P], abar_var[2][P], E[P][9][2], part[G][kPartial], loss[G].
struct Scratch {
    size_t abar, E, part, loss, total;
};
Scratch scratch_layout(long long P, int G) {
    Scratch s;
    s.abar = 0;
    s.E = s.abar + 4 * static_cast<size_t>(P);
    s.part = s.E + 18 * static_cast<size_t>(P);
    s.loss = s.part + static_cast<size_t>(G) * kPartial;
    s.total = s.loss + G;
    return s;
}

int grid_size() {
    int dev = 0, nsm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
    return 2 * nsm;
}

spl_status check_diff(const spl_params* prm, int nframes, const spl_hist* z, const float* h, float tau,
                      void* scratch, size_t bytes, int G, Scratch* sl) {
    spl_status st = check_params(prm, true);
    if (st != SPL_OK) return st;
    if (!z || !z->data || z->fmt != SPL_HIST_U16 || z->pitch < prm->T || (z->pitch % 8) != 0) {
        set_error("the differentiable filter takes uint16 histograms with pitch >= T, a multiple of 8");
        return SPL_EINVAL;
    }
    if (nframes < 1 || !h || !(tau > 0.f) || !isfinite(tau)) {
        set_error("need nframes >= 1, h and tau > 0");
        return SPL_EINVAL;
    }
    if (G <= 0) {
        set_error("no CUDA device");
        return SPL_ECUDA;
    }
    *sl = scratch_layout(static_cast<long long>(prm->H) * prm->W, G);
    if (!scratch || bytes < sl->total * sizeof(float)) {
        set_error("scratch must hold %zu bytes (spl_diff_scratch_size)", sl->total * sizeof(float));
        return SPL_EINVAL;
    }
    return SPL_OK;
}

DiffArgs make_args(const spl_params* q, const spl_hist* z, const float* h, float tau, int nframes) {
    DiffArgs a;
    memset(&a, 0, sizeof(a));
    a.z = static_cast<const uint16_t*>(z->data);
    a.pitch = z->pitch;
    a.h = h;
    a.H = q->H;
    a.W = q->W;
    a.T = q->T;
    a.L = q->L;
    a.peak = q->peak;
    a.dmin = q->dmin;
    a.D = q->dmax - q->dmin + 1;
    a.u0 = q->dmin - q->peak;
    a.beta = q->beta;
    a.lam = static_cast<float>((static_cast<double>(q->beta) + 1.0) / q->beta);
    a.lam2 = static_cast<float>((static_cast<double>(q->beta) + 1.0) / q->beta * 1.4426950408889634);
    a.sigma_rw2 = q->sigma_rw2;
    a.flat_m = 0.5f * static_cast<float>(q->dmin + q->dmax);
    const double span = static_cast<double>(q->dmax - q->dmin);
    a.flat_v = static_cast<float>(span * span / 12.0);
    a.tau = tau;
    a.inv_np = static_cast<float>(1.0 / (static_cast<double>(nframes) * q->H * q->W));
    for (int k = 0; k < 9; ++k) a.nu[k] = q->nu[k];
    return a;
}

// Warps per CTA (up to 8) whose slices fit in 200 KB of shared memory.
// Warps per CTA: the grid is two CTAs per SM, so size a CTA to let both be resident (half of about 200 KB of
// shared memory each) when one warp's slice allows it; otherwise one CTA per SM.
int warps_for(const DSlice& ds) {
    const size_t per = sizeof(float) * ds.words;
    const int two = static_cast<int>((100u * 1024u) / per);
    const int w = two >= 1 ? two : static_cast<int>((200u * 1024u) / per);
    return w > 8 ? 8 : w;
}

cudaError_t setup_kernel_smem(const void* kern, size_t smem) {
    return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
}

}  // namespace
}  // namespace spl

using namespace spl;

extern "C" {

spl_status spl_diff_scratch_size(const spl_params* prm, size_t* bytes) {
    set_error("%s", "");
    if (!prm || !bytes) {
        set_error("prm and bytes are required");
        return SPL_EINVAL;
    }
    const int G = grid_size();
    if (G <= 0) {
        set_error("no CUDA device");
        return SPL_ECUDA;
    }
    *bytes = scratch_layout(static_cast<long long>(prm->H) * prm->W, G).total * sizeof(float);
    return SPL_OK;
}

spl_status spl_diff_forward(const spl_params* prm, int nframes, const spl_hist* z, const float* h, float tau,
                            const float* d_ref, float* mu_states, float* var_states, float* dsoft, float* loss,
                            void* scratch, size_t scratch_bytes, void* stream) {
    set_error("%s", "");
    const int G = grid_size();
    Scratch sl;
    spl_status st = check_diff(prm, nframes, z, h, tau, scratch, scratch_bytes, G, &sl);
    if (st != SPL_OK) return st;
    if (!mu_states || !var_states || (loss && !d_ref)) {
        set_error("mu_states and var_states are required; loss needs d_ref");
        return SPL_EINVAL;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    float* base = static_cast<float*>(scratch);
    const long long P = static_cast<long long>(prm->H) * prm->W;
    DiffArgs a = make_args(prm, z, h, tau, nframes);
    const DSlice ds = make_dslice(prm->T, a.D);
    const int nw = warps_for(ds);
    if (nw < 1) {
        set_error("T = %d, D = %d need more shared memory per warp than a CTA has", prm->T, a.D);
        return SPL_EUNSUPPORTED;
    }
    const size_t smem = sizeof(float) * ds.words * nw;
    cudaError_t e = setup_kernel_smem(reinterpret_cast<const void*>(k_diff_forward), smem);
    if (e == cudaSuccess) e = cudaMemsetAsync(base + sl.loss, 0, sizeof(float) * G, s);
    for (int n = 0; n < nframes && e == cudaSuccess; ++n) {
        a.z = static_cast<const uint16_t*>(z->data) + n * P * z->pitch;
        a.mu_prev = mu_states + n * P;
        a.var_prev = var_states + n * P;
        a.mu_out = mu_states + (n + 1) * P;
        a.var_out = var_states + (n + 1) * P;
        a.dsoft = dsoft ? dsoft + n * P : nullptr;
        a.d_ref = d_ref ? d_ref + n * P : nullptr;
        a.loss_part = base + sl.loss;
        k_diff_forward<<<G, 32 * nw, smem, s>>>(a, ds);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess && loss) {
        k_diff_loss<<<1, 32, 0, s>>>(base + sl.loss, G, a.inv_np, loss);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) {
        set_error("spl_diff_forward: %s", cudaGetErrorString(e));
        return SPL_ECUDA;
    }
    return SPL_OK;
}

spl_status spl_diff_backward(const spl_params* prm, int nframes, const spl_hist* z, const float* h, float tau,
                             const float* d_ref, const float* mu_states, const float* var_states, float* grad_h,
                             float* grad_beta, float* grad_nu, void* scratch, size_t scratch_bytes, void* stream) {
    set_error("%s", "");
    const int G = grid_size();
    Scratch sl;
    spl_status st = check_diff(prm, nframes, z, h, tau, scratch, scratch_bytes, G, &sl);
    if (st != SPL_OK) return st;
    if (!d_ref || !mu_states || !var_states || !grad_h || !grad_beta || !grad_nu) {
        set_error("d_ref, mu_states, var_states, grad_h, grad_beta and grad_nu are required");
        return SPL_EINVAL;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    float* base = static_cast<float*>(scratch);
    const long long P = static_cast<long long>(prm->H) * prm->W;
    DiffArgs a = make_args(prm, z, h, tau, nframes);
    const DSlice ds = make_dslice(prm->T, a.D);
    const int nw = warps_for(ds);
    if (nw < 1) {
        set_error("T = %d, D = %d need more shared memory per warp than a CTA has", prm->T, a.D);
        return SPL_EUNSUPPORTED;
    }
    const size_t smem = sizeof(float) * ds.words * nw;
    float* abar = base + sl.abar;  // [2][2][P]: (mu, var) x ping-pong
    cudaError_t e = setup_kernel_smem(reinterpret_cast<const void*>(k_diff_backward), smem);
    if (e == cudaSuccess) e = cudaMemsetAsync(base + sl.part, 0, sizeof(float) * G * kPartial, s);
    for (int n = nframes - 1; n >= 0 && e == cudaSuccess; --n) {
        const int cur = n & 1;  // adjoint buffers of state n+1 (this frame's output)
        a.z = static_cast<const uint16_t*>(z->data) + n * P * z->pitch;
        a.mu_prev = mu_states + n * P;
        a.var_prev = var_states + n * P;
        a.d_ref = d_ref + n * P;
        a.abar_mu = n == nframes - 1 ? nullptr : abar + (2 * cur) * P;
        a.abar_var = n == nframes - 1 ? nullptr : abar + (2 * cur + 1) * P;
        a.E = base + sl.E;
        a.part = base + sl.part;
        k_diff_backward<<<G, 32 * nw, smem, s>>>(a, ds);
        e = cudaGetLastError();
        if (e == cudaSuccess && n > 0) {
            const int nxt = cur ^ 1;
            const int blocks = static_cast<int>((P + 255) / 256);
            k_diff_gather<<<blocks, 256, 0, s>>>(prm->H, prm->W, base + sl.E, abar + (2 * nxt) * P,
                                                 abar + (2 * nxt + 1) * P);
            e = cudaGetLastError();
        }
    }
    if (e == cudaSuccess) {
        k_diff_finalize<<<1, 256, 0, s>>>(base + sl.part, G, h, prm->L, prm->beta, grad_h, grad_beta, grad_nu);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) {
        set_error("spl_diff_backward: %s", cudaGetErrorString(e));
        return SPL_ECUDA;
    }
    return SPL_OK;
}

}  // extern "C"
