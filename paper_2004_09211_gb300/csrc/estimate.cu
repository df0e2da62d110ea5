// Fused per-pixel kernel: robust data term (Eq. beta_div2), pseudo-posterior on the depth grid
// (Eq. approx_post) with the spatio-temporal Gaussian-mixture prior (Eq. predict), moment matching
// (Eq. KL_div), and the background/reflectivity estimate (Sec. II-E).
//
// Mapping. One warp owns one pixel at a time (persistent grid-stride loop over pixels). The warp streams the
// pixel's histogram row from HBM once, with 16-byte loads, into its shared-memory slice, and keeps per-chunk
// photon counts (a chunk is the 8 bins of one 16-byte load, 4 for float counts) as a prefix sum.
//
// Correlation. C(d) = sum_j g_j z[d - peak + j] with g = h^beta. A pixel with few non-empty bins (the usual
// case for photon-starved data) is correlated from a compacted list of its non-empty bins (exact zero skip);
// a dense pixel uses the direct sum over taps. Both give the exact sum of the same products in FP32.
//
// Pruned epilogue. The candidates are processed in blocks of 32 (one per lane). For each block the kernel
// first bounds its log2 pseudo-posterior from above: lambda*log2(e)*max(g)*(photons in the block's window)
// plus the largest value the log2 prior can take on the block's depth interval. The block with the largest
// bound is evaluated exactly; its maximum is a lower bound LB of the global maximum. Every block whose upper
// bound is below LB - 64 (log2 units) holds only weights below 2^-64 relative to the maximum and is skipped;
// with at most 8192 candidates at distance at most 8192 bins, the skipped mass changes the moments by less
// than 8192^3 * 2^-64 < 3e-8 (bins^2). The argmax always lies in an evaluated block. All other blocks are
// evaluated exactly, so argmax, mean and variance are those of the full grid to FP32 accuracy.
#include <cuda_fp16.h>
#include <math.h>

#include "spl_internal.h"

namespace spl {
namespace {

constexpr float kLog2e = 1.4426950408889634f;
constexpr float kLog2TwoPi = 2.6514961294723187f;  // log2(2 pi)
constexpr int kMaxComp = 10;                        // 9 stencil entries + 1 merged weakly informative one
constexpr int kNnzSparse = 256;                     // zero-skip correlation up to this many non-empty bins
constexpr float kPrune2 = 64.f;                     // log2 margin below the best value for skipping a block

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

// Shared-memory slice of one warp (all offsets in 4-byte words; every array starts 16-byte aligned).
struct Slice {
    int nch;     // chunks per row
    int zs;      // dense counts as float, nch * CB words
    int ent;     // non-empty bins (bin, count) as uint2, kNnzSparse entries
    int cps;     // photon-count prefix over chunks, nch + 1 words
    int cpe;     // entry-index prefix over chunks, nch + 1 words
    int ubs;     // per-block upper bounds, NB words
    int cs;      // log2 pseudo-posterior (or C) per candidate, NB * 32 words
    int words;   // total
};

__host__ __device__ __forceinline__ int round4(int x) { return (x + 3) & ~3; }

__host__ __device__ __forceinline__ Slice make_slice(int T, int D, int cb) {
    Slice s;
    s.nch = (T + cb - 1) / cb;
    const int nb = (D + 31) / 32;
    s.zs = 0;
    s.ent = round4(s.nch * cb);
    s.cps = s.ent + 2 * kNnzSparse;
    s.cpe = s.cps + round4(s.nch + 1);
    s.ubs = s.cpe + round4(s.nch + 1);
    s.cs = s.ubs + round4(nb);
    s.words = s.cs + nb * 32;
    return s;
}

// Loads chunk i (16 bytes) of pixel p's row and converts it to floats; bins >= T read as 0.
template <int FMT>
__device__ __forceinline__ void load_chunk(const EstimateArgs& a, long long p, int i, float* f) {
    if (FMT == SPL_HIST_F32) {
        const float4 v = __ldcs(reinterpret_cast<const float4*>(static_cast<const float*>(a.z) + p * a.pitch) + i);
        f[0] = v.x;
        f[1] = v.y;
        f[2] = v.z;
        f[3] = v.w;
#pragma unroll
        for (int k = 0; k < 4; ++k)
            if (i * 4 + k >= a.T) f[k] = 0.f;
    } else {
        const uint4 v = __ldcs(reinterpret_cast<const uint4*>(static_cast<const uint16_t*>(a.z) + p * a.pitch) + i);
        const unsigned w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            if (FMT == SPL_HIST_U16) {
                // exact integer -> float through the 2^23 exponent trick (two full-rate ops per count)
                f[2 * k] = __int_as_float(0x4B000000 | (w[k] & 0xffffu)) - 8388608.f;
                f[2 * k + 1] = __int_as_float(0x4B000000 | (w[k] >> 16)) - 8388608.f;
            } else {
                f[2 * k] = __half2float(__ushort_as_half(static_cast<unsigned short>(w[k] & 0xffffu)));
                f[2 * k + 1] = __half2float(__ushort_as_half(static_cast<unsigned short>(w[k] >> 16)));
            }
        }
#pragma unroll
        for (int k = 0; k < 8; ++k)
            if (i * 8 + k >= a.T) f[k] = 0.f;
    }
}

// In-place exclusive prefix sum of n values (float array x and int array y) of a warp's slice, with the
// total written at index n.
__device__ __forceinline__ void warp_scan2(float* x, int* y, int n, int lane) {
    const int seg = (n + 31) >> 5;
    const int b = lane * seg, e = min(b + seg, n);
    float sx = 0.f;
    int sy = 0;
    for (int i = b; i < e; ++i) {
        sx += x[i];
        sy += y[i];
    }
    float ix = sx;
    int iy = sy;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const float tx = __shfl_up_sync(0xffffffffu, ix, o);
        const int ty = __shfl_up_sync(0xffffffffu, iy, o);
        if (lane >= o) {
            ix += tx;
            iy += ty;
        }
    }
    float rx = ix - sx;  // exclusive offsets of this lane's segment
    int ry = iy - sy;
    for (int i = b; i < e; ++i) {
        const float vx = x[i];
        const int vy = y[i];
        x[i] = rx;
        y[i] = ry;
        rx += vx;
        ry += vy;
    }
    if (lane == 31) {
        x[n] = ix;
        y[n] = iy;
    }
    __syncwarp();
}

// Mixture prior in log2 units: component c contributes 2^(ca[c] - ck[c] (d - cm[c])^2).
struct Prior {
    float ca[kMaxComp], ck[kMaxComp], cm[kMaxComp], cv[kMaxComp], cw[kMaxComp];
    int n;
};

// Adds weight w to the component N(m, v), merging it with an identical one already present.
__device__ __forceinline__ void prior_add(Prior& pr, float w, float m, float v) {
    bool merged = false;
#pragma unroll
    for (int i = 0; i < kMaxComp; ++i)
        if (i < pr.n && !merged && pr.cm[i] == m && pr.cv[i] == v) {
            pr.cw[i] += w;
            merged = true;
        }
    if (merged) return;
#pragma unroll
    for (int i = 0; i < kMaxComp; ++i)
        if (i == pr.n) {
            pr.cm[i] = m;
            pr.cv[i] = v;
            pr.cw[i] = w;
        }
    ++pr.n;
}

__device__ __forceinline__ void prior_finish(Prior& pr) {
#pragma unroll
    for (int i = 0; i < kMaxComp; ++i)
        if (i < pr.n) {
            pr.ca[i] = lg2(pr.cw[i]) - 0.5f * (kLog2TwoPi + lg2(pr.cv[i]));
            pr.ck[i] = kLog2e / (2.f * pr.cv[i]);
        }
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
                flat_w += w;  // every weakly informative entry is the same Gaussian
        }
        if (flat_w > 0.f) prior_add(pr, flat_w, a.flat_m, a.flat_v + a.sigma_rw2);
    }
    prior_finish(pr);
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

// C(d) for the candidate c = 32 b + lane of block b (clamped to the last candidate for lanes past D).
__device__ __forceinline__ float block_cost(const float* __restrict__ gs, const float* zs, const uint2* ent,
                                            const int* cpe, bool sparse, int b, int lane, int D, int L, int u0,
                                            int cb) {
    const int c = min(32 * b + lane, D - 1);
    const int t0 = u0 + c;  // first bin of this candidate's template
    if (sparse) {
        const int s_bin = u0 + 32 * b;
        const int e_bin = u0 + min(32 * b + 31, D - 1) + L - 1;
        const int e0 = cpe[s_bin / cb], e1 = cpe[e_bin / cb + 1];
        float acc = 0.f;
        for (int e = e0; e < e1; ++e) {
            const uint2 en = ent[e];
            const unsigned j = en.x - static_cast<unsigned>(t0);
            if (j < static_cast<unsigned>(L)) acc = fmaf(__uint_as_float(en.y), gs[j], acc);
        }
        return acc;
    }
    const float* zz = zs + t0;
    float acc0 = 0.f, acc1 = 0.f;
    int j = 0;
    for (; j + 4 <= L; j += 4) {
        const float4 g4 = *reinterpret_cast<const float4*>(gs + j);
        acc0 = fmaf(g4.x, zz[j], acc0);
        acc1 = fmaf(g4.y, zz[j + 1], acc1);
        acc0 = fmaf(g4.z, zz[j + 2], acc0);
        acc1 = fmaf(g4.w, zz[j + 3], acc1);
    }
    for (; j < L; ++j) acc0 = fmaf(gs[j], zz[j], acc0);
    return acc0 + acc1;
}

template <int FMT, bool COST_ONLY>
__global__ void __launch_bounds__(256) k_estimate(const EstimateArgs a) {
    extern __shared__ __align__(16) float dyn[];
    __shared__ __align__(16) float gs[SPL_MAX_TAPS];  // g_j = h_j^beta (0 for taps <= 0)
    __shared__ float as[SPL_MAX_TAPS];                 // h_j / sum(h): normalised template (intensity model)
    __shared__ float s_hsum, s_gmax;
    constexpr int CB = FMT == SPL_HIST_F32 ? 4 : 8;

    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    for (int j = threadIdx.x; j < SPL_MAX_TAPS; j += blockDim.x) {
        const float hj = j < a.L ? a.h[j] : 0.f;
        gs[j] = hj > 0.f ? powf(hj, a.beta) : 0.f;
        as[j] = hj > 0.f ? hj : 0.f;
    }
    __syncthreads();
    if (warp == 0) {
        float s = 0.f, g = 0.f;
        for (int j = lane; j < a.L; j += 32) {
            s += as[j];
            g = fmaxf(g, gs[j]);
        }
        s = warp_sum(s);
        g = warp_max(g);
        if (lane == 0) {
            s_hsum = s;
            s_gmax = g;
        }
    }
    __syncthreads();
    const float hsum = s_hsum, gmax = s_gmax;
    if (hsum > 0.f)
        for (int j = threadIdx.x; j < a.L; j += blockDim.x) as[j] /= hsum;
    __syncthreads();

    const int T = a.T, L = a.L, D = a.D, u0 = a.dmin - a.peak, NB = (D + 31) >> 5;
    const Slice sl = make_slice(T, D, CB);
    float* base = dyn + static_cast<size_t>(warp) * sl.words;
    float* zs = base + sl.zs;
    uint2* ent = reinterpret_cast<uint2*>(base + sl.ent);
    float* cps = base + sl.cps;
    int* cpe = reinterpret_cast<int*>(base + sl.cpe);
    float* ubs = base + sl.ubs;
    float* cs = base + sl.cs;
    const long long P = static_cast<long long>(a.H) * a.W;

    for (long long p = static_cast<long long>(blockIdx.x) * nwarps + warp; p < P;
         p += static_cast<long long>(gridDim.x) * nwarps) {
        const bool faulty = !COST_ONLY && a.faulty && a.faulty[p];

        // ---- 1. histogram row -> shared memory, per-chunk photon and non-empty-bin counts ----
        float K = 0.f;
        int nnz = 0;
        if (!faulty) {
            for (int i = lane; i < sl.nch; i += 32) {
                float f[CB];
                load_chunk<FMT>(a, p, i, f);
                float s = 0.f;
                int c = 0;
#pragma unroll
                for (int k = 0; k < CB; ++k) {
                    s += f[k];
                    c += f[k] != 0.f;
                }
                if (CB == 8) {
                    reinterpret_cast<float4*>(zs)[2 * i] = make_float4(f[0], f[1], f[2], f[3]);
                    reinterpret_cast<float4*>(zs)[2 * i + 1] = make_float4(f[4 % CB], f[5 % CB], f[6 % CB], f[7 % CB]);
                } else {
                    reinterpret_cast<float4*>(zs)[i] = make_float4(f[0], f[1], f[2], f[3]);
                }
                cps[i] = s;
                cpe[i] = c;
                K += s;
                nnz += c;
            }
            K = warp_sum(K);
            nnz = static_cast<int>(warp_sum(static_cast<float>(nnz)));
            __syncwarp();
            warp_scan2(cps, cpe, sl.nch, lane);
        }
        const bool sparse = !faulty && nnz <= kNnzSparse;
        if (sparse) {
            // compact the non-empty bins, in bin order, at the offsets the scan produced
            for (int i = lane; i < sl.nch; i += 32) {
                int o = cpe[i];
                if (cpe[i + 1] == o) continue;
#pragma unroll
                for (int k = 0; k < CB; ++k) {
                    const float v = zs[i * CB + k];
                    if (v != 0.f) ent[o++] = make_uint2(static_cast<unsigned>(i * CB + k), __float_as_uint(v));
                }
            }
            __syncwarp();
        }

        if (COST_ONLY) {
            float best = -INFINITY;
            int bidx = 0x7fffffff;
            for (int b = 0; b < NB; ++b) {
                const float acc = block_cost(gs, zs, ent, cpe, sparse, b, lane, D, L, u0, CB);
                const int c = 32 * b + lane;
                if (c < D) {
                    if (a.cost) __stcs(a.cost + p * D + c, acc);
                    if (acc > best) {
                        best = acc;
                        bidx = c;
                    }
                }
            }
            if (a.argmax) {
                warp_argmax(best, bidx);
                if (lane == 0) a.argmax[p] = a.dmin + bidx;
            }
            __syncwarp();
            continue;
        }

        // ---- 2. prior and per-block upper bounds of the log2 pseudo-posterior ----
        Prior pr;
        build_prior(a, p, pr);
        const float lam2 = a.lam2;
        float ubest = -INFINITY;
        int ub_b = 0x7fffffff;
        for (int b = lane; b < NB; b += 32) {
            const int s_bin = u0 + 32 * b;
            const int last = min(32 * b + 31, D - 1);
            const int e_bin = u0 + last + L - 1;
            const float nb = faulty ? 0.f : cps[e_bin / CB + 1] - cps[s_bin / CB];
            const float ub = lam2 * gmax * nb * 1.0001f +
                             log2_prior_bound(pr, static_cast<float>(a.dmin + 32 * b), static_cast<float>(a.dmin + last));
            ubs[b] = ub;
            if (ub > ubest) {
                ubest = ub;
                ub_b = b;
            }
        }
        warp_argmax(ubest, ub_b);
        if (ub_b >= NB) ub_b = 0;  // every bound was NaN (invalid inputs): keep the block index in range
        __syncwarp();

        // ---- 3. exact log2 pseudo-posterior on every block that can matter, and its argmax ----
        float best = -INFINITY;
        int bidx = 0x7fffffff;
        auto eval_block = [&](int b) {
            const float acc = faulty ? 0.f : block_cost(gs, zs, ent, cpe, sparse, b, lane, D, L, u0, CB);
            const int c = 32 * b + lane;
            float l = fmaf(lam2, acc, log2_prior(pr, static_cast<float>(a.dmin + c)));
            if (c >= D) l = -INFINITY;
            cs[c] = l;
            if (l > best || (l == best && c < bidx)) {
                best = l;
                bidx = c;
            }
        };
        eval_block(ub_b);
        const float thr = warp_max(best) - kPrune2;
        for (int w0 = 0; w0 < NB; w0 += 32) {
            unsigned m = __ballot_sync(0xffffffffu, w0 + lane < NB && ubs[w0 + lane] >= thr);
            if (w0 <= ub_b && ub_b < w0 + 32) m &= ~(1u << (ub_b - w0));
            while (m) {
                const int b = w0 + __ffs(m) - 1;
                m &= m - 1;
                eval_block(b);
            }
        }
        warp_argmax(best, bidx);
        if (bidx == 0x7fffffff) bidx = 0;  // every ell was NaN (invalid inputs): keep indices in range
        __syncwarp();

        // ---- 4. moments of the normalised weights 2^(ell - max), centred on the argmax ----
        float s0 = 0.f, s1 = 0.f, s2 = 0.f;
        for (int w0 = 0; w0 < NB; w0 += 32) {
            unsigned m = __ballot_sync(0xffffffffu, w0 + lane < NB && ubs[w0 + lane] >= thr);
            if (w0 <= ub_b && ub_b < w0 + 32) m |= 1u << (ub_b - w0);
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
        const float mu = static_cast<float>(a.dmin + bidx) + m1;
        const float var = fmaxf(s2 / s0 - m1 * m1, 0.f);
        if (lane == 0) {
            a.mu[p] = mu;
            a.var[p] = var;
            if (a.argmax) a.argmax[p] = a.dmin + bidx;
        }

        // ---- 5. background b and reflectivity r (Sec. II-E) ----
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
                // psi(f) = sum_W z (a - u) / (u + f (a - u)) - Kout / (1 - f) is decreasing on [0, 1):
                // safeguarded Newton on psi with the bracket [lo, hi] kept around its root.
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
                    // start from the box-template estimate (window excess over the flat background)
                    const float fr = static_cast<float>(L) * u;
                    f = fr < 1.f ? (kin - K * fr) / (K * (1.f - fr)) : 0.5f;
                    f = fminf(fmaxf(f, 0.02f), 0.98f);
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
                        const bool done = fabsf(fn - f) <= 1e-6f * fn || hi - lo <= 1e-7f * hi;
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

// Bytes of dynamic shared memory one warp needs.
size_t warp_bytes(const EstimateArgs& a) {
    const int cb = a.fmt == SPL_HIST_F32 ? 4 : 8;
    return sizeof(float) * static_cast<size_t>(make_slice(a.T, a.D, cb).words);
}

// Launch geometry of one (kernel, shape): warps per CTA chosen to maximise resident warps per SM (shared
// memory per warp grows with T and D), grid = resident CTAs on every SM (persistent), capped by the work.
template <int FMT, bool COST_ONLY>
cudaError_t launch_t(const EstimateArgs& a, cudaStream_t s) {
    auto kern = k_estimate<FMT, COST_ONLY>;
    const size_t per_warp = warp_bytes(a);
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    static int configured[64] = {0};
    if (dev < 64 && !configured[dev]) {
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024);
        if (e != cudaSuccess) return e;
        configured[dev] = 1;
    }
    int nsm = 0;
    e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    int best_wpc = 0, best_ctas = 0, best_warps = 0;
    for (int wpc = 8; wpc >= 1; --wpc) {
        const size_t smem = per_warp * wpc;
        if (smem > 220 * 1024) continue;
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
