// Fused per-pixel kernel: robust data term (Eq. beta_div2), pseudo-posterior on the depth grid
// (Eq. approx_post) with the spatio-temporal Gaussian-mixture prior (Eq. predict), moment matching
// (Eq. KL_div), and the background/reflectivity estimate (Sec. II-E).
//
// Mapping. One warp owns one pixel at a time (persistent grid-stride loop over pixels). The warp streams the
// pixel's histogram row from HBM once with 16-byte loads into its shared-memory slice and keeps a prefix sum
// of photon counts per 16-byte chunk (8 bins; 4 for float counts).
//
// Correlation. C(d) = sum_j g_j z[d - peak + j] (g = h^beta) for every candidate, into shared memory. A row
// with few non-empty bins (photon-starved data) is scattered from a compacted list of those bins (exact zero
// skip: each lane accumulates a contiguous run of candidates from the bins that reach it); a denser row uses
// a register-blocked direct sum (8 candidates per lane, taps in groups of 4).
//
// Epilogue. ell(d) = lambda C(d) + log f(d) in log2 units. Candidates are grouped in blocks of 32. Each block
// gets an upper bound of ell (lambda log2(e) max(g) times the photons in the block's window, plus the prior's
// largest value on the block). The block with the largest bound is evaluated exactly; its best value LB is a
// lower bound of the maximum, and every block whose bound is below LB - 64 is dropped: its weights are below
// 2^-64 of the maximum, so the moments move by less than 8192^3 * 2^-64 < 3e-8 bins^2.
//   * Few surviving blocks (a concentrated posterior): each is evaluated exactly in the log domain.
//   * Many (a broad posterior): the weights 2^(ell - ref) are formed directly in the linear domain over the
//     surviving range, each lane walking a contiguous run of candidates. The data factor costs one exp2 per
//     candidate; each mixture component is advanced by the exact two-multiply recurrence of a Gaussian on a
//     unit grid (value ratio, then ratio of ratios), restarted from exact exponentials every 16 candidates.
//     All values are scaled by fixed upper bounds so nothing overflows; a value that underflows is below
//     2^-126 while the largest weight is required to be at least 2^-60 (checked), so the dropped mass is
//     below 2^-62 per candidate. When that check or the component-width condition (variance >= 1.5 bins^2,
//     so 16 steps cannot underflow a component near its own peak) fails, the exact log-domain path runs.
// Moments are then taken in a second pass centred on the argmax (no cancellation between S2/S0 and the
// squared offset of the mean).
#include <cuda_fp16.h>
#include <math.h>

#include "spl_internal.h"

namespace spl {
namespace {

constexpr float kLog2e = 1.4426950408889634f;
constexpr float kLog2TwoPi = 2.6514961294723187f;  // log2(2 pi)
constexpr int kMaxComp = 10;                        // 9 stencil entries + 1 merged weakly informative one
constexpr int kNnzSparse = 320;                     // zero-skip correlation up to this many non-empty bins
constexpr float kPrune2 = 64.f;                     // log2 margin below the best value for dropping a block
constexpr int kFewBlocks = 6;                       // at most this many surviving blocks: exact log path
constexpr int kRestart = 16;                        // exact restart interval of the mixture recurrences

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
    int nch;     // 16-byte chunks per row
    int raw;     // the next pixel's row as loaded (cp.async target), nch * 4 words
    int zs;      // dense counts as float, nch * CB words + 16 zero words (read past the row by the dense sum)
    int ent;     // non-empty bins (bin, count) as uint2, kNnzSparse entries
    int cps;     // photon-count prefix over chunks, nch + 1 words
    int cpe;     // non-empty-bin prefix over chunks, nch + 1 words
    int ubs;     // per-block upper bounds, NB words
    int cs;      // C, then ell or weights, per candidate: NB * 32 words
    int words;   // total
};

__host__ __device__ __forceinline__ int round4(int x) { return (x + 3) & ~3; }

__host__ __device__ __forceinline__ Slice make_slice(int T, int D, int cb) {
    Slice s;
    s.nch = (T + cb - 1) / cb;
    const int nb = (D + 31) / 32;
    s.raw = 0;
    s.zs = s.nch * 4;
    s.ent = s.zs + round4(s.nch * cb) + 16;
    s.cps = s.ent + 2 * kNnzSparse;
    s.cpe = s.cps + round4(s.nch + 1);
    s.ubs = s.cpe + round4(s.nch + 1);
    s.cs = s.ubs + round4(nb);
    s.words = s.cs + nb * 32;
    return s;
}

// ------------------------------------------------------------------------------------------------------------
// Input staging: the histogram row and the neighbour states of the NEXT pixel are requested while the current
// pixel is processed, so HBM and L2 latency overlap compute.
// ------------------------------------------------------------------------------------------------------------

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
    const unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(smem));
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// Requests pixel p's row (nch 16-byte chunks) into raw.
__device__ __forceinline__ void request_row(const EstimateArgs& a, long long p, float* raw, int nch, int esz,
                                            int lane) {
    const char* row = static_cast<const char*>(a.z) + p * a.pitch * esz;
    for (int i = lane; i < nch; i += 32) cp_async16(raw + 4 * i, row + 16 * i);
}

// Converts 16-byte chunk i of the staged row to floats; bins >= T read as 0.
template <int FMT>
__device__ __forceinline__ void convert_chunk(const float* raw, int i, int T, float* f) {
    if (FMT == SPL_HIST_F32) {
        const float4 v = reinterpret_cast<const float4*>(raw)[i];
        f[0] = v.x;
        f[1] = v.y;
        f[2] = v.z;
        f[3] = v.w;
#pragma unroll
        for (int k = 0; k < 4; ++k)
            if (i * 4 + k >= T) f[k] = 0.f;
    } else {
        const uint4 v = reinterpret_cast<const uint4*>(raw)[i];
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
            if (i * 8 + k >= T) f[k] = 0.f;
    }
}

// One pixel's prior inputs, one stencil entry per lane (lanes 0-8; lane 0 for a per-pixel Gaussian prior).
struct Nbr {
    float m, v;
    int info;    // entry is inside the frame, present and not faulty
    int faulty;  // lane 0: the pixel itself is faulty
};

__device__ __forceinline__ Nbr request_nbr(const EstimateArgs& a, long long p, long long P, int lane) {
    Nbr r;
    r.m = r.v = 0.f;
    r.info = r.faulty = 0;
    if (p >= P) return r;
    if (a.prior_mode == PRIOR_GAUSS) {
        if (lane == 0) {
            r.m = a.pmu[p];
            r.v = a.pvar[p];
            r.info = 1;
        }
    } else if (a.prior_mode == PRIOR_STENCIL && lane < 9) {
        const int y = static_cast<int>(p / a.W), x = static_cast<int>(p - static_cast<long long>(y) * a.W);
        const int yy = y + lane / 3 - 1, xx = x + lane % 3 - 1;
        if (yy >= 0 && yy < a.H && xx >= 0 && xx < a.W) {
            const long long i = static_cast<long long>(yy) * a.W + xx;
            // independent loads (no load waits on another), selected when consumed
            const float m = a.pmu[i], v = a.pvar[i];
            const int pres = a.present_in ? a.present_in[i] : 1;
            const int fl = a.faulty ? a.faulty[i] : 0;
            r.m = m;
            r.v = v;
            r.info = (pres != 0) && (fl == 0);
        }
    }
    if (a.faulty && lane == 0) r.faulty = a.faulty[p] != 0;
    return r;
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

// ------------------------------------------------------------------------------------------------------------
// Prior (Eq. predict) in log2 units: component c contributes 2^(ca[c] - ck[c] (d - cm[c])^2)
// ------------------------------------------------------------------------------------------------------------

struct Prior {
    float ca[kMaxComp], ck[kMaxComp], cm[kMaxComp];
    float minv;  // smallest component variance
    int n;
};

// Lane-parallel construction: lane k (< 9) owns stencil entry k. Entries with identical Gaussians (every
// weakly informative one, and equal neighbour states) are merged by matching their (mean, variance) bits and
// summing their weights; the distinct components are then broadcast to every lane in lane order.
__device__ __forceinline__ void build_prior(const EstimateArgs& a, const Nbr& nb, int lane, Prior& pr) {
    float w = 0.f, m = 0.f, v = 1.f;
    if (a.prior_mode == PRIOR_GAUSS) {
        if (lane == 0) {
            w = 1.f;
            m = nb.m;
            v = nb.v;
        }
    } else if (a.prior_mode == PRIOR_STENCIL && lane < 9) {
        w = a.nu[lane];
        if (nb.info) {
            m = nb.m;
            v = nb.v + a.sigma_rw2;
        } else {
            m = a.flat_m;
            v = a.flat_v + a.sigma_rw2;
        }
    }
    const bool act = w > 0.f;
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
        const int src = lead ? __ffs(lead) - 1 : 0;
        lead &= lead - 1;
        pr.ca[i] = __shfl_sync(0xffffffffu, ca_l, src);
        pr.ck[i] = __shfl_sync(0xffffffffu, ck_l, src);
        pr.cm[i] = __shfl_sync(0xffffffffu, m, src);
        const float vi = __shfl_sync(0xffffffffu, v, src);
        if (i < pr.n) pr.minv = fminf(pr.minv, vi);
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
// Correlation C(d) for every candidate into cs[0 .. 32 NB); each routine returns max_d C(d) (warp-uniform)
// ------------------------------------------------------------------------------------------------------------

__device__ __forceinline__ void zero_words(float* x, int n4, int lane) {
    for (int i = lane; i < n4; i += 32) reinterpret_cast<float4*>(x)[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    __syncwarp();
}

// Sparse rows: lane l owns the contiguous run [r0, r1) of candidates and adds z_t g_{t-u0-c} into each
// candidate c of its run for every non-empty bin t whose taps reach the run (the bins come from the compacted
// list, the chunk prefix gives the first and last relevant entries). No other lane writes the run, so the
// accumulation needs no synchronisation.
__device__ __forceinline__ float corr_runs(const float* __restrict__ gs, const uint2* ent, const int* cpe,
                                           float* cs, int D, int L, int u0, int cb, int lane) {
    const int run = (D + 31) >> 5;
    const int r0 = lane * run, r1 = min(r0 + run, D);
    for (int c = r0; c < r1; ++c) cs[c] = 0.f;
    float mx = 0.f;
    if (r0 < r1) {
        const int e_lo = cpe[(u0 + r0) / cb];
        const int e_hi = cpe[(u0 + r1 - 1 + L - 1) / cb + 1];
        for (int e = e_lo; e < e_hi; ++e) {
            const uint2 en = ent[e];
            const float zc = __uint_as_float(en.y);
            const int tc = static_cast<int>(en.x) - u0;  // candidate whose tap 0 falls on this bin
            const int lo = max(tc - L + 1, r0), hi = min(tc, r1 - 1);
            for (int c = lo; c <= hi; ++c) {
                const float v = fmaf(zc, gs[tc - c], cs[c]);
                cs[c] = v;
                mx = fmaxf(mx, v);
            }
        }
    }
    __syncwarp();
    return warp_max(mx);
}

// Dense rows: a lane computes 8 consecutive candidates per 256-candidate super-block. Super-blocks start at
// candidate -(u0 & 3) so every lane's window starts on a 16-byte boundary of zs (candidates < 0 are dropped).
// Windows may read up to 11 words past the last bin of the row: zs carries 16 zero words there.
__device__ __forceinline__ float corr_dense(const float* __restrict__ gs, const float* zs, float* cs, int D, int L,
                                            int u0, int lane) {
    float mx = 0.f;
    for (int cb = -(u0 & 3); cb < D; cb += 256) {
        const int cl = cb + 8 * lane;
        if (cl < D && cl + 7 >= 0) {
            const float4* z4 = reinterpret_cast<const float4*>(zs + u0 + cl);
            const float4* g4 = reinterpret_cast<const float4*>(gs);
            float acc[8];
#pragma unroll
            for (int r = 0; r < 8; ++r) acc[r] = 0.f;
            float4 c0 = z4[0], c1 = z4[1];
            for (int jg = 0; jg < L; jg += 4) {
                const float4 nx = z4[jg / 4 + 2];
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
                if (cl + r >= 0 && cl + r < D) {
                    cs[cl + r] = acc[r];
                    mx = fmaxf(mx, acc[r]);
                }
        }
    }
    __syncwarp();
    return warp_max(mx);
}

// C(d) for all candidates of one pixel (row in zs, prefix sums in cps/cpe). Returns max C.
template <int CB>
__device__ __forceinline__ float correlate(const float* __restrict__ gs, const float* zs, uint2* ent,
                                           const int* cpe, float* cs, int nch, bool empty, int nnz, int NB, int D,
                                           int L, int u0, int lane) {
    if (empty) {
        zero_words(cs, NB * 8, lane);
        return 0.f;
    }
    if (nnz <= kNnzSparse) {
        for (int i = lane; i < nch; i += 32) {  // compact the non-empty bins, in bin order
            int o = cpe[i];
            if (cpe[i + 1] == o) continue;
#pragma unroll
            for (int k = 0; k < CB; ++k) {
                const float v = zs[i * CB + k];
                if (v != 0.f) ent[o++] = make_uint2(static_cast<unsigned>(i * CB + k), __float_as_uint(v));
            }
        }
        __syncwarp();
        return corr_runs(gs, ent, cpe, cs, D, L, u0, CB, lane);
    }
    return corr_dense(gs, zs, cs, D, L, u0, lane);
}

// ------------------------------------------------------------------------------------------------------------
// The kernel
// ------------------------------------------------------------------------------------------------------------

template <int FMT, bool COST_ONLY>
__global__ void __launch_bounds__(256) k_estimate(const EstimateArgs a) {
    extern __shared__ __align__(16) float dyn[];
    __shared__ __align__(16) float gs[SPL_MAX_TAPS + 4];  // g_j = h_j^beta (0 for taps <= 0 and for j >= L)
    __shared__ float as[SPL_MAX_TAPS];                     // h_j / sum(h): normalised template (intensity)
    __shared__ float s_hsum, s_gmax;
    constexpr int CB = FMT == SPL_HIST_F32 ? 4 : 8;

    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    for (int j = threadIdx.x; j < SPL_MAX_TAPS + 4; j += blockDim.x) {
        const float hj = j < a.L ? a.h[j] : 0.f;
        gs[j] = hj > 0.f ? powf(hj, a.beta) : 0.f;
        if (j < SPL_MAX_TAPS) as[j] = hj > 0.f ? hj : 0.f;
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
    float* raw = base + sl.raw;
    float* zs = base + sl.zs;
    uint2* ent = reinterpret_cast<uint2*>(base + sl.ent);
    float* cps = base + sl.cps;
    int* cpe = reinterpret_cast<int*>(base + sl.cpe);
    float* ubs = base + sl.ubs;
    float* cs = base + sl.cs;
    const long long P = static_cast<long long>(a.H) * a.W;
    const long long stride = static_cast<long long>(gridDim.x) * nwarps;
    constexpr int ESZ = FMT == SPL_HIST_F32 ? 4 : 2;
    if (lane < 4) reinterpret_cast<float4*>(zs + sl.nch * CB)[lane] = make_float4(0.f, 0.f, 0.f, 0.f);

    long long p = static_cast<long long>(blockIdx.x) * nwarps + warp;
    if (p < P) request_row(a, p, raw, sl.nch, ESZ, lane);
    cp_async_commit();
    Nbr nb_next = request_nbr(a, p, P, lane);

    for (; p < P; p += stride) {
        const Nbr nb = nb_next;
        const bool faulty = !COST_ONLY && __shfl_sync(0xffffffffu, nb.faulty, 0) != 0;
        cp_async_wait_all();
        __syncwarp();

        // ---- 1. staged row -> floats in shared memory, per-chunk photon and non-empty-bin counts ----
        float K = 0.f;
        int nnz = 0;
        if (!faulty) {
            for (int i = lane; i < sl.nch; i += 32) {
                float f[CB];
                convert_chunk<FMT>(raw, i, T, f);
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
        }
        __syncwarp();  // the staged row is consumed: stage the next pixel's inputs behind this pixel's work
        {
            const long long pn = p + stride;
            if (pn < P) request_row(a, pn, raw, sl.nch, ESZ, lane);
            cp_async_commit();
            nb_next = request_nbr(a, pn, P, lane);
        }
        if (!faulty) warp_scan2(cps, cpe, sl.nch, lane);
        const bool empty = faulty || nnz == 0;

        // ---- 2. C(d) for every candidate ----
        const float cmax = correlate<CB>(gs, zs, ent, cpe, cs, sl.nch, empty, nnz, NB, D, L, u0, lane);

        if (COST_ONLY) {
            float best = -INFINITY;
            int bidx = 0x7fffffff;
            for (int c = lane; c < D; c += 32) {
                const float acc = cs[c];
                if (a.cost) __stcs(a.cost + p * D + c, acc);
                if (acc > best) {
                    best = acc;
                    bidx = c;
                }
            }
            if (a.argmax) {
                warp_argmax(best, bidx);
                if (lane == 0) a.argmax[p] = a.dmin + bidx;
            }
            __syncwarp();
            continue;
        }

        // ---- 3. prior and per-block upper bounds of the log2 pseudo-posterior ----
        Prior pr;
        build_prior(a, nb, lane, pr);
        const float lam2 = a.lam2;
        float ubest = -INFINITY;
        int ub_b = 0x7fffffff;
        for (int b = lane; b < NB; b += 32) {
            const int s_bin = u0 + 32 * b;
            const int last = min(32 * b + 31, D - 1);
            const int e_bin = u0 + last + L - 1;
            const float nb = empty ? 0.f : cps[e_bin / CB + 1] - cps[s_bin / CB];
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

        // exact best value of the block with the largest bound: a lower bound of the maximum
        float lb;
        int cstar;  // its best candidate: the centre of the one-pass moments below
        {
            const int c = 32 * ub_b + lane;
            float l = -INFINITY;
            if (c < D) l = fmaf(lam2, cs[c], log2_prior(pr, static_cast<float>(a.dmin + c)));
            cstar = c < D ? c : 0x7fffffff;
            warp_argmax(l, cstar);
            lb = l;
            if (cstar >= D) cstar = min(32 * ub_b, D - 1);
        }
        const float thr = lb - kPrune2;
        int nsurv = 0, bfirst = NB, blast = -1;
        for (int w0 = 0; w0 < NB; w0 += 32) {
            const unsigned m =
                __ballot_sync(0xffffffffu, (w0 + lane < NB && ubs[w0 + lane] >= thr) || w0 + lane == ub_b);
            if (m) {
                nsurv += __popc(m);
                bfirst = min(bfirst, w0 + __ffs(m) - 1);
                blast = w0 + 31 - __clz(m);
            }
        }

        float best = -INFINITY;
        int bidx = 0x7fffffff;
        float mu_out = 0.f;
        bool done = false;

        // ---- 4a. linear-domain weights over the surviving range (when its exactness conditions hold) ----
        if ((blast - bfirst + 1) <= max(8, 2 * nsurv) && !(pr.minv < 1.5f)) {
            {
                float sref = pr.n > 0 ? -INFINITY : 0.f;
#pragma unroll
                for (int i = 0; i < kMaxComp; ++i)
                    if (i < pr.n) sref = fmaxf(sref, pr.ca[i]);
                const float xref = lam2 * cmax;  // lambda log2(e) max_d C(d)
                const int c_lo = 32 * bfirst, c_hi = min(32 * blast + 31, D - 1);
                const int run = (c_hi - c_lo + 32) >> 5;
                const int r0 = c_lo + lane * run, r1 = min(r0 + run, c_hi + 1);
                float v[kMaxComp], q[kMaxComp], kk[kMaxComp];
#pragma unroll
                for (int i = 0; i < kMaxComp; ++i) {
                    v[i] = q[i] = 0.f;
                    kk[i] = i < pr.n ? ex2(-2.f * pr.ck[i]) : 0.f;
                }
                float s0 = 0.f, s1 = 0.f, s2 = 0.f;
                for (int c = r0; c < r1; ++c) {
                    const float d = static_cast<float>(a.dmin + c);
                    if (((c - r0) & (kRestart - 1)) == 0) {  // exact restart of every component
#pragma unroll
                        for (int i = 0; i < kMaxComp; ++i)
                            if (i < pr.n) {
                                const float e = d - pr.cm[i];
                                v[i] = ex2(pr.ca[i] - pr.ck[i] * e * e - sref);
                                q[i] = ex2(fminf(-pr.ck[i] * (2.f * e + 1.f), 100.f));
                            }
                    }
                    float m = pr.n == 0 ? 1.f : 0.f;
#pragma unroll
                    for (int i = 0; i < kMaxComp; ++i)
                        if (i < pr.n) {
                            m += v[i];
                            v[i] *= q[i];
                            q[i] *= kk[i];
                        }
                    const float w = ex2(fmaf(lam2, cs[c], -xref)) * m;
                    cs[c] = w;
                    if (w > best) {
                        best = w;
                        bidx = c;
                    }
                    const float dd = static_cast<float>(c - cstar);
                    s0 += w;
                    s1 = fmaf(w, dd, s1);
                    s2 = fmaf(w * dd, dd, s2);
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
                    if (m1 * m1 > 4.f * var + 1.f) {
                        // the centre is far from the mean: second pass centred on the rounded mean
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
                    mu_out = static_cast<float>(a.dmin) + ctr + m1;
                    if (lane == 0) {
                        a.mu[p] = mu_out;
                        a.var[p] = fmaxf(var, 0.f);
                        if (a.argmax) a.argmax[p] = a.dmin + bidx;
                    }
                    done = true;
                } else {
                    // the weights overwrote C on the surviving range: recompute it for the exact path
                    correlate<CB>(gs, zs, ent, cpe, cs, sl.nch, empty, nnz, NB, D, L, u0, lane);
                }
            }
        }

        // ---- 4b. concentrated posterior (or fallback): exact log-domain ell on the surviving blocks ----
        if (!done) {
            best = -INFINITY;
            bidx = 0x7fffffff;
            for (int w0 = 0; w0 < NB; w0 += 32) {
                unsigned m =
                    __ballot_sync(0xffffffffu, (w0 + lane < NB && ubs[w0 + lane] >= thr) || w0 + lane == ub_b);
                while (m) {
                    const int b = w0 + __ffs(m) - 1;
                    m &= m - 1;
                    const int c = 32 * b + lane;
                    float l = -INFINITY;
                    if (c < D) l = fmaf(lam2, cs[c], log2_prior(pr, static_cast<float>(a.dmin + c)));
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
                unsigned m =
                    __ballot_sync(0xffffffffu, (w0 + lane < NB && ubs[w0 + lane] >= thr) || w0 + lane == ub_b);
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
            mu_out = static_cast<float>(a.dmin + bidx) + m1;
            if (lane == 0) {
                a.mu[p] = mu_out;
                a.var[p] = fmaxf(s2 / s0 - m1 * m1, 0.f);
                if (a.argmax) a.argmax[p] = a.dmin + bidx;
            }
        }

        // ---- 5. background b and reflectivity r (Sec. II-E) ----
        if (a.refl) {
            const float mu = mu_out;
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
                        float g = 0.f, gp = 0.f;
#pragma unroll
                        for (int q = 0; q < SPL_MAX_TAPS / 32; ++q) {
                            if (zj[q] > 0.f) {
                                const float e = __fdividef(aj[q] - u, fmaf(f, aj[q] - u, u));
                                g = fmaf(zj[q], e, g);
                                gp = fmaf(zj[q] * e, e, gp);
                            }
                        }
                        g = warp_sum(g);
                        gp = warp_sum(gp);
                        const float om = 1.f - f;
                        const float rom = __fdividef(1.f, om);
                        g = fmaf(-kout, rom, g);
                        gp = fmaf(kout * rom, rom, gp);
                        if (g > 0.f) lo = f; else hi = f;
                        float fn = f + __fdividef(g, gp);  // Newton step on psi (psi' = -gp)
                        if (!(fn > lo && fn < hi)) fn = 0.5f * (lo + hi);
                        const bool conv = fabsf(fn - f) <= 1e-6f * fn || hi - lo <= 1e-7f * hi;
                        f = fn;
                        if (conv) break;
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
    cp_async_wait_all();  // no copy may still target this CTA's shared memory when it exits
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
