// Fused per-pixel kernel over photon-count histograms: robust data term (Eq. beta_div2), pseudo-posterior on the
// depth grid (Eq. approx_post) with the spatio-temporal Gaussian-mixture prior (Eq. predict) and moment matching
// (Eq. KL_div). It leaves each pixel's photon count in bg; the background/reflectivity estimate (Sec. II-E) is a
// separate launch (intensity.cu).
//
// Mapping. One warp owns one pixel at a time (persistent grid-stride loop over pixels). While a pixel is
// processed, the next pixel's histogram row is copied into the warp's shared-memory slice with cp.async and its
// neighbour states are loaded into registers, so HBM and L2 latency overlap compute.
//
// Per pixel: (1) the non-empty 16-byte chunks of the staged row are listed (one load and one test per chunk), then
// their bins are counted (photons K, non-empty bins) 32 chunks at a time; (2) a row with few non-empty bins
// (photon-starved data) keeps them as a (bin, count) list in bin order: each block of 32 candidates gets the photon
// count of its window as its data bound, and C(d) = sum_j g_j z[d - peak + j] (g = h^beta) is scattered from the
// list, lane = tap; a denser row is correlated by a register-blocked direct sum (8 candidates per lane, taps in
// groups of 4) whose largest C bounds every block. Both forms add the products of one candidate in tap order, so
// they give bitwise the same C. (3) The pseudo-posterior (posterior.cuh) drops the blocks whose weights are
// provably below 2^-64 of the largest and weighs the rest.
#include <cuda_fp16.h>
#include <math.h>

#include <atomic>

#include "pixel.cuh"
#include "posterior.cuh"
#include "spl_internal.h"

namespace spl {
namespace {

using namespace px;

constexpr int kTapNnz = 128;  // zero-skip correlation up to this many non-empty bins (list capacity), dense above

// Shared-memory slice of one warp (all offsets in 4-byte words; every array starts 16-byte aligned).
struct Slice {
    int nch;     // 16-byte chunks per row
    int rawsz;   // words per staging buffer: nch * 4 + 16 zero words (windows read up to 11 bins past T)
    int raw;     // two staging buffers (cp.async targets): the current pixel's row and the next one's
    int ebin;    // non-empty bins of a listed row, in bin order (kTapNnz words)
    int eval;    // their counts (kTapNnz words)
    int bnd;     // per-block data bound of a listed row: photons whose windows reach the block, NB words
    int ubs;     // per-block upper bounds of ell, NB words
    int cs;      // C, then ell or weights, per candidate: NB * 32 words (first the list of non-empty chunks)
    int words;   // total
};

__host__ __device__ __forceinline__ int round4(int x) { return (x + 3) & ~3; }

__host__ __device__ __forceinline__ Slice make_slice(int T, int D, int cb) {
    Slice s;
    s.nch = (T + cb - 1) / cb;
    const int nb = (D + 31) / 32;
    s.rawsz = s.nch * 4 + 16;
    s.raw = 0;
    s.ebin = 2 * s.rawsz;
    s.eval = s.ebin + kTapNnz;
    s.bnd = s.eval + kTapNnz;
    s.ubs = s.bnd + round4(nb);
    s.cs = s.ubs + round4(nb);
    s.words = s.cs + (nb * 32 > round4(s.nch) ? nb * 32 : round4(s.nch));
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

// Count in bin t of the staged row (t < T).
template <int FMT>
__device__ __forceinline__ float bin_value(const float* raw, int t) {
    if (FMT == SPL_HIST_F32) return raw[t];
    const unsigned short v = reinterpret_cast<const unsigned short*>(raw)[t];
    if (FMT == SPL_HIST_U16) return __int_as_float(0x4B000000 | v) - 8388608.f;
    return __half2float(__ushort_as_half(v));
}

// Counts of bins t .. t+3 of the staged row (t a multiple of 4).
template <int FMT>
__device__ __forceinline__ float4 bin4(const float* raw, int t) {
    if (FMT == SPL_HIST_F32) return reinterpret_cast<const float4*>(raw)[t >> 2];
    const uint2 v = reinterpret_cast<const uint2*>(raw)[t >> 2];
    if (FMT == SPL_HIST_U16)
        return make_float4(__int_as_float(0x4B000000 | (v.x & 0xffffu)) - 8388608.f,
                           __int_as_float(0x4B000000 | (v.x >> 16)) - 8388608.f,
                           __int_as_float(0x4B000000 | (v.y & 0xffffu)) - 8388608.f,
                           __int_as_float(0x4B000000 | (v.y >> 16)) - 8388608.f);
    return make_float4(__half2float(__ushort_as_half(static_cast<unsigned short>(v.x & 0xffffu))),
                       __half2float(__ushort_as_half(static_cast<unsigned short>(v.x >> 16))),
                       __half2float(__ushort_as_half(static_cast<unsigned short>(v.y & 0xffffu))),
                       __half2float(__ushort_as_half(static_cast<unsigned short>(v.y >> 16))));
}

// One pixel's prior inputs, one stencil entry per lane (lanes 0-8; lane 0 for a per-pixel Gaussian prior).
struct Nbr {
    float m, v;
    int info;    // entry is inside the frame, present and not faulty
    int faulty;  // lane 0: the pixel itself is faulty
};

__device__ __forceinline__ Nbr request_nbr(const EstimateArgs& a, long long p, int y, int x, long long P, int lane) {
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

// ------------------------------------------------------------------------------------------------------------
// Row scan and the data term C(d)
// ------------------------------------------------------------------------------------------------------------

// The non-empty 16-byte chunks of the staged row (bins T and above are zero), listed in chunk order into
// nzc[0 .. M): 32 consecutive chunks per step (lane = chunk, one load and one test each), appended by ballot, so
// photon-starved rows cost little here. Returns M (warp-uniform).
__device__ __forceinline__ int nonempty_chunks(const float* raw, int nch, int* nzc, int lane) {
    int M = 0;
    const unsigned below = (1u << lane) - 1u;
    for (int i0 = 0; i0 < nch; i0 += 32) {
        const int i = i0 + lane;
        bool nz = false;
        if (i < nch) {
            const uint4 v = reinterpret_cast<const uint4*>(raw)[i];
            nz = (v.x | v.y | v.z | v.w) != 0u;
        }
        const unsigned m = __ballot_sync(0xffffffffu, nz);
        if (nz) nzc[M + __popc(m & below)] = i;
        M += __popc(m);
    }
    __syncwarp();
    return M;
}

// Photons K and non-empty bins nnz of the listed chunks (32 chunks per round, lane = chunk). While the running
// count stays within kTapNnz the non-empty bins are also listed as (bin, count) in ebin/eval, in bin order.
template <int FMT, int CB>
__device__ __forceinline__ void count_and_list(const float* raw, const int* nzc, int M, int T, int* ebin, float* eval,
                                               int lane, float& K, int& nnz) {
    float ks = 0.f;
    int base = 0;
    for (int k0 = 0; k0 < M; k0 += 32) {
        const int k = k0 + lane;
        float f[CB];
        int n = 0, i = 0;
        if (k < M) {
            i = nzc[k];
            convert_chunk<FMT>(raw, i, T, f);
#pragma unroll
            for (int j = 0; j < CB; ++j) {
                n += f[j] != 0.f;
                ks += f[j];
            }
        }
        int incl = n;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, incl, d);
            if (lane >= d) incl += t;
        }
        const int tot = __shfl_sync(0xffffffffu, incl, 31);
        if (k < M && base + tot <= kTapNnz) {  // warp-uniform round total: the list is either complete or unused
            int o = base + incl - n;
#pragma unroll
            for (int j = 0; j < CB; ++j)
                if (f[j] != 0.f) {
                    ebin[o] = i * CB + j;
                    eval[o] = f[j];
                    ++o;
                }
        }
        base += tot;
    }
    __syncwarp();
    K = warp_sum(ks);
    nnz = base;
}

// C on candidates [c_lo, c_hi] of a listed row, lane = tap: lane l owns the taps j = l + 32 k (k < NTG) and adds
// z_t g_j into candidate t - u0 - j for each listed bin t in turn (bins whose windows miss the range are skipped).
// The candidates of one bin are distinct across lanes and taps and the warp synchronises between bins, so every
// C(d) is summed in bin order, i.e. in tap order, as by the dense sum. The range must be zero on entry. Returns max
// C.
template <int NTG>
__device__ __forceinline__ float scatter_range(const float* __restrict__ gs, const int* ebin, const float* eval,
                                               int nnz, float* cs, int c_lo, int c_hi, int u0, int L, int lane) {
    float g[NTG];
#pragma unroll
    for (int k = 0; k < NTG; ++k) g[k] = gs[lane + 32 * k];
    const int off = -u0 - lane;
    const unsigned span = static_cast<unsigned>(c_hi - c_lo);
    float mx = 0.f;
    for (int e = 0; e < nnz; ++e) {
        const int t = ebin[e];
        if (t - u0 - L + 1 > c_hi) break;  // this bin and every later one lie past the range
        if (t - u0 < c_lo) continue;       // warp-uniform: the bin's window ends before the range
        const int c = t + off;
        const float z = eval[e];
#pragma unroll
        for (int k = 0; k < NTG; ++k) {
            const int ck = c - 32 * k;
            if (static_cast<unsigned>(ck - c_lo) <= span) {
                const float v = fmaf(z, g[k], cs[ck]);
                cs[ck] = v;
                mx = fmaxf(mx, v);
            }
        }
        __syncwarp();
    }
    return warp_max(mx);
}

// C on every candidate of a listed row (zero-filled, then scattered lane = tap); returns max C.
__device__ __forceinline__ float listed_all(const float* __restrict__ gs, const int* ebin, const float* eval, int nnz,
                                           float* cs, int NB, int D, int L, int u0, int lane) {
    zero_words(cs, NB * 8, lane);
    switch ((L + 31) >> 5) {
        case 1: return scatter_range<1>(gs, ebin, eval, nnz, cs, 0, D - 1, u0, L, lane);
        case 2: return scatter_range<2>(gs, ebin, eval, nnz, cs, 0, D - 1, u0, L, lane);
        case 3: return scatter_range<3>(gs, ebin, eval, nnz, cs, 0, D - 1, u0, L, lane);
        default: return scatter_range<4>(gs, ebin, eval, nnz, cs, 0, D - 1, u0, L, lane);
    }
}

// Photons of the listed bins that reach each block: entry (t, z) adds z to the blocks holding candidates
// t - u0 - L + 1 .. t - u0. bnd[0 .. NB) must be zero on entry.
__device__ __forceinline__ void block_photons(const int* ebin, const float* eval, int nnz, float* bnd, int D, int L,
                                              int u0, int lane) {
    for (int e = lane; e < nnz; e += 32) {
        const int chi = min(ebin[e] - u0, D - 1), clo = max(ebin[e] - u0 - L + 1, 0);
        if (chi < clo) continue;
        for (int b = clo >> 5; b <= (chi >> 5); ++b) atomicAdd(&bnd[b], eval[e]);
    }
    __syncwarp();
}

// Dense rows: a lane computes 8 consecutive candidates per 256-candidate super-block. Super-blocks start at
// candidate -(u0 & 3) so every lane's window starts on a 4-bin boundary (candidates < 0 are dropped). Windows
// may read up to 11 bins past the row: the staging buffer is zero there (bins T..pitch-1 are zeroed too).
// Returns max C (warp-uniform).
template <int FMT>
__device__ __forceinline__ float corr_dense(const float* __restrict__ gs, const float* raw, float* cs, int D, int L,
                                            int u0, int lane) {
    float mx = 0.f;
    for (int cb = -(u0 & 3); cb < D; cb += 256) {
        const int cl = cb + 8 * lane;
        if (cl < D && cl + 7 >= 0) {
            const int t0 = u0 + cl;
            const float4* g4 = reinterpret_cast<const float4*>(gs);
            float acc[8];
#pragma unroll
            for (int r = 0; r < 8; ++r) acc[r] = 0.f;
            float4 c0 = bin4<FMT>(raw, t0), c1 = bin4<FMT>(raw, t0 + 4);
            for (int jg = 0; jg < L; jg += 4) {
                const float4 nx = bin4<FMT>(raw, t0 + jg + 8);
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

// C everywhere again after the linear-domain weights overwrote it (the rare fallback to the log-domain path):
// out of line, so the hot loop's code stays small.
template <int FMT>
__device__ __noinline__ void recompute_all(const float* __restrict__ gs, const float* raw, const int* ebin,
                                           const float* eval, int nnz, float* cs, bool empty, bool sparse, int NB,
                                           int D, int L, int u0, int lane) {
    if (empty) {
        zero_words(cs, NB * 8, lane);
    } else if (sparse) {
        listed_all(gs, ebin, eval, nnz, cs, NB, D, L, u0, lane);
    } else {
        corr_dense<FMT>(gs, raw, cs, D, L, u0, lane);
    }
}

// ------------------------------------------------------------------------------------------------------------
// The kernel
// ------------------------------------------------------------------------------------------------------------

template <int FMT, bool COST_ONLY>
__global__ void __launch_bounds__(256) k_estimate(const EstimateArgs a) {
    extern __shared__ __align__(16) float dyn[];
    __shared__ __align__(16) float gs[SPL_MAX_TAPS + 4];  // g_j = h_j^beta (0 for taps <= 0 and for j >= L)
    __shared__ float s_gmax;
    constexpr int CB = FMT == SPL_HIST_F32 ? 4 : 8;

    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    for (int j = threadIdx.x; j < SPL_MAX_TAPS + 4; j += blockDim.x) {
        const float hj = j < a.L ? a.h[j] : 0.f;
        gs[j] = hj > 0.f ? powf(hj, a.beta) : 0.f;
    }
    __syncthreads();
    if (warp == 0) {
        float g = 0.f;
        for (int j = lane; j < a.L; j += 32) g = fmaxf(g, gs[j]);
        g = warp_max(g);
        if (lane == 0) s_gmax = g;
    }
    __syncthreads();
    const float gmax = s_gmax;

    const int T = a.T, L = a.L, D = a.D, u0 = a.dmin - a.peak, NB = (D + 31) >> 5;
    const Slice sl = make_slice(T, D, CB);
    float* base = dyn + static_cast<size_t>(warp) * sl.words;
    int* ebin = reinterpret_cast<int*>(base + sl.ebin);
    float* eval = base + sl.eval;
    float* bnd = base + sl.bnd;
    float* ubs = base + sl.ubs;
    float* cs = base + sl.cs;
    const long long P = static_cast<long long>(a.H) * a.W;
    const long long stride = static_cast<long long>(gridDim.x) * nwarps;
    constexpr int ESZ = FMT == SPL_HIST_F32 ? 4 : 2;
    if (lane < 8) {  // zero padding after each staging buffer (cp.async never writes it)
        float* pad = base + sl.raw + (lane >> 2) * sl.rawsz + sl.nch * 4;
        reinterpret_cast<float4*>(pad)[lane & 3] = make_float4(0.f, 0.f, 0.f, 0.f);
    }

    long long p = static_cast<long long>(blockIdx.x) * nwarps + warp;
    // pixel coordinates of p and of the grid stride (P < 2^31), advanced without a division per pixel
    int py = 0, px = 0;
    if (p < P) {
        py = static_cast<int>(p) / a.W;
        px = static_cast<int>(p) - py * a.W;
    }
    const int sy = static_cast<int>(stride / a.W), sx = static_cast<int>(stride - static_cast<long long>(sy) * a.W);
    if (p < P) request_row(a, p, base + sl.raw, sl.nch, ESZ, lane);
    cp_async_commit();
    Nbr nb_next = request_nbr(a, p, py, px, P, lane);

    for (int buf = 0; p < P; p += stride, buf ^= 1) {
        const Nbr nb = nb_next;
        const bool faulty = !COST_ONLY && __shfl_sync(0xffffffffu, nb.faulty, 0) != 0;
        float* raw = base + sl.raw + buf * sl.rawsz;
        cp_async_wait_all();
        __syncwarp();
        {  // stage the next pixel's row into the other buffer and its neighbour states into registers
            const long long pn = p + stride;
            px += sx;
            py += sy;
            if (px >= a.W) {
                px -= a.W;
                ++py;
            }
            if (pn < P) request_row(a, pn, base + sl.raw + (buf ^ 1) * sl.rawsz, sl.nch, ESZ, lane);
            cp_async_commit();
            nb_next = request_nbr(a, pn, py, px, P, lane);
        }
        // bins T .. pitch-1 are not data: make them zero (the chunk test and the dense windows read them)
        for (int t = T + lane; t < sl.nch * CB; t += 32) {
            if (FMT == SPL_HIST_F32) raw[t] = 0.f;
            else reinterpret_cast<unsigned short*>(raw)[t] = 0;
        }
        __syncwarp();

        // ---- 1. photons and non-empty bins of the staged row ----
        float K = 0.f;
        int nnz = 0;
        if (!faulty) {
            const int M = nonempty_chunks(raw, sl.nch, reinterpret_cast<int*>(cs), lane);
            count_and_list<FMT, CB>(raw, reinterpret_cast<const int*>(cs), M, T, ebin, eval, lane, K, nnz);
        }
        const bool empty = faulty || nnz == 0;
        const bool sparse = nnz <= kTapNnz;

        // ---- 2. C on every candidate: from the bin list (few non-empty bins; each block also gets the photons
        // that reach it, its data bound) or by the dense sum (whose largest C bounds every block) ----
        float cmax = 0.f;
        if (empty) {
            zero_words(cs, NB * 8, lane);
        } else if (sparse) {
            zero_words(bnd, (NB + 3) >> 2, lane);
            block_photons(ebin, eval, nnz, bnd, D, L, u0, lane);
            cmax = listed_all(gs, ebin, eval, nnz, cs, NB, D, L, u0, lane);
        } else {
            cmax = corr_dense<FMT>(gs, raw, cs, D, L, u0, lane);
        }

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

        // ---- 3. prior (Eq. predict) from the staged neighbour states ----
        Prior pr;
        {
            float w = 0.f, m = 0.f, v = 1.f;
            if (a.prior_mode == PRIOR_GAUSS) {
                if (lane == 0) {
                    w = 1.f;
                    m = nb.m;
                    v = nb.v;
                }
            } else if (a.prior_mode == PRIOR_STENCIL && lane < 9) {
                w = a.nu[lane];
                m = nb.info ? nb.m : a.flat_m;
                v = (nb.info ? nb.v : a.flat_v) + a.sigma_rw2;
            }
            build_prior(w, m, v, lane, pr);
        }

        // ---- 4. argmax, mean and variance of the pseudo-posterior (Eq. approx_post, Eq. KL_div) ----
        Grid grid;
        grid.D = D;
        grid.NB = NB;
        grid.dmin = a.dmin;
        grid.u0 = u0;
        grid.L = L;
        grid.lam2 = a.lam2;
        grid.gmax = gmax;
        const float lam2 = a.lam2;
        const int ub_b = block_bounds(
            grid, pr, ubs,
            [&](int b) {
                if (empty) return 0.f;
                if (sparse) return lam2 * gmax * bnd[b] * 1.0001f;
                return lam2 * cmax * 1.0001f;
            },
            lane);
        int bidx;
        float mu, var;
        posterior_eval(grid, pr, cmax, cs, ubs, ub_b,
                       [&]() {
                           recompute_all<FMT>(gs, raw, ebin, eval, nnz, cs, empty, sparse, NB, D, L, u0, lane);
                       },
                       lane, bidx, mu, var);
        if (lane == 0) {
            a.mu[p] = mu;
            a.var[p] = var;
            if (a.argmax) a.argmax[p] = a.dmin + bidx;
        }

        // ---- 5. background b and reflectivity r (Sec. II-E): a separate launch (intensity.cu) solves them; the
        // photon count goes to bg for it ----
        if (a.refl && lane == 0) a.bg[p] = K;
        __syncwarp();
    }
    cp_async_wait_all();  // no copy may still target this CTA's shared memory when it exits
}

// ------------------------------------------------------------------------------------------------------------
// Pixels set aside by the tensor-core filter step on uint16 histograms
// ------------------------------------------------------------------------------------------------------------

// The tensor-core kernel (uint16 frames of spl_filter_step, spl_filter_step_detect and spl_depth_estimate) converts
// uint16 counts to FP16 exactly only below 1024; a 128-pixel block holding a larger count gets mu = NaN instead of
// its results. This kernel computes those pixels again with the steps of
// k_estimate (without its prefetching: the case is rare), one warp per pixel. A warp tests the mu of 32
// consecutive pixels at once and takes the marked ones in turn; a CTA whose pixels hold no mark returns before
// any set-up, so a frame with none costs one load per pixel.
__global__ void __launch_bounds__(256) k_estimate_redo(const EstimateArgs a) {
    constexpr int FMT = SPL_HIST_U16, CB = 8;
    extern __shared__ __align__(16) float dyn[];
    __shared__ __align__(16) float gs[SPL_MAX_TAPS + 4];
    __shared__ float s_gmax;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const long long P = static_cast<long long>(a.H) * a.W;
    {  // the CTA's pixels first: nothing marked (the usual case) means nothing to set up
        int any = 0;
        for (long long g0 = (static_cast<long long>(blockIdx.x) * nwarps + warp) * 32; g0 < P && !any;
             g0 += static_cast<long long>(gridDim.x) * nwarps * 32)
            any = __any_sync(0xffffffffu, g0 + lane < P && isnan(a.mu[g0 + lane]));
        if (!__syncthreads_or(any)) return;
    }
    for (int j = threadIdx.x; j < SPL_MAX_TAPS + 4; j += blockDim.x) {
        const float hj = j < a.L ? a.h[j] : 0.f;
        gs[j] = hj > 0.f ? powf(hj, a.beta) : 0.f;
    }
    __syncthreads();
    if (warp == 0) {
        float g = 0.f;
        for (int j = lane; j < a.L; j += 32) g = fmaxf(g, gs[j]);
        g = warp_max(g);
        if (lane == 0) s_gmax = g;
    }
    __syncthreads();
    const float gmax = s_gmax;
    const int T = a.T, L = a.L, D = a.D, u0 = a.dmin - a.peak, NB = (D + 31) >> 5;
    const Slice sl = make_slice(T, D, CB);
    float* base = dyn + static_cast<size_t>(warp) * sl.words;
    int* ebin = reinterpret_cast<int*>(base + sl.ebin);
    float* eval = base + sl.eval;
    float* bnd = base + sl.bnd;
    float* ubs = base + sl.ubs;
    float* cs = base + sl.cs;
    float* raw = base + sl.raw;
    if (lane < 4) reinterpret_cast<float4*>(raw + sl.nch * 4)[lane] = make_float4(0.f, 0.f, 0.f, 0.f);
    for (long long g0 = (static_cast<long long>(blockIdx.x) * nwarps + warp) * 32; g0 < P;
         g0 += static_cast<long long>(gridDim.x) * nwarps * 32) {
        unsigned marked = __ballot_sync(0xffffffffu, g0 + lane < P && isnan(a.mu[g0 + lane]));
        while (marked) {
            const long long p = g0 + __ffs(marked) - 1;
            marked &= marked - 1;
            const int py = static_cast<int>(p / a.W), px = static_cast<int>(p - static_cast<long long>(py) * a.W);
            request_row(a, p, raw, sl.nch, 2, lane);
            cp_async_commit();
            const Nbr nb = request_nbr(a, p, py, px, P, lane);
            cp_async_wait_all();
            __syncwarp();
            for (int t = T + lane; t < sl.nch * CB; t += 32) reinterpret_cast<unsigned short*>(raw)[t] = 0;
            __syncwarp();
            const bool faulty = __shfl_sync(0xffffffffu, nb.faulty, 0) != 0;
            float K = 0.f;
            int nnz = 0;
            if (!faulty) {
                const int M = nonempty_chunks(raw, sl.nch, reinterpret_cast<int*>(cs), lane);
                count_and_list<FMT, CB>(raw, reinterpret_cast<const int*>(cs), M, T, ebin, eval, lane, K, nnz);
            }
            const bool empty = faulty || nnz == 0;
            const bool sparse = nnz <= kTapNnz;
            float cmax = 0.f;
            if (empty) {
                zero_words(cs, NB * 8, lane);
            } else if (sparse) {
                zero_words(bnd, (NB + 3) >> 2, lane);
                block_photons(ebin, eval, nnz, bnd, D, L, u0, lane);
                cmax = listed_all(gs, ebin, eval, nnz, cs, NB, D, L, u0, lane);
            } else {
                cmax = corr_dense<FMT>(gs, raw, cs, D, L, u0, lane);
            }
            Prior pr;
            {  // as k_estimate: the filter step's stencil (Eq. predict), one Gaussian, or the flat prior
                float w = 0.f, m = 0.f, v = 1.f;
                if (a.prior_mode == PRIOR_GAUSS) {
                    if (lane == 0) {
                        w = 1.f;
                        m = nb.m;
                        v = nb.v;
                    }
                } else if (a.prior_mode == PRIOR_STENCIL && lane < 9) {
                    w = a.nu[lane];
                    m = nb.info ? nb.m : a.flat_m;
                    v = (nb.info ? nb.v : a.flat_v) + a.sigma_rw2;
                }
                build_prior(w, m, v, lane, pr);
            }
            Grid grid;
            grid.D = D;
            grid.NB = NB;
            grid.dmin = a.dmin;
            grid.u0 = u0;
            grid.L = L;
            grid.lam2 = a.lam2;
            grid.gmax = gmax;
            const float lam2 = a.lam2;
            const int ub_b = block_bounds(
                grid, pr, ubs,
                [&](int b) {
                    if (empty) return 0.f;
                    if (sparse) return lam2 * gmax * bnd[b] * 1.0001f;
                    return lam2 * cmax * 1.0001f;
                },
                lane);
            int bidx;
            float mu, var;
            posterior_eval(grid, pr, cmax, cs, ubs, ub_b,
                                  [&]() {
                                      recompute_all<FMT>(gs, raw, ebin, eval, nnz, cs, empty, sparse, NB, D, L, u0,
                                                         lane);
                                  },
                                  lane, bidx, mu, var);
            if (lane == 0) {
                a.mu[p] = mu;
                a.var[p] = var;
                if (a.argmax) a.argmax[p] = a.dmin + bidx;
                if (a.refl) a.bg[p] = K;
            }
            __syncwarp();
        }
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
    static std::atomic<int> configured[64];  // per device: the shared-memory limit has been raised
    if (dev >= 64 || !configured[dev].load(std::memory_order_acquire)) {
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024);
        if (e != cudaSuccess) return e;
        if (dev < 64) configured[dev].store(1, std::memory_order_release);
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

// The pixels the tensor-core filter step set aside (uint16 input): a persistent grid of up to 8 warps per CTA and
// resident CTAs on every SM, each warp testing 32 pixels at a time.
cudaError_t launch_estimate_redo(const EstimateArgs& a, cudaStream_t s) {
    const size_t per_warp = warp_bytes(a);
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    static std::atomic<int> configured[64];
    if (dev >= 64 || !configured[dev].load(std::memory_order_acquire)) {
        e = cudaFuncSetAttribute(k_estimate_redo, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024);
        if (e != cudaSuccess) return e;
        if (dev < 64) configured[dev].store(1, std::memory_order_release);
    }
    int nsm = 0;
    if ((e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    int wpc = static_cast<int>((220 * 1024) / per_warp);
    if (wpc > 8) wpc = 8;
    if (wpc < 1) return cudaErrorInvalidConfiguration;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_estimate_redo, wpc * 32, per_warp * wpc);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    const long long P = static_cast<long long>(a.H) * a.W;
    long long ctas = (P + 32LL * wpc - 1) / (32LL * wpc);
    const long long cap = static_cast<long long>(nsm) * per_sm;
    if (ctas > cap) ctas = cap;
    k_estimate_redo<<<static_cast<unsigned>(ctas), wpc * 32, per_warp * wpc, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_estimate(const EstimateArgs& a, bool cost_only, cudaStream_t s) {
    cudaError_t e;
    switch (a.fmt) {
        case SPL_HIST_U16:
            e = cost_only ? launch_t<SPL_HIST_U16, true>(a, s) : launch_t<SPL_HIST_U16, false>(a, s);
            break;
        case SPL_HIST_F16:
            e = cost_only ? launch_t<SPL_HIST_F16, true>(a, s) : launch_t<SPL_HIST_F16, false>(a, s);
            break;
        case SPL_HIST_F32:
            e = cost_only ? launch_t<SPL_HIST_F32, true>(a, s) : launch_t<SPL_HIST_F32, false>(a, s);
            break;
        default:
            return cudaErrorInvalidValue;
    }
    if (e != cudaSuccess || cost_only || !a.refl) return e;
    return launch_intensity(a, s);  // reads K from bg, writes refl and bg
}

}  // namespace spl
