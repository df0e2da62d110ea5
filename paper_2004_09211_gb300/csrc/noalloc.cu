// Allocation-free variant of the batched photon-list step, for callers that cannot allocate device memory
// through CUDA (for example a host application whose device memory is entirely handed out by another
// framework's pool, or code that must not trigger a cudaMalloc inside a latency-critical loop).
//
// The plan-based path (batch.cu) keeps its work-queue head and its unit list in memory allocated by
// spl_batch_create. This variant needs no plan: the caller passes the sequence descriptors in device memory it
// already owns, and the only working memory -- the work-queue head and the per-sequence prefix of work units --
// lives in a fixed-size file-scope device array, g_noalloc_scratch, which every GPU that loads the library holds
// until the process exits. Work units are taken in sequence order (the plan-based path sorts them by cost).
// The per-pixel arithmetic is that of pixel.cuh and posterior.cuh, as in the plan-based kernel.
#include <math.h>
#include <stdio.h>

#include <mutex>

#include "pixel.cuh"
#include "photons.cuh"
#include "posterior.cuh"
#include "spl_internal.h"

namespace spl {
namespace {

using namespace px;

// [0]: work-queue head; [1 + s]: first work unit of sequence s (s = 0 .. nseq), i.e. a prefix of unit counts.
// Host code must not pass g_noalloc_scratch itself to a kernel (on the host it names a stand-in, not device
// memory): it uses the device address obtained with cudaGetSymbolAddress.
static __device__ __align__(256) unsigned g_noalloc_scratch[2 + SPL_NOALLOC_MAX_SEQ];

struct NSlice {
    int gs, as, bnd, ubs, cs, words;  // taps h^beta, template, per-block photon counts, bounds, C
};

__host__ __device__ __forceinline__ NSlice make_nslice(int maxD) {
    NSlice s;
    const int nb = (maxD + 31) / 32;
    s.gs = 0;
    s.as = s.gs + SPL_MAX_TAPS + 4;
    s.bnd = s.as + SPL_MAX_TAPS;
    s.ubs = s.bnd + ((nb + 3) & ~3);
    s.cs = s.ubs + ((nb + 3) & ~3);
    s.words = s.cs + (nb * 32 > SPL_MAX_TAPS ? nb * 32 : SPL_MAX_TAPS);  // cs doubles as the window histogram
    return s;
}

// Clears the queue head and writes the unit prefix: one warp, 32 sequences per step, each step an inclusive warp
// scan of the unit counts plus the running total of the steps before it.
__global__ void k_noalloc_setup(const spl_seq_desc* __restrict__ seqs, int nseq, int tile, unsigned* scratch) {
    if (blockIdx.x != 0 || threadIdx.x >= 32) return;
    const int lane = threadIdx.x;
    if (lane == 0) scratch[0] = 0u;
    unsigned carry = 0;
    for (int s0 = 0; s0 < nseq; s0 += 32) {
        const int s = s0 + lane;
        unsigned n = 0;
        if (s < nseq) {
            const long long P = static_cast<long long>(seqs[s].prm.H) * seqs[s].prm.W;
            n = static_cast<unsigned>((P + tile - 1) / tile);
        }
        unsigned inc = n;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned t = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += t;
        }
        if (s < nseq) scratch[1 + s] = carry + inc - n;
        carry += __shfl_sync(0xffffffffu, inc, 31);
    }
    if (lane == 0) scratch[1 + nseq] = carry;
}

__global__ void __launch_bounds__(256) k_noalloc_batch(const spl_seq_desc* __restrict__ seqs, int nseq, int tile,
                                                       unsigned* scratch, uint32_t* status, NSlice sl, int maxD) {
    extern __shared__ __align__(16) float dyn[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    float* base = dyn + static_cast<size_t>(warp) * sl.words;
    float* gs = base + sl.gs;
    float* as = base + sl.as;
    float* bnd = base + sl.bnd;
    float* ubs = base + sl.ubs;
    float* cs = base + sl.cs;
    const unsigned* prefix = scratch + 1;
    const unsigned nunits = prefix[nseq];

    while (true) {
        unsigned u = 0;
        if (lane == 0) u = atomicAdd(scratch, 1u);
        u = __shfl_sync(0xffffffffu, u, 0);
        if (u >= nunits) break;
        int lo = 0, hi = nseq - 1;  // last sequence whose first unit is <= u
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (prefix[mid] <= u) lo = mid; else hi = mid - 1;
        }
        const int sidx = lo;
        const spl_seq_desc& sq = seqs[sidx];
        const spl_params prm = sq.prm;
        const spl_seq_frame f = sq.f;
        const int P = prm.H * prm.W;
        const int p_begin = static_cast<int>(u - prefix[sidx]) * tile;
        const int p_end = min(P, p_begin + tile);
        const int T = prm.T, L = prm.L, D = prm.dmax - prm.dmin + 1, NB = (D + 31) >> 5;
        const int u0 = prm.dmin - prm.peak;
        if (D > maxD || D < 1 || L < 1 || L > SPL_MAX_TAPS || T < L) {
            // this device descriptor differs from the host copy the shared-memory slice was sized from: refuse the
            // unit rather than write past the warp's slice
            for (int p = p_begin + lane; p < p_end; p += 32) {
                f.mu_out[p] = f.var_out[p] = NAN;
                if (f.argmax) f.argmax[p] = -1;
                if (f.refl) f.refl[p] = f.bg[p] = NAN;
            }
            if (lane == 0 && status) atomicOr(status, SPL_BATCH_DESC_MISMATCH);
            continue;
        }
        const float lam2 = static_cast<float>((static_cast<double>(prm.beta) + 1.0) / prm.beta) * kLog2e;
        const float flat_m = 0.5f * static_cast<float>(prm.dmin + prm.dmax);
        const double span = static_cast<double>(prm.dmax - prm.dmin);
        const float flat_v = static_cast<float>(span * span / 12.0);

        float hs = 0.f, gm = 0.f;
        for (int j = lane; j < SPL_MAX_TAPS + 4; j += 32) {
            const float hj = j < L ? f.h[j] : 0.f;
            const float gj = hj > 0.f ? powf(hj, prm.beta) : 0.f;
            gs[j] = gj;
            if (j < SPL_MAX_TAPS) as[j] = hj > 0.f ? hj : 0.f;
            hs += hj > 0.f ? hj : 0.f;
            gm = fmaxf(gm, gj);
        }
        const float hsum = warp_sum(hs), gmax = warp_max(gm);
        __syncwarp();
        if (hsum > 0.f)
            for (int j = lane; j < L; j += 32) as[j] /= hsum;
        __syncwarp();

        Grid grid;
        grid.D = D;
        grid.NB = NB;
        grid.dmin = prm.dmin;
        grid.u0 = u0;
        grid.L = L;
        grid.lam2 = lam2;
        grid.gmax = gmax;

        for (int p = p_begin; p < p_end; ++p) {
            const bool faulty = f.faulty && f.faulty[p];
            const int off0 = f.offsets[p];
            const int K = faulty ? 0 : f.offsets[p + 1] - off0;
            if (K > SPL_MAX_PHOTONS) {
                if (lane == 0) {
                    if (status) atomicOr(status, SPL_BATCH_TOO_MANY);
                    f.mu_out[p] = f.var_out[p] = NAN;
                    if (f.argmax) f.argmax[p] = -1;
                    if (f.refl) f.refl[p] = f.bg[p] = NAN;
                }
                continue;
            }
            // C(d) for every candidate, and the photons that reach each block; out-of-range bins are dropped and
            // reported
            const int* pbins = f.bins + off0;
            int nk = 0;
            bool bad = false;
            const float cmax = corr_photon_list(gs, pbins, K, T, cs, bnd, NB, D, L, u0, lane, nk, bad);
            if (bad && lane == 0 && status) atomicOr(status, SPL_BATCH_BAD_BIN);

            Prior pr;
            {
                float w = 0.f, m = 0.f, v = 1.f;
                if (lane < 9) {
                    w = seqs[sidx].prm.nu[lane];
                    const int y = p / prm.W, x = p - y * prm.W;
                    const int yy = y + lane / 3 - 1, xx = x + lane % 3 - 1;
                    bool info = false;
                    if (yy >= 0 && yy < prm.H && xx >= 0 && xx < prm.W) {
                        const int i = yy * prm.W + xx;
                        info = (f.present_in ? f.present_in[i] != 0 : true) && !(f.faulty && f.faulty[i]);
                        if (info) {
                            m = f.mu_in[i];
                            v = f.var_in[i] + prm.sigma_rw2;
                        }
                    }
                    if (!info) {
                        m = flat_m;
                        v = flat_v + prm.sigma_rw2;
                    }
                }
                build_prior(w, m, v, lane, pr);
            }

            int bidx;
            float mu, var;
            const bool empty_row = nk == 0;
            const int ub_b = block_bounds(
                grid, pr, ubs, [&](int b) { return empty_row ? 0.f : grid.lam2 * grid.gmax * bnd[b] * 1.0001f; },
                lane);
            posterior_eval(grid, pr, cmax, cs, ubs, ub_b,
                           [&]() {  // rare fallback: C again, in the same order
                               int n2 = 0;
                               bool b2 = false;
                               corr_photon_list(gs, pbins, K, T, cs, nullptr, NB, D, L, u0, lane, n2, b2);
                           },
                           lane, bidx, mu, var);
            if (lane == 0) {
                f.mu_out[p] = mu;
                f.var_out[p] = var;
                if (f.argmax) f.argmax[p] = prm.dmin + bidx;
            }

            if (f.refl) {
                float r = 0.f, b = 0.f;
                const bool present = f.present_now ? f.present_now[p] != 0 : true;
                const float Kf = static_cast<float>(nk);
                if (faulty) {
                    r = b = 0.f;
                } else if (!present || nk == 0 || !(hsum > 0.f)) {
                    r = 0.f;
                    b = Kf / static_cast<float>(T);
                } else {
                    const int t0 = min(max(__float2int_rn(mu) - prm.peak, 0), T - L);
                    __syncwarp();
                    float* zwin = cs;
                    for (int j = lane; j < SPL_MAX_TAPS; j += 32) zwin[j] = 0.f;
                    __syncwarp();
                    window_photons(pbins, K, T, t0, L, zwin, lane);
                    __syncwarp();
                    float zj[SPL_MAX_TAPS / 32], aj[SPL_MAX_TAPS / 32];
#pragma unroll
                    for (int q = 0; q < SPL_MAX_TAPS / 32; ++q) {
                        const int j = lane + 32 * q;
                        zj[q] = j < L ? zwin[j] : 0.f;
                        aj[q] = j < L ? as[j] : 0.f;
                    }
                    intensity_mle<SPL_MAX_TAPS / 32>(zj, aj, Kf, L, T, hsum, r, b);
                }
                if (lane == 0) {
                    f.refl[p] = r;
                    f.bg[p] = b;
                }
            }
            __syncwarp();
        }
    }
}

// Device address of g_noalloc_scratch, looked up once per device (with that device current).
constexpr int kMaxDevices = 64;
unsigned* g_scratch_addr[kMaxDevices] = {};
std::mutex g_scratch_mu;

cudaError_t scratch_address(int dev, unsigned** out) {
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_scratch_mu);
    if (!g_scratch_addr[dev]) {
        void* ptr = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_addr[dev] = static_cast<unsigned*>(ptr);
    }
    *out = g_scratch_addr[dev];
    return cudaSuccess;
}

}  // namespace
}  // namespace spl

using namespace spl;

extern "C" spl_status spl_batch_step_noalloc(const spl_seq_desc* descs_host, const spl_seq_desc* descs_dev, int nseq,
                                             int tile, uint32_t* status, void* stream) {
    set_error("%s", "");
    if (!descs_host || !descs_dev) {
        set_error("descs_host and descs_dev are required");
        return SPL_EINVAL;
    }
    if (nseq < 1 || nseq > SPL_NOALLOC_MAX_SEQ) {
        set_error("nseq = %d is outside [1, %d], the capacity of the fixed scratch array of "
                  "spl_batch_step_noalloc", nseq, SPL_NOALLOC_MAX_SEQ);
        return SPL_EINVAL;
    }
    if (tile < 1 || tile > 4096) {
        set_error("tile = %d must be in [1, 4096]", tile);
        return SPL_EINVAL;
    }
    int maxD = 1;
    unsigned long long units = 0;
    for (int s = 0; s < nseq; ++s) {
        const spl_seq_desc& d = descs_host[s];
        spl_status st = check_params(&d.prm, true);
        if (st != SPL_OK) {
            char msg[600];
            snprintf(msg, sizeof(msg), "sequence %d: %s", s, spl_last_error());
            set_error("%s", msg);
            return st;
        }
        const spl_seq_frame& f = d.f;
        if (!f.h || !f.offsets || !f.bins || !f.mu_in || !f.var_in || !f.mu_out || !f.var_out) {
            set_error("sequence %d: h, offsets, bins, mu_in, var_in, mu_out and var_out are required", s);
            return SPL_EINVAL;
        }
        if (f.mu_out == f.mu_in || f.var_out == f.var_in || f.mu_out == f.var_in || f.var_out == f.mu_in) {
            set_error("sequence %d: outputs must not alias the previous-frame state", s);
            return SPL_EINVAL;
        }
        if ((f.refl == nullptr) != (f.bg == nullptr)) {
            set_error("sequence %d: give both refl and bg or neither", s);
            return SPL_EINVAL;
        }
        maxD = maxD > d.prm.dmax - d.prm.dmin + 1 ? maxD : d.prm.dmax - d.prm.dmin + 1;
        units += (static_cast<unsigned long long>(d.prm.H) * d.prm.W + tile - 1) / tile;
    }
    if (units >= (1ull << 32) - 1) {
        set_error("too many work units (%llu) for one call: use a larger tile", units);
        return SPL_EUNSUPPORTED;
    }
    int dev = 0, nsm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    unsigned* scratch = nullptr;
    if (e == cudaSuccess) e = scratch_address(dev, &scratch);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const NSlice sl = make_nslice(maxD);
    const size_t per_warp = sizeof(float) * static_cast<size_t>(sl.words);
    int wpc = 0, per_sm = 0;
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_noalloc_batch, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024);
    for (int w = 8; w >= 1 && e == cudaSuccess && wpc == 0; --w) {
        if (per_warp * w > 220 * 1024) continue;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_noalloc_batch, w * 32, per_warp * w);
        if (e == cudaSuccess && per_sm > 0) wpc = w;
    }
    if (e == cudaSuccess && wpc == 0) e = cudaErrorInvalidConfiguration;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (e == cudaSuccess) {
        k_noalloc_setup<<<1, 32, 0, s>>>(descs_dev, nseq, tile, scratch);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
        k_noalloc_batch<<<per_sm * nsm, wpc * 32, per_warp * wpc, s>>>(descs_dev, nseq, tile, scratch, status, sl,
                                                                         maxD);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) {
        set_error("spl_batch_step_noalloc: %s", cudaGetErrorString(e));
        return SPL_ECUDA;
    }
    return SPL_OK;
}
