// Batched online filter over many independent sequences whose photon data are time-of-arrival lists (CSR),
// in one persistent launch per frame and size class.
//
// Work units are (sequence, tile of consecutive pixels), ordered by decreasing estimated cost (pixels times
// candidate depths) so the largest are taken first. Each warp repeatedly takes the next unit from a device
// work-queue head (one atomicAdd by lane 0), loads that sequence's IRF into its own shared-memory tables,
// and processes the tile's pixels one at a time with the same per-pixel arithmetic as the histogram kernel
// (pixel.cuh, posterior.cuh). The data term uses the photon-sum form of Eq. beta_div2:
// C(d) = sum_k g[y_k - d + peak], formed lane = tap from the list in global memory (corr_photon_list, photons.cuh).
// Sequences are split into two size classes when that raises the shorter ones' resident warps (their shared-memory
// slices are sized for their own longest candidate grid); each class has its own launch and queue head. The queue
// heads are reset by one memset on the launch stream before every step, so a step is a memset node and one or two
// kernel nodes in a CUDA graph. The plan (unit list, descriptor tables, queue heads, status word) is
// allocated once at creation; nothing is allocated per step.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "pixel.cuh"
#include "photons.cuh"
#include "posterior.cuh"
#include "spl_internal.h"

namespace spl {
namespace {

using namespace px;

// Device descriptor of one sequence for one frame: parameters plus the caller's pointers.
struct DevSeq {
    spl_params prm;
    spl_seq_frame f;
};

struct Unit {
    int seq, p0, p1, pad;
};

// Per-warp shared-memory slice for a batch whose largest candidate count is maxD (offsets in words).
struct BSlice {
    int gs, as, bnd, ubs, cs, words;  // taps h^beta, template, per-block photon counts, bounds, C
};

__host__ __device__ __forceinline__ int r4(int x) { return (x + 3) & ~3; }

__host__ __device__ __forceinline__ BSlice make_bslice(int maxD) {
    BSlice s;
    const int nb = (maxD + 31) / 32;
    s.gs = 0;
    s.as = s.gs + SPL_MAX_TAPS + 4;
    s.bnd = s.as + SPL_MAX_TAPS;
    s.ubs = s.bnd + r4(nb);
    s.cs = s.ubs + r4(nb);
    s.words = s.cs + (nb * 32 > SPL_MAX_TAPS ? nb * 32 : SPL_MAX_TAPS);  // cs doubles as the window histogram
    return s;
}

__global__ void __launch_bounds__(256) k_batch(const DevSeq* __restrict__ seqs, const Unit* __restrict__ units,
                                               int nunits, unsigned* __restrict__ head, unsigned* __restrict__ status,
                                               BSlice sl) {
    extern __shared__ __align__(16) float dyn[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    float* base = dyn + static_cast<size_t>(warp) * sl.words;
    float* gs = base + sl.gs;
    float* as = base + sl.as;
    float* bnd = base + sl.bnd;
    float* ubs = base + sl.ubs;
    float* cs = base + sl.cs;

    while (true) {
        unsigned u = 0;
        if (lane == 0) u = atomicAdd(head, 1u);
        u = __shfl_sync(0xffffffffu, u, 0);
        if (u >= static_cast<unsigned>(nunits)) break;
        const Unit un = units[u];
        const DevSeq& sq = seqs[un.seq];
        const spl_params prm = sq.prm;
        const spl_seq_frame f = sq.f;
        const int T = prm.T, L = prm.L, D = prm.dmax - prm.dmin + 1, NB = (D + 31) >> 5;
        const int u0 = prm.dmin - prm.peak;
        const float lam2 = static_cast<float>((static_cast<double>(prm.beta) + 1.0) / prm.beta) * kLog2e;
        const float flat_m = 0.5f * static_cast<float>(prm.dmin + prm.dmax);
        const double span = static_cast<double>(prm.dmax - prm.dmin);
        const float flat_v = static_cast<float>(span * span / 12.0);

        // IRF tables of this sequence: g = h^beta and the normalised template h / sum(h)
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

        for (int p = un.p0; p < un.p1; ++p) {
            const bool faulty = f.faulty && f.faulty[p];
            const int off0 = f.offsets[p];
            const int K = faulty ? 0 : f.offsets[p + 1] - off0;
            if (K > SPL_MAX_PHOTONS) {
                if (lane == 0) {
                    atomicOr(status, SPL_BATCH_TOO_MANY);
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
            if (bad && lane == 0) atomicOr(status, SPL_BATCH_BAD_BIN);

            // prior from the previous frame's states of this sequence (Eq. predict)
            Prior pr;
            {
                float w = 0.f, m = 0.f, v = 1.f;
                if (lane < 9) {
                    w = seqs[un.seq].prm.nu[lane];  // global read: no local copy of the array
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

            const bool empty_row = nk == 0;
            int bidx;
            float mu, var;
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

            // background and reflectivity (Sec. II-E) from the photons in the template window
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
                    float* zwin = cs;  // the candidate scratch is free again: window histogram
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

}  // namespace
}  // namespace spl

// ------------------------------------------------------------------------------------------------------------
// Host side of the plan
// ------------------------------------------------------------------------------------------------------------

struct spl_batch {
    int device = 0, nseq = 0, nslots = 0, nsm = 0;
    std::vector<spl_params> prm;
    spl::DevSeq* d_seqs = nullptr;   // [nslots][nseq]
    spl::Unit* d_units = nullptr;    // [max units]
    unsigned* d_head = nullptr;      // [nslots][2] work-queue heads, one per class
    unsigned* d_status = nullptr;    // condition flags
    int max_units = 0, nunits = 0, tile = 32;
    // Two classes of sequences by candidate count, each with its own per-warp slice and launch geometry: the
    // sequences with at most split_D candidates would otherwise carry the slice sized for the longest grid and
    // keep fewer warps resident. nclass = 1 when the split would not raise their resident warps.
    int nclass = 1, split_D = 0;
    int ubeg[2] = {0, 0}, ucnt[2] = {0, 0};  // each class's range of the unit list
    int maxD[2] = {1, 1};                    // each class's longest candidate grid
    int wpc[2] = {8, 8}, ctas[2] = {0, 0};
    size_t smem[2] = {0, 0};
    spl::BSlice sl[2];
    std::vector<int> slot_set;       // slot has been filled by spl_batch_set
};

namespace spl {
namespace {

constexpr int kTiles[] = {8, 16, 32, 64, 128};

// The work units of the plan, class 0 (more than split_D candidates) first, then class 1, each in decreasing cost
// order (candidates per pixel); cnt receives the two classes' unit counts.
std::vector<Unit> make_units(const std::vector<spl_params>& prm, int tile, int split_D, int* cnt) {
    std::vector<Unit> u;
    std::vector<std::pair<long long, int>> order;  // (cost per pixel, seq)
    for (int s = 0; s < static_cast<int>(prm.size()); ++s)
        order.push_back({static_cast<long long>(prm[s].dmax - prm[s].dmin + 1), s});
    std::stable_sort(order.begin(), order.end(), [](const auto& a, const auto& b) { return a.first > b.first; });
    cnt[0] = cnt[1] = 0;
    for (const auto& o : order) {
        const int s = o.second;
        const int P = prm[s].H * prm[s].W;
        const int c = o.first > split_D ? 0 : 1;
        for (int p0 = 0; p0 < P; p0 += tile) {
            u.push_back(Unit{s, p0, std::min(P, p0 + tile), 0});
            ++cnt[c];
        }
    }
    return u;
}

cudaError_t upload_units(spl_batch* b, int tile) {
    int cnt[2];
    std::vector<Unit> u = make_units(b->prm, tile, b->nclass > 1 ? b->split_D : 0, cnt);
    if (static_cast<int>(u.size()) > b->max_units) return cudaErrorInvalidValue;
    cudaError_t e = cudaMemcpy(b->d_units, u.data(), sizeof(Unit) * u.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return e;
    b->nunits = static_cast<int>(u.size());
    b->ubeg[0] = 0;
    b->ucnt[0] = cnt[0];
    b->ubeg[1] = cnt[0];
    b->ucnt[1] = cnt[1];
    b->tile = tile;
    return cudaSuccess;
}

// One step: the two queue heads of the slot cleared by one memset, then one persistent launch per class (a memset
// node and one or two kernel nodes in a CUDA graph).
cudaError_t launch_batch(spl_batch* b, int slot, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(b->d_head + 2 * slot, 0, 2 * sizeof(unsigned), s);
    for (int c = 0; c < b->nclass && e == cudaSuccess; ++c) {
        if (b->ucnt[c] == 0) continue;
        k_batch<<<b->ctas[c], b->wpc[c] * 32, b->smem[c], s>>>(b->d_seqs + static_cast<size_t>(slot) * b->nseq,
                                                               b->d_units + b->ubeg[c], b->ucnt[c],
                                                               b->d_head + 2 * slot + c, b->d_status, b->sl[c]);
        e = cudaGetLastError();
    }
    return e;
}

// Warps per CTA that maximise resident warps for slice sl (one wave of resident CTAs); best = warps per SM.
cudaError_t batch_geometry(const BSlice& sl, int nsm, int& wpc, int& ctas, size_t& smem, int& best) {
    const size_t per_warp = sizeof(float) * static_cast<size_t>(sl.words);
    best = 0;
    for (int w = 8; w >= 1; --w) {
        if (per_warp * w > 220 * 1024) continue;
        int per_sm = 0;
        const cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batch, w * 32, per_warp * w);
        if (e != cudaSuccess) return e;
        if (per_sm * w > best) {
            best = per_sm * w;
            wpc = w;
            ctas = per_sm * nsm;
            smem = per_warp * w;
        }
    }
    return best == 0 ? cudaErrorInvalidConfiguration : cudaSuccess;
}

void free_plan(spl_batch* b) {
    if (!b) return;
    cudaFree(b->d_seqs);
    cudaFree(b->d_units);
    cudaFree(b->d_head);
    cudaFree(b->d_status);
    delete b;
}

}  // namespace
}  // namespace spl

using namespace spl;

extern "C" {

spl_status spl_batch_create(const spl_params* prms, int nseq, int nslots, spl_batch** out) {
    set_error("%s", "");
    if (!out) {
        set_error("out is NULL");
        return SPL_EINVAL;
    }
    *out = nullptr;
    if (!prms || nseq < 1 || nslots < 1) {
        set_error("need prms, nseq >= 1 and nslots >= 1 (got nseq %d, nslots %d)", nseq, nslots);
        return SPL_EINVAL;
    }
    int maxD = 1;
    long long max_units = 0;
    std::vector<int> Ds;
    for (int s = 0; s < nseq; ++s) {
        spl_status st = check_params(&prms[s], true);
        if (st != SPL_OK) {
            char msg[600];
            snprintf(msg, sizeof(msg), "sequence %d: %s", s, spl_last_error());
            set_error("%s", msg);
            return st;
        }
        maxD = std::max(maxD, prms[s].dmax - prms[s].dmin + 1);
        Ds.push_back(prms[s].dmax - prms[s].dmin + 1);
        max_units += (static_cast<long long>(prms[s].H) * prms[s].W + kTiles[0] - 1) / kTiles[0];
    }
    if (max_units > (1LL << 30)) {
        set_error("too many pixels in the batch");
        return SPL_EUNSUPPORTED;
    }
    spl_batch* b = new spl_batch();
    b->nseq = nseq;
    b->nslots = nslots;
    b->prm.assign(prms, prms + nseq);
    b->slot_set.assign(nslots, 0);
    b->max_units = static_cast<int>(max_units);
    // class 1: the sequences with at most half the longest grid's candidates, sliced for their own longest
    b->split_D = maxD / 2;
    int maxD1 = 0;
    for (int d : Ds)
        if (d <= b->split_D) maxD1 = std::max(maxD1, d);
    b->maxD[0] = maxD;
    b->maxD[1] = std::max(maxD1, 1);
    b->sl[0] = make_bslice(b->maxD[0]);
    b->sl[1] = make_bslice(b->maxD[1]);
    b->nclass = maxD1 > 0 ? 2 : 1;
    cudaError_t e = cudaGetDevice(&b->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&b->nsm, cudaDevAttrMultiProcessorCount, b->device);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_seqs, sizeof(DevSeq) * static_cast<size_t>(nseq) * nslots);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_units, sizeof(Unit) * static_cast<size_t>(b->max_units));
    if (e == cudaSuccess) e = cudaMalloc(&b->d_head, 2 * sizeof(unsigned) * nslots);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_status, sizeof(unsigned));
    if (e == cudaSuccess) e = cudaMemset(b->d_status, 0, sizeof(unsigned));
    if (e == cudaSuccess) e = cudaMemset(b->d_seqs, 0, sizeof(DevSeq) * static_cast<size_t>(nseq) * nslots);
    // launch geometry per class: warps per CTA maximising resident warps, one wave of resident CTAs; the split is
    // kept only where it raises the short sequences' resident warps
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_batch, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024);
    int best0 = 0, best1 = 0;
    if (e == cudaSuccess) e = batch_geometry(b->sl[0], b->nsm, b->wpc[0], b->ctas[0], b->smem[0], best0);
    if (e == cudaSuccess && b->nclass == 2) {
        e = batch_geometry(b->sl[1], b->nsm, b->wpc[1], b->ctas[1], b->smem[1], best1);
        if (e == cudaSuccess && best1 <= best0) b->nclass = 1;
    }
    if (e == cudaSuccess) e = upload_units(b, 32);
    if (e != cudaSuccess) {
        const bool oom = e == cudaErrorMemoryAllocation;
        set_error("spl_batch_create: %s", cudaGetErrorString(e));
        free_plan(b);
        return oom ? SPL_ENOMEM : SPL_ECUDA;
    }
    *out = b;
    return SPL_OK;
}

void spl_batch_destroy(spl_batch* b) { free_plan(b); }

spl_status spl_batch_set(spl_batch* b, int slot, const spl_seq_frame* frames) {
    set_error("%s", "");
    if (!b || !frames || slot < 0 || slot >= b->nslots) {
        set_error("invalid plan, frames or slot %d", slot);
        return SPL_EINVAL;
    }
    std::vector<DevSeq> d(b->nseq);
    for (int s = 0; s < b->nseq; ++s) {
        const spl_seq_frame& f = frames[s];
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
        d[s].prm = b->prm[s];
        d[s].f = f;
    }
    cudaError_t e = cudaMemcpy(b->d_seqs + static_cast<size_t>(slot) * b->nseq, d.data(), sizeof(DevSeq) * d.size(),
                               cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        set_error("spl_batch_set: %s", cudaGetErrorString(e));
        return SPL_ECUDA;
    }
    b->slot_set[slot] = 1;
    return SPL_OK;
}

spl_status spl_batch_step(spl_batch* b, int slot, void* stream) {
    if (!b || slot < 0 || slot >= b->nslots) {
        set_error("invalid plan or slot %d", slot);
        return SPL_EINVAL;
    }
    if (!b->slot_set[slot]) {
        set_error("slot %d has no frame descriptors (call spl_batch_set first)", slot);
        return SPL_EINVAL;
    }
    const cudaError_t e = launch_batch(b, slot, static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) {
        set_error("spl_batch_step: %s", cudaGetErrorString(e));
        return SPL_ECUDA;
    }
    return SPL_OK;
}

spl_status spl_batch_tune(spl_batch* b, int slot, void* stream) {
    if (!b || slot < 0 || slot >= b->nslots || !b->slot_set[slot]) {
        set_error("invalid plan or slot %d (filled by spl_batch_set?)", slot);
        return SPL_EINVAL;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaEvent_t e0, e1;
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    int best_tile = b->tile;
    float best_ms = INFINITY;
    for (int t : kTiles) {
        if (e != cudaSuccess) break;
        e = upload_units(b, t);
        if (e == cudaSuccess) e = launch_batch(b, slot, s);  // warm-up
        float tot = 0.f;
        for (int rep = 0; rep < 3 && e == cudaSuccess; ++rep) {
            e = cudaEventRecord(e0, s);
            if (e == cudaSuccess) e = launch_batch(b, slot, s);
            if (e == cudaSuccess) e = cudaEventRecord(e1, s);
            if (e == cudaSuccess) e = cudaEventSynchronize(e1);
            float ms = 0.f;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
            tot += ms;
        }
        if (e == cudaSuccess && tot < best_ms) {
            best_ms = tot;
            best_tile = t;
        }
    }
    if (e == cudaSuccess) e = upload_units(b, best_tile);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess) {
        set_error("spl_batch_tune: %s", cudaGetErrorString(e));
        return SPL_ECUDA;
    }
    return SPL_OK;
}

spl_status spl_batch_info(const spl_batch* b, int* tile, int* units, int* ctas, int* warps_per_cta) {
    if (!b) {
        set_error("plan is NULL");
        return SPL_EINVAL;
    }
    if (tile) *tile = b->tile;
    if (units) *units = b->nunits;
    if (ctas) *ctas = b->ctas[0];
    if (warps_per_cta) *warps_per_cta = b->wpc[0];
    return SPL_OK;
}

spl_status spl_batch_class_info(const spl_batch* b, int cls, int* nclass, int* units, int* ctas, int* warps_per_cta,
                                int* max_candidates) {
    if (!b) {
        set_error("plan is NULL");
        return SPL_EINVAL;
    }
    if (cls < 0 || cls >= b->nclass) {
        set_error("spl_batch_class_info: class %d of a plan with %d", cls, b->nclass);
        return SPL_EINVAL;
    }
    if (nclass) *nclass = b->nclass;
    if (units) *units = b->ucnt[cls];
    if (ctas) *ctas = b->ctas[cls];
    if (warps_per_cta) *warps_per_cta = b->wpc[cls];
    if (max_candidates) *max_candidates = b->maxD[cls];
    return SPL_OK;
}

spl_status spl_batch_status(spl_batch* b, uint32_t* flags) {
    if (!b || !flags) {
        set_error("plan or flags is NULL");
        return SPL_EINVAL;
    }
    unsigned v = 0;
    cudaError_t e = cudaMemcpy(&v, b->d_status, sizeof(unsigned), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemset(b->d_status, 0, sizeof(unsigned));
    if (e != cudaSuccess) {
        set_error("spl_batch_status: %s", cudaGetErrorString(e));
        return SPL_ECUDA;
    }
    *flags = v;
    return SPL_OK;
}

}  // extern "C"
