// The data term of the photon-list kernels (batch.cu, noalloc.cu): C(d) from a pixel's photon time-of-arrival
// list, the photon-sum form of Eq. beta_div2 (a photon in bin y adds g_j = h_j^beta to candidate y - u0 - j for
// every tap j), one warp per pixel.
#pragma once

#include "pixel.cuh"
#include "spl.h"

namespace spl {
namespace px {

// C over every candidate into cs[0 .. 32 NB) from the K photon bins at `bins` (global memory). The list is read in
// coalesced chunks of 32 and each photon, in list order, broadcast to the warp by shuffle; lane l owns taps
// l + 32 k and adds g_j to candidate y - u0 - j. The candidates of one photon are distinct across lanes and taps
// and the warp synchronises between photons, so every C(d) is summed in list order. Bins outside [0, T) are
// skipped (bad: some lane saw one). With bnd, bnd[b] counts the photons whose template window reaches block b of
// 32 candidates (candidates y - u0 - L + 1 .. y - u0 meet it), the data bound of the pruning. Returns max C;
// nk = the photons used.
__device__ __forceinline__ float corr_photon_list(const float* __restrict__ gs, const int* __restrict__ bins, int K,
                                                  int T, float* cs, float* bnd, int NB, int D, int L, int u0, int lane,
                                                  int& nk, bool& bad) {
    constexpr int KG = SPL_MAX_TAPS / 32;
    zero_words(cs, NB * 8, lane);
    if (bnd) zero_words(bnd, (NB + 3) >> 2, lane);
    float g[KG];
#pragma unroll
    for (int k = 0; k < KG; ++k) g[k] = gs[lane + 32 * k];
    const int ntg = (L + 31) >> 5;
    float mx = 0.f;
    int n = 0;
    bool out = false;
    for (int k0 = 0; k0 < K; k0 += 32) {
        int y = -1;
        if (k0 + lane < K) {
            y = bins[k0 + lane];
            if (y < 0 || y >= T) {
                out = true;
                y = -1;
            }
        }
        unsigned m = __ballot_sync(0xffffffffu, y >= 0);
        n += __popc(m);
        while (m) {
            const int ye = __shfl_sync(0xffffffffu, y, __ffs(m) - 1);
            m &= m - 1;
            const int c = ye - u0 - lane;
#pragma unroll
            for (int k = 0; k < KG; ++k) {
                const int ck = c - 32 * k;
                if (k < ntg && static_cast<unsigned>(ck) < static_cast<unsigned>(D)) {
                    const float v = cs[ck] + g[k];
                    cs[ck] = v;
                    mx = fmaxf(mx, v);
                }
            }
            if (bnd) {  // at most five blocks (L <= 128): lane j takes the j-th
                const int clo = max(ye - u0 - L + 1, 0), chi = min(ye - u0, D - 1);
                if (clo <= chi) {
                    const int b = (clo >> 5) + lane;
                    if (b <= (chi >> 5)) bnd[b] += 1.f;
                }
            }
            __syncwarp();
        }
    }
    nk = n;
    bad = __any_sync(0xffffffffu, out);
    return warp_max(mx);
}

// Photons of the list in bins t0 .. t0 + L - 1 into the window histogram zwin[0 .. L) (zeroed by the caller);
// bins outside [0, T) are skipped as in corr_photon_list.
__device__ __forceinline__ void window_photons(const int* __restrict__ bins, int K, int T, int t0, int L, float* zwin,
                                               int lane) {
    for (int k = lane; k < K; k += 32) {
        const int y = bins[k];
        const int j = y - t0;
        if (y >= 0 && y < T && j >= 0 && j < L) atomicAdd(&zwin[j], 1.f);
    }
}

}  // namespace px
}  // namespace spl
