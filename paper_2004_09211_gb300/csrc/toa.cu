// Histograms from photon time-of-arrival lists: z_p[t] = the number of pixel p's photons detected in bin t, the
// histogram on which the histogram form of Eq. beta_div2 (C(d) = z^T s_d^beta) and Eq. lik_bg_poisson are
// written (Sec. II-A: y_{p,n} is the set of a pixel's ToA, binned on the N_T bins of Eq. lik_ideal_poisson).
//
// One warp per pixel, its counters (32-bit, T rounded up to 8 of them) in the warp's slice of shared memory: the
// lanes add the pixel's photons with shared-memory atomics (any order gives the same counts), then write the row
// as uint16 with one coalesced 8-byte store per 4 elements (zeros past the counters), zeroing the slice in the
// same pass for the warp's next pixel. DRAM traffic per pixel: the row written once (2 * pitch bytes) plus its
// photons read once (2 bytes each) and its two offsets.
//
// Device-detected conditions (bits of the status word read by spl_toa_status):
//   bit 0  a photon with a bin >= T was dropped;
//   bit 1  a bin held more than 65535 photons and was written as 65535;
//   bit 2  a pixel's offsets were not 0 <= offsets[p] <= offsets[p + 1] <= nphotons: its row is written as zeros
//          and none of its photons is read.
#include <stdint.h>

#include "spl_internal.h"

namespace spl {

__device__ unsigned g_toa_status;

namespace {

constexpr int kMaxWarps = 8;

__global__ void __launch_bounds__(kMaxWarps * 32) k_toa_hist(const int32_t* __restrict__ offsets,
                                                             const uint16_t* __restrict__ bins, long long nph, int T,
                                                             long long pitch, long long P, uint16_t* __restrict__ out) {
    extern __shared__ uint4 s_cnt4[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, wpc = blockDim.x >> 5;
    const int tw = (T + 7) & ~7;  // counters per warp
    unsigned* cnt = reinterpret_cast<unsigned*>(s_cnt4) + warp * tw;
    uint4* c4 = reinterpret_cast<uint4*>(cnt);
    const int nc4 = tw >> 2;             // groups of four counters (one 8-byte store each)
    const long long n4 = pitch >> 2;     // 8-byte stores per row
    for (int i = lane; i < nc4; i += 32) c4[i] = make_uint4(0u, 0u, 0u, 0u);
    __syncwarp();
    unsigned flags = 0;
    const long long stride = static_cast<long long>(gridDim.x) * wpc;
    // The next pixel's offsets and first 32 photons are loaded while the current one is counted and written, so
    // the two dependent loads (offsets, then bins) of a pixel overlap the previous pixel's work.
    long long p = static_cast<long long>(blockIdx.x) * wpc + warp;
    long long b = 0, e = 0;
    unsigned t0 = 0xffffffffu;  // this lane's first photon of the pixel (none: above every bin)
    if (p < P) {
        b = offsets[p];
        e = offsets[p + 1];
        if (b >= 0 && b <= e && e <= nph && b + lane < e) t0 = bins[b + lane];
    }
    for (; p < P; p += stride) {
        const long long pn = p + stride;
        long long bn = 0, en = 0;
        if (pn < P) {
            bn = offsets[pn];
            en = offsets[pn + 1];
        }
        if (b >= 0 && b <= e && e <= nph) {
            if (b + lane < e) {
                if (t0 < static_cast<unsigned>(T)) atomicAdd(&cnt[t0], 1u);
                else flags |= 1u;
            }
            for (long long k = b + 32 + lane; k < e; k += 32) {
                const unsigned t = bins[k];
                if (t < static_cast<unsigned>(T)) atomicAdd(&cnt[t], 1u);
                else flags |= 1u;
            }
        } else {
            flags |= 4u;
        }
        __syncwarp();
        // the next pixel's first photons, issued before this pixel's row is written
        const unsigned t0n =
            (pn < P && bn >= 0 && bn <= en && en <= nph && bn + lane < en) ? bins[bn + lane] : 0xffffffffu;
        // four counters per lane at unit stride (conflict-free 16-byte shared loads and stores), written as four
        // uint16 with one 8-byte store per lane (coalesced: 256 bytes per warp instruction)
        uint2* o = reinterpret_cast<uint2*>(out + p * pitch);
        for (long long i = nc4 + lane; i < n4; i += 32) o[i] = make_uint2(0u, 0u);
#pragma unroll 4
        for (int i = lane; i < nc4; i += 32) {
            const uint4 a = c4[i];
            c4[i] = make_uint4(0u, 0u, 0u, 0u);
            flags |= (a.x | a.y | a.z | a.w) > 0xffffu ? 2u : 0u;
            o[i] = make_uint2(min(a.x, 0xffffu) | (min(a.y, 0xffffu) << 16),
                              min(a.z, 0xffffu) | (min(a.w, 0xffffu) << 16));
        }
        __syncwarp();
        b = bn;
        e = en;
        t0 = t0n;
    }
    flags = __reduce_or_sync(0xffffffffu, flags);
    if (lane == 0 && flags) atomicOr(&g_toa_status, flags);
}

}  // namespace

cudaError_t toa_status_read(unsigned* out) {
    cudaError_t e = cudaMemcpyFromSymbol(out, g_toa_status, sizeof(unsigned));
    if (e != cudaSuccess) return e;
    const unsigned zero = 0;
    return cudaMemcpyToSymbol(g_toa_status, &zero, sizeof(unsigned));
}

// Warps per CTA: as many as fit in 96 KB of shared memory ((T + 7) & ~7 32-bit counters each), at most 8; a
// persistent grid of the resident CTAs on every SM, or fewer when the frame has fewer pixels.
cudaError_t launch_toa_hist(const int32_t* offsets, const uint16_t* bins, long long nph, int T, long long pitch,
                            long long P, uint16_t* out, cudaStream_t s) {
    const long long slice = 4LL * ((T + 7) & ~7);
    int wpc = static_cast<int>((96 * 1024) / slice);
    wpc = wpc < 1 ? 1 : (wpc > kMaxWarps ? kMaxWarps : wpc);
    const size_t smem = static_cast<size_t>(slice) * wpc;
    cudaError_t e = cudaFuncSetAttribute(k_toa_hist, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(smem));
    if (e != cudaSuccess) return e;
    int dev = 0, nsm = 0, per_sm = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_toa_hist, wpc * 32, smem)) != cudaSuccess)
        return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    const long long need = (P + wpc - 1) / wpc, full = static_cast<long long>(nsm) * per_sm;
    const int grid = static_cast<int>(need < full ? need : full);
    k_toa_hist<<<grid, wpc * 32, smem, s>>>(offsets, bins, nph, T, pitch, P, out);
    return cudaGetLastError();
}

}  // namespace spl
