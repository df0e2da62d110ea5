// Mixed-precision robust data term on the 5th-generation tensor cores (tcgen05 + TMA, sm_103a).
//
// C(d) = sum_j g_j z[d - peak + j] (Eq. beta_div2, histogram form) for 128 pixels x 64 candidates per MMA tile,
// written as a banded-Toeplitz product: with a0 = (dmin - peak) rounded down to a multiple of 8 and
// delta = dmin - peak - a0, candidate tile t (candidates 64 t .. 64 t + 63) is
//     C[p, 64 t + n] = sum_k Z[p, a0 + 64 t + k] G[k, n],   G[k, n] = g[k - n - delta] (0 outside 0..L-1),
// for k = 0 .. Kw - 1, Kw = 64 + L - 1 + delta rounded up to 16. A = the counts window (FP16; integer counts up
// to 2048 are exact), B = G, the same for every tile. To keep FP32-level accuracy with 16-bit operands, G is
// scaled by 2^15 and split into an FP16 high part and an FP16 low part (the rounding residual); both products
// accumulate into one FP32 accumulator in tensor memory (the products of exact counts and FP16 values are exact
// in FP32), and the epilogue multiplies by 2^-15. The relative error of each g is then about 2^-22.
//
// Pipeline (one persistent CTA per SM, 6 warps):
//   warp 4 (TMA producer): streams 64-bin slabs of the 128-pixel block (16 KB, 128-byte swizzled; the tensor map
//     zero-fills bins >= T and pixels >= P) into a ring of 6 slabs. A candidate tile's window spans
//     ceil(Kw / 64) consecutive slabs and consecutive tiles share all but one, so each slab is loaded once.
//   warp 5 (MMA issuer, one lane): per candidate tile, Kw / 16 K-steps x 2 (high and low part of G) into one of
//     two TMEM accumulators (128 lanes x 64 fp32 columns each); tcgen05.commit releases the accumulator to the
//     epilogue and the oldest slab back to the producer.
//   warps 0-3 (epilogue): thread = pixel = TMEM lane; tcgen05.ld of its 64 candidates, then the per-candidate work.
// Every wait on an mbarrier is bounded; one that runs out sets a status flag and all roles stop at their next
// wait; tensor memory is released before the CTA exits.
#include <math.h>
#include <stdint.h>

#include "spl_internal.h"
#include "tc_common.cuh"

namespace spl {
namespace {

using namespace tc;

constexpr int kM = 128;               // pixels per block (MMA M, TMEM lanes)
constexpr int kN = 64;                // candidates per tile (MMA N, TMEM columns per accumulator)
constexpr int kSlab = 64;             // bins per slab (128-byte rows)
constexpr int kRing = 6;              // slabs in flight
constexpr int kMaxBSlabs = 4;         // ceil(208 / 64): largest window (L = 128, delta = 7)
constexpr int kThreads = 192;         // warps 0-3 epilogue, warp 4 producer, warp 5 MMA
constexpr float kScale = 32768.f;     // 2^15
constexpr size_t kSlabBytes = kM * kSlab * 2;        // 16 KB
constexpr size_t kBSlabBytes = kN * kSlab * 2;       // 8 KB
constexpr size_t kSmemBytes = 1024 + kRing * kSlabBytes + 2 * kMaxBSlabs * kBSlabBytes;
constexpr uint32_t kIdesc = idesc_f16(kM, kN);

struct TcArgs {
    int P, T, L, D, a0, delta, kw, ntiles, nslab, npt;
    float beta;
    const float* h;
    float* cost;      // [P][D] (nullable)
    int* argmax;      // [P] (nullable): dmin + index of the largest C
    int dmin;
    unsigned* status; // bit 0: an mbarrier wait ran out
};

__global__ void __launch_bounds__(kThreads, 1) k_cost_tc(const __grid_constant__ CUtensorMap zmap, const TcArgs a) {
    extern __shared__ unsigned char smem_raw[];
    __shared__ __align__(8) unsigned long long bar[2 * kRing + 5];
    __shared__ uint32_t tmem_base;
    __shared__ int abort_flag;

    // 1024-byte aligned operand area: A ring, then B high / B low (each kMaxBSlabs slabs of 64 x 64)
    const unsigned base = (smem_u32(smem_raw) + 1023u) & ~1023u;
    unsigned char* gbase = smem_raw + (base - smem_u32(smem_raw));
    const unsigned ringA = base;
    const unsigned Bhi = base + kRing * kSlabBytes;
    const unsigned Blo = Bhi + kMaxBSlabs * kBSlabBytes;
    const unsigned full0 = smem_u32(&bar[0]), empty0 = smem_u32(&bar[kRing]);
    const unsigned accf0 = smem_u32(&bar[2 * kRing]), acce0 = smem_u32(&bar[2 * kRing + 2]);
    const unsigned drain = smem_u32(&bar[2 * kRing + 4]);
    volatile int* stop = &abort_flag;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    // ---- set-up: tensor memory (two accumulators), barriers, the Toeplitz operand (high and low parts) ----
    if (warp == 5) {
        tmem_alloc(smem_u32(&tmem_base), 2 * kN);
    }
    if (tid == 0) {
        for (int i = 0; i < kRing; ++i) {
            mbar_init(full0 + 8 * i, 1);   // producer's expect_tx arrive + TMA bytes
            mbar_init(empty0 + 8 * i, 1);  // MMA commit
        }
        for (int i = 0; i < 2; ++i) {
            mbar_init(accf0 + 8 * i, 1);   // MMA commit
            mbar_init(acce0 + 8 * i, 4);   // one arrive per epilogue warp
        }
        mbar_init(drain, 1);
        abort_flag = 0;
    }
    const int nbs = (a.kw + kSlab - 1) / kSlab;
    for (int e = tid; e < nbs * kSlab * kN; e += kThreads) {
        const int k = e / kN, n = e - k * kN;
        const int j = k - n - a.delta;
        float g = 0.f;
        if (k < a.kw && j >= 0 && j < a.L) {
            const float hj = a.h[j];
            g = hj > 0.f ? powf(hj, a.beta) * kScale : 0.f;
        }
        const __half hi = __float2half_rn(g);
        const __half lo = __float2half_rn(g - __half2float(hi));
        const int b = k / kSlab, kk = k - b * kSlab;
        const unsigned off = b * static_cast<unsigned>(kBSlabBytes) + swz_offset(n, kk);
        *reinterpret_cast<__half*>(gbase + (Bhi - base) + off) = hi;
        *reinterpret_cast<__half*>(gbase + (Blo - base) + off) = lo;
    }
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");  // generic writes of B -> MMA reads
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = tmem_base;
    const int slabs_per_block = a.ntiles + a.nslab - 1;

    if (warp == 4) {
        // ================= TMA producer =================
        if (lane == 0) {
            unsigned cnt = 0;
            bool ok = true;
            for (int pt = blockIdx.x; pt < a.npt && ok && !*stop; pt += gridDim.x) {
                for (int s = 0; s < slabs_per_block; ++s, ++cnt) {
                    const unsigned slot = cnt % kRing, fill = cnt / kRing;
                    if (fill > 0 && !(ok = wait_bounded(empty0 + 8 * slot, (fill - 1) & 1u, stop, a.status))) break;
                    mbar_expect_tx(full0 + 8 * slot, static_cast<unsigned>(kSlabBytes));
                    tma_load_2d(ringA + slot * static_cast<unsigned>(kSlabBytes), &zmap, a.a0 + kSlab * s, pt * kM,
                                full0 + 8 * slot);
                }
            }
            // copies still in flight land before the CTA may exit (bounded; in normal runs they have all landed)
            for (unsigned i = cnt > kRing ? cnt - kRing : 0; i < cnt; ++i)
                wait_quiet(full0 + 8 * (i % kRing), (i / kRing) & 1u);
        }
    } else if (warp == 5) {
        // ================= MMA issuer =================
        if (lane == 0) {
            unsigned slab0 = 0;  // global index of the first slab of the current block
            unsigned waited = 0; // slabs whose "full" barrier has been waited for
            unsigned g = 0;      // global tile counter (accumulator parity)
            bool ok = true;
            for (int pt = blockIdx.x; pt < a.npt && ok; pt += gridDim.x) {
                for (int t = 0; t < a.ntiles && ok; ++t, ++g) {
                    const unsigned acc = g & 1u, use = g >> 1;
                    if (use > 0 && !(ok = wait_bounded(acce0 + 8 * acc, (use - 1) & 1u, stop, a.status))) break;
                    fence_after();
                    const uint32_t d = tmem + acc * kN;
                    for (int j = 0; j < a.nslab && ok; ++j) {
                        const unsigned gs = slab0 + t + j;
                        while (waited <= gs && ok) {
                            ok = wait_bounded(full0 + 8 * (waited % kRing), (waited / kRing) & 1u, stop, a.status);
                            ++waited;
                        }
                        if (!ok) break;
                        fence_after();
                        const unsigned aslab = ringA + (gs % kRing) * static_cast<unsigned>(kSlabBytes);
                        const int k_end = min(kSlab * (j + 1), a.kw);
                        for (int k = kSlab * j; k < k_end; k += 16) {
                            const unsigned koff = (k - kSlab * j) * 2;  // bytes within the 128-byte row
                            const uint64_t ad = desc_sw128(aslab + koff);
                            const uint64_t bh = desc_sw128(Bhi + j * static_cast<unsigned>(kBSlabBytes) + koff);
                            const uint64_t bl = desc_sw128(Blo + j * static_cast<unsigned>(kBSlabBytes) + koff);
                            mma_f16<kIdesc>(d, ad, bh, k > 0 ? 1u : 0u);
                            mma_f16<kIdesc>(d, ad, bl, 1u);
                        }
                    }
                    if (!ok) break;
                    mma_commit(accf0 + 8 * acc);
                    // the first slab of this tile's window is not needed by later tiles of the block
                    mma_commit(empty0 + 8 * ((slab0 + t) % kRing));
                }
                // the block's trailing slabs are released too
                for (int j = 1; j < a.nslab && ok; ++j) mma_commit(empty0 + 8 * ((slab0 + a.ntiles - 1 + j) % kRing));
                slab0 += slabs_per_block;
            }
            // every MMA this thread issued has completed before tensor memory is released
            mma_commit(drain);
            wait_quiet(drain, 0);
        }
    } else {
        // ================= epilogue: thread = pixel = TMEM lane =================
        unsigned g = 0;
        bool ok = true;
        const uint32_t lane_addr = tmem + (static_cast<uint32_t>(warp * 32) << 16);
        for (int pt = blockIdx.x; pt < a.npt && ok; pt += gridDim.x) {
            const int p = pt * kM + tid;
            float best = -INFINITY;
            int bidx = 0;
            for (int t = 0; t < a.ntiles; ++t, ++g) {
                const unsigned acc = g & 1u, use = g >> 1;
                // the warp leaves together: tcgen05.ld below is warp-collective
                ok = __all_sync(0xffffffffu, wait_bounded(accf0 + 8 * acc, use & 1u, stop, a.status));
                if (!ok) break;
                fence_after();
#pragma unroll
                for (int q = 0; q < kN / 16; ++q) {
                    float v[16];
                    tmem_ld16(lane_addr + acc * kN + q * 16, v);
                    tmem_wait_ld();
                    const int c0 = kN * t + 16 * q;
                    if (p < a.P) {
#pragma unroll
                        for (int i = 0; i < 16; ++i) {
                            const float C = v[i] * (1.f / kScale);
                            const int c = c0 + i;
                            if (c < a.D) {
                                if (a.cost) a.cost[static_cast<long long>(p) * a.D + c] = C;
                                if (C > best) {
                                    best = C;
                                    bidx = c;
                                }
                            }
                        }
                    }
                }
                fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(acce0 + 8 * acc);
            }
            if (ok && a.argmax && p < a.P) a.argmax[p] = a.dmin + bidx;
        }
    }
    fence_before();
    __syncthreads();
    if (warp == 5) {
        fence_after();
        tmem_dealloc(tmem, 2 * kN);
    }
}

}  // namespace

// Condition flags of the tensor-core kernels (bit 0: an mbarrier wait ran out); read and cleared by
// spl_tc_status.
__device__ unsigned g_tc_status;

unsigned* tc_status_ptr() {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_tc_status) != cudaSuccess) return nullptr;
    return static_cast<unsigned*>(p);
}

cudaError_t tc_status_read(unsigned* out) {
    cudaError_t e = cudaMemcpyFromSymbol(out, g_tc_status, sizeof(unsigned));
    if (e != cudaSuccess) return e;
    const unsigned zero = 0;
    return cudaMemcpyToSymbol(g_tc_status, &zero, sizeof(unsigned));
}

cudaError_t launch_cost_tc(const spl_params* q, const void* z, long long pitch, const float* h, float* cost,
                           int* argmax, unsigned* status, cudaStream_t s) {
    TcArgs a;
    a.P = q->H * q->W;
    a.T = q->T;
    a.L = q->L;
    a.D = q->dmax - q->dmin + 1;
    const int u0 = q->dmin - q->peak;
    a.a0 = u0 & ~7;
    a.delta = u0 - a.a0;
    a.kw = ((kN + q->L - 1 + a.delta) + 15) & ~15;
    a.ntiles = (a.D + kN - 1) / kN;
    a.nslab = (a.kw + kSlab - 1) / kSlab;
    a.npt = (a.P + kM - 1) / kM;
    a.beta = q->beta;
    a.h = h;
    a.cost = cost;
    a.argmax = argmax;
    a.dmin = q->dmin;
    a.status = status;
    CUtensorMap map;
    cudaError_t e = hist_map(&map, z, pitch, q->T, a.P);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_cost_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(kSmemBytes));
    if (e != cudaSuccess) return e;
    int dev = 0, nsm = 0;
    e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    const int grid = a.npt < nsm ? a.npt : nsm;
    k_cost_tc<<<grid, kThreads, kSmemBytes, s>>>(map, a);
    return cudaGetLastError();
}

}  // namespace spl
