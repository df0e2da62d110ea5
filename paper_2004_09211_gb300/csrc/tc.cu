// Mixed-precision robust data term on the 5th-generation tensor cores (tcgen05, sm_103a).
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
// Shared memory holds both operands in the no-swizzle K-major core-matrix layout (8 rows x 16 bytes per core
// matrix; SBO = 128 bytes between 8-row groups, LBO = bytes between 8-element K chunks). One thread issues the
// MMAs; completion is signalled through an mbarrier (tcgen05.commit); the accumulator (128 lanes x 64 fp32
// columns) is read with tcgen05.ld by the 4 warps, lane = pixel. Waits are bounded: a wait that runs out sets a
// status flag and the CTA stops cleanly (its tensor memory is still released).
#include <cuda_fp16.h>
#include <math.h>
#include <stdint.h>

#include "spl_internal.h"

namespace spl {
namespace {

constexpr int kM = 128;     // pixels per tile (MMA M, TMEM lanes)
constexpr int kN = 64;      // candidates per tile (MMA N, TMEM columns)
constexpr int kMaxKw = 208; // 64 + 127 + 7 rounded up to 16
constexpr float kScale = 32768.f;  // 2^15
constexpr unsigned kSpinLimit = 1u << 26;

__device__ __forceinline__ unsigned smem_u32(const void* p) {
    return static_cast<unsigned>(__cvta_generic_to_shared(p));
}

// Shared-memory matrix descriptor (no swizzle, K-major): start, leading (K) and stride (8-row group) offsets.
__device__ __forceinline__ uint64_t make_desc(unsigned saddr, unsigned lbo, unsigned sbo) {
    uint64_t d = 0;
    d |= static_cast<uint64_t>((saddr & 0x3FFFFu) >> 4);
    d |= static_cast<uint64_t>((lbo & 0x3FFFFu) >> 4) << 16;
    d |= static_cast<uint64_t>((sbo & 0x3FFFFu) >> 4) << 32;
    d |= static_cast<uint64_t>(1) << 46;  // descriptor version for this architecture
    return d;                             // base offset 0, layout type 0 (no swizzle)
}

// Instruction descriptor: FP32 accumulator, FP16 A and B, both K-major, N = 64, M = 128.
constexpr uint32_t kIdesc = (1u << 4) | (static_cast<uint32_t>(kN >> 3) << 17) | (static_cast<uint32_t>(kM >> 4) << 24);

__device__ __forceinline__ void mma_f16(uint32_t tmem, uint64_t a, uint64_t b, uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem),
        "l"(a), "l"(b), "r"(kIdesc), "r"(accumulate));
}

__device__ __forceinline__ void mma_commit(unsigned mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(mbar)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(unsigned mbar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(mbar), "r"(parity)
        : "memory");
    return ok != 0;
}

// 16 consecutive fp32 accumulator columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15}, [%16];\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(smem_u32(smem)), "l"(gmem) : "memory");
}

struct TcArgs {
    const __half* z;  // [P][pitch] FP16 counts
    long long pitch;
    const float* h;
    int P, T, L, D, u0, a0, delta, kw, ntiles;
    float beta;
    float* cost;      // [P][D] (nullable)
    int* argmax;      // [P] (nullable): dmin + index of the largest C
    int dmin;
    unsigned* status; // bit 0: an mbarrier wait ran out
};

__global__ void __launch_bounds__(128, 1) k_cost_tc(const TcArgs a) {
    extern __shared__ __align__(1024) unsigned char smem[];
    __half* As = reinterpret_cast<__half*>(smem);                  // [kw/8][128][8]
    __half* Bh = As + kMaxKw * kM;                                  // [kw/8][64][8]
    __half* Bl = Bh + kMaxKw * kN;
    __shared__ __align__(8) unsigned long long mbar;
    __shared__ uint32_t tmem_base;
    __shared__ int abort_flag;

    const int tid = threadIdx.x, warp = tid >> 5;
    const int p0 = blockIdx.x * kM;
    const int kc = a.kw / 8;  // 8-element K chunks per tile

    // ---- one-time set-up: tensor memory, mbarrier, the Toeplitz operand B (hi and lo parts) ----
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(&tmem_base)),
                     "r"(kN)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(&mbar)) : "memory");
        abort_flag = 0;
    }
    for (int e = tid; e < a.kw * kN; e += blockDim.x) {
        const int k = e / kN, n = e - k * kN;
        const int j = k - n - a.delta;
        float g = 0.f;
        if (j >= 0 && j < a.L) {
            const float hj = a.h[j];
            g = hj > 0.f ? powf(hj, a.beta) * kScale : 0.f;
        }
        const __half hi = __float2half_rn(g);
        const __half lo = __float2half_rn(g - __half2float(hi));
        const int off = (k >> 3) * (kN * 8) + (n >> 3) * 64 + (n & 7) * 8 + (k & 7);
        Bh[off] = hi;
        Bl[off] = lo;
    }
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    const uint32_t tmem = tmem_base;

    const int row = tid;  // this thread's pixel (tile row = TMEM lane)
    const int p = p0 + row;
    float best = -INFINITY;
    int bidx = 0;
    unsigned phase = 0;

    for (int t = 0; t < a.ntiles; ++t) {
        // ---- A window: chunks of 8 bins starting at a0 + 64 t, 128 pixels, core-matrix layout ----
        for (int i = tid; i < kc * kM; i += blockDim.x) {
            const int c = i / kM, r = i - c * kM;
            const int bin = a.a0 + kN * t + 8 * c;
            __half* dst = As + c * (kM * 8) + (r >> 3) * 64 + (r & 7) * 8;
            if (p0 + r < a.P && bin < a.T) {
                cp_async16(dst, a.z + static_cast<long long>(p0 + r) * a.pitch + bin);
            } else {
                *reinterpret_cast<uint4*>(dst) = make_uint4(0u, 0u, 0u, 0u);
            }
        }
        asm volatile("cp.async.wait_all;\n" ::: "memory");
        // bins at or past T inside a loaded chunk are not data: zero them
        if ((a.T & 7) != 0) {
            const int c_last = (a.T - a.a0 - kN * t) >> 3;  // chunk holding bin T (may be out of this tile)
            if (c_last >= 0 && c_last < kc) {
                __half* dst = As + c_last * (kM * 8) + (row >> 3) * 64 + (row & 7) * 8;
                for (int k = (a.T - a.a0 - kN * t) & 7; k < 8; ++k) dst[k] = __float2half_rn(0.f);
            }
        }
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");  // generic-proxy writes -> MMA reads
        __syncthreads();

        // ---- MMAs: one thread issues kw/16 K-steps, each with the high and the low part of B ----
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
            for (int s = 0; s < a.kw / 16; ++s) {
                const uint64_t ad = make_desc(smem_u32(As + 2 * s * (kM * 8)), kM * 16, 128);
                const uint64_t bh = make_desc(smem_u32(Bh + 2 * s * (kN * 8)), kN * 16, 128);
                const uint64_t bl = make_desc(smem_u32(Bl + 2 * s * (kN * 8)), kN * 16, 128);
                mma_f16(tmem, ad, bh, s > 0 ? 1u : 0u);
                mma_f16(tmem, ad, bl, 1u);
            }
            mma_commit(smem_u32(&mbar));
        }
        // ---- wait for the accumulator (bounded) ----
        bool ok = false;
        for (unsigned it = 0; it < kSpinLimit; ++it)
            if (mbar_try_wait(smem_u32(&mbar), phase)) {
                ok = true;
                break;
            }
        phase ^= 1u;
        if (!ok) {
            abort_flag = 1;
            if (a.status) atomicOr(a.status, 1u);
        }
        __syncthreads();
        if (abort_flag) break;
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");

        // ---- epilogue: this pixel's 64 candidates ----
        const uint32_t lane_addr = tmem + (static_cast<uint32_t>(warp * 32) << 16);
#pragma unroll
        for (int q = 0; q < kN / 16; ++q) {
            float v[16];
            tmem_ld16(lane_addr + q * 16, v);
            asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
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
        asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
        __syncthreads();  // accumulator and A buffer free for the next tile
    }
    if (a.argmax && p < a.P) a.argmax[p] = a.dmin + bidx;
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(kN) : "memory");
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

size_t tc_smem_bytes() { return sizeof(__half) * (static_cast<size_t>(kMaxKw) * kM + 2 * static_cast<size_t>(kMaxKw) * kN); }

cudaError_t launch_cost_tc(const spl_params* q, const void* z, long long pitch, const float* h, float* cost,
                           int* argmax, unsigned* status, cudaStream_t s) {
    TcArgs a;
    a.z = static_cast<const __half*>(z);
    a.pitch = pitch;
    a.h = h;
    a.P = q->H * q->W;
    a.T = q->T;
    a.L = q->L;
    a.D = q->dmax - q->dmin + 1;
    a.u0 = q->dmin - q->peak;
    a.a0 = a.u0 & ~7;
    a.delta = a.u0 - a.a0;
    a.kw = ((kN + q->L - 1 + a.delta) + 15) & ~15;
    a.ntiles = (a.D + kN - 1) / kN;
    a.beta = q->beta;
    a.cost = cost;
    a.argmax = argmax;
    a.dmin = q->dmin;
    a.status = status;
    const size_t smem = tc_smem_bytes();
    cudaError_t e = cudaFuncSetAttribute(k_cost_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
    if (e != cudaSuccess) return e;
    const int blocks = (a.P + kM - 1) / kM;
    k_cost_tc<<<blocks, 128, smem, s>>>(a);
    return cudaGetLastError();
}

}  // namespace spl
