// Arithmetic-throughput probes: the denominators of the ALU rooflines that the depth kernels are quoted
// against. The paper has no counterpart; these kernels measure the GPU, not the method.
//
// Each probe runs `iters` iterations of 8 independent dependency chains per thread of one instruction kind, on a
// persistent grid (blocks_per_sm x SMs blocks of 256 threads), so the pipe of that kind, not latency, bounds
// the rate. Every block records the SM clocks it spent (clock64) so that the caller can report operations per
// clock per SM without trusting a sampled clock, and one value per thread is stored so no chain is dead code.
#include <stdint.h>

#include "spl_internal.h"

namespace spl {
namespace {

constexpr int kChains = 8;
constexpr int kThreads = 256;

__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

template <int KIND>
__global__ void __launch_bounds__(kThreads) k_probe(int iters, float seed, float* sink,
                                                    unsigned long long* cycles) {
    const long long t0 = clock64();
    float a[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = seed + 1e-3f * static_cast<float>(threadIdx.x * kChains + k);
    if (KIND == SPL_PROBE_FFMA) {
        const float m = 0.999f, c = 1e-4f * seed;
        for (int i = 0; i < iters; ++i) {
#pragma unroll
            for (int r = 0; r < 16; ++r)
#pragma unroll
                for (int k = 0; k < kChains; ++k) a[k] = fmaf(a[k], m, c);
        }
    } else if (KIND == SPL_PROBE_FFMA2) {
        unsigned long long v[kChains / 2];
#pragma unroll
        for (int k = 0; k < kChains / 2; ++k)
            v[k] = (static_cast<unsigned long long>(__float_as_uint(a[2 * k + 1])) << 32) | __float_as_uint(a[2 * k]);
        const unsigned long long m = (static_cast<unsigned long long>(__float_as_uint(0.999f)) << 32) |
                                     __float_as_uint(0.999f);
        const float cf = 1e-4f * seed;
        const unsigned long long c = (static_cast<unsigned long long>(__float_as_uint(cf)) << 32) | __float_as_uint(cf);
        for (int i = 0; i < iters; ++i) {
#pragma unroll
            for (int r = 0; r < 16; ++r)
#pragma unroll
                for (int k = 0; k < kChains / 2; ++k)
                    asm volatile("fma.rn.f32x2 %0, %0, %1, %2;" : "+l"(v[k]) : "l"(m), "l"(c));
        }
#pragma unroll
        for (int k = 0; k < kChains / 2; ++k) {
            a[2 * k] = __uint_as_float(static_cast<unsigned>(v[k]));
            a[2 * k + 1] = __uint_as_float(static_cast<unsigned>(v[k] >> 32));
        }
    } else {  // SPL_PROBE_EX2: x <- 2^-x stays in [0.5, 1)
        for (int i = 0; i < iters; ++i) {
#pragma unroll
            for (int r = 0; r < 16; ++r)
#pragma unroll
                for (int k = 0; k < kChains; ++k) a[k] = ex2_approx(-a[k]);
        }
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += a[k];
    sink[static_cast<size_t>(blockIdx.x) * blockDim.x + threadIdx.x] = s;
    __syncthreads();
    if (threadIdx.x == 0) cycles[blockIdx.x] = static_cast<unsigned long long>(clock64() - t0);
}

}  // namespace
}  // namespace spl

extern "C" SPL_API spl_status spl_probe_throughput(int kind, int blocks_per_sm, int iters, float* sink,
                                                   unsigned long long* cycles, int* blocks, long long* ops_per_thread,
                                                   void* stream) {
    using namespace spl;
    if (kind < SPL_PROBE_FFMA || kind > SPL_PROBE_EX2) {
        set_error("unknown probe kind %d", kind);
        return SPL_EINVAL;
    }
    if (blocks_per_sm < 1 || blocks_per_sm > 8 || iters < 1 || !blocks || !ops_per_thread) {
        set_error("blocks_per_sm must be 1..8, iters >= 1, blocks and ops_per_thread non-NULL");
        return SPL_EINVAL;
    }
    int dev = 0, nsm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) !=
                                                  cudaSuccess) {
        set_error("no CUDA device");
        return SPL_ECUDA;
    }
    *blocks = nsm * blocks_per_sm;
    // one FMA = 2 flops is not counted here: the unit is instructions per lane (an f32x2 op counts as 2)
    *ops_per_thread = static_cast<long long>(iters) * 16 * kChains;
    if (!sink || !cycles) return SPL_OK;  // size query
    const cudaStream_t s = static_cast<cudaStream_t>(stream);
    const float seed = 0.75f;
    switch (kind) {
        case SPL_PROBE_FFMA: k_probe<SPL_PROBE_FFMA><<<*blocks, kThreads, 0, s>>>(iters, seed, sink, cycles); break;
        case SPL_PROBE_FFMA2: k_probe<SPL_PROBE_FFMA2><<<*blocks, kThreads, 0, s>>>(iters, seed, sink, cycles); break;
        default: k_probe<SPL_PROBE_EX2><<<*blocks, kThreads, 0, s>>>(iters, seed, sink, cycles); break;
    }
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_error("probe launch failed: %s", cudaGetErrorString(e));
        return SPL_ECUDA;
    }
    return SPL_OK;
}
