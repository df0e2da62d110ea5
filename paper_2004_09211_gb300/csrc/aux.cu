// Small per-pixel kernels around the fused step: the initial state of Algorithm 1 and the presence-prior
// propagation of Eq. prior_detect.
#include <math.h>

#include "spl_internal.h"

namespace spl {
namespace {

__global__ void k_state_init(long long P, float m, float v, float* mu, float* var) {
    for (long long p = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; p < P;
         p += static_cast<long long>(gridDim.x) * blockDim.x) {
        mu[p] = m;
        var[p] = v;
    }
}

constexpr float kLogitMax = 16.1180956f;  // log(1e7 - 1)

struct Nu {
    float w[9];
};

// pi0 = sigmoid(sum_k nu_k logit(pi[p + k])) with out-of-view neighbours and faulty pixels at 0.5. pi is
// limited to [1e-7, 1 - 1e-7] through the equivalent clamp of its logit to +-log(1e7 - 1): 1 - 1e-7 has no
// exact float, while the logit bound is the same in every precision.
__global__ void k_pi_propagate(int H, int W, Nu nu, const float* __restrict__ pi_in,
                               const uint8_t* __restrict__ faulty, float* __restrict__ pi_out) {
    const long long P = static_cast<long long>(H) * W;
    for (long long p = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; p < P;
         p += static_cast<long long>(gridDim.x) * blockDim.x) {
        if (faulty && faulty[p]) {
            pi_out[p] = 0.5f;
            continue;
        }
        const int y = static_cast<int>(p / W), x = static_cast<int>(p - static_cast<long long>(y) * W);
        float acc = 0.f;
#pragma unroll
        for (int k = 0; k < 9; ++k) {
            const int yy = y + k / 3 - 1, xx = x + k % 3 - 1;
            float v = 0.5f;
            if (yy >= 0 && yy < H && xx >= 0 && xx < W) {
                const long long i = static_cast<long long>(yy) * W + xx;
                v = (faulty && faulty[i]) ? 0.5f : pi_in[i];
            }
            float lg = logf(v) - log1pf(-v);   // 1 - v is exact for v >= 0.5
            lg = fminf(fmaxf(lg, -kLogitMax), kLogitMax);
            acc = fmaf(nu.w[k], lg, acc);
        }
        pi_out[p] = 1.f / (1.f + expf(-acc));
    }
}

int grid_for(long long n, int block) {
    long long g = (n + block - 1) / block;
    if (g > 152 * 16) g = 152 * 16;
    if (g < 1) g = 1;
    return static_cast<int>(g);
}

}  // namespace

cudaError_t launch_state_init(int P, float m, float v, float* mu, float* var, cudaStream_t s) {
    k_state_init<<<grid_for(P, 256), 256, 0, s>>>(P, m, v, mu, var);
    return cudaGetLastError();
}

cudaError_t launch_pi_propagate(int H, int W, const float* nu, const float* pi_in, const uint8_t* faulty,
                                float* pi_out, cudaStream_t s) {
    Nu n;
    for (int k = 0; k < 9; ++k) n.w[k] = nu[k];
    const long long P = static_cast<long long>(H) * W;
    k_pi_propagate<<<grid_for(P, 256), 256, 0, s>>>(H, W, n, pi_in, faulty, pi_out);
    return cudaGetLastError();
}

}  // namespace spl
