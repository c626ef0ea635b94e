// Stein update + Adam (Eq. stein_icp_phi, the RBF kernels that follow it, and
// Sec. V), plus the FP64 particle moments.  The translation and rotation
// blocks are independent (own kernel, bandwidth, gradient and Adam
// components), so the update runs as two CTAs of 1024 threads, one per block.
//
// Per iteration, for K particles theta_j with mean ICP gradients gbar_j:
//   G_j   = -N gbar_j + grad log prior(theta_j)          (Eq. posterior)
//   D^t_jl = |theta_j,1:3 - theta_l,1:3|^2,  D^r_jl = sum_a wrap(theta_j,a - theta_l,a)^2
//   h     = median over all K*K entries / ln(K+1)        (median heuristic; 1 if 0)
//   phi_i = (1/K) sum_j [ k(j,i) G_j + (2/h) (theta_i - theta_j) k(j,i) ]   per block
//   Adam on g = -phi.
// wrap(x) = atan2(sin x, cos x) is evaluated as the equal x - 2 pi round(x / 2 pi)
// with a two-term 2 pi (Cody-Waite reduction), which avoids three transcendental
// calls per pair.
//
// The medians are exact order statistics of the fp32 distances: a radix select
// over their bit patterns (non-negative floats order like unsigned ints), with
// the distances recomputed from shared-memory particles on every pass.
#include <float.h>

#include "common.cuh"
#include "stein_device.cuh"

namespace sicp {
namespace {

using namespace sd;

// CTA b updates block b (translation, rotation) of every particle.
__global__ void __launch_bounds__(kThreads) k_stein_adam(SteinArgs a) { stein_adam_one_block(a, blockIdx.x); }

__global__ void k_moments(const float* __restrict__ th, int K, double* __restrict__ out) {
    __shared__ double mean[6];
    const int tid = threadIdx.x;
    if (tid < 6) {
        double s = 0.0;
        for (int j = 0; j < K; ++j) s += (double)th[6 * j + tid];
        mean[tid] = s / (double)K;
    }
    __syncthreads();
    if (tid < 36) {
        const int a = tid / 6, b = tid % 6;
        double s = 0.0;
        for (int j = 0; j < K; ++j) s += ((double)th[6 * j + a] - mean[a]) * ((double)th[6 * j + b] - mean[b]);
        out[6 + tid] = (K > 1) ? s / (double)(K - 1) : 0.0;
    }
    if (tid < 6) out[tid] = mean[tid];
}

}  // namespace

cudaError_t kernel_attrs_init() {
    return cudaFuncSetAttribute(k_stein_adam, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
}

cudaError_t launch_stein_adam(const SteinArgs& a, cudaStream_t s) {
    const size_t pairs = (size_t)a.K * (a.K - 1) / 2;
    const size_t smem = sizeof(float) * (18 * (size_t)a.K + (pairs <= (size_t)kCacheFloats ? pairs : 0));
    k_stein_adam<<<2, kThreads, smem, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_moments(const float* theta, int32_t K, double* out42, cudaStream_t s) {
    k_moments<<<1, 64, 0, s>>>(theta, K, out42);
    return cudaGetLastError();
}

}  // namespace sicp
