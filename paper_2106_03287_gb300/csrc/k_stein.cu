// Stein update + Adam (Eq. stein_icp_phi, the RBF kernels that follow it, and
// Sec. V), plus the FP64 particle moments.  The translation and rotation
// blocks are independent (own kernel, bandwidth, gradient and Adam
// components), so each block has its own CTAs of 1024 threads: P of them
// (P = ceil(K / 32), at most 32), each taking the Stein direction and the
// Adam step of a share of the particles after computing the block's bandwidth
// itself (the same value in every CTA).
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
// The medians are exact order statistics of the fp32 distances.  Within a
// registration run the selection starts from the previous iteration's median:
// one pass counts the distances below a bracket around it and bins those
// inside; the two middle ranks are then found among the few values of their
// bins.  Otherwise (first iteration, or a rank outside the bracket) a radix
// select over the bit patterns (non-negative floats order like unsigned ints)
// finds them.
#include <float.h>

#include <algorithm>

#include "common.cuh"
#include "stein_device.cuh"

namespace sicp {
namespace {

using namespace sd;

// CTAs [b P, (b + 1) P) update block b (translation, rotation), CTA q of them
// the particles [q Kq, (q + 1) Kq).
__global__ void __launch_bounds__(kThreads) k_stein_adam(SteinArgs a, int P) {
    stein_adam_one_block(a, blockIdx.x / P, blockIdx.x % P, P);
}

// Independent SGD-ICP runs: for every particle j and component c, G = -N gbar
// + grad log prior and Adam on g = -phi with phi = G, computed as the Stein
// kernel computes them for K = 1 (the same partial sums in the same order;
// the K = 1 Stein sum adds +0 to G and multiplies by 1), so each particle
// follows exactly the run it would follow alone.  chunks == 1: one thread per
// component; else one warp per component, lanes over the chunks.
__global__ void k_adam_independent(SteinArgs a) {
    const int lane = threadIdx.x & 31;
    const int64_t n = 6 * (int64_t)a.K;
    const int64_t idx = a.chunks == 1 ? (int64_t)blockIdx.x * blockDim.x + threadIdx.x
                                      : ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (idx >= n) return;
    const int j = (int)(idx / 6), c = (int)(idx % 6);
    float gb;
    if (a.chunks == 1) {
        gb = a.partial[idx];
    } else {
        float s = 0.f;
        for (int ch = lane; ch < a.chunks; ch += 32) s += a.partial[((int64_t)ch * a.K + j) * 6 + c];
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
        if (lane != 0) return;
        gb = s;
    }
    const float x = a.theta[idx];
    float pr = 0.f;
    if (a.prior == 1) pr = (c < 3) ? -(x - a.mu[c]) / a.sigma[c] : -a.kappa[c - 3] * sinf(x - a.mu[c]);
    const float G = fmaf(-a.N, gb * a.inv_m, pr);
    const float phi = (G + 0.f) * 1.f;
    if (a.out_phi) a.out_phi[idx] = phi;
    const float omb1 = 1.f - a.beta1, omb2 = 1.f - a.beta2;
    const float c1 = -expm1f((float)a.t * log1pf(-omb1));
    const float c2 = -expm1f((float)a.t * log1pf(-omb2));
    const float g = -phi;
    const float mo = fmaf(a.beta1, a.adam_m[idx], omb1 * g);
    const float ve = fmaf(a.beta2, a.adam_v[idx], omb2 * g * g);
    a.adam_m[idx] = mo;
    a.adam_v[idx] = ve;
    const float mh = mo / c1, vh = ve / c2;
    a.theta[idx] = x - a.lr * mh / (sqrtf(vh) + a.eps);
}

// Mean and covariance (two passes, float64) over kMomThreads threads: thread t
// takes the particles j = t, t + kMomThreads, ... in order, the warps combine
// their lanes with a fixed butterfly and thread 0 the warps in order, so the
// result is deterministic.  (FP64 is the slow unit of this GPU; a few threads
// walking all K particles took about 28 us for K = 100.)
constexpr int kMomThreads = 256;

template <int N>
__device__ __forceinline__ void block_sum_d(double (&v)[N], double (*part)[kMomThreads / 32]) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int i = 0; i < N; ++i) {
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) v[i] += __shfl_xor_sync(0xffffffffu, v[i], off);
        if (lane == 0) part[i][warp] = v[i];
    }
    __syncthreads();
    if (threadIdx.x == 0) {
#pragma unroll
        for (int i = 0; i < N; ++i) {
            double s = 0.0;
            for (int w = 0; w < kMomThreads / 32; ++w) s += part[i][w];
            part[i][0] = s;
        }
    }
    __syncthreads();
}

__global__ void __launch_bounds__(kMomThreads) k_moments(const float* __restrict__ th, int K, double* __restrict__ out) {
    __shared__ double part[21][kMomThreads / 32];
    __shared__ double mean[6];
    const int tid = threadIdx.x;
    double m[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    for (int j = tid; j < K; j += kMomThreads)
#pragma unroll
        for (int a = 0; a < 6; ++a) m[a] += (double)th[6 * j + a];
    block_sum_d(m, part);
    if (tid < 6) mean[tid] = part[tid][0] / (double)K;
    __syncthreads();
    double c[21];
#pragma unroll
    for (int i = 0; i < 21; ++i) c[i] = 0.0;
    for (int j = tid; j < K; j += kMomThreads) {
        double d[6];
#pragma unroll
        for (int a = 0; a < 6; ++a) d[a] = (double)th[6 * j + a] - mean[a];
        int i = 0;
#pragma unroll
        for (int a = 0; a < 6; ++a)
#pragma unroll
            for (int b = a; b < 6; ++b) c[i++] += d[a] * d[b];
    }
    block_sum_d(c, part);
    if (tid < 36) {
        const int a = tid / 6, b = tid % 6;
        const int lo = a < b ? a : b, hi = a < b ? b : a;
        const int i = lo * 6 - lo * (lo - 1) / 2 + (hi - lo);   // upper-triangle index of (lo, hi)
        out[6 + tid] = (K > 1) ? part[i][0] / (double)(K - 1) : 0.0;
    }
    if (tid < 6) out[tid] = mean[tid];
}

// The same with circular statistics for the three angles: the mean of angle
// a is atan2(sum sin, sum cos) (0 when both sums vanish), and the covariance
// is that of [theta_t - mean_t ; wrap(theta_r - mean_r)], wrap(x) = atan2(sin
// x, cos x), for particles whose angles straddle +-pi.
__device__ __forceinline__ double wrap_d(double x) { return atan2(sin(x), cos(x)); }

__global__ void k_moments_circular(const float* __restrict__ th, int K, double* __restrict__ out) {
    __shared__ double mean[6];
    const int tid = threadIdx.x;
    if (tid < 3) {
        double s = 0.0;
        for (int j = 0; j < K; ++j) s += (double)th[6 * j + tid];
        mean[tid] = s / (double)K;
    } else if (tid < 6) {
        double ss = 0.0, sc = 0.0;
        for (int j = 0; j < K; ++j) {
            const double x = (double)th[6 * j + tid];
            ss += sin(x);
            sc += cos(x);
        }
        mean[tid] = (ss == 0.0 && sc == 0.0) ? 0.0 : atan2(ss, sc);
    }
    __syncthreads();
    if (tid < 36) {
        const int a = tid / 6, b = tid % 6;
        double s = 0.0;
        for (int j = 0; j < K; ++j) {
            double da = (double)th[6 * j + a] - mean[a], db = (double)th[6 * j + b] - mean[b];
            if (a >= 3) da = wrap_d(da);
            if (b >= 3) db = wrap_d(db);
            s += da * db;
        }
        out[6 + tid] = (K > 1) ? s / (double)(K - 1) : 0.0;
    }
    if (tid < 6) out[tid] = mean[tid];
}

}  // namespace

cudaError_t kernel_attrs_init() {
    return cudaFuncSetAttribute(k_stein_adam, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
}

// CTAs per block: at most 32 particles each (one warp per particle), at most 32 CTAs.
int stein_ctas_per_block(int32_t K) { return std::min(32, std::max(1, (K + 31) / 32)); }

cudaError_t launch_stein_adam(const SteinArgs& a, cudaStream_t s) {
    const size_t pairs = (size_t)a.K * (a.K - 1) / 2;
    const size_t smem = sizeof(float) * (18 * (size_t)a.K + (pairs <= (size_t)kCacheFloats ? pairs : 0));
    const int P = (a.arrive && a.err) ? stein_ctas_per_block(a.K) : 1;
    // With P > 1 the CTAs of a block wait for one another, so all 2P <= 64 of
    // them must be resident together.  They are: everything before them in the
    // stream completes without waiting for them, and the next kernel is
    // scheduled only once every one of them has passed its pdl_wait.  (A
    // cooperative launch would state it; it is not combined with the
    // programmatic serialisation here.)  The wait is bounded all the same.
    return launch_pdl(k_stein_adam, dim3(2 * P), dim3(kThreads), smem, s, a, P);
}

cudaError_t launch_adam_independent(const SteinArgs& a, cudaStream_t s) {
    const int64_t threads = a.chunks == 1 ? 6 * (int64_t)a.K : 32 * 6 * (int64_t)a.K;
    k_adam_independent<<<(unsigned)((threads + 255) / 256), 256, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_moments(const float* theta, int32_t K, double* out42, cudaStream_t s) {
    k_moments<<<1, kMomThreads, 0, s>>>(theta, K, out42);
    return cudaGetLastError();
}

cudaError_t launch_moments_circular(const float* theta, int32_t K, double* out42, cudaStream_t s) {
    k_moments_circular<<<1, 64, 0, s>>>(theta, K, out42);
    return cudaGetLastError();
}

}  // namespace sicp
