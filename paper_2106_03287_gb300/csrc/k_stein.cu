// Stein update + Adam, fused in one CTA (Eq. stein_icp_phi, the RBF kernels
// that follow it, and Sec. V), plus the FP64 particle moments.
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

namespace sicp {
namespace {

constexpr int kThreads = 1024;
constexpr float kTwoPiHi = 6.28318548202514648f;      // float nearest 2 pi
constexpr float kTwoPiLo = -1.74845553146951576e-7f;  // 2 pi - kTwoPiHi
constexpr float kInvTwoPi = 0.159154943091895336f;

__device__ __forceinline__ float wrapf(float x) {
    const float r = rintf(x * kInvTwoPi);
    return fmaf(-r, kTwoPiLo, fmaf(-r, kTwoPiHi, x));
}

__device__ __forceinline__ float pair_d2(const float* th, int j, int l, int block) {
    const float* a = th + 6 * j + 3 * block;
    const float* b = th + 6 * l + 3 * block;
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        float d = a[c] - b[c];
        if (block) d = wrapf(d);
        s = fmaf(d, d, s);
    }
    return s;
}

// Exact value of rank `rank` (0-based) among the K*K distances of `block`.
__device__ unsigned select_rank(const float* th, int K, int block, unsigned rank, unsigned* hist,
                                unsigned* s_out) {
    const int tid = threadIdx.x, lane = tid & 31;
    const int n = K * K;
    unsigned prefix = 0, mask = 0, rem = rank + 1;
    for (int shift = 24; shift >= 0; shift -= 8) {
        for (int i = tid; i < 256; i += blockDim.x) hist[i] = 0;
        __syncthreads();
        for (int p = tid; p < n; p += blockDim.x) {
            unsigned b = __float_as_uint(pair_d2(th, p / K, p % K, block));
            if ((b & mask) == prefix) atomicAdd(&hist[(b >> shift) & 255u], 1u);
        }
        __syncthreads();
        if (tid < 32) {
            unsigned c[8], tot = 0;
#pragma unroll
            for (int q = 0; q < 8; ++q) { c[q] = hist[lane * 8 + q]; tot += c[q]; }
            unsigned incl = tot;
#pragma unroll
            for (int off = 1; off < 32; off <<= 1) {
                unsigned v = __shfl_up_sync(0xffffffffu, incl, off);
                if (lane >= off) incl += v;
            }
            unsigned excl = incl - tot;
            if (excl < rem && rem <= incl) {
                unsigned acc = excl;
                for (int q = 0; q < 8; ++q) {
                    if (rem <= acc + c[q]) {
                        s_out[0] = prefix | ((unsigned)(lane * 8 + q) << shift);
                        s_out[1] = rem - acc;
                        break;
                    }
                    acc += c[q];
                }
            }
        }
        __syncthreads();
        prefix = s_out[0];
        rem = s_out[1];
        mask |= 0xffu << shift;
        __syncthreads();
    }
    return prefix;
}

// Median (mean of the two middle order statistics for an even count) / ln(K+1).
__device__ float bandwidth(const float* th, int K, int block, unsigned* hist, unsigned* s_u,
                           float* s_f) {
    const unsigned n = (unsigned)K * (unsigned)K;
    const unsigned r_lo = (n - 1) / 2, r_hi = n / 2;
    const unsigned v_lo = select_rank(th, K, block, r_lo, hist, s_u);
    float med = __uint_as_float(v_lo);
    if (r_hi != r_lo) {
        // rank r_hi is v_lo again if more than r_hi values are <= v_lo, else the next larger value
        if (threadIdx.x == 0) { s_u[2] = 0; s_u[3] = 0x7f800000u; }
        __syncthreads();
        unsigned cnt = 0, mn = 0x7f800000u;
        for (int p = threadIdx.x; p < (int)n; p += blockDim.x) {
            unsigned b = __float_as_uint(pair_d2(th, p / K, p % K, block));
            if (b <= v_lo) ++cnt; else mn = min(mn, b);
        }
        atomicAdd(&s_u[2], cnt);
        atomicMin(&s_u[3], mn);
        __syncthreads();
        const float v_hi = (s_u[2] > r_hi) ? med : __uint_as_float(s_u[3]);
        med = 0.5f * (med + v_hi);
        __syncthreads();
    }
    (void)s_f;
    return med > 0.f ? med / logf((float)K + 1.f) : 1.f;
}

__global__ void __launch_bounds__(kThreads) k_stein_adam(SteinArgs a) {
    extern __shared__ float sm[];
    float* th = sm;               // K x 6
    float* G = sm + 6 * a.K;      // K x 6
    __shared__ unsigned hist[256];
    __shared__ unsigned s_u[4];
    __shared__ float s_f[4];
    const int K = a.K, tid = threadIdx.x;

    for (int idx = tid; idx < 6 * K; idx += blockDim.x) {
        const int j = idx / 6, c = idx % 6;
        const float x = a.theta[idx];
        th[idx] = x;
        float s = 0.f;
        for (int ch = 0; ch < a.chunks; ++ch) s += a.partial[((int64_t)ch * K + j) * 6 + c];
        float pr = 0.f;
        if (a.prior == 1) pr = (c < 3) ? -(x - a.mu[c]) / a.sigma[c] : -a.kappa[c - 3] * sinf(x - a.mu[c]);
        G[idx] = fmaf(-a.N, s * a.inv_m, pr);
    }
    __syncthreads();

    const float h_t = bandwidth(th, K, 0, hist, s_u, s_f);
    const float h_r = bandwidth(th, K, 1, hist, s_u, s_f);
    const float inv_ht = 1.f / h_t, inv_hr = 1.f / h_r;
    const float two_ht = 2.f / h_t, two_hr = 2.f / h_r;
    if (tid == 0 && a.out_h) { a.out_h[0] = h_t; a.out_h[1] = h_r; }

    // S lanes per particle (power of two <= 32), each summing over j = lane (mod S)
    int S = 32;
    while (S > 1 && K * S > (int)blockDim.x) S >>= 1;
    const int groups = blockDim.x / S;
    const int g_id = tid / S, g_lane = tid % S;
    const int rounds = (K + groups - 1) / groups;
    const float invK = 1.f / (float)K;
    const float omb1 = 1.f - a.beta1, omb2 = 1.f - a.beta2;   // exact for beta in [0.5, 1]
    const float c1 = -expm1f((float)a.t * log1pf(-omb1));    // 1 - beta1^t
    const float c2 = -expm1f((float)a.t * log1pf(-omb2));    // 1 - beta2^t
    for (int r = 0; r < rounds; ++r) {
        const int i = r * groups + g_id;
        const bool valid = i < K;
        float acc[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        if (valid) {
            const float* ti = th + 6 * i;
            for (int j = g_lane; j < K; j += S) {
                const float* tj = th + 6 * j;
                const float* Gj = G + 6 * j;
                float dt[3], dr[3], Dt = 0.f, Dr = 0.f;
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    dt[c] = ti[c] - tj[c];
                    Dt = fmaf(dt[c], dt[c], Dt);
                    dr[c] = wrapf(ti[3 + c] - tj[3 + c]);
                    Dr = fmaf(dr[c], dr[c], Dr);
                }
                const float kt = expf(-Dt * inv_ht), kr = expf(-Dr * inv_hr);
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    acc[c] += kt * fmaf(two_ht, dt[c], Gj[c]);
                    acc[3 + c] += kr * fmaf(two_hr, dr[c], Gj[3 + c]);
                }
            }
        }
#pragma unroll
        for (int c = 0; c < 6; ++c)
            for (int off = S >> 1; off > 0; off >>= 1) acc[c] += __shfl_xor_sync(0xffffffffu, acc[c], off, S);
        if (valid && g_lane == 0) {
#pragma unroll
            for (int c = 0; c < 6; ++c) {
                const int idx = 6 * i + c;
                const float phi = acc[c] * invK;
                if (a.out_phi) a.out_phi[idx] = phi;
                const float g = -phi;
                const float mo = fmaf(a.beta1, a.adam_m[idx], omb1 * g);
                const float ve = fmaf(a.beta2, a.adam_v[idx], omb2 * g * g);
                a.adam_m[idx] = mo;
                a.adam_v[idx] = ve;
                const float mh = mo / c1, vh = ve / c2;
                a.theta[idx] = th[idx] - a.lr * mh / (sqrtf(vh) + a.eps);
            }
        }
    }
}

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
    const size_t smem = sizeof(float) * 12 * (size_t)a.K;
    k_stein_adam<<<1, kThreads, smem, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_moments(const float* theta, int32_t K, double* out42, cudaStream_t s) {
    k_moments<<<1, 64, 0, s>>>(theta, K, out42);
    return cudaGetLastError();
}

}  // namespace sicp
