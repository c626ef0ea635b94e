// sicp_icp_grad_noalloc: the mean ICP gradient with the exhaustive FP32
// search, for callers that cannot allocate device memory.  It needs no
// context: every input and output is the caller's device buffer, and the
// kernel's scratch (per-chunk partial sums and an arrival counter) lives in a
// file-scope __device__ array that every GPU loading this library holds until
// the process exits.
//
// The arithmetic matches the context path of sicp_icp_grad with
// SICP_NN_BRUTE_FP32: the same chunking of the minibatch, the same distance
// function and lowest-index tie rule, the same in-CTA reduction order and the
// same chunk-order fold, so the two give the same gradients.
#include <float.h>

#include <mutex>

#include "common.cuh"

namespace sicp {
namespace {

constexpr int kNaMaxK = 256;
constexpr int kNaMaxM = 1024;
constexpr int kNaMaxThreads = 256;                                   // minibatch entries per CTA, at most
constexpr int kNaMaxChunks = (kNaMaxM + kNaMaxThreads - 1) / kNaMaxThreads;
constexpr int kNaTile = 2048;
constexpr int kMaxDevices = 64;

// Scratch: partial sums [chunk][K][6], then one arrival counter per particle.
constexpr size_t kNaPartialFloats = (size_t)kNaMaxChunks * kNaMaxK * 6;
constexpr size_t kNaScratchBytes = kNaPartialFloats * sizeof(float) + kNaMaxK * sizeof(unsigned);
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNaScratchBytes];

struct NaArgs {
    const float* ref;       // M x 3
    int M;
    const float* src;       // N x 3
    int64_t N;
    const int32_t* mb;      // m (an entry outside [0, N) contributes nothing)
    int m;
    const float* theta;     // K x 6
    int K;
    float* gbar;            // K x 6
    float inv_m;
    float* partial;         // device address of the scratch partials
    unsigned* done;         // device address of the scratch counters
};

__device__ __forceinline__ void na_block_sum6(float g[6], float (*red)[6]) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int a = 0; a < 6; ++a) {
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) g[a] += __shfl_down_sync(0xffffffffu, g[a], off);
    }
    if (lane == 0) {
#pragma unroll
        for (int a = 0; a < 6; ++a) red[warp][a] = g[a];
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const int nw = blockDim.x >> 5;
        for (int a = 0; a < 6; ++a) {
            float s = 0.f;
            for (int w = 0; w < nw; ++w) s += red[w][a];
            g[a] = s;
        }
    }
}

// grid (chunks, K): CTA (c, j) handles minibatch entries [c*blockDim, (c+1)*blockDim) of particle j;
// the last CTA of particle j folds its chunk partials into gbar[j].
__global__ void __launch_bounds__(kNaMaxThreads) k_grad_brute_noalloc(NaArgs a) {
    __shared__ float4 tile[kNaTile];
    __shared__ Pose P;
    __shared__ float red[kNaMaxThreads / 32][6];
    __shared__ unsigned s_last;
    const int j = blockIdx.y;
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (threadIdx.x == 0) make_pose(a.theta + 6 * j, P);
    __syncthreads();
    const int i = k < a.m ? a.mb[k] : -1;
    const bool valid = i >= 0 && (int64_t)i < a.N;   // an index outside the source reads nothing
    float3 s = make_float3(0.f, 0.f, 0.f);
    if (valid) s = make_float3(a.src[3 * (int64_t)i], a.src[3 * (int64_t)i + 1], a.src[3 * (int64_t)i + 2]);
    const float3 q = apply_pose(P, s);
    float best = FLT_MAX;
    int bi = 0x7fffffff;
    for (int base = 0; base < a.M; base += kNaTile) {
        const int cnt = min(kNaTile, a.M - base);
        __syncthreads();
        for (int t = threadIdx.x; t < cnt; t += blockDim.x) {
            const int64_t r = (int64_t)base + t;
            tile[t] = make_float4(a.ref[3 * r], a.ref[3 * r + 1], a.ref[3 * r + 2], 0.f);
        }
        __syncthreads();
#pragma unroll 8
        for (int t = 0; t < cnt; ++t) {
            const float d = dist2(tile[t], q);
            if (d < best) {
                best = d;
                bi = base + t;
            }
        }
    }
    float g[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    if (valid && bi != 0x7fffffff) {
        const float3 r = make_float3(a.ref[3 * (int64_t)bi], a.ref[3 * (int64_t)bi + 1], a.ref[3 * (int64_t)bi + 2]);
        grad_terms(P, s, make_float3(q.x - r.x, q.y - r.y, q.z - r.z), g);
    }
    na_block_sum6(g, red);
    if (threadIdx.x == 0) {
        float* dst = a.partial + ((int64_t)blockIdx.x * a.K + j) * 6;
        for (int c = 0; c < 6; ++c) dst[c] = g[c];
        __threadfence();
        s_last = atomicAdd(a.done + j, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    if (threadIdx.x < 6) {
        float sum = 0.f;
        for (int ch = 0; ch < (int)gridDim.x; ++ch) sum += __ldcg(a.partial + ((int64_t)ch * a.K + j) * 6 + threadIdx.x);
        a.gbar[j * 6 + threadIdx.x] = sum * a.inv_m;
    }
    if (threadIdx.x == 0) a.done[j] = 0u;
}

// Device address of the scratch array, looked up once per device.
struct NaSetup {
    std::once_flag once;
    cudaError_t err = cudaSuccess;
    void* addr = nullptr;
};
NaSetup g_setup[kMaxDevices];

}  // namespace
}  // namespace sicp

using namespace sicp;

extern "C" int sicp_icp_grad_noalloc(const float* ref_xyz, int64_t M, const float* src_xyz, int64_t N,
                                     const int32_t* mb, int32_t m, const float* particles, int32_t K,
                                     float* out_gbar, void* cuda_stream) {
    if (!ref_xyz || !src_xyz || !mb || !particles || !out_gbar) return SICP_EINVAL;
    if (M < 1 || M > (1 << 30) || N < 1 || N > 0x7fffffff || m < 1 || m > kNaMaxM || K < 1 || K > kNaMaxK)
        return SICP_EINVAL;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        return SICP_ECUDA;
    }
    NaSetup& S = g_setup[dev];
    std::call_once(S.once, [&S]() { S.err = cudaGetSymbolAddress(&S.addr, g_noalloc_scratch); });
    if (S.err != cudaSuccess || !S.addr) return SICP_ECUDA;
    const cudaStream_t stream = (cudaStream_t)cuda_stream;
    NaArgs a;
    a.ref = ref_xyz;
    a.M = (int)M;
    a.src = src_xyz;
    a.N = N;
    a.mb = mb;
    a.m = m;
    a.theta = particles;
    a.K = K;
    a.gbar = out_gbar;
    a.inv_m = 1.f / (float)m;
    a.partial = (float*)S.addr;
    a.done = (unsigned*)((unsigned char*)S.addr + kNaPartialFloats * sizeof(float));
    // the arrival counters must start at zero
    if (cudaMemsetAsync(a.done, 0, sizeof(unsigned) * (size_t)K, stream) != cudaSuccess) {
        cudaGetLastError();
        return SICP_ECUDA;
    }
    const GradLayout L = grad_layout(m);
    dim3 grid(L.chunks, K);
    k_grad_brute_noalloc<<<grid, L.threads, 0, stream>>>(a);
    if (cudaGetLastError() != cudaSuccess) return SICP_ECUDA;
    return SICP_OK;
}
