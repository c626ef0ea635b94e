// Exhaustive FP32 nearest-neighbour search (Eq. correspondences: the
// reference point minimising the Euclidean distance to the transformed source
// point) and the fused per-particle gradient kernel built on it
// (Eqs. trans_gradient and rotation_gradient).
//
// The reference (float4: x, y, z, index bits) is streamed through shared
// memory in tiles; every thread scans each tile against its own query with
// broadcast reads.  Tiles are visited in index order and a candidate replaces
// the incumbent only if strictly closer, so ties resolve to the lowest index.
#include <float.h>

#include "common.cuh"

namespace sicp {
namespace {

constexpr int kTile = 2048;          // 32 KB of float4 per tile
constexpr int kGradMaxThreads = 256; // queries per CTA in the fused kernel (at most)
constexpr int kNNThreads = 256;

__device__ __forceinline__ void scan_tile(const float4* __restrict__ tile, int cnt, int base,
                                          float3 q, float& best, int& bi) {
#pragma unroll 8
    for (int k = 0; k < cnt; ++k) {
        float d = dist2(tile[k], q);
        if (d < best) { best = d; bi = base + k; }
    }
}

__device__ __forceinline__ void brute_search(const float4* __restrict__ ref, int M, float4* tile,
                                             float3 q, float& best, int& bi) {
    best = FLT_MAX;
    bi = 0x7fffffff;
    for (int base = 0; base < M; base += kTile) {
        const int cnt = min(kTile, M - base);
        __syncthreads();
        for (int k = threadIdx.x; k < cnt; k += blockDim.x) tile[k] = ref[base + k];
        __syncthreads();
        scan_tile(tile, cnt, base, q, best, bi);
    }
}

__global__ void __launch_bounds__(kNNThreads) k_nn_brute(const float4* __restrict__ ref, int M,
                                                         const float* __restrict__ q, int64_t n,
                                                         int32_t* __restrict__ idx,
                                                         float* __restrict__ d2) {
    __shared__ float4 tile[kTile];
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    float3 qq = make_float3(0.f, 0.f, 0.f);
    if (i < n) qq = make_float3(q[3 * i], q[3 * i + 1], q[3 * i + 2]);
    float best;
    int bi;
    brute_search(ref, M, tile, qq, best, bi);
    if (i < n) {
        idx[i] = bi != 0x7fffffff ? bi : -1;
        if (d2) d2[i] = best;
    }
}

// Block-wide deterministic sum of 6 values per thread; result valid in thread 0.
__device__ __forceinline__ void block_sum6(float g[6], float (*red)[6]) {
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

// grid (chunks, K): CTA (c, j) handles minibatch entries [c*blockDim, (c+1)*blockDim) of particle j.
__global__ void __launch_bounds__(kGradMaxThreads) k_grad_brute(GradArgs a, const float4* __restrict__ ref,
                                                                int M) {
    __shared__ float4 tile[kTile];
    __shared__ Pose P;
    __shared__ float red[kGradMaxThreads / 32][6];
    const int j = blockIdx.y;
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    pdl_wait();      // the particles of the previous Stein step
    pdl_trigger();   // only after the wait: see pdl_wait
    if (threadIdx.x == 0) make_pose(a.theta + 6 * j, P);
    __syncthreads();
    const bool valid = k < a.m;
    float3 s = make_float3(0.f, 0.f, 0.f);
    if (valid) {
        float4 s4 = a.src[SICP_IDX(a.mb[(int64_t)j * a.mb_stride + k], a.n_src, kChkSrc)];
        s = make_float3(s4.x, s4.y, s4.z);
    }
    const float3 q = apply_pose(P, s);
    float best;
    int bi;
    brute_search(ref, M, tile, q, best, bi);
    float g[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    const bool found = bi != 0x7fffffff;      // false only for a non-finite distance
    if (valid && found) {
        const float4 r = ref[bi];
        float3 d = make_float3(q.x - r.x, q.y - r.y, q.z - r.z);
        if (a.normals) d = plane_residual(__ldg(a.normals + SICP_IDX(bi, a.n_ref, kChkRef)), d);
        grad_terms(P, s, d, g);
    }
    if (valid && a.out_nn) a.out_nn[(int64_t)j * a.m + k] = found ? bi : -1;
    block_sum6(g, red);
    if (threadIdx.x == 0) {
        float* dst = a.partial + ((int64_t)blockIdx.x * a.K + j) * 6;
        for (int c = 0; c < 6; ++c) dst[c] = g[c];
    }
}

}  // namespace

GradLayout grad_layout(int32_t m) {
    GradLayout L;
    L.chunks = (m + kGradMaxThreads - 1) / kGradMaxThreads;
    const int per = (m + L.chunks - 1) / L.chunks;
    L.threads = ((per + 31) / 32) * 32;
    return L;
}

cudaError_t launch_nn_brute(const float4* ref, int64_t M, const float* q, int64_t n, int32_t* idx,
                            float* d2, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    const int64_t blocks = (n + kNNThreads - 1) / kNNThreads;
    k_nn_brute<<<(unsigned)blocks, kNNThreads, 0, s>>>(ref, (int)M, q, n, idx, d2);
    return cudaGetLastError();
}

cudaError_t launch_grad_brute(const GradArgs& a, const float4* ref, int64_t M, cudaStream_t s) {
    const GradLayout L = grad_layout(a.m);
    dim3 grid(L.chunks, a.K);
    return launch_pdl(k_grad_brute, grid, dim3(L.threads), 0, s, a, ref, (int)M);
}

}  // namespace sicp
