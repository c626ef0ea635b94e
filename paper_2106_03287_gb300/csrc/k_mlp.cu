// Learned closest-point field: an MLP that maps a query to the displacement to
// its nearest reference point plus a confidence, trained on queries labelled
// by the exact grid search and served in place of that search during the early
// iterations of a run (falling back to the exact search where the confidence
// is low).  Both training and inference run on the fifth-generation tensor
// cores: bf16 operands in shared memory, fp32 accumulators in tensor memory.
//
// Model.  q~ = (q - c) / s with c the centre of the reference bounding box and
// s = 0.6 x its largest extent.  Features (112): q~, then sin and cos of
// w_f q~_a, w_f = pi 2^(8f/15), f = 0..15 (index 3 + 6f + 2a), then zeros.
// Layers 112 -> 128 (ReLU) -> 128 (ReLU) -> 16; outputs 0..2 are the
// displacement d~ (normalised units), output 3 the confidence logit z.
// Loss per sample: |d~ - d~*|^2 + lam (softplus(z) - c* z) with the constant
// target c* = exp(-|d~ - d~*|^2 / delta~^2).
//
// Tiles.  A CTA of 256 threads handles 128 samples: row r = thread % 128 is a
// sample (tensor-memory lane r); the two halves of the CTA split each row's
// columns.  Every operand tile is stored K-major in 8 x 8 core matrices; the
// same tiles serve as MN-major operands for the weight gradients
// (dW = delta^T x activation), so nothing is transposed.
//
// Training step on a batch: per tile, forward (3 MMAs) -> output deltas ->
// E2 = d3 W3 -> d2 = E2 * [h2 > 0] -> E1 = d2 W2 and dW2 = d2^T h1 -> d1 =
// E1 * [h1 > 0] -> dW1 = d1^T x; dW3 and the bias gradients on the CUDA cores.
// Per-tile gradients are reduced over tiles in fixed order, then Adam updates
// fp32 master weights and rewrites the bf16 weight images the MMAs read.
#include <cuda_bf16.h>
#include <float.h>
#include <math.h>

#include <stdio.h>
#include <string.h>

#include <vector>

#include "common.cuh"
#include "nvtx.cuh"
#include "grid_search.cuh"
#include "tc.cuh"

namespace sicp {
namespace {

using namespace gs;

constexpr int kDin = 112, kH = 128, kDout = 16, kRows = 128;
constexpr int kMlpThreads = 256;
constexpr int oW1 = 0, ob1 = kH * kDin, oW2 = ob1 + kH, ob2 = oW2 + kH * kH, oW3 = ob2 + kH, ob3 = oW3 + kDout * kH;
constexpr int kNParam = ob3 + kDout;                              // 33,040
constexpr int kImgW1 = 0, kImgW2 = kH * kDin * 2, kImgW3 = kImgW2 + kH * kH * 2, kImgBytes = kImgW3 + kDout * kH * 2;
constexpr long long kMbarPolls = 1ll << 24;

// shared-memory layout (bytes); every operand tile starts on a 128-byte boundary
constexpr int sOffW = 0;                          // weight images, kImgBytes
constexpr int sOffX = kImgBytes;                  // 128 x 112 bf16
constexpr int sOffH1 = sOffX + kRows * kDin * 2;  // 128 x 128
constexpr int sOffH2 = sOffH1 + kRows * kH * 2;   // 128 x 128 (delta1 after use)
constexpr int sOffD2 = sOffH2 + kRows * kH * 2;   // 128 x 128
constexpr int sOffD3 = sOffD2 + kRows * kH * 2;   // 128 x 16 bf16
constexpr int sOffD3f = sOffD3 + kRows * kDout * 2;  // 128 x 16 fp32, row-major
constexpr int sOffBias = sOffD3f + kRows * kDout * 4;  // b1, b2, b3 fp32
constexpr int kTrainSmem = sOffBias + (kH + kH + kDout) * 4;

__device__ __forceinline__ float feat_freq(int f) { return 3.14159265358979323846f * exp2f(8.f * (float)f / 15.f); }

// Feature k (0..111) of normalised query qn.
__device__ __forceinline__ float feature(int k, float3 qn) {
    if (k < 3) return k == 0 ? qn.x : (k == 1 ? qn.y : qn.z);
    if (k >= 99) return 0.f;
    const int r = k - 3, f = r / 6, a = (r % 6) >> 1;
    const float v = a == 0 ? qn.x : (a == 1 ? qn.y : qn.z);
    const float w = feat_freq(f) * v;
    return (r & 1) ? cosf(w) : sinf(w);
}

// Store 8 consecutive bf16 values of row r, columns [c0, c0+8) of a K-major tile (c0 % 8 == 0).
__device__ __forceinline__ void store8(unsigned char* tile, int r, int c0, int K, const float v[8]) {
    uint4 u;
    __nv_bfloat162 p0 = __floats2bfloat162_rn(v[0], v[1]), p1 = __floats2bfloat162_rn(v[2], v[3]);
    __nv_bfloat162 p2 = __floats2bfloat162_rn(v[4], v[5]), p3 = __floats2bfloat162_rn(v[6], v[7]);
    u.x = *reinterpret_cast<uint32_t*>(&p0);
    u.y = *reinterpret_cast<uint32_t*>(&p1);
    u.z = *reinterpret_cast<uint32_t*>(&p2);
    u.w = *reinterpret_cast<uint32_t*>(&p3);
    *reinterpret_cast<uint4*>(tile + tc::kmajor_offset(r, c0, K)) = u;
}

__device__ __forceinline__ float load_bf16(const unsigned char* tile, int r, int c, int K) {
    const uint16_t b = *reinterpret_cast<const uint16_t*>(tile + tc::kmajor_offset(r, c, K));
    return __uint_as_float((uint32_t)b << 16);
}

// Descriptors of a K-major operand (rows x K) and of an MN-major use of a tile
// stored [K rows][MN columns]; ks = index of the 16-wide K step.
__device__ __forceinline__ uint64_t desc_k(const unsigned char* t, int ks, int K) {
    return tc::smem_desc(tc::smem_u32(t) + ks * 256, 128, K * 16, false);
}
__device__ __forceinline__ uint64_t desc_mn(const unsigned char* t, int ks, int MN) {
    return tc::smem_desc(tc::smem_u32(t) + ks * 2 * (MN / 8) * 128, (MN / 8) * 128, 128, false);
}
__device__ __forceinline__ uint32_t idesc(int M, int N, bool a_mn, bool b_mn) {
    return tc::idesc_bf16(M, N) | ((uint32_t)a_mn << 15) | ((uint32_t)b_mn << 16);
}

struct TmemCtl {
    uint64_t* mbar;
    uint32_t base;
    uint32_t phase;
    int* err;
};

// Issue-side: thread 0 commits; all threads wait for completion.  False if the wait gave up.
// The result is the same on every thread (warp-collective tensor-memory loads
// follow under it).
__device__ __forceinline__ bool mma_wait(TmemCtl& T) {
    bool ok = tc::mbar_wait(T.mbar, T.phase, kMbarPolls);
    T.phase ^= 1u;
    ok = __syncthreads_and(ok) != 0;
    if (!ok && threadIdx.x == 0) atomicOr(T.err, 1);
    tc::fence_after_sync();
    return ok;
}

__device__ __forceinline__ void to_tensor_core() {
    tc::fence_async_shared();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
}

__device__ __forceinline__ uint32_t lane_addr(uint32_t base, int col) {
    const int warp = threadIdx.x >> 5;
    return base + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)col;
}

// Forward of the tile in sX: H1, H2 in shared memory, the 16 outputs of row r
// (only for the first half, threadIdx.x < 128) in out[].  False on a wait failure.
__device__ bool forward_tile(unsigned char* sm, const float* bias, TmemCtl& T, float out[kDout]) {
    unsigned char* sX = sm + sOffX;
    unsigned char* sH1 = sm + sOffH1;
    unsigned char* sH2 = sm + sOffH2;
    const unsigned char* sW1 = sm + sOffW + kImgW1;
    const unsigned char* sW2 = sm + sOffW + kImgW2;
    const unsigned char* sW3 = sm + sOffW + kImgW3;
    const int row = threadIdx.x & 127, half = threadIdx.x >> 7;
    to_tensor_core();
    if (threadIdx.x == 0) {
        for (int ks = 0; ks < kDin / 16; ++ks)
            tc::mma_bf16(T.base, desc_k(sX, ks, kDin), desc_k(sW1, ks, kDin), idesc(128, kH, false, false), ks > 0);
        tc::mma_commit(T.mbar);
    }
    if (!mma_wait(T)) return false;
    for (int c0 = 64 * half; c0 < 64 * half + 64; c0 += 16) {
        float v[16];
        tc::tmem_ld16(lane_addr(T.base, c0), v);
        for (int j = 0; j < 16; ++j) v[j] = fmaxf(v[j] + bias[c0 + j], 0.f);
        store8(sH1, row, c0, kH, v);
        store8(sH1, row, c0 + 8, kH, v + 8);
    }
    to_tensor_core();
    if (threadIdx.x == 0) {
        for (int ks = 0; ks < kH / 16; ++ks)
            tc::mma_bf16(T.base + 128, desc_k(sH1, ks, kH), desc_k(sW2, ks, kH), idesc(128, kH, false, false), ks > 0);
        tc::mma_commit(T.mbar);
    }
    if (!mma_wait(T)) return false;
    for (int c0 = 64 * half; c0 < 64 * half + 64; c0 += 16) {
        float v[16];
        tc::tmem_ld16(lane_addr(T.base + 128, c0), v);
        for (int j = 0; j < 16; ++j) v[j] = fmaxf(v[j] + bias[kH + c0 + j], 0.f);
        store8(sH2, row, c0, kH, v);
        store8(sH2, row, c0 + 8, kH, v + 8);
    }
    to_tensor_core();
    if (threadIdx.x == 0) {
        for (int ks = 0; ks < kH / 16; ++ks)
            tc::mma_bf16(T.base + 256, desc_k(sH2, ks, kH), desc_k(sW3, ks, kH), idesc(128, kDout, false, false), ks > 0);
        tc::mma_commit(T.mbar);
    }
    if (!mma_wait(T)) return false;
    if (half == 0) {
        tc::tmem_ld16(lane_addr(T.base + 256, 0), out);
        for (int j = 0; j < kDout; ++j) out[j] += bias[2 * kH + j];
    } else {
        // the tensor-memory load is warp-collective: the second half reads too and discards
        float tmp[16];
        tc::tmem_ld16(lane_addr(T.base + 256, 0), tmp);
    }
    return true;
}

// Features of this thread's half of row `row` into sX.
__device__ __forceinline__ void write_features(unsigned char* sX, int row, int half, float3 qn) {
    for (int c0 = 56 * half; c0 < 56 * half + 56; c0 += 8) {
        float v[8];
        for (int j = 0; j < 8; ++j) v[j] = feature(c0 + j, qn);
        store8(sX, row, c0, kDin, v);
    }
}

__device__ __forceinline__ void copy_weights(unsigned char* sm, const unsigned char* __restrict__ img,
                                             const float* __restrict__ params, float* bias) {
    const uint4* src = reinterpret_cast<const uint4*>(img);
    uint4* dst = reinterpret_cast<uint4*>(sm + sOffW);
    for (int i = threadIdx.x; i < kImgBytes / 16; i += blockDim.x) dst[i] = __ldg(src + i);
    for (int i = threadIdx.x; i < kH; i += blockDim.x) {
        bias[i] = params[ob1 + i];
        bias[kH + i] = params[ob2 + i];
    }
    if (threadIdx.x < kDout) bias[2 * kH + threadIdx.x] = params[ob3 + threadIdx.x];
}

__device__ __forceinline__ float sigmoidf_(float z) { return 1.f / (1.f + expf(-z)); }
__device__ __forceinline__ float softplusf_(float z) { return z > 0.f ? z + log1pf(expf(-z)) : log1pf(expf(z)); }

struct TrainArgs {
    const float* qn;          // [n][3] normalised queries
    const float* dstar;       // [n][3] normalised displacement targets
    int64_t first;            // first sample of the batch
    int rows;                 // samples in the batch (multiple of 128)
    float lam, inv_delta2;
    const unsigned char* img; // bf16 weight images
    const float* params;      // fp32 master parameters (biases are read from here)
    float* part;              // [tiles][kNParam] per-tile gradient sums
    float* loss_part;         // [tiles]
    int* err;
};

__global__ void __launch_bounds__(kMlpThreads, 1) k_mlp_train(TrainArgs a) {
    extern __shared__ __align__(128) unsigned char sm[];
    __shared__ uint64_t mbar;
    __shared__ uint32_t tbase;
    __shared__ float red[8];
    float* bias = reinterpret_cast<float*>(sm + sOffBias);
    unsigned char* sX = sm + sOffX;
    unsigned char* sH1 = sm + sOffH1;
    unsigned char* sH2 = sm + sOffH2;
    unsigned char* sD2 = sm + sOffD2;
    unsigned char* sD3 = sm + sOffD3;
    float* sD3f = reinterpret_cast<float*>(sm + sOffD3f);
    const unsigned char* sW2 = sm + sOffW + kImgW2;
    const unsigned char* sW3 = sm + sOffW + kImgW3;
    const int warp = threadIdx.x >> 5, row = threadIdx.x & 127, half = threadIdx.x >> 7;
    const int64_t s = a.first + (int64_t)blockIdx.x * kRows + row;
    if (warp == 0) tc::tmem_alloc(&tbase, 512);
    if (threadIdx.x == 0) {
        tc::mbar_init(&mbar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    copy_weights(sm, a.img, a.params, bias);
    const float3 qn = make_float3(a.qn[3 * s], a.qn[3 * s + 1], a.qn[3 * s + 2]);
    write_features(sX, row, half, qn);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    TmemCtl T{&mbar, tbase, 0u, a.err};
    float out[kDout];
    bool ok = forward_tile(sm, bias, T, out);
    // output deltas (first half: one sample per thread)
    float loss = 0.f;
    if (half == 0) {
        float d3[kDout];
        for (int j = 0; j < kDout; ++j) d3[j] = 0.f;
        if (ok) {
            const float t0 = a.dstar[3 * s], t1 = a.dstar[3 * s + 1], t2 = a.dstar[3 * s + 2];
            const float e0 = out[0] - t0, e1 = out[1] - t1, e2 = out[2] - t2;
            const float err2 = e0 * e0 + e1 * e1 + e2 * e2;
            const float cs = expf(-err2 * a.inv_delta2);
            const float z = out[3];
            loss = err2 + a.lam * (softplusf_(z) - cs * z);
            d3[0] = 2.f * e0;
            d3[1] = 2.f * e1;
            d3[2] = 2.f * e2;
            d3[3] = a.lam * (sigmoidf_(z) - cs);
        }
        for (int j = 0; j < kDout; ++j) sD3f[row * kDout + j] = d3[j];
        store8(sD3, row, 0, kDout, d3);
        store8(sD3, row, 8, kDout, d3 + 8);
    }
    to_tensor_core();
    // E2 = d3 W3 (W3 as MN-major: stored [o][i])
    if (threadIdx.x == 0 && ok) {
        tc::mma_bf16(T.base, desc_k(sD3, 0, kDout), desc_mn(sW3, 0, kH), idesc(128, kH, false, true), false);
        tc::mma_commit(T.mbar);
    }
    float* part = a.part + (int64_t)blockIdx.x * kNParam;
    // dW3 and db3 on the CUDA cores while the MMA runs: rows o < 4 are the live outputs
    {
        const int i = threadIdx.x & 127, o0 = 2 * half;
        float acc0 = 0.f, acc1 = 0.f;
        for (int b = 0; b < kRows; ++b) {
            const float h = load_bf16(sH2, b, i, kH);
            acc0 = fmaf(sD3f[b * kDout + o0], h, acc0);
            acc1 = fmaf(sD3f[b * kDout + o0 + 1], h, acc1);
        }
        part[oW3 + o0 * kH + i] = acc0;
        part[oW3 + (o0 + 1) * kH + i] = acc1;
        for (int o = 4 + half; o < kDout; o += 2) part[oW3 + o * kH + i] = 0.f;
        if (threadIdx.x < kDout) {
            float sb = 0.f;
            for (int b = 0; b < kRows; ++b) sb += sD3f[b * kDout + threadIdx.x];
            part[ob3 + threadIdx.x] = sb;
        }
    }
    if (ok) ok = mma_wait(T);
    // d2 = E2 * [h2 > 0] -> sD2
    if (ok) {
        for (int c0 = 64 * half; c0 < 64 * half + 64; c0 += 16) {
            float v[16];
            tc::tmem_ld16(lane_addr(T.base, c0), v);
            for (int j = 0; j < 16; ++j) v[j] = load_bf16(sH2, row, c0 + j, kH) > 0.f ? v[j] : 0.f;
            store8(sD2, row, c0, kH, v);
            store8(sD2, row, c0 + 8, kH, v + 8);
        }
    }
    to_tensor_core();
    // E1 = d2 W2 (W2 as MN-major: stored [j][i]); dW2 = d2^T h1 (both MN-major)
    if (threadIdx.x == 0 && ok) {
        for (int ks = 0; ks < kH / 16; ++ks)
            tc::mma_bf16(T.base + 128, desc_k(sD2, ks, kH), desc_mn(sW2, ks, kH), idesc(128, kH, false, true), ks > 0);
        for (int ks = 0; ks < kRows / 16; ++ks)
            tc::mma_bf16(T.base + 256, desc_mn(sD2, ks, kH), desc_mn(sH1, ks, kH), idesc(128, kH, true, true), ks > 0);
        tc::mma_commit(T.mbar);
    }
    // db2 (column sums of d2) while the MMAs run
    if (threadIdx.x < kH) {
        float sb = 0.f;
        for (int b = 0; b < kRows; ++b) sb += load_bf16(sD2, b, threadIdx.x, kH);
        part[ob2 + threadIdx.x] = sb;
    }
    if (ok) ok = mma_wait(T);
    unsigned char* sD1 = sH2;   // h2 is no longer needed
    if (ok) {
        for (int c0 = 64 * half; c0 < 64 * half + 64; c0 += 16) {
            float v[16];
            tc::tmem_ld16(lane_addr(T.base + 128, c0), v);
            for (int j = 0; j < 16; ++j) v[j] = load_bf16(sH1, row, c0 + j, kH) > 0.f ? v[j] : 0.f;
            store8(sD1, row, c0, kH, v);
            store8(sD1, row, c0 + 8, kH, v + 8);
            float w[16];
            tc::tmem_ld16(lane_addr(T.base + 256, c0), w);     // dW2 row j = row, columns i
            for (int j = 0; j < 16; ++j) part[oW2 + row * kH + c0 + j] = w[j];
        }
    }
    to_tensor_core();
    // dW1 = d1^T x (both MN-major; x has 112 columns)
    if (threadIdx.x == 0 && ok) {
        for (int ks = 0; ks < kRows / 16; ++ks)
            tc::mma_bf16(T.base + 384, desc_mn(sD1, ks, kH), desc_mn(sX, ks, kDin), idesc(128, kDin, true, true), ks > 0);
        tc::mma_commit(T.mbar);
    }
    if (threadIdx.x < kH) {
        float sb = 0.f;
        for (int b = 0; b < kRows; ++b) sb += load_bf16(sD1, b, threadIdx.x, kH);
        part[ob1 + threadIdx.x] = sb;
    }
    if (ok) ok = mma_wait(T);
    if (ok) {
        const int c_lo = half ? 64 : 0, c_hi = half ? kDin : 64;
        for (int c0 = c_lo; c0 < c_hi; c0 += 16) {
            float w[16];
            tc::tmem_ld16(lane_addr(T.base + 384, c0), w);
            for (int j = 0; j < 16; ++j) part[oW1 + row * kDin + c0 + j] = w[j];
        }
    } else {
        for (int i = threadIdx.x; i < kNParam; i += blockDim.x) part[i] = 0.f;
    }
    // tile loss (deterministic: warp sums, then the first thread)
    for (int off = 16; off > 0; off >>= 1) loss += __shfl_down_sync(0xffffffffu, loss, off);
    if ((threadIdx.x & 31) == 0) red[warp] = loss;
    tc::fence_before_sync();
    __syncthreads();
    if (threadIdx.x == 0) {
        float l = 0.f;
        for (int w = 0; w < 8; ++w) l += red[w];
        a.loss_part[blockIdx.x] = l;
    }
    if (warp == 0) tc::tmem_dealloc(tbase, 512);
}

// Sum the per-tile gradients in tile order, scale by 1/n and take one Adam
// step on the fp32 master parameters; rewrite the bf16 weight images.
__global__ void k_mlp_update(const float* __restrict__ part, int tiles, float inv_n, float* __restrict__ params,
                             float* __restrict__ am, float* __restrict__ av, const int* __restrict__ step,
                             float lr, float b1, float b2, float eps, unsigned char* __restrict__ img,
                             float* __restrict__ grad_out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= kNParam) return;
    float g = 0.f;
    for (int t = 0; t < tiles; ++t) g += part[(int64_t)t * kNParam + i];
    g *= inv_n;
    if (grad_out) grad_out[i] = g;
    if (!am) return;                                     // gradient only
    const int tt = *step + 1;
    const float c1 = -expm1f((float)tt * log1pf(-(1.f - b1)));
    const float c2 = -expm1f((float)tt * log1pf(-(1.f - b2)));
    const float mo = fmaf(b1, am[i], (1.f - b1) * g);
    const float ve = fmaf(b2, av[i], (1.f - b2) * g * g);
    am[i] = mo;
    av[i] = ve;
    const float p = params[i] - lr * (mo / c1) / (sqrtf(ve / c2) + eps);
    params[i] = p;
    const __nv_bfloat16 pb = __float2bfloat16_rn(p);
    if (i < ob1) *reinterpret_cast<__nv_bfloat16*>(img + kImgW1 + tc::kmajor_offset(i / kDin, i % kDin, kDin)) = pb;
    else if (i >= oW2 && i < ob2) {
        const int k = i - oW2;
        *reinterpret_cast<__nv_bfloat16*>(img + kImgW2 + tc::kmajor_offset(k / kH, k % kH, kH)) = pb;
    } else if (i >= oW3 && i < ob3) {
        const int k = i - oW3;
        *reinterpret_cast<__nv_bfloat16*>(img + kImgW3 + tc::kmajor_offset(k / kH, k % kH, kH)) = pb;
    }
}

__global__ void k_step_inc(int* step) { *step += 1; }

// bf16 weight images from fp32 parameters.
__global__ void k_mlp_images(const float* __restrict__ params, unsigned char* __restrict__ img) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= kNParam) return;
    const __nv_bfloat16 pb = __float2bfloat16_rn(params[i]);
    if (i < ob1) *reinterpret_cast<__nv_bfloat16*>(img + kImgW1 + tc::kmajor_offset(i / kDin, i % kDin, kDin)) = pb;
    else if (i >= oW2 && i < ob2) {
        const int k = i - oW2;
        *reinterpret_cast<__nv_bfloat16*>(img + kImgW2 + tc::kmajor_offset(k / kH, k % kH, kH)) = pb;
    } else if (i >= oW3 && i < ob3) {
        const int k = i - oW3;
        *reinterpret_cast<__nv_bfloat16*>(img + kImgW3 + tc::kmajor_offset(k / kH, k % kH, kH)) = pb;
    }
}

struct Pose6 {
    float v[6];
};

// Training queries: even samples around reference points (normal offsets
// whose standard deviation is log-uniform in [sd_n / 50, sd_n], normalised
// units), odd samples uniform in the unit cube; stored normalised and in
// metres (the latter for labelling).
__global__ void k_surr_samples(const float4* __restrict__ ref, int M, int64_t n, uint64_t seed, float3 c, float s,
                               float sd_n, float* __restrict__ qn, float* __restrict__ qw) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t base = sm64_at(seed, (uint64_t)i + 1);
        float u[6];
        for (int k = 0; k < 6; ++k) u[k] = ((float)(sm64_at(base, k + 1) >> 40) + 0.5f) * (1.f / 16777216.f);
        float3 p;
        if ((i & 1) == 0) {
            const float4 r = ref[min((int)(u[0] * (float)M), M - 1)];
            const float sd = sd_n * exp2f(-5.64385619f * u[5]);   // 2^-log2(50) = 1/50
            const float g0 = sd * sqrtf(-2.f * logf(u[1])), g1 = sd * sqrtf(-2.f * logf(u[3]));
            float s0, c0, s1, c1;
            sincospif(2.f * u[2], &s0, &c0);
            sincospif(2.f * u[4], &s1, &c1);
            p = make_float3((r.x - c.x) / s + g0 * c0, (r.y - c.y) / s + g0 * s0, (r.z - c.z) / s + g1 * c1);
        } else {
            p = make_float3(2.f * u[0] - 1.f, 2.f * u[1] - 1.f, 2.f * u[2] - 1.f);
        }
        qn[3 * i] = p.x;
        qn[3 * i + 1] = p.y;
        qn[3 * i + 2] = p.z;
        qw[3 * i] = c.x + s * p.x;
        qw[3 * i + 1] = c.y + s * p.y;
        qw[3 * i + 2] = c.z + s * p.z;
    }
}

// Training queries of a registration run: source point s (uniform over the
// source cloud) moved by a pose theta drawn uniformly from the box lo..hi of
// the run's initial particles, q = R(theta) s + u -- the queries that the
// run's own iterations put to the search, as the particles move from their
// initial spread towards the answer.  Stored normalised and in metres.
__global__ void k_surr_samples_run(const float4* __restrict__ src, int64_t N, Pose6 lo, Pose6 hi, int64_t n,
                                   uint64_t seed, float3 c, float s, float* __restrict__ qn, float* __restrict__ qw) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t base = sm64_at(seed, (uint64_t)i + 1);
        float u[7];
        for (int k = 0; k < 7; ++k) u[k] = ((float)(sm64_at(base, k + 1) >> 40) + 0.5f) * (1.f / 16777216.f);
        const float4 s4 = src[min((int64_t)(u[0] * (float)N), N - 1)];
        float th[6];
        for (int a = 0; a < 6; ++a) th[a] = fmaf(hi.v[a] - lo.v[a], u[1 + a], lo.v[a]);
        Pose P;
        make_pose(th, P);
        const float3 q = apply_pose(P, make_float3(s4.x, s4.y, s4.z));
        qw[3 * i] = q.x;
        qw[3 * i + 1] = q.y;
        qw[3 * i + 2] = q.z;
        qn[3 * i] = (q.x - c.x) / s;
        qn[3 * i + 1] = (q.y - c.y) / s;
        qn[3 * i + 2] = (q.z - c.z) / s;
    }
}

// Normalised displacement targets from the exact correspondences.
__global__ void k_surr_targets(const float4* __restrict__ ref, const float* __restrict__ qw,
                               const int32_t* __restrict__ idx, int64_t n, float inv_s, float* __restrict__ dstar) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float4 r = ref[idx[i]];
        dstar[3 * i] = (r.x - qw[3 * i]) * inv_s;
        dstar[3 * i + 1] = (r.y - qw[3 * i + 1]) * inv_s;
        dstar[3 * i + 2] = (r.z - qw[3 * i + 2]) * inv_s;
    }
}

// ---- inference: 256 rows per CTA, two 128-row blocks sharing the weights ----
//
// Thread t owns row t (row block t / 128, tensor-memory lane t % 128).  The
// features of a block and its second activation share a buffer (the features
// are dead once the first MMA of the block has completed).
constexpr int kPairRows = 2 * kRows;
constexpr int pOffXH = kImgBytes;                      // 2 x 32 KB: features, then h2
constexpr int pOffH1 = pOffXH + 2 * kRows * kH * 2;    // 2 x 32 KB
constexpr int pOffQ = pOffH1 + 2 * kRows * kH * 2;     // 256 float4
constexpr int pOffBias = pOffQ + kPairRows * 16;
constexpr int kPairSmem = pOffBias + (kH + kH + kDout) * 4;
constexpr int kPairTmemCols = 256;

__device__ __forceinline__ uint32_t pair_lane_addr(uint32_t base, int rb, int col) {
    const int warp = threadIdx.x >> 5;
    return base + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)(rb * kH + col);
}

// One dense layer's epilogue for this thread's row: bias, ReLU, bf16 into `dst`.
__device__ __forceinline__ void pair_epilogue(uint32_t tbase, int rb, int row, const float* bias, unsigned char* dst) {
#pragma unroll 1
    for (int c0 = 0; c0 < kH; c0 += 16) {
        float v[16];
        tc::tmem_ld16(pair_lane_addr(tbase, rb, c0), v);
#pragma unroll
        for (int j = 0; j < 16; ++j) v[j] = fmaxf(v[j] + bias[c0 + j], 0.f);
        store8(dst, row, c0, kH, v);
        store8(dst, row, c0 + 8, kH, v + 8);
    }
}

// Forward of both row blocks; the features are already in the X/H2 buffers.
// out[] receives this thread's 16 outputs (biases added).  False on a wait failure.
__device__ bool forward_pair(unsigned char* sm, const float* bias, TmemCtl& T, float out[kDout]) {
    const unsigned char* sW1 = sm + kImgW1;
    const unsigned char* sW2 = sm + kImgW2;
    const unsigned char* sW3 = sm + kImgW3;
    const int rb = threadIdx.x >> 7, row = threadIdx.x & 127;
    unsigned char* myXH = sm + pOffXH + rb * (kRows * kH * 2);
    unsigned char* myH1 = sm + pOffH1 + rb * (kRows * kH * 2);
    to_tensor_core();
    if (threadIdx.x == 0) {
        for (int b = 0; b < 2; ++b) {
            const unsigned char* X = sm + pOffXH + b * (kRows * kH * 2);
            for (int ks = 0; ks < kDin / 16; ++ks)
                tc::mma_bf16(T.base + b * kH, desc_k(X, ks, kDin), desc_k(sW1, ks, kDin), idesc(128, kH, false, false),
                             ks > 0);
        }
        tc::mma_commit(T.mbar);
    }
    if (!mma_wait(T)) return false;
    pair_epilogue(T.base, rb, row, bias, myH1);
    to_tensor_core();
    if (threadIdx.x == 0) {
        for (int b = 0; b < 2; ++b) {
            const unsigned char* H1 = sm + pOffH1 + b * (kRows * kH * 2);
            for (int ks = 0; ks < kH / 16; ++ks)
                tc::mma_bf16(T.base + b * kH, desc_k(H1, ks, kH), desc_k(sW2, ks, kH), idesc(128, kH, false, false),
                             ks > 0);
        }
        tc::mma_commit(T.mbar);
    }
    if (!mma_wait(T)) return false;
    pair_epilogue(T.base, rb, row, bias + kH, myXH);
    to_tensor_core();
    if (threadIdx.x == 0) {
        for (int b = 0; b < 2; ++b) {
            const unsigned char* H2 = sm + pOffXH + b * (kRows * kH * 2);
            for (int ks = 0; ks < kH / 16; ++ks)
                tc::mma_bf16(T.base + b * kH, desc_k(H2, ks, kH), desc_k(sW3, ks, kH), idesc(128, kDout, false, false),
                             ks > 0);
        }
        tc::mma_commit(T.mbar);
    }
    if (!mma_wait(T)) return false;
    tc::tmem_ld16(pair_lane_addr(T.base, rb, 0), out);
#pragma unroll
    for (int j = 0; j < kDout; ++j) out[j] += bias[2 * kH + j];
    return true;
}

// All 112 features of this thread's row.  The angle pi w_f v is evaluated as
// sincospi(2^(8f/15) v), which needs no large-argument reduction.
__device__ __forceinline__ void write_features_row(unsigned char* X, int row, float3 qn) {
    float v[8];
    v[0] = qn.x;
    v[1] = qn.y;
    v[2] = qn.z;
    int n = 3, c0 = 0;
    const float a3[3] = {qn.x, qn.y, qn.z};
#pragma unroll 1
    for (int f = 0; f < 16; ++f) {
        const float sc = exp2f(8.f * (float)f / 15.f);
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            float sn, cs;
            sincospif(sc * a3[a], &sn, &cs);
            v[n++] = sn;
            if (n == 8) { store8(X, row, c0, kDin, v); c0 += 8; n = 0; }
            v[n++] = cs;
            if (n == 8) { store8(X, row, c0, kDin, v); c0 += 8; n = 0; }
        }
    }
    // 99 features written; pad to 112 with zeros
    for (; n < 8; ++n) v[n] = 0.f;
    store8(X, row, c0, kDin, v);
    c0 += 8;
    const float z[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    for (; c0 < kDin; c0 += 8) store8(X, row, c0, kDin, z);
}

__device__ __forceinline__ void pair_setup(unsigned char* sm, uint64_t* mbar, uint32_t* tbase,
                                           const unsigned char* img, const float* params, float* bias) {
    if ((threadIdx.x >> 5) == 0) tc::tmem_alloc(tbase, kPairTmemCols);
    if (threadIdx.x == 0) {
        tc::mbar_init(mbar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    copy_weights(sm, img, params, bias);
}

struct InferArgs {
    const float* q;           // [n][3] metres
    int64_t n;
    float3 c;
    float s;
    const unsigned char* img;
    const float* params;
    float* disp;              // [n][3] metres
    float* conf;              // [n]
    int* err;
};

__global__ void __launch_bounds__(kMlpThreads, 1) k_mlp_infer(InferArgs a) {
    extern __shared__ __align__(128) unsigned char sm[];
    __shared__ uint64_t mbar;
    __shared__ uint32_t tbase;
    float* bias = reinterpret_cast<float*>(sm + pOffBias);
    const int rb = threadIdx.x >> 7, row = threadIdx.x & 127;
    const int64_t i = (int64_t)blockIdx.x * kPairRows + threadIdx.x;
    pair_setup(sm, &mbar, &tbase, a.img, a.params, bias);
    float3 qn = make_float3(0.f, 0.f, 0.f);
    if (i < a.n) qn = make_float3((a.q[3 * i] - a.c.x) / a.s, (a.q[3 * i + 1] - a.c.y) / a.s, (a.q[3 * i + 2] - a.c.z) / a.s);
    write_features_row(sm + pOffXH + rb * (kRows * kH * 2), row, qn);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    TmemCtl T{&mbar, tbase, 0u, a.err};
    float out[kDout];
    const bool ok = forward_pair(sm, bias, T, out);
    if (i < a.n) {
        a.disp[3 * i] = ok ? a.s * out[0] : 0.f;
        a.disp[3 * i + 1] = ok ? a.s * out[1] : 0.f;
        a.disp[3 * i + 2] = ok ? a.s * out[2] : 0.f;
        a.conf[i] = ok ? sigmoidf_(out[3]) : 0.f;
    }
    tc::fence_before_sync();
    __syncthreads();
    if ((threadIdx.x >> 5) == 0) tc::tmem_dealloc(tbase, kPairTmemCols);
}

struct SurrGradArgs {
    const float4* src;
    int64_t n_src;            // source points (bounds checks)
    const int32_t* mb;        // m indices
    int m;
    const float* theta;       // K x 6
    int K;
    float3 c;
    float s;
    float min_conf;
    const unsigned char* img;
    const float* params;
    float* qterms;            // [K][m][6] gradient terms per query, particle-major
    int* fb_list;             // queries left to the exact search
    int* fb_count;            // their number (zero on entry)
    unsigned long long* stats;  // [8] or null: slot 6 surrogate queries, slot 7 queries left to the exact search
    int* err;
};

// 256 (particle, minibatch entry) queries of one iteration, query g = j m + k:
// the surrogate's displacement where it is confident and inside the trained
// cube, giving that query's gradient terms; the others go on a list for the
// exact search.
__global__ void __launch_bounds__(kMlpThreads, 1) k_grad_surrogate(SurrGradArgs a) {
    extern __shared__ __align__(128) unsigned char sm[];
    __shared__ uint64_t mbar;
    __shared__ uint32_t tbase;
    __shared__ int nfall, fbase;
    __shared__ int fall[kPairRows];
    float* bias = reinterpret_cast<float*>(sm + pOffBias);
    const int rb = threadIdx.x >> 7, row = threadIdx.x & 127;
    const int Q = a.K * a.m;
    const int g = blockIdx.x * kPairRows + threadIdx.x;
    const bool live = g < Q;
    const int j = live ? g / a.m : 0, k = live ? g % a.m : 0;
    if (threadIdx.x == 0) nfall = 0;
    pair_setup(sm, &mbar, &tbase, a.img, a.params, bias);
    Pose P;
    make_pose(a.theta + 6 * j, P);
    float3 s3 = make_float3(0.f, 0.f, 0.f);
    if (live) {
        const float4 s4 = __ldg(a.src + SICP_IDX(__ldg(a.mb + k), a.n_src, kChkSrc));
        s3 = make_float3(s4.x, s4.y, s4.z);
    }
    const float3 q = apply_pose(P, s3);
    const float3 qn = make_float3((q.x - a.c.x) / a.s, (q.y - a.c.y) / a.s, (q.z - a.c.z) / a.s);
    write_features_row(sm + pOffXH + rb * (kRows * kH * 2), row, qn);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    TmemCtl T{&mbar, tbase, 0u, a.err};
    float out[kDout];
    const bool ok = forward_pair(sm, bias, T, out);
    if (live) {
        const bool inside = fabsf(qn.x) <= 1.f && fabsf(qn.y) <= 1.f && fabsf(qn.z) <= 1.f;   // the trained cube
        const float cf = sigmoidf_(out[3]);
        if (ok && inside && cf >= a.min_conf && isfinite(out[0] + out[1] + out[2])) {
            // r^ = q + s d~, so the residual q - r^ is -s d~
            float t[6];
            grad_terms(P, s3, make_float3(-a.s * out[0], -a.s * out[1], -a.s * out[2]), t);
            float* dst = a.qterms + (int64_t)g * 6;
#pragma unroll
            for (int c = 0; c < 6; ++c) dst[c] = t[c];
        } else {
            fall[atomicAdd(&nfall, 1)] = g;
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    if ((threadIdx.x >> 5) == 0) tc::tmem_dealloc(tbase, kPairTmemCols);
    if (threadIdx.x == 0) fbase = nfall ? atomicAdd(a.fb_count, nfall) : 0;
    __syncthreads();
    for (int f = threadIdx.x; f < nfall; f += blockDim.x) a.fb_list[fbase + f] = fall[f];
    if (a.stats && threadIdx.x == 0) {
        const int nl = min(kPairRows, Q - (int)blockIdx.x * kPairRows);
        atomicAdd(a.stats + 6, (unsigned long long)nl);
        atomicAdd(a.stats + 7, (unsigned long long)nfall);
    }
}

struct FallbackArgs {
    const float4* src;
    int64_t n_src;            // source points (bounds checks)
    int64_t nq;               // queries of the iteration, K m (bounds checks)
    const int32_t* mb;
    int m;
    const float* theta;
    GridSearch S;
    const int* fb_list;
    const int* fb_count;
    float* qterms;
    unsigned long long* stats;
};

// The exact grid search for the listed queries, one warp per query; writes
// their gradient terms.
__global__ void __launch_bounds__(128, 8) k_grad_fallback(FallbackArgs a) {
    const int lane = threadIdx.x & 31;
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nw = (gridDim.x * blockDim.x) >> 5;
    const int n = *a.fb_count;
    Work w;
    for (int f = gw; f < n; f += nw) {
        const int g = (int)SICP_IDX(__ldg(a.fb_list + f), a.nq, kChkFallback);
        const int j = g / a.m, k = g % a.m;
        Pose P;
        make_pose(a.theta + 6 * j, P);
        const float4 s4 = __ldg(a.src + SICP_IDX(__ldg(a.mb + k), a.n_src, kChkSrc));
        const float3 s3 = make_float3(s4.x, s4.y, s4.z);
        const float3 q = apply_pose(P, s3);
        Best B;
        grid_search(a.S, q, B, w);
        if (lane == 0) {
            float t[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
            if (B.i != kNone) grad_terms(P, s3, make_float3(q.x - B.p.x, q.y - B.p.y, q.z - B.p.z), t);
            float* dst = a.qterms + (int64_t)g * 6;
#pragma unroll
            for (int c = 0; c < 6; ++c) dst[c] = t[c];
        }
    }
    if (a.stats) add_stats(a.stats, w);
}

}  // namespace

// ---------------------------------------------------------------- host side

struct Surrogate {
    Buf params, am, av, img, part, loss_part, losses, step, qn, qw, dstar, idx, grad, saved;
    Buf fb;   // fallback count (first int, padded to 16 ints) then the fallback list
    float3 c = {0, 0, 0};
    float s = 1.f;
    bool trained = false;
    int64_t n_train = 0;
    ~Surrogate() {
        Buf* bs[] = {&params, &am, &av, &img, &part, &loss_part, &losses, &step, &qn, &qw, &dstar, &idx, &grad, &saved, &fb};
        for (Buf* b : bs)
            if (b->p) cudaFree(b->p);
    }
};

void surrogate_destroy(Surrogate* s) { delete s; }

cudaError_t surrogate_kernel_attrs() {
    cudaError_t e = cudaFuncSetAttribute(k_mlp_train, cudaFuncAttributeMaxDynamicSharedMemorySize, kTrainSmem);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_mlp_infer, cudaFuncAttributeMaxDynamicSharedMemorySize, kPairSmem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_grad_surrogate, cudaFuncAttributeMaxDynamicSharedMemorySize, kPairSmem);
    return e;
}

bool surrogate_ready(const sicp_ctx* ctx) { return ctx->surr && ctx->surr->trained; }

void surrogate_invalidate(sicp_ctx* ctx) {
    if (ctx->surr) ctx->surr->trained = false;
    ++ctx->surr_gen;
}

namespace {

constexpr int kMaxTrainRows = 65536;   // samples per gradient pass (per-tile partials: 132 KB per 128 samples)

int surr_alloc(sicp_ctx* ctx) {
    if (!ctx->surr) ctx->surr = new Surrogate();
    Surrogate& S = *ctx->surr;
    int rc;
    if ((rc = ensure(ctx, S.params, sizeof(float) * kNParam))) return rc;
    if ((rc = ensure(ctx, S.am, sizeof(float) * kNParam))) return rc;
    if ((rc = ensure(ctx, S.av, sizeof(float) * kNParam))) return rc;
    if ((rc = ensure(ctx, S.img, kImgBytes))) return rc;
    if ((rc = ensure(ctx, S.step, sizeof(int) * 4))) return rc;
    if ((rc = ensure(ctx, S.grad, sizeof(float) * kNParam))) return rc;
    if ((rc = ensure(ctx, S.saved, sizeof(float) * kNParam + kImgBytes))) return rc;
    if ((rc = ensure(ctx, S.losses, sizeof(float) * 4))) return rc;
    return SICP_OK;
}

// Normalisation: centre of the reference bounding box, 0.6 x its largest extent.
void surr_norm_from_reference(sicp_ctx* ctx) {
    Surrogate& S = *ctx->surr;
    S.c = make_float3(0.5f * (ctx->ref_lo.x + ctx->ref_hi.x), 0.5f * (ctx->ref_lo.y + ctx->ref_hi.y),
                      0.5f * (ctx->ref_lo.z + ctx->ref_hi.z));
    const float ext = fmaxf(ctx->ref_hi.x - ctx->ref_lo.x, fmaxf(ctx->ref_hi.y - ctx->ref_lo.y, ctx->ref_hi.z - ctx->ref_lo.z));
    S.s = ext > 0.f ? 0.6f * ext : 1.f;
}

// Per-tile gradients of `rows` samples starting at `first` into S.part, tile
// losses into S.loss_part (both sized by the caller for rows / 128 tiles).
cudaError_t launch_train_tiles(Surrogate& S, const float* qn, const float* dstar, int64_t first, int rows, float lam,
                               float delta, int* err, cudaStream_t s) {
    TrainArgs a;
    a.qn = qn;
    a.dstar = dstar;
    a.first = first;
    a.rows = rows;
    a.lam = lam;
    a.inv_delta2 = 1.f / (delta * delta);
    a.img = (const unsigned char*)S.img.p;
    a.params = (const float*)S.params.p;
    a.part = (float*)S.part.p;
    a.loss_part = (float*)S.loss_part.p;
    a.err = err;
    k_mlp_train<<<rows / kRows, kMlpThreads, kTrainSmem, s>>>(a);
    return cudaGetLastError();
}

__global__ void k_sum_loss(const float* __restrict__ loss_part, int tiles, float inv_n, float* __restrict__ out) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        float s = 0.f;
        for (int t = 0; t < tiles; ++t) s += loss_part[t];
        *out = s * inv_n;
    }
}

unsigned blocks_n(int64_t n, int threads) {
    int64_t b = (n + threads - 1) / threads;
    return (unsigned)(b < 1 ? 1 : (b > 8192 ? 8192 : b));
}

// He-normal initial weights from a counter-based stream (splitmix64 pairs,
// Box-Muller); biases zero; only the four live outputs get weights.
void init_params(std::vector<float>& p, uint64_t seed) {
    p.assign(kNParam, 0.f);
    auto normal = [&](uint64_t k) {
        const uint64_t a = sm64_at(seed, 2 * k + 1), b = sm64_at(seed, 2 * k + 2);
        const double u1 = ((double)(a >> 11) + 0.5) * (1.0 / 9007199254740992.0);
        const double u2 = (double)(b >> 11) * (1.0 / 9007199254740992.0);
        return sqrt(-2.0 * log(u1)) * cos(6.283185307179586 * u2);
    };
    uint64_t k = 0;
    for (int i = 0; i < kH * kDin; ++i) p[oW1 + i] = (float)(normal(k++) * sqrt(2.0 / kDin));
    for (int i = 0; i < kH * kH; ++i) p[oW2 + i] = (float)(normal(k++) * sqrt(2.0 / kH));
    for (int o = 0; o < 4; ++o)
        for (int i = 0; i < kH; ++i) p[oW3 + o * kH + i] = (float)(normal(k++) * 0.01);
}

cudaError_t launch_images(Surrogate& S, cudaStream_t s) {
    k_mlp_images<<<(kNParam + 255) / 256, 256, 0, s>>>((const float*)S.params.p, (unsigned char*)S.img.p);
    return cudaGetLastError();
}

}  // namespace

int surrogate_prepare(sicp_ctx* ctx, int64_t queries) {
    Surrogate& S = *ctx->surr;
    void* before = S.fb.p;
    int rc = ensure(ctx, S.fb, sizeof(int) * (size_t)(queries + 16));
    if (rc) return rc;
    if (S.fb.p != before) ++ctx->surr_gen;   // captured graphs hold the old pointer
    SICP_CUDA(cudaMemsetAsync(S.fb.p, 0, sizeof(int) * 16, ctx->stream));
    return SICP_OK;
}

cudaError_t surrogate_launch_grad(sicp_ctx* ctx, const float4* src, const int32_t* mb, int m, const float* theta,
                                  int K, float min_conf, float* qterms, float* gbar, unsigned long long* stats,
                                  int* err, int* fb_keep) {
    Surrogate& S = *ctx->surr;
    int* fb_count = (int*)S.fb.p;
    int* fb_list = fb_count + 16;
    SurrGradArgs a;
    a.src = src;
    a.n_src = ctx->src_n;
    a.mb = mb;
    a.m = m;
    a.theta = theta;
    a.K = K;
    a.c = S.c;
    a.s = S.s;
    a.min_conf = min_conf;
    a.img = (const unsigned char*)S.img.p;
    a.params = (const float*)S.params.p;
    a.qterms = qterms;
    a.fb_list = fb_list;
    a.fb_count = fb_count;
    a.stats = stats;
    a.err = err;
    const int64_t tiles = ((int64_t)K * m + kPairRows - 1) / kPairRows;
    k_grad_surrogate<<<(unsigned)tiles, kMlpThreads, kPairSmem, ctx->stream>>>(a);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    FallbackArgs f;
    f.src = src;
    f.n_src = ctx->src_n;
    f.nq = (int64_t)K * m;
    f.mb = mb;
    f.m = m;
    f.theta = theta;
    f.S = ctx->search;
    f.fb_list = fb_list;
    f.fb_count = fb_count;
    f.qterms = qterms;
    f.stats = stats;
    k_grad_fallback<<<(unsigned)(ctx->num_sms * 8), 128, 0, ctx->stream>>>(f);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    return launch_qterms_to_gbar(qterms, K, m, 1.f / (float)m, gbar, fb_count, ctx->stream, fb_keep);
}

}  // namespace sicp

using namespace sicp;

namespace {

struct DevScope {
    int prev = -1;
    explicit DevScope(int d) {
        cudaGetDevice(&prev);
        if (prev != d) cudaSetDevice(d);
    }
    ~DevScope() {
        int cur = -1;
        cudaGetDevice(&cur);
        if (prev >= 0 && cur != prev) cudaSetDevice(prev);
    }
};

int read_err_flag(sicp_ctx* ctx, int* out) {
    int flags[4] = {0, 0, 0, 0};
    SICP_CUDA(cudaMemcpyAsync(flags, ctx->flags.p, sizeof flags, cudaMemcpyDeviceToHost, ctx->stream));
    SICP_CUDA(cudaStreamSynchronize(ctx->stream));
    *out = flags[3];
    return SICP_OK;
}

}  // namespace

namespace {

// Where the training queries come from: the fixed distribution around the
// reference (src null), or a run's source points under poses from its
// particles' box.
struct RunSampling {
    const float4* src = nullptr;
    int64_t N = 0;
    Pose6 lo{}, hi{};
};

int surrogate_train_impl(sicp_ctx* ctx, int64_t n_queries, uint64_t seed, int32_t epochs, int32_t batch, float lr,
                         float* out_loss, const RunSampling& run) {
    if (ctx->M < 1) return set_err(ctx, SICP_ENOREF, "no reference cloud set");
    if (n_queries < kRows || n_queries > ((int64_t)1 << 26) || epochs < 1 || epochs > 100000 || batch < kRows ||
        batch > kMaxTrainRows || batch % kRows || !(lr > 0.f) || !isfinite(lr))
        return set_err(ctx, SICP_EINVAL,
                       "surrogate training needs 128 <= n <= 2^26, 1 <= epochs <= 1e5, batch a multiple of 128 "
                       "in [128, %d] and lr > 0",
                       kMaxTrainRows);
    const int64_t n = (n_queries / batch) * batch;
    if (n < batch) return set_err(ctx, SICP_EINVAL, "n_queries must be at least one batch");
    DevScope ds(ctx->device);
    int rc = surr_alloc(ctx);
    if (rc) return rc;
    Surrogate& S = *ctx->surr;
    cudaStream_t s = ctx->stream;
    S.trained = false;
    ++ctx->surr_gen;
    surr_norm_from_reference(ctx);
    const int steps = (int)(n / batch);
    const int tiles = batch / kRows;
    if ((rc = ensure(ctx, S.qn, sizeof(float) * 3 * n))) return rc;
    if ((rc = ensure(ctx, S.qw, sizeof(float) * 3 * n))) return rc;
    if ((rc = ensure(ctx, S.dstar, sizeof(float) * 3 * n))) return rc;
    if ((rc = ensure(ctx, S.idx, sizeof(int32_t) * n))) return rc;
    if ((rc = ensure(ctx, S.losses, sizeof(float) * (size_t)steps))) return rc;
    if ((rc = ensure(ctx, S.part, sizeof(float) * (size_t)tiles * kNParam))) return rc;
    if ((rc = ensure(ctx, S.loss_part, sizeof(float) * tiles))) return rc;
    // initial weights and Adam state
    std::vector<float> p0;
    init_params(p0, seed ^ 0x5eedULL);
    SICP_CUDA(cudaMemcpyAsync(S.params.p, p0.data(), sizeof(float) * kNParam, cudaMemcpyHostToDevice, s));
    SICP_CUDA(cudaMemsetAsync(S.am.p, 0, sizeof(float) * kNParam, s));
    SICP_CUDA(cudaMemsetAsync(S.av.p, 0, sizeof(float) * kNParam, s));
    SICP_CUDA(cudaMemsetAsync(S.step.p, 0, sizeof(int) * 4, s));
    SICP_CUDA(launch_images(S, s));
    // labelled samples: exact correspondences from the grid search
    if (run.src)
        k_surr_samples_run<<<blocks_n(n, 256), 256, 0, s>>>(run.src, run.N, run.lo, run.hi, n, seed, S.c, S.s,
                                                             (float*)S.qn.p, (float*)S.qw.p);
    else
        k_surr_samples<<<blocks_n(n, 256), 256, 0, s>>>(ctx->ref4, (int)ctx->M, n, seed, S.c, S.s, 0.1f,
                                                         (float*)S.qn.p, (float*)S.qw.p);
    SICP_CUDA(cudaGetLastError());
    SICP_CUDA(launch_nn_grid(ctx->search, (const float*)S.qw.p, n, (int32_t*)S.idx.p, nullptr, nullptr, s));
    k_surr_targets<<<blocks_n(n, 256), 256, 0, s>>>(ctx->ref4, (const float*)S.qw.p, (const int32_t*)S.idx.p, n,
                                                     1.f / S.s, (float*)S.dstar.p);
    SICP_CUDA(cudaGetLastError());
    SICP_CUDA(cudaMemsetAsync(ctx->flags.p, 0, 4 * sizeof(int), s));
    int* err = (int*)ctx->flags.p + 3;
    const float lam = 0.1f, delta = 0.01f;
    // one epoch captured in a graph and replayed `epochs` times
    cudaGraph_t graph;
    cudaGraphExec_t exec = nullptr;
    SICP_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = cudaSuccess;
    for (int b = 0; b < steps && e == cudaSuccess; ++b) {
        e = launch_train_tiles(S, (const float*)S.qn.p, (const float*)S.dstar.p, (int64_t)b * batch, batch, lam, delta,
                               err, s);
        if (e != cudaSuccess) break;
        k_mlp_update<<<(kNParam + 255) / 256, 256, 0, s>>>((const float*)S.part.p, tiles, 1.f / (float)batch,
                                                           (float*)S.params.p, (float*)S.am.p, (float*)S.av.p,
                                                           (const int*)S.step.p, lr, 0.9f, 0.999f, 1e-8f,
                                                           (unsigned char*)S.img.p, nullptr);
        k_sum_loss<<<1, 32, 0, s>>>((const float*)S.loss_part.p, tiles, 1.f / (float)batch, (float*)S.losses.p + b);
        k_step_inc<<<1, 1, 0, s>>>((int*)S.step.p);
        e = cudaGetLastError();
    }
    cudaError_t e2 = cudaStreamEndCapture(s, &graph);
    if (e != cudaSuccess) {
        if (e2 == cudaSuccess) cudaGraphDestroy(graph);
        return cuda_err(ctx, e, "surrogate training launch");
    }
    if (e2 != cudaSuccess) return cuda_err(ctx, e2, "cudaStreamEndCapture (surrogate training)");
    e = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return cuda_err(ctx, e, "cudaGraphInstantiate (surrogate training)");
    for (int ep = 0; ep < epochs && e == cudaSuccess; ++ep) e = cudaGraphLaunch(exec, s);
    std::vector<float> losses(steps);
    int flags[4] = {0, 0, 0, 0};
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(losses.data(), S.losses.p, sizeof(float) * steps, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(flags, ctx->flags.p, sizeof flags, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaGraphExecDestroy(exec);
    if (e != cudaSuccess) return cuda_err(ctx, e, "surrogate training");
    if (flags[3]) return set_err(ctx, SICP_ETIMEOUT, "a tensor-core wait of the surrogate training gave up");
    S.trained = true;
    S.n_train = n;
    if (out_loss) {
        double sum = 0.0;
        for (float l : losses) sum += l;
        *out_loss = (float)(sum / steps);   // mean batch loss over the last epoch
    }
    return SICP_OK;
}

}  // namespace

extern "C" int sicp_surrogate_train(sicp_ctx* ctx, int64_t n_queries, uint64_t seed, int32_t epochs, int32_t batch,
                                    float lr, float* out_loss) {
    sicp::NvtxRange nvtx_("surrogate_train");
    if (!ctx) return SICP_EINVAL;
    ctx->err.clear();
    return surrogate_train_impl(ctx, n_queries, seed, epochs, batch, lr, out_loss, RunSampling{});
}

extern "C" int sicp_surrogate_train_run(sicp_ctx* ctx, const float* src_xyz, int64_t N, const float* particles,
                                        int32_t K, int64_t n_queries, uint64_t seed, int32_t epochs, int32_t batch,
                                        float lr, float* out_loss, int on_device) {
    sicp::NvtxRange nvtx_("surrogate_train");
    if (!ctx) return SICP_EINVAL;
    ctx->err.clear();
    if (!src_xyz || !particles || N < 1 || N > 0x7fffffff || K < 1 || K > 2048)
        return set_err(ctx, SICP_EINVAL, "run sampling needs a source (1 <= N < 2^31) and 1 <= K <= 2048 particles");
    DevScope ds(ctx->device);
    std::vector<float> th(6 * (size_t)K);
    if (on_device) {
        SICP_CUDA(cudaMemcpyAsync(th.data(), particles, sizeof(float) * th.size(), cudaMemcpyDeviceToHost, ctx->stream));
        SICP_CUDA(cudaStreamSynchronize(ctx->stream));
    } else {
        memcpy(th.data(), particles, sizeof(float) * th.size());
    }
    RunSampling run;
    for (int a = 0; a < 6; ++a) {
        run.lo.v[a] = run.hi.v[a] = th[a];
        for (int32_t j = 1; j < K; ++j) {
            run.lo.v[a] = fminf(run.lo.v[a], th[6 * j + a]);
            run.hi.v[a] = fmaxf(run.hi.v[a], th[6 * j + a]);
        }
        if (!isfinite(run.lo.v[a]) || !isfinite(run.hi.v[a])) return set_err(ctx, SICP_EINVAL, "non-finite particle");
    }
    const void* d_src = src_xyz;
    if (!on_device) {
        int rc = ensure(ctx, ctx->tmp_in, sizeof(float) * 3 * (size_t)N);
        if (rc) return rc;
        SICP_CUDA(cudaMemcpyAsync(ctx->tmp_in.p, src_xyz, sizeof(float) * 3 * (size_t)N, cudaMemcpyHostToDevice,
                                  ctx->stream));
        d_src = ctx->tmp_in.p;
    }
    int rc = ensure(ctx, ctx->src4, sizeof(float4) * (size_t)N);
    if (rc) return rc;
    SICP_CUDA(cudaMemsetAsync(ctx->flags.p, 0, 4 * sizeof(int), ctx->stream));
    SICP_CUDA(launch_pack_points((const float*)d_src, N, (float4*)ctx->src4.p, (int*)ctx->flags.p, ctx->stream));
    ctx->src_n = N;
    int bad = 0;
    {
        int flags[4];
        SICP_CUDA(cudaMemcpyAsync(flags, ctx->flags.p, sizeof flags, cudaMemcpyDeviceToHost, ctx->stream));
        SICP_CUDA(cudaStreamSynchronize(ctx->stream));
        bad = flags[0];
    }
    if (bad) return set_err(ctx, SICP_EINVAL, "non-finite source point");
    run.src = (const float4*)ctx->src4.p;
    run.N = N;
    return surrogate_train_impl(ctx, n_queries, seed, epochs, batch, lr, out_loss, run);
}

extern "C" int sicp_surrogate_params(sicp_ctx* ctx, int set, float* params, float* norm4) {
    if (!ctx) return SICP_EINVAL;
    ctx->err.clear();
    if (!params || !norm4) return set_err(ctx, SICP_EINVAL, "null pointer");
    if (set) {
        for (int i = 0; i < kNParam; ++i)
            if (!isfinite(params[i])) return set_err(ctx, SICP_EINVAL, "non-finite parameter");
        for (int a = 0; a < 3; ++a)
            if (!isfinite(norm4[a])) return set_err(ctx, SICP_EINVAL, "non-finite centre");
        if (!(norm4[3] > 0.f) || !isfinite(norm4[3])) return set_err(ctx, SICP_EINVAL, "scale must be positive");
    } else if (!surrogate_ready(ctx)) {
        return set_err(ctx, SICP_ENOSURROGATE, "no trained surrogate on this context");
    }
    DevScope ds(ctx->device);
    int rc = surr_alloc(ctx);
    if (rc) return rc;
    Surrogate& S = *ctx->surr;
    cudaStream_t s = ctx->stream;
    if (set) {
        SICP_CUDA(cudaMemcpyAsync(S.params.p, params, sizeof(float) * kNParam, cudaMemcpyHostToDevice, s));
        SICP_CUDA(launch_images(S, s));
        S.c = make_float3(norm4[0], norm4[1], norm4[2]);
        S.s = norm4[3];
        S.trained = true;
        ++ctx->surr_gen;
    } else {
        SICP_CUDA(cudaMemcpyAsync(params, S.params.p, sizeof(float) * kNParam, cudaMemcpyDeviceToHost, s));
        norm4[0] = S.c.x;
        norm4[1] = S.c.y;
        norm4[2] = S.c.z;
        norm4[3] = S.s;
    }
    SICP_CUDA(cudaStreamSynchronize(s));
    return SICP_OK;
}

extern "C" int sicp_surrogate_loss_grad(sicp_ctx* ctx, const float* params, const float* qn, const float* dstar,
                                        int64_t n, float lam, float delta, float* out_loss, float* out_grad) {
    if (!ctx) return SICP_EINVAL;
    ctx->err.clear();
    if (!params || !qn || !dstar || !out_grad) return set_err(ctx, SICP_EINVAL, "null pointer");
    if (n < kRows || n % kRows || n > kMaxTrainRows || !(delta > 0.f) || !isfinite(delta) || !isfinite(lam))
        return set_err(ctx, SICP_EINVAL, "loss_grad needs n a multiple of 128 in [128, %d], finite lam, delta > 0",
                       kMaxTrainRows);
    for (int i = 0; i < kNParam; ++i)
        if (!isfinite(params[i])) return set_err(ctx, SICP_EINVAL, "non-finite parameter");
    DevScope ds(ctx->device);
    int rc = surr_alloc(ctx);
    if (rc) return rc;
    Surrogate& S = *ctx->surr;
    cudaStream_t s = ctx->stream;
    const int tiles = (int)(n / kRows);
    if ((rc = ensure(ctx, S.qn, sizeof(float) * 3 * n))) return rc;
    if ((rc = ensure(ctx, S.dstar, sizeof(float) * 3 * n))) return rc;
    if ((rc = ensure(ctx, S.part, sizeof(float) * (size_t)tiles * kNParam))) return rc;
    if ((rc = ensure(ctx, S.loss_part, sizeof(float) * tiles))) return rc;
    // the given parameters replace the context's only for this call
    float* sp = (float*)S.saved.p;
    SICP_CUDA(cudaMemcpyAsync(sp, S.params.p, sizeof(float) * kNParam, cudaMemcpyDeviceToDevice, s));
    SICP_CUDA(cudaMemcpyAsync(sp + kNParam, S.img.p, kImgBytes, cudaMemcpyDeviceToDevice, s));
    SICP_CUDA(cudaMemcpyAsync(S.params.p, params, sizeof(float) * kNParam, cudaMemcpyHostToDevice, s));
    SICP_CUDA(cudaMemcpyAsync(S.qn.p, qn, sizeof(float) * 3 * n, cudaMemcpyHostToDevice, s));
    SICP_CUDA(cudaMemcpyAsync(S.dstar.p, dstar, sizeof(float) * 3 * n, cudaMemcpyHostToDevice, s));
    SICP_CUDA(cudaMemsetAsync(ctx->flags.p, 0, 4 * sizeof(int), s));
    cudaError_t e = launch_images(S, s);
    if (e == cudaSuccess)
        e = launch_train_tiles(S, (const float*)S.qn.p, (const float*)S.dstar.p, 0, (int)n, lam, delta,
                               (int*)ctx->flags.p + 3, s);
    if (e == cudaSuccess) {
        k_mlp_update<<<(kNParam + 255) / 256, 256, 0, s>>>((const float*)S.part.p, tiles, 1.f / (float)n, nullptr,
                                                           nullptr, nullptr, nullptr, 0.f, 0.f, 0.f, 0.f, nullptr,
                                                           (float*)S.grad.p);
        k_sum_loss<<<1, 32, 0, s>>>((const float*)S.loss_part.p, tiles, 1.f / (float)n, (float*)S.losses.p);
        e = cudaGetLastError();
    }
    // put the context's parameters back whatever happened above
    cudaError_t r1 = cudaMemcpyAsync(S.params.p, sp, sizeof(float) * kNParam, cudaMemcpyDeviceToDevice, s);
    cudaError_t r2 = cudaMemcpyAsync(S.img.p, sp + kNParam, kImgBytes, cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) return cuda_err(ctx, e, "surrogate loss/gradient launch");
    if (r1 != cudaSuccess || r2 != cudaSuccess) return cuda_err(ctx, r1 != cudaSuccess ? r1 : r2, "restore");
    SICP_CUDA(cudaMemcpyAsync(out_grad, S.grad.p, sizeof(float) * kNParam, cudaMemcpyDeviceToHost, s));
    if (out_loss) SICP_CUDA(cudaMemcpyAsync(out_loss, S.losses.p, sizeof(float), cudaMemcpyDeviceToHost, s));
    int tc_err = 0;
    if ((rc = read_err_flag(ctx, &tc_err))) return rc;
    if (tc_err) return set_err(ctx, SICP_ETIMEOUT, "a tensor-core wait gave up");
    return SICP_OK;
}

extern "C" int sicp_surrogate_infer(sicp_ctx* ctx, const float* q, int64_t n, float* out_disp, float* out_conf,
                                    int on_device) {
    if (!ctx) return SICP_EINVAL;
    ctx->err.clear();
    if (n < 0 || n > ((int64_t)1 << 28)) return set_err(ctx, SICP_EINVAL, "query count out of range");
    if (n == 0) return SICP_OK;
    if (!q || !out_disp || !out_conf) return set_err(ctx, SICP_EINVAL, "null pointer");
    if (!surrogate_ready(ctx)) return set_err(ctx, SICP_ENOSURROGATE, "no trained surrogate on this context");
    DevScope ds(ctx->device);
    Surrogate& S = *ctx->surr;
    cudaStream_t s = ctx->stream;
    const float* dq = q;
    float *dd = out_disp, *dc = out_conf;
    int rc;
    if (!on_device) {
        if ((rc = ensure(ctx, ctx->tmp_in, sizeof(float) * 3 * n))) return rc;
        if ((rc = ensure(ctx, ctx->tmp_out, sizeof(float) * 4 * n))) return rc;
        SICP_CUDA(cudaMemcpyAsync(ctx->tmp_in.p, q, sizeof(float) * 3 * n, cudaMemcpyHostToDevice, s));
        dq = (const float*)ctx->tmp_in.p;
        dd = (float*)ctx->tmp_out.p;
        dc = dd + 3 * n;
    }
    SICP_CUDA(cudaMemsetAsync(ctx->flags.p, 0, 4 * sizeof(int), s));
    InferArgs a;
    a.q = dq;
    a.n = n;
    a.c = S.c;
    a.s = S.s;
    a.img = (const unsigned char*)S.img.p;
    a.params = (const float*)S.params.p;
    a.disp = dd;
    a.conf = dc;
    a.err = (int*)ctx->flags.p + 3;
    k_mlp_infer<<<(unsigned)((n + kPairRows - 1) / kPairRows), kMlpThreads, kPairSmem, s>>>(a);
    SICP_CUDA(cudaGetLastError());
    if (!on_device) {
        SICP_CUDA(cudaMemcpyAsync(out_disp, dd, sizeof(float) * 3 * n, cudaMemcpyDeviceToHost, s));
        SICP_CUDA(cudaMemcpyAsync(out_conf, dc, sizeof(float) * n, cudaMemcpyDeviceToHost, s));
    }
    int tc_err = 0;
    if ((rc = read_err_flag(ctx, &tc_err))) return rc;
    if (tc_err) return set_err(ctx, SICP_ETIMEOUT, "a tensor-core wait gave up");
    return SICP_OK;
}

// ---------------------------------------------------------------- weight file
//
// Little-endian file: "SICPSURR", u32 version (1), u32 parameter count
// (33,040), float norm4[4] (centre, scale), float params[33040] (the order of
// sicp_surrogate_params), u32 FNV-1a checksum of every byte after the magic
// and before the checksum.

namespace {

constexpr char kMagic[8] = {'S', 'I', 'C', 'P', 'S', 'U', 'R', 'R'};
constexpr uint32_t kFileVersion = 1;

uint32_t fnv1a(const unsigned char* p, size_t n, uint32_t h = 2166136261u) {
    for (size_t i = 0; i < n; ++i) {
        h ^= p[i];
        h *= 16777619u;
    }
    return h;
}

}  // namespace

extern "C" int sicp_surrogate_save(sicp_ctx* ctx, const char* path) {
    if (!ctx) return SICP_EINVAL;
    ctx->err.clear();
    if (!path) return set_err(ctx, SICP_EINVAL, "null path");
    std::vector<float> body(4 + kNParam);
    int rc = sicp_surrogate_params(ctx, 0, body.data() + 4, body.data());
    if (rc) return rc;
    std::vector<unsigned char> buf(8 + 8 + sizeof(float) * body.size() + 4);
    unsigned char* w = buf.data();
    memcpy(w, kMagic, 8);
    const uint32_t hdr[2] = {kFileVersion, (uint32_t)kNParam};
    memcpy(w + 8, hdr, 8);
    memcpy(w + 16, body.data(), sizeof(float) * body.size());
    const uint32_t sum = fnv1a(w + 8, buf.size() - 12);
    memcpy(w + buf.size() - 4, &sum, 4);
    FILE* f = fopen(path, "wb");
    if (!f) return set_err(ctx, SICP_EINVAL, "cannot open %s for writing", path);
    const size_t n = fwrite(buf.data(), 1, buf.size(), f);
    const int cl = fclose(f);
    if (n != buf.size() || cl != 0) return set_err(ctx, SICP_EINVAL, "write to %s failed", path);
    return SICP_OK;
}

extern "C" int sicp_surrogate_load(sicp_ctx* ctx, const char* path) {
    if (!ctx) return SICP_EINVAL;
    ctx->err.clear();
    if (!path) return set_err(ctx, SICP_EINVAL, "null path");
    FILE* f = fopen(path, "rb");
    if (!f) return set_err(ctx, SICP_EINVAL, "cannot open %s", path);
    const size_t want = 8 + 8 + sizeof(float) * (4 + kNParam) + 4;
    std::vector<unsigned char> buf(want + 1);
    const size_t n = fread(buf.data(), 1, buf.size(), f);
    fclose(f);
    if (n != want) return set_err(ctx, SICP_EINVAL, "%s: %zu bytes, a weight file has %zu", path, n, want);
    if (memcmp(buf.data(), kMagic, 8) != 0) return set_err(ctx, SICP_EINVAL, "%s: not a surrogate weight file", path);
    uint32_t hdr[2], sum;
    memcpy(hdr, buf.data() + 8, 8);
    memcpy(&sum, buf.data() + want - 4, 4);
    if (hdr[0] != kFileVersion || hdr[1] != (uint32_t)kNParam)
        return set_err(ctx, SICP_EINVAL, "%s: version %u with %u parameters, expected %u with %d", path, hdr[0], hdr[1],
                       kFileVersion, kNParam);
    if (fnv1a(buf.data() + 8, want - 12) != sum) return set_err(ctx, SICP_EINVAL, "%s: checksum mismatch", path);
    std::vector<float> body(4 + kNParam);
    memcpy(body.data(), buf.data() + 16, sizeof(float) * body.size());
    return sicp_surrogate_params(ctx, 1, body.data() + 4, body.data());
}
