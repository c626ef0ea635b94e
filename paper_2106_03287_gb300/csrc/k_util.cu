// Small utility kernels: input packing and checks, the chunk reduction that
// turns partial gradient sums into gbar, a bounding box and an exclusive scan
// used by the grid build.
#include <stdlib.h>
#include <string.h>

#include "common.cuh"

namespace sicp {
namespace {

__global__ void k_pack_points(const float* __restrict__ xyz, int64_t n, float4* __restrict__ out,
                              int* __restrict__ flags) {
    int bad = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float x = xyz[3 * i], y = xyz[3 * i + 1], z = xyz[3 * i + 2];
        bad |= !(isfinite(x) && isfinite(y) && isfinite(z));
        out[i] = make_float4(x, y, z, __int_as_float((int)i));
    }
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(flags, 1);
}

__global__ void k_check_finite(const float* __restrict__ x, int64_t n, int* __restrict__ flags) {
    int bad = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        bad |= !isfinite(x[i]);
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(flags, 1);
}

// flags[0] |= 1 on a value that is non-finite or negative
__global__ void k_check_nonneg(const float* __restrict__ x, int64_t n, int* __restrict__ flags) {
    int bad = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        bad |= !(isfinite(x[i]) && x[i] >= 0.f);
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(flags, 1);
}

__global__ void k_check_index(const int32_t* __restrict__ idx, int64_t n, int64_t N, int* __restrict__ flags) {
    int bad = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        bad |= (idx[i] < 0 || idx[i] >= N);
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(flags + 1, 1);
}

__global__ void k_partial_to_gbar(const float* __restrict__ partial, int chunks, int K, float inv_m,
                                  float* __restrict__ gbar) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= 6 * K) return;
    float s = 0.f;
    for (int c = 0; c < chunks; ++c) s += partial[(int64_t)c * 6 * K + i];
    gbar[i] = s * inv_m;
}

__device__ __forceinline__ unsigned float_to_ordered(float f) {
    const unsigned b = __float_as_uint(f);
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}

__global__ void k_bbox(const float4* __restrict__ p, int64_t n, unsigned* __restrict__ lohi) {
    float lo[3] = {3.4e38f, 3.4e38f, 3.4e38f}, hi[3] = {-3.4e38f, -3.4e38f, -3.4e38f};
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float4 v = p[i];
        lo[0] = fminf(lo[0], v.x); lo[1] = fminf(lo[1], v.y); lo[2] = fminf(lo[2], v.z);
        hi[0] = fmaxf(hi[0], v.x); hi[1] = fmaxf(hi[1], v.y); hi[2] = fmaxf(hi[2], v.z);
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        for (int off = 16; off > 0; off >>= 1) {
            lo[a] = fminf(lo[a], __shfl_xor_sync(0xffffffffu, lo[a], off));
            hi[a] = fmaxf(hi[a], __shfl_xor_sync(0xffffffffu, hi[a], off));
        }
    }
    if ((threadIdx.x & 31) == 0) {
        for (int a = 0; a < 3; ++a) {
            atomicMin(lohi + a, float_to_ordered(lo[a]));
            atomicMax(lohi + 3 + a, float_to_ordered(hi[a]));
        }
    }
}

constexpr int kScanThreads = 1024;
constexpr int kScanPer = 4;
constexpr int kScanBlock = kScanThreads * kScanPer;

// Block-wide exclusive scan of one value per thread; returns the exclusive
// prefix and writes the block total to *total.
__device__ __forceinline__ int block_exclusive(int v, int* warp_sums, int* total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int incl = v;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const int w = __shfl_up_sync(0xffffffffu, incl, off);
        if (lane >= off) incl += w;
    }
    if (lane == 31) warp_sums[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        const int nw = blockDim.x >> 5;
        int s = lane < nw ? warp_sums[lane] : 0, si = s;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const int w = __shfl_up_sync(0xffffffffu, si, off);
            if (lane >= off) si += w;
        }
        if (lane < nw) warp_sums[lane] = si - s;
        if (lane == 31) *total = si;
    }
    __syncthreads();
    return warp_sums[warp] + incl - v;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_blocks(const int32_t* __restrict__ in, int64_t n,
                                                              int32_t* __restrict__ out, int32_t* __restrict__ sums) {
    __shared__ int warp_sums[32];
    __shared__ int total;
    const int64_t base = (int64_t)blockIdx.x * kScanBlock + (int64_t)threadIdx.x * kScanPer;
    int v[kScanPer], s = 0;
#pragma unroll
    for (int k = 0; k < kScanPer; ++k) {
        v[k] = (base + k < n) ? in[base + k] : 0;
        s += v[k];
    }
    int run = block_exclusive(s, warp_sums, &total);
#pragma unroll
    for (int k = 0; k < kScanPer; ++k) {
        if (base + k < n) out[base + k] = run;
        run += v[k];
    }
    if (threadIdx.x == 0) sums[blockIdx.x] = total;
}

// Exclusive scan of the block totals in place (one CTA, any count), plus the grand total.
__global__ void __launch_bounds__(kScanThreads) k_scan_sums(int32_t* __restrict__ sums, int nb,
                                                            int32_t* __restrict__ out_total) {
    __shared__ int warp_sums[32];
    __shared__ int total;
    int carry = 0;
    for (int b0 = 0; b0 < nb; b0 += kScanThreads) {
        const int b = b0 + threadIdx.x;
        const int v = b < nb ? sums[b] : 0;
        const int ex = block_exclusive(v, warp_sums, &total);
        if (b < nb) sums[b] = carry + ex;
        carry += total;
        __syncthreads();
    }
    if (threadIdx.x == 0) *out_total = carry;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_add(int32_t* __restrict__ out, int64_t n,
                                                           const int32_t* __restrict__ sums) {
    const int add = sums[blockIdx.x];
    const int64_t base = (int64_t)blockIdx.x * kScanBlock;
    for (int k = threadIdx.x; k < kScanBlock; k += kScanThreads)
        if (base + k < n) out[base + k] += add;
}

unsigned grid_1d(int64_t n, int threads, int cap = 4096) {
    int64_t b = (n + threads - 1) / threads;
    if (b < 1) b = 1;
    if (b > cap) b = cap;
    return (unsigned)b;
}

// gbar[j] = inv_m * (sum over k of qterms[j][k]) in a fixed order.  CTA j
// reads particle j's m x 6 terms as rows of 192 floats (32 minibatch entries
// x 6 components, coalesced): thread (e, c) sums component c of entries
// e, e + 32, ...; then warp c adds the 32 partial sums of component c with a
// fixed butterfly.  Clears the fallback count for the next iteration.
constexpr int kGbarThreads = 192;
__global__ void __launch_bounds__(kGbarThreads) k_qterms_to_gbar(const float* __restrict__ qterms, int K, int m,
                                                                 float inv_m, float* __restrict__ gbar, int* fb_count,
                                                                 int* fb_keep) {
    __shared__ float part[6][33];
    const int j = blockIdx.x, t = threadIdx.x;
    pdl_trigger();   // the Stein step may be scheduled now (it waits for this grid)
    pdl_wait();
    if (j == 0 && t == 0 && fb_count) {
        if (fb_keep) *fb_keep = *fb_count;
        *fb_count = 0;
    }
    const int e = t / 6, c = t % 6;
    const float* row = qterms + (int64_t)j * m * 6;
    // up to 16 values in flight per thread, then added in the order of k
    float acc = 0.f;
    for (int k0 = e; k0 < m; k0 += 32 * 16) {
        float v[16];
#pragma unroll
        for (int i = 0; i < 16; ++i) v[i] = k0 + 32 * i < m ? __ldg(row + 6 * (k0 + 32 * i) + c) : 0.f;
#pragma unroll
        for (int i = 0; i < 16; ++i)
            if (k0 + 32 * i < m) acc += v[i];
    }
    part[c][e] = acc;
    __syncthreads();
    const int w = t >> 5, lane = t & 31;
    if (w < 6) {
        float v = part[w][lane];
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
        if (lane == 0) gbar[6 * j + w] = v * inv_m;
    }
}

}  // namespace

bool pdl_enabled() {
    static const bool on = getenv("SICP_NO_PDL") == nullptr;
    return on;
}

cudaError_t launch_pack_points(const float* xyz, int64_t n, float4* out, int* flags, cudaStream_t s) {
    k_pack_points<<<grid_1d(n, 256), 256, 0, s>>>(xyz, n, out, flags);
    return cudaGetLastError();
}

cudaError_t launch_check_finite(const float* x, int64_t n, int* flags, cudaStream_t s) {
    k_check_finite<<<grid_1d(n, 256), 256, 0, s>>>(x, n, flags);
    return cudaGetLastError();
}

cudaError_t launch_check_nonneg(const float* x, int64_t n, int* flags, cudaStream_t s) {
    k_check_nonneg<<<grid_1d(n, 256), 256, 0, s>>>(x, n, flags);
    return cudaGetLastError();
}

cudaError_t launch_check_index(const int32_t* idx, int64_t n, int64_t N, int* flags, cudaStream_t s) {
    k_check_index<<<grid_1d(n, 256), 256, 0, s>>>(idx, n, N, flags);
    return cudaGetLastError();
}

cudaError_t launch_partial_to_gbar(const float* partial, int chunks, int32_t K, float inv_m, float* gbar,
                                   cudaStream_t s) {
    k_partial_to_gbar<<<(6 * K + 255) / 256, 256, 0, s>>>(partial, chunks, K, inv_m, gbar);
    return cudaGetLastError();
}

cudaError_t launch_qterms_to_gbar(const float* qterms, int32_t K, int32_t m, float inv_m, float* gbar, int* fb_count,
                                  cudaStream_t s, int* fb_keep) {
    if (K <= 0) return cudaSuccess;
    return launch_pdl(k_qterms_to_gbar, dim3(K), dim3(kGbarThreads), 0, s, qterms, K, m, inv_m, gbar, fb_count,
                      fb_keep);
}

cudaError_t launch_bbox(const float4* p, int64_t n, unsigned* lohi, cudaStream_t s) {
    k_bbox<<<grid_1d(n, 256, 1024), 256, 0, s>>>(p, n, lohi);
    return cudaGetLastError();
}

float ordered_to_float(unsigned u) {
    const unsigned b = (u & 0x80000000u) ? (u & 0x7fffffffu) : ~u;
    float f;
    memcpy(&f, &b, 4);
    return f;
}

size_t scan_sums_size(int64_t n) { return (size_t)((n + kScanBlock - 1) / kScanBlock) + 1; }

cudaError_t launch_exclusive_scan(const int32_t* in, int64_t n, int32_t* out, int32_t* sums, cudaStream_t s) {
    const int nb = (int)((n + kScanBlock - 1) / kScanBlock);
    if (nb < 1) {
        return cudaMemsetAsync(out, 0, sizeof(int32_t), s);
    }
    k_scan_blocks<<<nb, kScanThreads, 0, s>>>(in, n, out, sums);
    k_scan_sums<<<1, kScanThreads, 0, s>>>(sums, nb, out + n);
    k_scan_add<<<nb, kScanThreads, 0, s>>>(out, n, sums);
    return cudaGetLastError();
}

}  // namespace sicp
