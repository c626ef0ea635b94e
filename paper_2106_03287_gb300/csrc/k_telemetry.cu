// Per-iteration telemetry of a registration run (sicp_set_telemetry).  The
// paper has no such output; it serves to watch a run: one row per iteration
// with the particles' mean and spread at the start of the iteration, the mean
// distance from the iteration's queries to their correspondences, and the
// share of queries the learned closest-point field answered.
//
// Two launches per iteration, between the gradient and the Stein step (the
// particles are still those the iteration started from):
//   k_tel_part  one CTA per particle: its m queries' distances, summed in a
//               fixed order (strided per thread, then a tree);
//   k_tel_row   one CTA: mean and standard deviation of the particles in
//               float64, the distance sums over particles, the row.
// Both are deterministic, and neither writes anything the run reads.
#include <math.h>

#include "common.cuh"

namespace sicp {
namespace {

constexpr int kPartThreads = 128;
constexpr int kRowThreads = 256;

__global__ void __launch_bounds__(kPartThreads) k_tel_part(TelArgs a) {
    __shared__ Pose P;
    __shared__ float sd[kPartThreads], sc[kPartThreads];
    const int j = blockIdx.x, tid = threadIdx.x;
    if (tid == 0) make_pose(a.theta + 6 * j, P);
    __syncthreads();
    const int32_t* mb = a.mb + (int64_t)j * a.mb_stride;
    float dsum = 0.f, cnt = 0.f;
    for (int k = tid; k < a.m; k += kPartThreads) {
        const int64_t q = (int64_t)j * a.m + k;
        if (a.nn) {   // exact iteration: distance to the nearest reference point
            const int32_t r = a.nn[q];
            if (r >= 0) {
                const float4 s4 = __ldg(a.src + SICP_IDX(__ldg(mb + k), a.n_src, kChkSrc));
                const float3 x = apply_pose(P, make_float3(s4.x, s4.y, s4.z));
                const float4 c = __ldg(a.ref4 + SICP_IDX(r, a.n_ref, kChkRef));
                const float dx = x.x - c.x, dy = x.y - c.y, dz = x.z - c.z;
                dsum += sqrtf(fmaf(dx, dx, fmaf(dy, dy, dz * dz)));
                cnt += 1.f;
            }
        } else {      // learned iteration: the residual the query's gradient terms carry
            const float* e = a.qterms + 6 * q;
            dsum += sqrtf(fmaf(e[0], e[0], fmaf(e[1], e[1], e[2] * e[2])));
            cnt += 1.f;
        }
    }
    sd[tid] = dsum;
    sc[tid] = cnt;
    __syncthreads();
    for (int h = kPartThreads / 2; h > 0; h >>= 1) {
        if (tid < h) {
            sd[tid] += sd[tid + h];
            sc[tid] += sc[tid + h];
        }
        __syncthreads();
    }
    if (tid == 0) {
        a.part[j] = sd[0];
        a.part[a.K + j] = sc[0];
    }
}

// Sum of v over the CTA in a fixed order (every thread calls it; all get the sum).
__device__ double block_sum(double v, double* red) {
    const int tid = threadIdx.x;
    red[tid] = v;
    __syncthreads();
    for (int h = kRowThreads / 2; h > 0; h >>= 1) {
        if (tid < h) red[tid] += red[tid + h];
        __syncthreads();
    }
    const double s = red[0];
    __syncthreads();
    return s;
}

__global__ void __launch_bounds__(kRowThreads) k_tel_row(TelArgs a) {
    __shared__ double red[kRowThreads];
    __shared__ double mean[6];
    const int tid = threadIdx.x, K = a.K;
    for (int c = 0; c < 6; ++c) {
        double s = 0.0;
        for (int j = tid; j < K; j += kRowThreads) s += (double)a.theta[6 * j + c];
        s = block_sum(s, red);
        if (tid == 0) mean[c] = s / (double)K;
    }
    __syncthreads();
    for (int c = 0; c < 6; ++c) {
        double s = 0.0;
        for (int j = tid; j < K; j += kRowThreads) {
            const double d = (double)a.theta[6 * j + c] - mean[c];
            s += d * d;
        }
        s = block_sum(s, red);
        if (tid == 0) {
            a.row[c] = (float)mean[c];
            a.row[6 + c] = K > 1 ? (float)sqrt(s / (double)(K - 1)) : 0.f;
        }
    }
    double ds = 0.0, dc = 0.0;
    for (int j = tid; j < K; j += kRowThreads) {
        ds += (double)a.part[j];
        dc += (double)a.part[K + j];
    }
    ds = block_sum(ds, red);
    dc = block_sum(dc, red);
    if (tid == 0) {
        const double q = (double)K * (double)a.m;
        a.row[12] = dc > 0.0 ? (float)(ds / dc) : 0.f;
        a.row[13] = a.fb ? (float)(1.0 - (double)*a.fb / q) : 0.f;
        a.row[14] = (float)a.t_abs;
        a.row[15] = (float)(dc / q);
    }
}

}  // namespace

cudaError_t launch_telemetry(const TelArgs& a, cudaStream_t s) {
    if (a.K <= 0) return cudaSuccess;
    k_tel_part<<<(unsigned)a.K, kPartThreads, 0, s>>>(a);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_tel_row<<<1, kRowThreads, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace sicp
