// Minibatch selection (Sec. III-B: SGD-ICP draws m source points per
// iteration; one minibatch is shared by all particles, as Eq. stein_icp_phi
// uses a single M).  The minibatch of iteration t is the set of m source
// indices whose splitmix64 keys are smallest, in ascending index order.
//
// One CTA per iteration.  The m-th smallest key is found by an exact radix
// select over the 64-bit keys (8-bit digits from the top, a 256-bin shared
// histogram per pass, keys recomputed each pass instead of stored), and the
// selected indices are then compacted in index order with a block scan.
#include "common.cuh"

namespace sicp {
namespace {

constexpr int kThreads = 1024;

// The minibatch of iteration t into row[0..m) by the whole CTA (kThreads threads).
__device__ __forceinline__ void minibatch_row(uint64_t seed, int64_t t, int64_t N, int32_t m,
                                              int32_t* __restrict__ row) {
    __shared__ unsigned hist[256];
    __shared__ uint64_t s_prefix;
    __shared__ unsigned s_rem;
    __shared__ int s_done;
    __shared__ unsigned warp_cnt[32];

    const int tid = threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5;
    const uint64_t base = sm64_at(seed, (uint64_t)t + 1);

    uint64_t prefix = 0, mask = 0;
    unsigned rem = (unsigned)m;       // rank (1-based) still wanted among keys matching prefix
    for (int shift = 56; shift >= 0; shift -= 8) {
        for (int i = tid; i < 256; i += kThreads) hist[i] = 0;
        __syncthreads();
        for (int64_t i = tid; i < N; i += kThreads) {
            uint64_t k = sm64_at(base, (uint64_t)i + 1);
            if ((k & mask) == prefix) atomicAdd(&hist[(k >> shift) & 255u], 1u);
        }
        __syncthreads();
        if (warp == 0) {
            unsigned c[8], tot = 0;
#pragma unroll
            for (int b = 0; b < 8; ++b) { c[b] = hist[lane * 8 + b]; tot += c[b]; }
            unsigned incl = tot;
#pragma unroll
            for (int off = 1; off < 32; off <<= 1) {
                unsigned v = __shfl_up_sync(0xffffffffu, incl, off);
                if (lane >= off) incl += v;
            }
            unsigned excl = incl - tot;
            if (excl < rem && rem <= incl) {
                unsigned acc = excl;
                for (int b = 0; b < 8; ++b) {
                    if (rem <= acc + c[b]) {
                        unsigned r2 = rem - acc;
                        s_prefix = prefix | ((uint64_t)(lane * 8 + b) << shift);
                        s_rem = r2;
                        s_done = (r2 == c[b]);   // every key in this bucket is selected
                        break;
                    }
                    acc += c[b];
                }
            }
        }
        __syncthreads();
        prefix = s_prefix;
        rem = s_rem;
        mask |= (uint64_t)0xff << shift;
        const int done = s_done;
        __syncthreads();
        if (done) break;
    }

    // selected: (key & mask) <= prefix, compacted in ascending index order
    unsigned written = 0;
    for (int64_t i0 = 0; i0 < N; i0 += kThreads) {
        const int64_t i = i0 + tid;
        bool sel = false;
        if (i < N) sel = (sm64_at(base, (uint64_t)i + 1) & mask) <= prefix;
        unsigned bal = __ballot_sync(0xffffffffu, sel);
        if (lane == 0) warp_cnt[warp] = __popc(bal);
        __syncthreads();
        if (warp == 0) {
            unsigned v = warp_cnt[lane], incl = v;
#pragma unroll
            for (int off = 1; off < 32; off <<= 1) {
                unsigned w = __shfl_up_sync(0xffffffffu, incl, off);
                if (lane >= off) incl += w;
            }
            warp_cnt[lane] = incl - v;      // exclusive warp offsets
            if (lane == 31) s_rem = incl;   // total this round
        }
        __syncthreads();
        if (sel) {
            unsigned pos = written + warp_cnt[warp] + __popc(bal & ((1u << lane) - 1u));
            if (pos < (unsigned)m) row[pos] = (int32_t)i;
        }
        written += s_rem;
        __syncthreads();
    }
}

__global__ void __launch_bounds__(kThreads) k_minibatch(uint64_t seed, int64_t t0, int64_t N, int32_t m,
                                                        int32_t* __restrict__ out) {
    minibatch_row(seed, t0 + blockIdx.x, N, m, out + (int64_t)blockIdx.x * m);
}

// grid (T, R): independent run j uses seed + j; row [j][t] of iteration t0 + t.
__global__ void __launch_bounds__(kThreads) k_minibatch_runs(uint64_t seed, int64_t t0, int32_t T, int64_t N,
                                                             int32_t m, int32_t* __restrict__ out) {
    const int j = blockIdx.y, t = blockIdx.x;
    minibatch_row(seed + (uint64_t)j, t0 + t, N, m, out + ((int64_t)j * T + t) * m);
}

// grid (T, P): problem p uses seed + p, its own source size and row [p][t].
__global__ void __launch_bounds__(kThreads) k_minibatch_batched(uint64_t seed, int32_t T, int32_t m,
                                                                const int64_t* __restrict__ src_off,
                                                                int32_t* __restrict__ out) {
    const int p = blockIdx.y, t = blockIdx.x;
    minibatch_row(seed + (uint64_t)p, t, src_off[p + 1] - src_off[p], m, out + ((int64_t)p * T + t) * m);
}

}  // namespace

cudaError_t launch_minibatch_batched(uint64_t seed, int32_t T, int32_t m, int32_t P, const int64_t* src_off,
                                     int32_t* out, cudaStream_t s) {
    if (T <= 0 || P <= 0) return cudaSuccess;
    k_minibatch_batched<<<dim3(T, P), kThreads, 0, s>>>(seed, T, m, src_off, out);
    return cudaGetLastError();
}

cudaError_t launch_minibatch_runs(uint64_t seed, int64_t t0, int32_t T, int64_t N, int32_t m, int32_t R,
                                  int32_t* out, cudaStream_t s) {
    if (T <= 0 || R <= 0) return cudaSuccess;
    k_minibatch_runs<<<dim3(T, R), kThreads, 0, s>>>(seed, t0, T, N, m, out);
    return cudaGetLastError();
}

cudaError_t launch_minibatch(uint64_t seed, int64_t t0, int32_t T, int64_t N, int32_t m,
                             int32_t* out, cudaStream_t s) {
    if (T <= 0) return cudaSuccess;
    k_minibatch<<<T, kThreads, 0, s>>>(seed, t0, N, m, out);
    return cudaGetLastError();
}

}  // namespace sicp
