// Minibatch selection (Sec. III-B: SGD-ICP draws m source points per
// iteration; one minibatch is shared by all particles, as Eq. stein_icp_phi
// uses a single M).  The minibatch of iteration t is the set of m source
// indices whose splitmix64 keys are smallest, in ascending index order.
//
// One CTA of 256 threads per iteration.  The m-th smallest key is found by
// an exact radix select over the 64-bit keys (12-bit digits from the top, so
// that two passes settle almost every row, then 12, 12, 12, 12 and 4 bits; a
// 4096-bin shared histogram per pass; keys recomputed each pass instead of
// stored).  The selected indices are then compacted in index order: thread
// tid owns the contiguous indices [tid per, (tid + 1) per), counts its
// selected keys, and one block scan gives every thread its output offset.
#include <math.h>

#include "common.cuh"

namespace sicp {
namespace {

constexpr int kThreads = 256;
constexpr int kBins = 4096;                    // 12-bit digits
constexpr int kBinsPer = kBins / kThreads;     // bins summed by one thread

// Exclusive prefix of v over the CTA; *total receives the sum.  `wtot` is
// kThreads / 32 words of shared scratch.
__device__ __forceinline__ unsigned block_excl_scan(unsigned v, unsigned* wtot, unsigned* total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned incl = v;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const unsigned x = __shfl_up_sync(0xffffffffu, incl, off);
        if (lane >= off) incl += x;
    }
    if (lane == 31) wtot[warp] = incl;
    __syncthreads();
    unsigned base = 0, all = 0;
    for (int w = 0; w < kThreads / 32; ++w) {
        const unsigned x = wtot[w];
        if (w < warp) base += x;
        all += x;
    }
    __syncthreads();   // wtot may be reused right after
    *total = all;
    return base + incl - v;
}

// The minibatch of iteration t into row[0..m) by the whole CTA (kThreads threads).
// hk: null, or N words of shared memory that keep the top 32 bits of every
// key from the first pass, so that the passes and the selection that only
// look at bits 63..32 read them instead of hashing again (a row whose select
// settles within the top 24 bits, which is almost every row, hashes each key
// once).
__device__ __forceinline__ void minibatch_row(uint64_t seed, int64_t t, int64_t N, int32_t m,
                                              int32_t* __restrict__ row, uint32_t* hk) {
    __shared__ unsigned hist[kBins];
    __shared__ unsigned wtot[kThreads / 32];
    __shared__ uint64_t s_prefix;
    __shared__ unsigned s_rem;
    __shared__ int s_done;

    const int tid = threadIdx.x;
    const uint64_t base = sm64_at(seed, (uint64_t)t + 1);
    const int64_t per = (N + kThreads - 1) / kThreads;
    const int64_t c0 = min(N, (int64_t)tid * per), c1 = min(N, c0 + per);

    uint64_t prefix = 0, mask = 0;
    unsigned rem = (unsigned)m;   // rank (1-based) still wanted among keys matching prefix
    // The first pass counts only the keys whose top 12 bits lie below `lim`:
    // the keys are uniform, so the m smallest lie there with a wide margin
    // (m + 8 sqrt(m) + 16 expected keys), and every bin below `lim` is counted
    // whole.  Should that pass count fewer than m keys, it is repeated over all
    // keys, so the selection stays exact.
    int lim = kBins;
    {
        const float frac = ((float)m + 8.f * sqrtf((float)m) + 16.f) / (float)N;
        if (frac < 0.5f) lim = min(kBins, (int)(frac * (float)kBins) + 2);
    }
    // With the keys stored and at most 64 of them per thread, the keys below the
    // cut are also marked in a per-thread mask: only they can match a later
    // prefix or be selected (a key at or above the cut has a larger top digit
    // than the m-th smallest), so the later passes visit only them.
    const bool cmode = hk && per <= 64;
    uint64_t cand = 0;
    auto key_at = [&](int64_t i, bool top_only) -> uint64_t {
        return top_only ? (uint64_t)hk[i] << 32 : sm64_at(base, (uint64_t)i + 1);
    };
    for (int shift = 52;;) {
        const int width = shift > 0 ? 12 : 4;   // digits 63..52, .., 15..4, then 3..0
        const uint64_t dmask = ((uint64_t)1 << width) - 1;
        for (int i = tid; i < kBins; i += kThreads) hist[i] = 0;
        __syncthreads();
        if (shift == 52) {
            cand = 0;
            for (int64_t i = c0; i < c1; ++i) {
                const uint64_t k = sm64_at(base, (uint64_t)i + 1);
                if (hk) hk[i] = (uint32_t)(k >> 32);
                const unsigned d = (unsigned)(k >> 52);
                if (d < (unsigned)lim) {
                    atomicAdd(&hist[d], 1u);
                    if (cmode) cand |= 1ull << (i - c0);
                }
            }
        } else if (cmode) {   // the digit lies in the top 32 bits while shift >= 32
            for (uint64_t bits = cand; bits; bits &= bits - 1) {
                const int64_t i = c0 + __ffsll((long long)bits) - 1;
                const uint64_t k = key_at(i, shift >= 32);
                if ((k & mask) == prefix) atomicAdd(&hist[(k >> shift) & dmask], 1u);
            }
        } else {
            for (int64_t i = c0; i < c1; ++i) {
                const uint64_t k = key_at(i, hk && shift >= 32);
                if ((k & mask) == prefix) atomicAdd(&hist[(k >> shift) & dmask], 1u);
            }
        }
        __syncthreads();
        // the bin holding rank `rem`: each thread sums kBinsPer consecutive bins
        unsigned cnt[kBinsPer], tot = 0;
#pragma unroll
        for (int b = 0; b < kBinsPer; ++b) {
            cnt[b] = hist[tid * kBinsPer + b];
            tot += cnt[b];
        }
        unsigned all;
        const unsigned excl = block_excl_scan(tot, wtot, &all);
        if (shift == 52 && lim < kBins && all < rem) {   // too few below the cut: count every key
            lim = kBins;
            continue;
        }
        if (excl < rem && rem <= excl + tot) {
            unsigned acc = excl;
#pragma unroll
            for (int b = 0; b < kBinsPer; ++b) {
                if (acc < rem && rem <= acc + cnt[b]) {
                    const unsigned r2 = rem - acc;
                    s_prefix = prefix | ((uint64_t)(tid * kBinsPer + b) << shift);
                    s_rem = r2;
                    s_done = (r2 == cnt[b]);   // every key in this bin is selected
                }
                acc += cnt[b];
            }
        }
        __syncthreads();
        prefix = s_prefix;
        rem = s_rem;
        mask |= dmask << shift;
        const int done = s_done;
        __syncthreads();
        if (done || shift == 0) break;
        shift = shift > 4 ? shift - 12 : 0;
    }

    // selected: (key & mask) <= prefix, exactly m keys: the keys of one row are
    // distinct (the inputs base + (i + 1) gamma differ for every index, gamma
    // being odd, and the splitmix64 finalizer is a bijection on 64 bits), so the
    // m-th smallest is unique; written in ascending index order
    const bool top = hk && (mask & 0xffffffffull) == 0;   // the selection needs only bits 63..32
    unsigned mine = 0;
    uint64_t sel = 0;
    if (cmode) {
        for (uint64_t bits = cand; bits; bits &= bits - 1) {
            const int j = __ffsll((long long)bits) - 1;
            if ((key_at(c0 + j, top) & mask) <= prefix) sel |= 1ull << j;
        }
        mine = (unsigned)__popcll(sel);
    } else {
        for (int64_t i = c0; i < c1; ++i) mine += (key_at(i, top) & mask) <= prefix;
    }
    unsigned all;
    unsigned pos = block_excl_scan(mine, wtot, &all);
    if (cmode) {
        for (uint64_t bits = sel; bits && pos < (unsigned)m; bits &= bits - 1)
            row[pos++] = (int32_t)(c0 + __ffsll((long long)bits) - 1);
    } else {
        for (int64_t i = c0; i < c1 && pos < (unsigned)m; ++i)
            if ((key_at(i, top) & mask) <= prefix) row[pos++] = (int32_t)i;
    }
}

// Rows of at most kStoreKeys keys keep their keys' top halves in dynamic
// shared memory (48 KB).
constexpr int64_t kStoreKeys = 12288;

__device__ __forceinline__ uint32_t* key_store(int64_t N) {
    extern __shared__ uint32_t dyn_keys[];
    return N <= kStoreKeys ? dyn_keys : nullptr;
}

size_t key_store_bytes(int64_t N) { return N <= kStoreKeys ? sizeof(uint32_t) * (size_t)N : 0; }

__global__ void __launch_bounds__(kThreads, 4) k_minibatch(uint64_t seed, int64_t t0, int64_t N, int32_t m,
                                                        int32_t* __restrict__ out) {
    minibatch_row(seed, t0 + blockIdx.x, N, m, out + (int64_t)blockIdx.x * m, key_store(N));
}

// grid (T, R): independent run j uses seed + j; row [j][t] of iteration t0 + t.
__global__ void __launch_bounds__(kThreads, 4) k_minibatch_runs(uint64_t seed, int64_t t0, int32_t T, int64_t N,
                                                             int32_t m, int32_t* __restrict__ out) {
    const int j = blockIdx.y, t = blockIdx.x;
    minibatch_row(seed + (uint64_t)j, t0 + t, N, m, out + ((int64_t)j * T + t) * m, key_store(N));
}

// grid (T, P): problem p uses seed + p, its own source size and row [p][t].
__global__ void __launch_bounds__(kThreads, 4) k_minibatch_batched(uint64_t seed, int32_t T, int32_t m,
                                                                const int64_t* __restrict__ src_off,
                                                                int32_t* __restrict__ out) {
    const int p = blockIdx.y, t = blockIdx.x;
    minibatch_row(seed + (uint64_t)p, t, src_off[p + 1] - src_off[p], m, out + ((int64_t)p * T + t) * m, nullptr);
}

}  // namespace

// The rows that keep their keys in shared memory use kStoreKeys words of
// dynamic shared memory on top of the static histogram: opted in once.
cudaError_t minibatch_kernel_attrs() {
    const int bytes = (int)(sizeof(uint32_t) * kStoreKeys);
    cudaError_t e = cudaFuncSetAttribute(k_minibatch, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(k_minibatch_runs, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

cudaError_t launch_minibatch_batched(uint64_t seed, int32_t T, int32_t m, int32_t P, const int64_t* src_off,
                                     int32_t* out, cudaStream_t s) {
    if (T <= 0 || P <= 0) return cudaSuccess;
    k_minibatch_batched<<<dim3(T, P), kThreads, 0, s>>>(seed, T, m, src_off, out);
    return cudaGetLastError();
}

cudaError_t launch_minibatch_runs(uint64_t seed, int64_t t0, int32_t T, int64_t N, int32_t m, int32_t R,
                                  int32_t* out, cudaStream_t s) {
    if (T <= 0 || R <= 0) return cudaSuccess;
    k_minibatch_runs<<<dim3(T, R), kThreads, key_store_bytes(N), s>>>(seed, t0, T, N, m, out);
    return cudaGetLastError();
}

cudaError_t launch_minibatch(uint64_t seed, int64_t t0, int32_t T, int64_t N, int32_t m,
                             int32_t* out, cudaStream_t s) {
    if (T <= 0) return cudaSuccess;
    k_minibatch<<<T, kThreads, key_store_bytes(N), s>>>(seed, t0, N, m, out);
    return cudaGetLastError();
}

}  // namespace sicp
