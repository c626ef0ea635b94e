// Stein + Adam device code shared by the single-problem kernel and the
// batched persistent kernel.  See k_stein.cu for the description.
#pragma once

#include <float.h>

#include "common.cuh"

namespace sicp {
namespace sd {
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

constexpr int kCacheFloats = 40000;   // pair distances of both blocks kept in shared memory (K <= 200)

// A team is a contiguous range of threads of the CTA with its own named barrier.
struct Team {
    int t0, n, bar;
};
__device__ __forceinline__ void team_sync(const Team& T) {
    asm volatile("bar.sync %0, %1;" ::"r"(T.bar), "r"(T.n) : "memory");
}

// Visit the K(K-1)/2 distances of unique pairs j < l of one block, team-uniformly:
// every thread of the team calls f(valid, value) the same number of times.
template <class F>
__device__ __forceinline__ void for_each_pair(const Team& T, const float* D, bool cached, const float* th, int K,
                                              int block, F f) {
    const int lt = threadIdx.x - T.t0;
    if (cached) {
        const int n = K * (K - 1) / 2;
        for (int base = 0; base < n; base += T.n) {
            const int p = base + lt;
            const bool v = p < n;
            f(v, v ? D[p] : 0.f);
        }
    } else {
        const int n = K * K;
        for (int base = 0; base < n; base += T.n) {
            const int p = base + lt;
            const int j = p / K, l = p % K;
            const bool v = p < n && j < l;
            f(v, v ? pair_d2(th, j, l, block) : 0.f);
        }
    }
}

// Exact value of rank `rank` (0-based) among non-negative floats: radix select
// over their bit patterns with 11-, 11- and 10-bit digits, counting with one
// shared atomic per distinct bin per warp.  visit(f) calls f(valid, value)
// for every value, the same number of times on every thread of the team.
template <class Visit>
__device__ unsigned radix_select(const Team& T, Visit visit, unsigned rank, unsigned* hist, unsigned* s_u,
                                 unsigned* wsum) {
    const int lane = threadIdx.x & 31, lt = threadIdx.x - T.t0, lw = lt >> 5;
    unsigned prefix = 0, mask = 0, rem = rank + 1;
    const int shifts[3] = {21, 10, 0}, widths[3] = {11, 11, 10};
    for (int pass = 0; pass < 3; ++pass) {
        const int shift = shifts[pass], nb = 1 << widths[pass];
        for (int i = lt; i < nb; i += T.n) hist[i] = 0;
        team_sync(T);
        visit([&](bool v, float x) {
            const unsigned b = __float_as_uint(x);
            const bool m = v && (b & mask) == prefix;
            const unsigned bin = m ? (b >> shift) & (unsigned)(nb - 1) : 0xffffffffu;
            const unsigned peers = __match_any_sync(0xffffffffu, bin);
            if (m && lane == __ffs(peers) - 1) atomicAdd(&hist[bin], (unsigned)__popc(peers));
        });
        team_sync(T);
        {
            // team-wide scan of the histogram: thread lt owns bins [lt*per, lt*per + per)
            const int per = nb / T.n;
            unsigned tot = 0;
            for (int q = 0; q < per; ++q) tot += hist[lt * per + q];
            unsigned incl = tot;
#pragma unroll
            for (int off = 1; off < 32; off <<= 1) {
                const unsigned v = __shfl_up_sync(0xffffffffu, incl, off);
                if (lane >= off) incl += v;
            }
            if (lane == 31) wsum[lw] = incl;
            team_sync(T);
            if (lw == 0) {
                const unsigned v = lane < (T.n >> 5) ? wsum[lane] : 0u;
                unsigned vi = v;
#pragma unroll
                for (int off = 1; off < 32; off <<= 1) {
                    const unsigned u = __shfl_up_sync(0xffffffffu, vi, off);
                    if (lane >= off) vi += u;
                }
                if (lane < (T.n >> 5)) wsum[lane] = vi - v;
            }
            team_sync(T);
            incl += wsum[lw];
            unsigned acc = incl - tot;
            if (acc < rem && rem <= incl) {
                for (int q = 0; q < per; ++q) {
                    const unsigned c = hist[lt * per + q];
                    if (rem <= acc + c) {
                        s_u[0] = prefix | ((unsigned)(lt * per + q) << shift);
                        s_u[1] = rem - acc;
                        break;
                    }
                    acc += c;
                }
            }
        }
        team_sync(T);
        prefix = s_u[0];
        rem = s_u[1];
        mask |= (unsigned)(nb - 1) << shift;
        team_sync(T);
    }
    return prefix;
}

// Rank `rank` among the unique pair distances of one block.
__device__ unsigned select_rank(const Team& T, const float* D, bool cached, const float* th, int K, int block,
                                unsigned rank, unsigned* hist, unsigned* s_u, unsigned* wsum) {
    return radix_select(
        T, [&](auto f) { for_each_pair(T, D, cached, th, K, block, f); }, rank, hist, s_u, wsum);
}

constexpr float kBracketRel = 0.25f;   // half-width of the bracket, relative to the previous median
constexpr int kBins = 2048;            // linear bins over the bracket
constexpr int kBinMax = 1024;          // values of one target bin ranked directly

// Warm start of the selection: the unique-pair distances of unique ranks
// u[0] <= u[1] (cached in D, n of them) are looked for in the bracket
// [lo, hi] = m_prev * (1 -+ kBracketRel) around the previous iteration's
// median.  One pass counts the values below lo and sorts those inside into
// kBins linear bins of the bracket; bin(x) = floor((x - lo) * kBins / (hi -
// lo)) is monotone in x in floating point, so a lower bin holds only smaller
// values.  A scan of the bin counts gives the bin of each target rank and its
// rank inside the bin; the values of that bin are then ranked directly.  True,
// with the two values in v[], when both ranks fall inside the bracket and each
// target bin holds at most kBinMax values; the caller takes the full selection
// otherwise.  Exact either way: the values found are the same order statistics.
__device__ bool bracket_select(const Team& T, const float* D, int n, const unsigned u[2], float m_prev, float* C,
                               unsigned* hist, unsigned* s_u, unsigned* wsum, float v[2]) {
    const int lane = threadIdx.x & 31, lt = threadIdx.x - T.t0, lw = lt >> 5;
    const float lo = m_prev * (1.f - kBracketRel), hi = m_prev * (1.f + kBracketRel);
    const float scale = (float)kBins / (hi - lo);
    auto bin_of = [&](float x) { return min(kBins - 1, (int)((x - lo) * scale)); };
    for (int b = lt; b < kBins; b += T.n) hist[b] = 0;
    if (lt == 0) s_u[0] = 0;   // values below the bracket
    team_sync(T);
    for (int base = 0; base < n; base += T.n) {
        const int p = base + lt;
        const float x = p < n ? D[p] : FLT_MAX;
        const unsigned below = __ballot_sync(0xffffffffu, p < n && x < lo);
        if (lane == 0 && below) atomicAdd(&s_u[0], (unsigned)__popc(below));
        if (p < n && x >= lo && x <= hi) atomicAdd(&hist[bin_of(x)], 1u);
    }
    team_sync(T);
    const unsigned c_lt = s_u[0];
    // team-wide scan of the bin counts: thread lt owns bins [lt*per, lt*per + per)
    const int per = kBins / T.n;
    unsigned tot = 0;
    for (int q = 0; q < per; ++q) tot += hist[lt * per + q];
    unsigned incl = tot;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const unsigned x = __shfl_up_sync(0xffffffffu, incl, off);
        if (lane >= off) incl += x;
    }
    if (lane == 31) wsum[lw] = incl;
    if (lt == 0) {
        s_u[1] = 0xffffffffu;   // bin of u[0] (none yet)
        s_u[3] = 0xffffffffu;   // bin of u[1]
    }
    team_sync(T);
    if (lw == 0) {
        const unsigned x = lane < (T.n >> 5) ? wsum[lane] : 0u;
        unsigned xi = x;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const unsigned y = __shfl_up_sync(0xffffffffu, xi, off);
            if (lane >= off) xi += y;
        }
        if (lane < (T.n >> 5)) wsum[lane] = xi - x;
    }
    team_sync(T);
    {
        unsigned acc = c_lt + wsum[lw] + incl - tot;   // values below this thread's first bin
        for (int q = 0; q < per; ++q) {
            const unsigned c = hist[lt * per + q];
#pragma unroll
            for (int w = 0; w < 2; ++w)
                if (acc <= u[w] && u[w] < acc + c) {
                    s_u[1 + 2 * w] = (unsigned)(lt * per + q);
                    s_u[2 + 2 * w] = u[w] - acc;
                }
            acc += c;
        }
    }
    team_sync(T);
    const unsigned b0 = s_u[1], r0 = s_u[2], b1 = s_u[3], r1 = s_u[4];
    const bool found = b0 != 0xffffffffu && b1 != 0xffffffffu && hist[b0] <= (unsigned)kBinMax &&
                       hist[b1] <= (unsigned)kBinMax;
    team_sync(T);
    if (!found) return false;
    // gather the values of the target bins (C[0 ..) for b0, C[kBinMax ..) for b1)
    if (lt == 0) {
        s_u[5] = 0;
        s_u[6] = 0;
    }
    team_sync(T);
    for (int base = 0; base < n; base += T.n) {
        const int p = base + lt;
        if (p < n) {
            const float x = D[p];
            if (x >= lo && x <= hi) {
                const unsigned b = (unsigned)bin_of(x);
                if (b == b0) C[atomicAdd(&s_u[5], 1u)] = x;
                if (b == b1 && b1 != b0) C[kBinMax + atomicAdd(&s_u[6], 1u)] = x;
            }
        }
    }
    team_sync(T);
    const unsigned e0 = s_u[5], e1 = b1 != b0 ? s_u[6] : e0;
    const float* E1 = b1 != b0 ? C + kBinMax : C;
    const unsigned rr[2] = {r0, r1};
    // value of local rank r in a bin: the x with #(< x) <= r < #(<= x)
    for (int w = 0; w < 2; ++w) {
        const float* E = w ? E1 : C;
        const unsigned e = w ? e1 : e0;
        for (int i = lt; i < (int)e; i += T.n) {
            const float x = E[i];
            unsigned less = 0, leq = 0;
            for (int k = 0; k < (int)e; ++k) {
                less += E[k] < x;
                leq += E[k] <= x;
            }
            if (less <= rr[w] && rr[w] < leq) s_u[7 + w] = __float_as_uint(x);
        }
    }
    team_sync(T);
    v[0] = __uint_as_float(s_u[7]);
    v[1] = __uint_as_float(s_u[8]);
    team_sync(T);
    return true;
}

// Median heuristic: median of all K*K squared distances of the block (the K
// zeros of the diagonal plus every unique pair twice; the mean of the two
// middle values for an even count) divided by ln(K+1); 1 if the median is 0.
// With m_prev > 0 and the distances cached, a warm start around the previous
// median is tried first; *med_out (if not null) receives the median itself.
__device__ float bandwidth(const Team& T, const float* th, int K, int block, float* D, bool cached,
                           unsigned* hist, unsigned* s_u, unsigned* wsum, float m_prev = 0.f, float* C = nullptr,
                           float* med_out = nullptr) {
    if (K < 2) return 1.f;
    const int lt = threadIdx.x - T.t0;
    if (cached) {
        // unique pairs j < l, row by row: warp w of the team takes rows w, w + warps, ...
        const int lane = threadIdx.x & 31, warps = T.n >> 5;
        for (int j = lt >> 5; j < K - 1; j += warps) {
            const int row = j * K - j * (j + 1) / 2 - j - 1;   // D index of (j, l) is row + l
            for (int l = j + 1 + lane; l < K; l += 32) D[row + l] = pair_d2(th, j, l, block);
        }
        team_sync(T);
    }
    const unsigned n = (unsigned)K * (unsigned)K;
    const unsigned r_lo = (n - 1) / 2, r_hi = n / 2, uK = (unsigned)K;
    if (cached && C && m_prev > 0.f && r_lo >= uK) {
        // full-multiset rank r >= K is unique rank (r - K) / 2
        const unsigned u[2] = {(r_lo - uK) / 2, (r_hi - uK) / 2};
        float v[2];
        if (bracket_select(T, D, K * (K - 1) / 2, u, m_prev, C, hist, s_u, wsum, v)) {
            const float med = r_hi != r_lo ? 0.5f * (v[0] + v[1]) : v[0];
            if (med_out) *med_out = med;
            return med > 0.f ? med / logf((float)K + 1.f) : 1.f;
        }
    }
    // full-multiset rank r maps to 0 for r < K, else to unique rank (r - K) / 2
    unsigned v_lo = 0;
    if (r_lo >= uK) v_lo = select_rank(T, D, cached, th, K, block, (r_lo - uK) / 2, hist, s_u, wsum);
    float med = __uint_as_float(v_lo);
    if (r_hi != r_lo) {
        // the next order statistic: v_lo again if enough values are <= v_lo, else the smallest value above it
        if (lt == 0) {
            s_u[2] = 0;
            s_u[3] = 0x7f800000u;
        }
        team_sync(T);
        unsigned cnt = 0, mn = 0x7f800000u;
        for_each_pair(T, D, cached, th, K, block, [&](bool v, float x) {
            if (!v) return;
            const unsigned b = __float_as_uint(x);
            if (b <= v_lo) ++cnt;
            else mn = min(mn, b);
        });
        atomicAdd(&s_u[2], cnt);
        atomicMin(&s_u[3], mn);
        team_sync(T);
        const unsigned below = uK + 2 * s_u[2];   // full count of values <= v_lo
        const float v_hi = (below > r_hi) ? med : __uint_as_float(s_u[3]);
        med = 0.5f * (med + v_hi);
        team_sync(T);
    }
    if (med_out) *med_out = med;
    return med > 0.f ? med / logf((float)K + 1.f) : 1.f;
}

// One Stein + Adam update of K particles by the whole CTA (1024 threads), with
// its shared memory laid out as described at the top of k_stein.cu.
__device__ __forceinline__ void stein_adam_block(const SteinArgs& a) {
    extern __shared__ float sm[];
    float* th = sm;               // K x 6
    float* G = sm + 6 * a.K;      // K x 6
    float* Ph = sm + 12 * a.K;    // K x 6: the Stein direction
    float* D = sm + 18 * a.K;     // unique pair distances of both blocks when they fit
    __shared__ unsigned hist[2][2048];
    __shared__ unsigned s_u[2][4];
    __shared__ unsigned wsum[2][32];
    __shared__ float s_h[2];
    const int K = a.K, tid = threadIdx.x;
    const int pairs = K * (K - 1) / 2;
    const bool cached = a.cache && 2 * pairs <= kCacheFloats;

    // G = -N gbar + grad log prior, gbar = inv_m * (sum of the chunk partials)
    if (a.chunks == 1) {
        for (int idx = tid; idx < 6 * K; idx += blockDim.x) {
            const float x = a.theta[idx], gb = a.partial[idx];
            const int c = idx % 6;
            if (a.out_gbar) a.out_gbar[idx] = gb * a.inv_m;
            th[idx] = x;
            float pr = 0.f;
            if (a.prior == 1) pr = (c < 3) ? -(x - a.mu[c]) / a.sigma[c] : -a.kappa[c - 3] * sinf(x - a.mu[c]);
            G[idx] = fmaf(-a.N, gb * a.inv_m, pr);
        }
    } else {
        // one warp per component, lanes over chunks, fixed butterfly order
        const int warp = tid >> 5, lane = tid & 31, nwarps = blockDim.x >> 5;
        for (int idx = warp; idx < 6 * K; idx += nwarps) {
            const int j = idx / 6, c = idx % 6;
            float s = 0.f;
            for (int ch = lane; ch < a.chunks; ch += 32) s += a.partial[((int64_t)ch * K + j) * 6 + c];
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
            if (lane == 0) {
                const float x = a.theta[idx];
                if (a.out_gbar) a.out_gbar[idx] = s * a.inv_m;
                th[idx] = x;
                float pr = 0.f;
                if (a.prior == 1) pr = (c < 3) ? -(x - a.mu[c]) / a.sigma[c] : -a.kappa[c - 3] * sinf(x - a.mu[c]);
                G[idx] = fmaf(-a.N, s * a.inv_m, pr);
            }
        }
    }
    __syncthreads();

    // the two halves of the CTA take the translation and rotation medians at the same time
    {
        const int half = tid >= (int)blockDim.x / 2;
        const Team T = {half * (int)blockDim.x / 2, (int)blockDim.x / 2, 1 + half};
        const float h = bandwidth(T, th, K, half, D + (cached ? half * pairs : 0), cached, hist[half], s_u[half],
                                  wsum[half]);
        if (tid == T.t0) s_h[half] = h;
    }
    __syncthreads();
    const float h_t = s_h[0], h_r = s_h[1];
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
            for (int c = 0; c < 6; ++c) Ph[6 * i + c] = acc[c] * invK;
        }
    }
    __syncthreads();
    // Adam on g = -phi, all components in parallel
    for (int idx = tid; idx < 6 * K; idx += blockDim.x) {
        const float phi = Ph[idx];
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

constexpr long long kArriveSpins = 1ll << 22;   // ~0.3 s of 64 ns polls

// The same update for one block only (b = 0: translation x, y, z; b = 1:
// rotation), by CTA q of P: the two blocks share nothing (each has its own
// kernel, bandwidth, gradient components and Adam components), and within a
// block CTA q takes the Stein direction and the Adam step of particles
// [q Kq, (q + 1) Kq), Kq = ceil(K / P).  Every CTA of the block computes the
// same bandwidth from all particles (identical arithmetic), so they exchange
// nothing but one arrival: a CTA writes theta only after all P CTAs of its
// block have read it (a.arrive[b] counts arrivals, a.gen * P of them by the end
// of update a.gen; bounded wait, a.err set on timeout, and then nothing is
// written).  P > 1 needs all CTAs co-resident (see launch_stein_adam).
__device__ __forceinline__ void stein_adam_one_block(const SteinArgs& a, int b, int q, int P) {
    extern __shared__ float sm[];
    float* th = sm;               // K x 6 (all components: pair_d2 indexes the full rows)
    float* G = sm + 6 * a.K;      // K x 6, columns 3b..3b+2 used
    float* Ph = sm + 12 * a.K;    // K x 6, columns 3b..3b+2 of this CTA's particles used
    float* D = sm + 18 * a.K;     // unique pair distances of block b when they fit
    __shared__ unsigned hist[2048];
    __shared__ unsigned s_u[9];
    __shared__ unsigned wsum[32];
    __shared__ float bracket[2 * kBinMax];
    __shared__ int s_fail;
    const int K = a.K, tid = threadIdx.x;
    const int pairs = K * (K - 1) / 2;
    const bool cached = pairs <= kCacheFloats;
    const int c0 = 3 * b;
    const int Kq = (K + P - 1) / P, i0 = min(K, q * Kq), i1 = min(K, i0 + Kq);

    // The particles and the previous median come from the previous Stein step,
    // which has completed before this grid is scheduled (see pdl_wait), so the
    // bandwidth is found before the wait for the gradients, overlapping the
    // end of the gradient kernel.  (Loads through L2: nothing stale from L1.)
    const float m_prev = a.med_state ? __ldcg(a.med_state + b) : 0.f;   // read before the arrival below
    if (tid == 0) s_fail = 0;
    for (int idx = tid; idx < 6 * K; idx += blockDim.x) th[idx] = __ldcg(a.theta + idx);
    __syncthreads();
    const Team T = {0, (int)blockDim.x, 1};
    // the Adam moments of this thread's first component (also from the previous Stein step)
    const int e0 = 3 * i0 + tid;
    const bool has0 = e0 < 3 * i1;
    const int idx0 = 6 * (e0 / 3) + c0 + e0 % 3;
    float am0 = 0.f, av0 = 0.f;
    if (has0) {
        am0 = __ldcg(a.adam_m + idx0);
        av0 = __ldcg(a.adam_v + idx0);
    }
    float med = 0.f;
    const float h = bandwidth(T, th, K, b, D, cached, hist, s_u, wsum, m_prev, bracket, &med);
    const float inv_h = 1.f / h, two_h = 2.f / h;

    pdl_wait();      // the gradients of this iteration
    pdl_trigger();   // the next gradient kernel may be scheduled (it waits for this grid)
    if (a.chunks == 1) {
        for (int e = tid; e < 3 * K; e += blockDim.x) {
            const int j = e / 3, c = c0 + e % 3, idx = 6 * j + c;
            const float x = th[idx], gb = a.partial[idx];
            float pr = 0.f;
            if (a.prior == 1) pr = (c < 3) ? -(x - a.mu[c]) / a.sigma[c] : -a.kappa[c - 3] * sinf(x - a.mu[c]);
            G[idx] = fmaf(-a.N, gb * a.inv_m, pr);
        }
    } else {
        const int warp = tid >> 5, lane = tid & 31, nwarps = blockDim.x >> 5;
        for (int e = warp; e < 3 * K; e += nwarps) {
            const int j = e / 3, c = c0 + e % 3, idx = 6 * j + c;
            float s = 0.f;
            for (int ch = lane; ch < a.chunks; ch += 32) s += a.partial[((int64_t)ch * K + j) * 6 + c];
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
            if (lane == 0) {
                const float x = th[idx];
                float pr = 0.f;
                if (a.prior == 1) pr = (c < 3) ? -(x - a.mu[c]) / a.sigma[c] : -a.kappa[c - 3] * sinf(x - a.mu[c]);
                G[idx] = fmaf(-a.N, s * a.inv_m, pr);
            }
        }
    }
    __syncthreads();
    if (P > 1 && tid == 0) atomicAdd(a.arrive + b, 1u);   // this CTA has read theta

    // S lanes per particle (power of two <= 32), each summing over j = lane (mod S)
    int S = 32;
    while (S > 1 && Kq * S > (int)blockDim.x) S >>= 1;
    const int groups = blockDim.x / S;
    const int g_id = tid / S, g_lane = tid % S;
    const int rounds = (i1 - i0 + groups - 1) / groups;
    const float invK = 1.f / (float)K;
    const float omb1 = 1.f - a.beta1, omb2 = 1.f - a.beta2;
    const float c1 = -expm1f((float)a.t * log1pf(-omb1));
    const float c2 = -expm1f((float)a.t * log1pf(-omb2));
    for (int r = 0; r < rounds; ++r) {
        const int i = i0 + r * groups + g_id;
        const bool valid = i < i1;
        float acc[3] = {0.f, 0.f, 0.f};
        if (valid) {
            const float* ti = th + 6 * i + c0;
            for (int j = g_lane; j < K; j += S) {
                const float* tj = th + 6 * j + c0;
                const float* Gj = G + 6 * j + c0;
                float d[3], Dd = 0.f;
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    d[c] = b ? wrapf(ti[c] - tj[c]) : ti[c] - tj[c];
                    Dd = fmaf(d[c], d[c], Dd);
                }
                const float k = expf(-Dd * inv_h);
#pragma unroll
                for (int c = 0; c < 3; ++c) acc[c] += k * fmaf(two_h, d[c], Gj[c]);
            }
        }
#pragma unroll
        for (int c = 0; c < 3; ++c)
            for (int off = S >> 1; off > 0; off >>= 1) acc[c] += __shfl_xor_sync(0xffffffffu, acc[c], off, S);
        if (valid && g_lane == 0) {
#pragma unroll
            for (int c = 0; c < 3; ++c) Ph[6 * i + c0 + c] = acc[c] * invK;
        }
    }
    __syncthreads();
    if (P > 1) {
        // every CTA of the block has read theta (and the previous median) once all have arrived
        if (tid == 0) {
            const unsigned target = a.gen * (unsigned)P + a.extra;
            const long long limit = a.max_spins > 0 ? a.max_spins : kArriveSpins;
            long long spins = 0;
            for (;;) {
                unsigned now;
                asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(now) : "l"(a.arrive + b) : "memory");
                if ((int)(now - target) >= 0) break;
                // give up after the limit, or at once when another wait of this call already gave up
                if (++spins > limit || *(volatile int*)a.err) {
                    s_fail = 1;
                    atomicExch(a.err, 1);
                    break;
                }
                __nanosleep(64);
            }
        }
        __syncthreads();
        if (s_fail) return;
    }
    if (q == 0 && tid == 0) {
        if (a.out_h) a.out_h[b] = h;
        if (a.med_state) a.med_state[b] = med;
    }
    for (int e = 3 * i0 + tid; e < 3 * i1; e += blockDim.x) {
        const int idx = 6 * (e / 3) + c0 + e % 3;
        const float phi = Ph[idx];
        if (a.out_phi) a.out_phi[idx] = phi;
        const float g = -phi;
        const bool first = e == e0;   // moments loaded before the wait
        const float mo = fmaf(a.beta1, first ? am0 : __ldcg(a.adam_m + idx), omb1 * g);
        const float ve = fmaf(a.beta2, first ? av0 : __ldcg(a.adam_v + idx), omb2 * g * g);
        a.adam_m[idx] = mo;
        a.adam_v[idx] = ve;
        const float mh = mo / c1, vh = ve / c2;
        a.theta[idx] = th[idx] - a.lr * mh / (sqrtf(vh) + a.eps);
    }
}

}  // namespace
}  // namespace sd
}  // namespace sicp
