// Batched Stein ICP: P independent registration problems of uneven sizes in
// one persistent, cooperative kernel launch captured in a CUDA graph.
//
// Layout: reference, source and particle arrays of all problems are packed
// back to back (CSR offsets).  Every problem gets its own two-level voxel
// grid, built for all problems at once by segmented kernels: a global cell
// array holds the problems' cells in problem order, so one exclusive scan of
// all cell counts gives every cell's position in the global sorted point
// array, and problem p's grid views simply point into the global arrays.
//
// The persistent kernel runs T iterations.  Each iteration:
//   gradient phase: every warp of the grid takes work items (problem,
//     particle, chunk of minibatch entries) in a fixed interleaved order and
//     runs the exact grid search and gradient terms of their queries, writing
//     one partial sum per item;
//   grid barrier;
//   Stein phase: each CTA takes whole problems and runs the Stein + Adam
//     update of that problem's particles (the same device code as the
//     single-problem kernel, summing the chunk partials in fixed order);
//   grid barrier.
// The grid barrier is a counter and generation word in global memory; every
// wait is bounded (about 10 s of polling) and gives up with an error flag the
// host reads, so a fault in scheduling cannot hang the device.
//
// Autotuning: sicp_autotune_batched times the persistent kernel over a few
// iterations for each candidate (grid cell-size factor, minibatch entries per
// work item) and keeps the fastest; results are cached per (GPU name, problem
// count, mean reference size) in a small JSON file when a path is given.
#include <float.h>
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <string>
#include <vector>

#include "common.cuh"
#include "nvtx.cuh"
#include "grid_search.cuh"
#include "stein_device.cuh"

namespace sicp {

cudaError_t launch_minibatch_batched(uint64_t seed, int32_t T, int32_t m, int32_t P, const int64_t* src_off,
                                     int32_t* out, cudaStream_t s);

namespace {

using namespace gs;

// CTA shapes of the persistent kernel the autotuner chooses from: 1024 threads, one CTA per SM, with
// the Stein phase's pair distances kept in shared memory; or 512 x 3 / 256 x 6 per SM without that
// cache (48 warps per SM for the search phase, the Stein phase recomputing the distances).
constexpr int kShapes = 3;
constexpr int kShapeThreads[kShapes] = {1024, 512, 256};
constexpr long long kMaxSpins = 1ll << 27;   // ~10 s of 64 ns polls

// Largest p with off[p] <= i, for off[0] = 0 <= i < off[P].
__device__ __forceinline__ int find_problem(const int64_t* __restrict__ off, int P, int64_t i) {
    int lo = 0, hi = P - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(off + mid) <= i) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// ---------------------------------------------------------------- batched build

__global__ void kb_pack(const float* __restrict__ xyz, int64_t n, const int64_t* __restrict__ off, int P,
                        float4* __restrict__ out, int* __restrict__ flags) {
    int bad = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int p = find_problem(off, P, i);
        const float x = xyz[3 * i], y = xyz[3 * i + 1], z = xyz[3 * i + 2];
        bad |= !(isfinite(x) && isfinite(y) && isfinite(z));
        out[i] = make_float4(x, y, z, __int_as_float((int)(i - off[p])));
    }
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(flags, 1);
}

// One CTA per problem: bounding box of its points into lohi[p][6].
__global__ void kb_bbox(const float4* __restrict__ pts, const int64_t* __restrict__ off, float* __restrict__ lohi) {
    __shared__ float red[6][32];
    const int p = blockIdx.x;
    float lo[3] = {FLT_MAX, FLT_MAX, FLT_MAX}, hi[3] = {-FLT_MAX, -FLT_MAX, -FLT_MAX};
    for (int64_t i = off[p] + threadIdx.x; i < off[p + 1]; i += blockDim.x) {
        const float4 v = pts[i];
        lo[0] = fminf(lo[0], v.x); lo[1] = fminf(lo[1], v.y); lo[2] = fminf(lo[2], v.z);
        hi[0] = fmaxf(hi[0], v.x); hi[1] = fmaxf(hi[1], v.y); hi[2] = fmaxf(hi[2], v.z);
    }
    for (int a = 0; a < 3; ++a)
        for (int o = 16; o > 0; o >>= 1) {
            lo[a] = fminf(lo[a], __shfl_xor_sync(kFull, lo[a], o));
            hi[a] = fmaxf(hi[a], __shfl_xor_sync(kFull, hi[a], o));
        }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0)
        for (int a = 0; a < 3; ++a) { red[a][w] = lo[a]; red[3 + a][w] = hi[a]; }
    __syncthreads();
    if (threadIdx.x < 6) {
        const int a = threadIdx.x, nw = blockDim.x >> 5;
        float r = red[a][0];
        for (int k = 1; k < nw; ++k) r = a < 3 ? fminf(r, red[a][k]) : fmaxf(r, red[a][k]);
        lohi[6 * p + a] = r;
    }
}

__global__ void kb_cell_assign(const float4* __restrict__ ref, int64_t n, const int64_t* __restrict__ ref_off, int P,
                               const GridView* __restrict__ views, const int64_t* __restrict__ cell_off,
                               int32_t* __restrict__ cell_of, int32_t* __restrict__ counts) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int p = find_problem(ref_off, P, i);
        const GridView g = views[p];
        const float4 v = ref[i];
        const int cx = cell_coord(v.x, g.origin.x, g.inv_cell, g.dims.x);
        const int cy = cell_coord(v.y, g.origin.y, g.inv_cell, g.dims.y);
        const int cz = cell_coord(v.z, g.origin.z, g.inv_cell, g.dims.z);
        const int64_t c = cell_off[p] + ((int64_t)cz * g.dims.y + cy) * g.dims.x + cx;
        cell_of[i] = (int32_t)c;
        atomicAdd(counts + c, 1);
    }
}

__global__ void kb_scatter(const float4* __restrict__ ref, int64_t n, const int32_t* __restrict__ cell_of,
                           const int32_t* __restrict__ cell_start, int32_t* __restrict__ cursor,
                           float4* __restrict__ out) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t c = cell_of[i];
        out[cell_start[c] + atomicAdd(cursor + c, 1)] = ref[i];
    }
}

// One warp per cell: place each point at its rank by index within the cell.
__global__ void kb_sort_cells(const int32_t* __restrict__ cell_start, int64_t ncells, const float4* __restrict__ in,
                              float4* __restrict__ out) {
    const int lane = threadIdx.x & 31;
    const int64_t wid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t c = wid; c < ncells; c += nw) {
        const int b = cell_start[c], e = cell_start[c + 1];
        for (int i = b + lane; i < e; i += 32) {
            const float4 v = in[i];
            const int key = __float_as_int(v.w);
            int rank = 0;
            for (int k = b; k < e; ++k) rank += __float_as_int(in[k].w) < key;
            out[b + rank] = v;
        }
    }
}

__device__ __forceinline__ float3 centre_of(const GridView& g, int x, int y, int z) {
    return make_float3(g.origin.x + ((float)x + 0.5f) * g.cell, g.origin.y + ((float)y + 0.5f) * g.cell,
                       g.origin.z + ((float)z + 0.5f) * g.cell);
}

__global__ void kb_seed_init(const GridView* __restrict__ views, const int64_t* __restrict__ cell_off, int P,
                             int64_t ncells, int32_t* __restrict__ seed) {
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < ncells; c += (int64_t)gridDim.x * blockDim.x) {
        const int p = find_problem(cell_off, P, c);
        const GridView g = views[p];
        const int64_t lc = c - cell_off[p];
        const int b = g.cell_start[lc], e = g.cell_start[lc + 1];
        int best = -1;
        if (e > b) {
            const int x = (int)(lc % g.dims.x), y = (int)((lc / g.dims.x) % g.dims.y),
                      z = (int)(lc / ((int64_t)g.dims.x * g.dims.y));
            const float3 ct = centre_of(g, x, y, z);
            float bd = FLT_MAX;
            for (int q = b; q < e; ++q) {
                const float d = dist2(g.sorted[q], ct);
                if (d < bd) {
                    bd = d;
                    best = q;
                }
            }
        }
        seed[c] = best;
    }
}

__global__ void kb_seed_step(const GridView* __restrict__ views, const int64_t* __restrict__ cell_off, int P,
                             int64_t ncells, int k, const int32_t* __restrict__ in, int32_t* __restrict__ out) {
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < ncells; c += (int64_t)gridDim.x * blockDim.x) {
        const int p = find_problem(cell_off, P, c);
        const GridView g = views[p];
        const int64_t base = cell_off[p], lc = c - base;
        const int x = (int)(lc % g.dims.x), y = (int)((lc / g.dims.x) % g.dims.y),
                  z = (int)(lc / ((int64_t)g.dims.x * g.dims.y));
        const float3 ct = centre_of(g, x, y, z);
        int best = in[c];
        float bd = best >= 0 ? dist2(g.sorted[best], ct) : FLT_MAX;
        for (int dz = -k; dz <= k; dz += k) {
            const int zz = z + dz;
            if (zz < 0 || zz >= g.dims.z) continue;
            for (int dy = -k; dy <= k; dy += k) {
                const int yy = y + dy;
                if (yy < 0 || yy >= g.dims.y) continue;
                for (int dx = -k; dx <= k; dx += k) {
                    const int xx = x + dx;
                    if (xx < 0 || xx >= g.dims.x || (dx == 0 && dy == 0 && dz == 0)) continue;
                    const int s = in[base + ((int64_t)zz * g.dims.y + yy) * g.dims.x + xx];
                    if (s < 0 || s == best) continue;
                    const float d = dist2(g.sorted[s], ct);
                    if (d < bd || (d == bd && s < best)) {
                        bd = d;
                        best = s;
                    }
                }
            }
        }
        out[c] = best;
    }
}

// ---------------------------------------------------------------- persistent kernel

struct BatchArgs {
    int P, T, m, kkc, C;                 // C = ceil(m / kkc) chunks per particle
    const GridSearch* S;                 // [P]
    const float4* src4;                  // packed sources, w = local index
    const int64_t* src_off;              // [P+1]
    const int32_t* mb;                   // [P][T][m]
    const int32_t* part_off;             // [P+1]
    const int64_t* item_off;             // [P+1]: K_p * C items per problem
    int64_t total_items;
    float* theta;                        // [sum K][6]
    float* am;
    float* av;
    float* partial;                      // problem p at C * part_off[p] * 6: [chunk][K_p][6]
    float lr, beta1, beta2, eps;
    int prior;
    float mu[6], sigma[3], kappa[3];
    unsigned* bar;                       // arrival count, generation
    int* err;
    unsigned long long* stats;           // search work counters or null
    // trace of iteration trace_t (-1: none): the particles and Adam moments it starts from
    // [sum K][6], its correspondences [sum K][m] and mean gradients and Stein directions [sum K][6]
    int trace_t;
    float *tr_theta, *tr_am, *tr_av, *tr_gbar, *tr_phi;
    int32_t* tr_nn;
    int cache;                           // Stein phase: pair distances in shared memory (1) or not (0)
    long long max_spins;                 // polls of a barrier wait before it gives up (0: kMaxSpins)
    unsigned extra;                      // arrivals a barrier waits for beyond the grid's CTAs (1 only in
                                         // the failure-detection check, where every wait must give up)
};

// Grid-wide barrier with a bounded wait; false if any CTA gave up waiting.
__device__ bool grid_barrier(unsigned* bar, int* err, long long max_spins, unsigned extra) {
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned* gen = bar + 1;
        const unsigned g = *gen;
        __threadfence();
        if (atomicAdd(bar, 1u) + 1u == gridDim.x + extra) {
            bar[0] = 0u;
            __threadfence();
            atomicAdd(bar + 1, 1u);
        } else {
            const long long limit = max_spins > 0 ? max_spins : kMaxSpins;
            long long spins = 0;
            while (*gen == g) {
                if (++spins > limit || *(volatile int*)err) {
                    atomicOr(err, 1);
                    break;
                }
                __nanosleep(64);
            }
        }
        __threadfence();
    }
    __syncthreads();
    return *(volatile int*)err == 0;
}

template <int kThreads, int kMinBlocks>
__global__ void __launch_bounds__(kThreads, kMinBlocks) kb_persistent(BatchArgs b) {
    __shared__ Pose P[kThreads / 32];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t W = (int64_t)gridDim.x * (kThreads / 32);
    for (int t = 0; t < b.T; ++t) {
        const bool tr = t == b.trace_t;
        if (tr) {   // the state this iteration starts from (theta changes only after the barrier)
            const int64_t n = 6 * (int64_t)b.part_off[b.P];
            for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
                b.tr_theta[i] = b.theta[i];
                b.tr_am[i] = b.am[i];
                b.tr_av[i] = b.av[i];
            }
        }
        // gradient phase: one warp per item, items interleaved over the whole grid
        for (int64_t it = (int64_t)blockIdx.x * (kThreads / 32) + warp; it < b.total_items; it += W) {
            const int p = (int)SICP_IDX(find_problem(b.item_off, b.P, it), b.P, kChkProblem);
            const int K = b.part_off[p + 1] - b.part_off[p];
            const int64_t r = it - b.item_off[p];
            const int c = (int)(r / K), j = (int)(r % K);
            const int jg = b.part_off[p] + j;
            if (lane == 0) make_pose(b.theta + 6 * jg, P[warp]);
            __syncwarp();
            const GridSearch& S = b.S[p];
            const int32_t* mbp = b.mb + ((int64_t)p * b.T + t) * b.m;
            const float4* srcp = b.src4 + b.src_off[p];
            float gr[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
            Work w;
            for (int kk = 0; kk < b.kkc; ++kk) {
                const int k = c * b.kkc + kk;
                if (k >= b.m) break;
                const float4 s4 =
                    __ldg(srcp + SICP_IDX(__ldg(mbp + k), b.src_off[p + 1] - b.src_off[p], kChkSrc));
                const float3 s = make_float3(s4.x, s4.y, s4.z);
                const float3 q = apply_pose(P[warp], s);
                Best B;
                grid_search(S, q, B, w);
                if (tr && lane == 0) b.tr_nn[(int64_t)jg * b.m + k] = B.i != kNone ? B.i : -1;
                if (lane == 0 && B.i != kNone) {
                    float tt[6];
                    grad_terms(P[warp], s, make_float3(q.x - B.p.x, q.y - B.p.y, q.z - B.p.z), tt);
#pragma unroll
                    for (int a = 0; a < 6; ++a) gr[a] += tt[a];
                }
            }
            if (lane == 0) {
                float* dst = b.partial + ((int64_t)b.C * b.part_off[p] + (int64_t)c * K + j) * 6;
#pragma unroll
                for (int a = 0; a < 6; ++a) dst[a] = gr[a];
            }
            if (b.stats) add_stats(b.stats, w);
            __syncwarp();
        }
        if (!grid_barrier(b.bar, b.err, b.max_spins, b.extra)) return;
        // Stein phase: whole problems per CTA
        for (int p = blockIdx.x; p < b.P; p += gridDim.x) {
            const int off = b.part_off[p];
            SteinArgs a;
            a.theta = b.theta + 6 * off;
            a.adam_m = b.am + 6 * off;
            a.adam_v = b.av + 6 * off;
            a.partial = b.partial + (int64_t)b.C * off * 6;
            a.chunks = b.C;
            a.inv_m = 1.f / (float)b.m;
            a.K = b.part_off[p + 1] - off;
            a.N = (float)(b.src_off[p + 1] - b.src_off[p]);
            a.t = t + 1;
            a.lr = b.lr;
            a.beta1 = b.beta1;
            a.beta2 = b.beta2;
            a.eps = b.eps;
            a.prior = b.prior;
            for (int q = 0; q < 6; ++q) a.mu[q] = b.mu[q];
            for (int q = 0; q < 3; ++q) {
                a.sigma[q] = b.sigma[q];
                a.kappa[q] = b.kappa[q];
            }
            a.out_phi = tr ? b.tr_phi + 6 * off : nullptr;
            a.out_gbar = tr ? b.tr_gbar + 6 * off : nullptr;
            a.out_h = nullptr;
            a.med_state = nullptr;
            a.arrive = nullptr;
            a.err = nullptr;
            a.gen = 0;
            a.max_spins = 0;
            a.extra = 0;
            a.cache = b.cache;
            sd::stein_adam_block(a);
            __syncthreads();
        }
        if (!grid_barrier(b.bar, b.err, b.max_spins, b.extra)) return;
    }
}

// One CTA per problem: FP64 mean and covariance into out[p][42].
__global__ void kb_moments(const float* __restrict__ theta, const int32_t* __restrict__ part_off,
                           double* __restrict__ out) {
    __shared__ double mean[6];
    const int p = blockIdx.x, tid = threadIdx.x;
    const float* th = theta + 6 * part_off[p];
    const int K = part_off[p + 1] - part_off[p];
    if (tid < 6) {
        double s = 0.0;
        for (int j = 0; j < K; ++j) s += (double)th[6 * j + tid];
        mean[tid] = s / (double)K;
    }
    __syncthreads();
    if (tid < 36) {
        const int a = tid / 6, c = tid % 6;
        double s = 0.0;
        for (int j = 0; j < K; ++j) s += ((double)th[6 * j + a] - mean[a]) * ((double)th[6 * j + c] - mean[c]);
        out[42 * p + 6 + tid] = (K > 1) ? s / (double)(K - 1) : 0.0;
    }
    if (tid < 6) out[42 * p + tid] = mean[tid];
}

unsigned nblocks(int64_t n, int threads, int cap = 8192) {
    int64_t b = (n + threads - 1) / threads;
    return (unsigned)(b < 1 ? 1 : (b > cap ? cap : b));
}

int3 level_dims(const float ext[3], double& c, int64_t max_cells) {
    int3 d;
    for (;;) {
        d.x = (int)fmin(floor(ext[0] / c) + 1.0, 1 << 20);
        d.y = (int)fmin(floor(ext[1] / c) + 1.0, 1 << 20);
        d.z = (int)fmin(floor(ext[2] / c) + 1.0, 1 << 20);
        const double n = (double)d.x * d.y * d.z;
        if (n <= (double)max_cells) return d;
        c *= cbrt(n / (double)max_cells) * 1.01;
    }
}

}  // namespace

// ---------------------------------------------------------------- host state

struct BatchState {
    Buf ref4, src4, mb, theta, am, av, partial, moments, stage, flags, bar;
    Buf ref_off, src_off, part_off, item_off, lohi;
    // per level: sorted points, cell_of, counts, cell_start, scan sums, views, cell offsets
    struct Level {
        Buf sorted, staging, cell_of, counts, cell_start, sums, views, cell_off, seed, seed_tmp;
        std::vector<GridView> hv;
        std::vector<int64_t> h_cell_off;
        int64_t ncells = 0;
    } lv[2];
    Buf searches;
    // built-reference signature and captured graph
    bool graph_valid = false;
    cudaGraphExec_t exec = nullptr;
    std::vector<unsigned char> key;
    float cell_factor = 0.5f;
    int kkc = 4;
    int shape = 0;                       // index into kShapeThreads
    int grid_ctas = 0;
    size_t smem = 0;
    // trace of one iteration (sicp_trace_batched): armed iteration, and what the last run recorded
    int trace_t = -1;
    bool trace_ready = false;
    int64_t trace_K = 0;
    int trace_m = 0;
    Buf tr;
    ~BatchState() {
        if (exec) cudaGraphExecDestroy(exec);
        Buf* bs[] = {&ref4, &src4, &mb, &theta, &am, &av, &partial, &moments, &stage, &flags, &bar,
                     &ref_off, &src_off, &part_off, &item_off, &lohi, &searches, &tr};
        for (Buf* x : bs)
            if (x->p) cudaFree(x->p);
        for (Level& L : lv) {
            Buf* ls[] = {&L.sorted, &L.staging, &L.cell_of, &L.counts, &L.cell_start, &L.sums,
                         &L.views, &L.cell_off, &L.seed, &L.seed_tmp};
            for (Buf* x : ls)
                if (x->p) cudaFree(x->p);
        }
    }
};

void batch_destroy(BatchState* b) { delete b; }

namespace {

// Build both grid levels of every problem from the packed references.
int build_batched(sicp_ctx* ctx, BatchState& B, int P, const std::vector<int64_t>& ref_off, float factor) {
    cudaStream_t s = ctx->stream;
    const int64_t M = ref_off[P];
    int rc;
    if ((rc = ensure(ctx, B.lohi, sizeof(float) * 6 * P))) return rc;
    kb_bbox<<<P, 256, 0, s>>>((const float4*)B.ref4.p, (const int64_t*)B.ref_off.p, (float*)B.lohi.p);
    SICP_CUDA(cudaGetLastError());
    std::vector<float> lohi(6 * (size_t)P);
    SICP_CUDA(cudaMemcpyAsync(lohi.data(), B.lohi.p, sizeof(float) * 6 * P, cudaMemcpyDeviceToHost, s));
    SICP_CUDA(cudaStreamSynchronize(s));
    for (int l = 0; l < 2; ++l) {
        BatchState::Level& L = B.lv[l];
        L.hv.assign(P, GridView{});
        L.h_cell_off.assign(P + 1, 0);
        for (int p = 0; p < P; ++p) {
            float ext[3];
            double X = 0.0, maxext = 0.0;
            for (int a = 0; a < 3; ++a) {
                ext[a] = lohi[6 * p + 3 + a] - lohi[6 * p + a];
                X = fmax(X, fmax(fabs((double)lohi[6 * p + a]), fabs((double)lohi[6 * p + 3 + a])));
                maxext = fmax(maxext, ext[a]);
            }
            const int64_t Mp = ref_off[p + 1] - ref_off[p];
            double c;
            if (l == 0) {
                if (maxext <= 0.0) {
                    c = 1.0;
                } else {
                    const double fl = maxext * 1e-3;
                    const double V = fmax(ext[0], fl) * fmax(ext[1], fl) * fmax(ext[2], fl);
                    c = factor * cbrt(V / (double)Mp);
                }
            } else {
                c = (double)B.lv[0].hv[p].cell * kCoarseFactor;
            }
            const int3 d = level_dims(ext, c, kMaxCells);
            GridView& v = L.hv[p];
            v.origin = make_float3(lohi[6 * p], lohi[6 * p + 1], lohi[6 * p + 2]);
            v.cell = (float)c;
            v.inv_cell = (float)(1.0 / c);
            v.tol = (float)(1e-6 * (X + c));
            v.dims = d;
            L.h_cell_off[p + 1] = L.h_cell_off[p] + (int64_t)d.x * d.y * d.z;
        }
        L.ncells = L.h_cell_off[P];
        if ((rc = ensure(ctx, L.sorted, sizeof(float4) * M))) return rc;
        if ((rc = ensure(ctx, L.staging, sizeof(float4) * M))) return rc;
        if ((rc = ensure(ctx, L.cell_of, sizeof(int32_t) * M))) return rc;
        if ((rc = ensure(ctx, L.counts, sizeof(int32_t) * (L.ncells + 1)))) return rc;
        if ((rc = ensure(ctx, L.cell_start, sizeof(int32_t) * (L.ncells + 1)))) return rc;
        if ((rc = ensure(ctx, L.sums, sizeof(int32_t) * scan_sums_size(L.ncells)))) return rc;
        if ((rc = ensure(ctx, L.views, sizeof(GridView) * P))) return rc;
        if ((rc = ensure(ctx, L.cell_off, sizeof(int64_t) * (P + 1)))) return rc;
        if (l == 0) {
            if ((rc = ensure(ctx, L.seed, sizeof(int32_t) * L.ncells))) return rc;
            if ((rc = ensure(ctx, L.seed_tmp, sizeof(int32_t) * L.ncells))) return rc;
        }
        for (int p = 0; p < P; ++p) {
            GridView& v = L.hv[p];
            v.sorted = (const float4*)L.sorted.p;
            v.nsorted = (int32_t)M;
            v.cell_start = (const int32_t*)L.cell_start.p + L.h_cell_off[p];
            v.seed = l == 0 ? (const int32_t*)L.seed.p + L.h_cell_off[p] : nullptr;
            v.seed4 = nullptr;
        }
        SICP_CUDA(cudaMemcpyAsync(L.views.p, L.hv.data(), sizeof(GridView) * P, cudaMemcpyHostToDevice, s));
        SICP_CUDA(cudaMemcpyAsync(L.cell_off.p, L.h_cell_off.data(), sizeof(int64_t) * (P + 1), cudaMemcpyHostToDevice, s));
        const GridView* dv = (const GridView*)L.views.p;
        const int64_t* dco = (const int64_t*)L.cell_off.p;
        SICP_CUDA(cudaMemsetAsync(L.counts.p, 0, sizeof(int32_t) * (L.ncells + 1), s));
        kb_cell_assign<<<nblocks(M, 256), 256, 0, s>>>((const float4*)B.ref4.p, M, (const int64_t*)B.ref_off.p, P, dv,
                                                       dco, (int32_t*)L.cell_of.p, (int32_t*)L.counts.p);
        SICP_CUDA(cudaGetLastError());
        SICP_CUDA(launch_exclusive_scan((const int32_t*)L.counts.p, L.ncells, (int32_t*)L.cell_start.p,
                                        (int32_t*)L.sums.p, s));
        SICP_CUDA(cudaMemsetAsync(L.counts.p, 0, sizeof(int32_t) * (L.ncells + 1), s));
        kb_scatter<<<nblocks(M, 256), 256, 0, s>>>((const float4*)B.ref4.p, M, (const int32_t*)L.cell_of.p,
                                                   (const int32_t*)L.cell_start.p, (int32_t*)L.counts.p,
                                                   (float4*)L.staging.p);
        SICP_CUDA(cudaGetLastError());
        kb_sort_cells<<<nblocks(L.ncells * 32, 256), 256, 0, s>>>((const int32_t*)L.cell_start.p, L.ncells,
                                                                  (const float4*)L.staging.p, (float4*)L.sorted.p);
        SICP_CUDA(cudaGetLastError());
        if (l == 0) {
            int32_t* a = (int32_t*)L.seed.p;
            int32_t* c = (int32_t*)L.seed_tmp.p;
            kb_seed_init<<<nblocks(L.ncells, 256), 256, 0, s>>>(dv, dco, P, L.ncells, a);
            SICP_CUDA(cudaGetLastError());
            int maxd = 1;
            for (const GridView& v : L.hv) maxd = std::max(maxd, std::max(v.dims.x, std::max(v.dims.y, v.dims.z)));
            int k = 1;
            while (k * 2 <= maxd / 2) k *= 2;
            std::vector<int> steps;
            for (; k >= 1; k /= 2) steps.push_back(k);
            steps.push_back(1);
            for (int st : steps) {
                kb_seed_step<<<nblocks(L.ncells, 256), 256, 0, s>>>(dv, dco, P, L.ncells, st, a, c);
                SICP_CUDA(cudaGetLastError());
                std::swap(a, c);
            }
            if (a != (int32_t*)L.seed.p)
                SICP_CUDA(cudaMemcpyAsync(L.seed.p, a, sizeof(int32_t) * L.ncells, cudaMemcpyDeviceToDevice, s));
        }
    }
    // per-problem search descriptors
    std::vector<GridSearch> hs(P);
    for (int p = 0; p < P; ++p) {
        hs[p].fine = B.lv[0].hv[p];
        hs[p].coarse = B.lv[1].hv[p];
        hs[p].tab = ctx->search.tab;
        hs[p].ref4 = (const float4*)B.ref4.p + ref_off[p];
        hs[p].M = (int)(ref_off[p + 1] - ref_off[p]);
        hs[p].reach = gs::kBatchedFineReach;
    }
    if ((rc = ensure(ctx, B.searches, sizeof(GridSearch) * P))) return rc;
    SICP_CUDA(cudaMemcpyAsync(B.searches.p, hs.data(), sizeof(GridSearch) * P, cudaMemcpyHostToDevice, s));
    return SICP_OK;
}

bool host_finite_b(const float* x, int64_t n) {
    for (int64_t i = 0; i < n; ++i)
        if (!isfinite(x[i])) return false;
    return true;
}

struct BatchInputs {
    int P;
    const int64_t* ref_off;
    const float* ref_xyz;
    const int64_t* src_off;
    const float* src_xyz;
    const int32_t* part_off;
    const float* particles_in;
};

int check_batch(sicp_ctx* ctx, const BatchInputs& in, const sicp_params& p) {
    if (in.P < 1 || in.P > 65535 || !in.ref_off || !in.src_off || !in.part_off || !in.ref_xyz || !in.src_xyz ||
        !in.particles_in)
        return set_err(ctx, SICP_EINVAL, "batched call needs 1 <= P <= 65535 and non-NULL arrays");
    if (in.ref_off[0] != 0 || in.src_off[0] != 0 || in.part_off[0] != 0)
        return set_err(ctx, SICP_EINVAL, "offset arrays must start at 0");
    for (int q = 0; q < in.P; ++q) {
        const int64_t M = in.ref_off[q + 1] - in.ref_off[q], N = in.src_off[q + 1] - in.src_off[q];
        const int32_t K = in.part_off[q + 1] - in.part_off[q];
        if (M < 1 || M > (1 << 30)) return set_err(ctx, SICP_EINVAL, "problem %d: reference size %lld", q, (long long)M);
        if (N < p.m || N > 0x7fffffff) return set_err(ctx, SICP_EINVAL, "problem %d: source size %lld < m", q, (long long)N);
        if (K < 1 || K > 2048) return set_err(ctx, SICP_EINVAL, "problem %d: particle count %d outside [1, 2048]", q, K);
    }
    if (p.T < 0 || p.m < 1) return set_err(ctx, SICP_EINVAL, "T must be >= 0 and m >= 1");
    if (p.nn_mode != SICP_NN_GRID) return set_err(ctx, SICP_EINVAL, "the batched path uses the grid search (SICP_NN_GRID)");
    return SICP_OK;
}

// Upload, build and (optionally) run T iterations; elapsed_ms (if not NULL)
// receives the persistent kernel's time measured with CUDA events.
int run_batched(sicp_ctx* ctx, const BatchInputs& in, const sicp_params& p, int on_device, float factor, int kkc,
                int shape_ix, bool use_graph, float* particles_out, double* mean6, double* cov36, float* elapsed_ms) {
    BatchState& B = *ctx->batch;
    cudaStream_t s = ctx->stream;
    const int P = in.P;
    std::vector<int64_t> ro(in.ref_off, in.ref_off + P + 1), so(in.src_off, in.src_off + P + 1);
    std::vector<int32_t> po(in.part_off, in.part_off + P + 1);
    const int64_t M = ro[P], N = so[P];
    const int64_t Ktot = po[P];
    int maxK = 1;
    for (int q = 0; q < P; ++q) maxK = std::max(maxK, po[q + 1] - po[q]);
    const int C = (p.m + kkc - 1) / kkc;
    std::vector<int64_t> io(P + 1, 0);
    for (int q = 0; q < P; ++q) io[q + 1] = io[q] + (int64_t)(po[q + 1] - po[q]) * C;
    int rc;
    if ((rc = ensure(ctx, B.ref4, sizeof(float4) * M))) return rc;
    if ((rc = ensure(ctx, B.src4, sizeof(float4) * N))) return rc;
    if ((rc = ensure(ctx, B.mb, sizeof(int32_t) * (size_t)P * (p.T > 0 ? p.T : 1) * p.m))) return rc;
    if ((rc = ensure(ctx, B.theta, sizeof(float) * 6 * Ktot))) return rc;
    if ((rc = ensure(ctx, B.am, sizeof(float) * 6 * Ktot))) return rc;
    if ((rc = ensure(ctx, B.av, sizeof(float) * 6 * Ktot))) return rc;
    if ((rc = ensure(ctx, B.partial, sizeof(float) * 6 * (size_t)C * Ktot))) return rc;
    if ((rc = ensure(ctx, B.moments, sizeof(double) * 42 * P))) return rc;
    if ((rc = ensure(ctx, B.flags, 4 * sizeof(int)))) return rc;
    if ((rc = ensure(ctx, B.bar, 4 * sizeof(unsigned)))) return rc;
    if ((rc = ensure(ctx, B.ref_off, sizeof(int64_t) * (P + 1)))) return rc;
    if ((rc = ensure(ctx, B.src_off, sizeof(int64_t) * (P + 1)))) return rc;
    if ((rc = ensure(ctx, B.part_off, sizeof(int32_t) * (P + 1)))) return rc;
    if ((rc = ensure(ctx, B.item_off, sizeof(int64_t) * (P + 1)))) return rc;
    SICP_CUDA(cudaMemcpyAsync(B.ref_off.p, ro.data(), sizeof(int64_t) * (P + 1), cudaMemcpyHostToDevice, s));
    SICP_CUDA(cudaMemcpyAsync(B.src_off.p, so.data(), sizeof(int64_t) * (P + 1), cudaMemcpyHostToDevice, s));
    SICP_CUDA(cudaMemcpyAsync(B.part_off.p, po.data(), sizeof(int32_t) * (P + 1), cudaMemcpyHostToDevice, s));
    SICP_CUDA(cudaMemcpyAsync(B.item_off.p, io.data(), sizeof(int64_t) * (P + 1), cudaMemcpyHostToDevice, s));
    // inputs: device pointers pass through, host arrays are staged
    const float *d_ref = in.ref_xyz, *d_src = in.src_xyz, *d_par = in.particles_in;
    if (!on_device) {
        const size_t bref = sizeof(float) * 3 * M, bsrc = sizeof(float) * 3 * N, bpar = sizeof(float) * 6 * Ktot;
        if ((rc = ensure(ctx, B.stage, bref + bsrc + bpar))) return rc;
        char* st = (char*)B.stage.p;
        SICP_CUDA(cudaMemcpyAsync(st, in.ref_xyz, bref, cudaMemcpyHostToDevice, s));
        SICP_CUDA(cudaMemcpyAsync(st + bref, in.src_xyz, bsrc, cudaMemcpyHostToDevice, s));
        SICP_CUDA(cudaMemcpyAsync(st + bref + bsrc, in.particles_in, bpar, cudaMemcpyHostToDevice, s));
        d_ref = (const float*)st;
        d_src = (const float*)(st + bref);
        d_par = (const float*)(st + bref + bsrc);
    }
    SICP_CUDA(cudaMemsetAsync(B.flags.p, 0, 4 * sizeof(int), s));
    kb_pack<<<nblocks(M, 256), 256, 0, s>>>(d_ref, M, (const int64_t*)B.ref_off.p, P, (float4*)B.ref4.p, (int*)B.flags.p);
    SICP_CUDA(cudaGetLastError());
    kb_pack<<<nblocks(N, 256), 256, 0, s>>>(d_src, N, (const int64_t*)B.src_off.p, P, (float4*)B.src4.p, (int*)B.flags.p);
    SICP_CUDA(cudaGetLastError());
    SICP_CUDA(launch_check_finite(d_par, 6 * Ktot, (int*)B.flags.p, s));
    SICP_CUDA(cudaMemcpyAsync(B.theta.p, d_par, sizeof(float) * 6 * Ktot, cudaMemcpyDeviceToDevice, s));
    SICP_CUDA(cudaMemsetAsync(B.am.p, 0, sizeof(float) * 6 * Ktot, s));
    SICP_CUDA(cudaMemsetAsync(B.av.p, 0, sizeof(float) * 6 * Ktot, s));
    if ((rc = build_batched(ctx, B, P, ro, factor))) return rc;

    // the persistent kernel's CTA shape (autotuned): 1024 threads with the Stein pair cache, or
    // 512 / 256 threads without it
    const int shape = shape_ix < 0 || shape_ix >= kShapes ? 0 : shape_ix;
    const int threads = kShapeThreads[shape];
    const bool cache = shape == 0;
    void (*kern)(BatchArgs) = shape == 0 ? kb_persistent<1024, 1> : shape == 1 ? kb_persistent<512, 3>
                                                                                 : kb_persistent<256, 6>;
    const size_t pairs = (size_t)maxK * (maxK - 1) / 2;
    const size_t smem =
        sizeof(float) * (18 * (size_t)maxK + (cache && 2 * pairs <= (size_t)sd::kCacheFloats ? 2 * pairs : 0));
    SICP_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    SICP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem));
    if (per_sm < 1) return set_err(ctx, SICP_ECUDA, "persistent kernel does not fit on an SM (smem %zu)", smem);
    const int ctas = per_sm * ctx->num_sms;

    BatchArgs a;
    memset(&a, 0, sizeof a);   // the bytes (padding too) key the captured graph
    a.P = P;
    a.T = p.T;
    a.m = p.m;
    a.kkc = kkc;
    a.C = C;
    a.S = (const GridSearch*)B.searches.p;
    a.src4 = (const float4*)B.src4.p;
    a.src_off = (const int64_t*)B.src_off.p;
    a.mb = (const int32_t*)B.mb.p;
    a.part_off = (const int32_t*)B.part_off.p;
    a.item_off = (const int64_t*)B.item_off.p;
    a.total_items = io[P];
    a.theta = (float*)B.theta.p;
    a.am = (float*)B.am.p;
    a.av = (float*)B.av.p;
    a.partial = (float*)B.partial.p;
    a.lr = p.lr;
    a.beta1 = p.beta1;
    a.beta2 = p.beta2;
    a.eps = p.eps;
    a.prior = p.prior;
    for (int q = 0; q < 6; ++q) a.mu[q] = p.prior_mu[q];
    for (int q = 0; q < 3; ++q) {
        a.sigma[q] = p.prior_sigma[q];
        a.kappa[q] = p.prior_kappa[q];
    }
    a.bar = (unsigned*)B.bar.p;
    a.cache = cache ? 1 : 0;
    a.trace_t = -1;
    const bool tracing = B.trace_t >= 0 && B.trace_t < p.T && !elapsed_ms;
    if (tracing) {
        const size_t st = sizeof(float) * 6 * (size_t)Ktot;
        if ((rc = ensure(ctx, B.tr, 5 * st + sizeof(int32_t) * (size_t)Ktot * p.m))) return rc;
        char* t0 = (char*)B.tr.p;
        a.trace_t = B.trace_t;
        a.tr_theta = (float*)t0;
        a.tr_am = (float*)(t0 + st);
        a.tr_av = (float*)(t0 + 2 * st);
        a.tr_gbar = (float*)(t0 + 3 * st);
        a.tr_phi = (float*)(t0 + 4 * st);
        a.tr_nn = (int32_t*)(t0 + 5 * st);
    }
    B.trace_ready = false;
    a.max_spins = ctx->wait_polls;
    a.extra = ctx->wait_never ? 1u : 0u;
    a.err = (int*)B.flags.p + 2;
    a.stats = ctx->stats_on ? (unsigned long long*)ctx->stats.p : nullptr;

    // with kernel timing on (sicp_profile), the launch's duration joins the
    // context's gradient-kernel totals
    float prof_ms = 0.f;
    const bool to_prof = !elapsed_ms && ctx->prof_stride > 0;
    if (to_prof) elapsed_ms = &prof_ms;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (elapsed_ms) {
        SICP_CUDA(cudaEventCreate(&e0));
        SICP_CUDA(cudaEventCreate(&e1));
    }
    auto record = [&]() -> int {
        SICP_CUDA(launch_minibatch_batched(p.seed, p.T, p.m, P, (const int64_t*)B.src_off.p, (int32_t*)B.mb.p, s));
        SICP_CUDA(cudaMemsetAsync(B.bar.p, 0, 4 * sizeof(unsigned), s));
        if (p.T > 0) {
            cudaLaunchConfig_t cfg = {};
            cfg.gridDim = dim3(ctas);
            cfg.blockDim = dim3(threads);
            cfg.dynamicSmemBytes = smem;
            cfg.stream = s;
            cudaLaunchAttribute attr[1];
            attr[0].id = cudaLaunchAttributeCooperative;
            attr[0].val.cooperative = 1;
            cfg.attrs = attr;
            cfg.numAttrs = 1;
            SICP_CUDA(cudaLaunchKernelEx(&cfg, kern, a));
        }
        kb_moments<<<P, 64, 0, s>>>((const float*)B.theta.p, (const int32_t*)B.part_off.p, (double*)B.moments.p);
        SICP_CUDA(cudaGetLastError());
        return SICP_OK;
    };
    if (e0) SICP_CUDA(cudaEventRecord(e0, s));
    if (use_graph) {
        std::vector<unsigned char> key(sizeof(BatchArgs) + sizeof(int) * 3 + sizeof(uint64_t));
        memcpy(key.data(), &a, sizeof(BatchArgs));
        memcpy(key.data() + sizeof(BatchArgs), &ctas, sizeof(int));
        const int sm_i = (int)smem;
        memcpy(key.data() + sizeof(BatchArgs) + sizeof(int), &sm_i, sizeof(int));
        memcpy(key.data() + sizeof(BatchArgs) + 2 * sizeof(int), &threads, sizeof(int));
        memcpy(key.data() + sizeof(BatchArgs) + 3 * sizeof(int), &p.seed, sizeof(uint64_t));
        if (!(B.graph_valid && B.key == key)) {
            if (B.exec) cudaGraphExecDestroy(B.exec);
            B.exec = nullptr;
            B.graph_valid = false;
            cudaGraph_t graph;
            SICP_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
            rc = record();
            cudaError_t e = cudaStreamEndCapture(s, &graph);
            if (rc) {
                if (e == cudaSuccess) cudaGraphDestroy(graph);
                return rc;
            }
            if (e != cudaSuccess) return cuda_err(ctx, e, "cudaStreamEndCapture (batched)");
            e = cudaGraphInstantiate(&B.exec, graph, 0);
            cudaGraphDestroy(graph);
            if (e != cudaSuccess) return cuda_err(ctx, e, "cudaGraphInstantiate (batched)");
            B.key = key;
            B.graph_valid = true;
        }
        SICP_CUDA(cudaGraphLaunch(B.exec, s));
    } else {
        if ((rc = record())) return rc;
    }
    if (e1) SICP_CUDA(cudaEventRecord(e1, s));
    int flags[4];
    SICP_CUDA(cudaMemcpyAsync(flags, B.flags.p, 4 * sizeof(int), cudaMemcpyDeviceToHost, s));
    SICP_CUDA(cudaStreamSynchronize(s));
    if (elapsed_ms) {
        cudaEventElapsedTime(elapsed_ms, e0, e1);
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        if (to_prof) {
            ctx->prof[0] += prof_ms;
            ctx->prof[1] += 1.0;
        }
    }
    if (flags[0]) return set_err(ctx, SICP_EINVAL, "non-finite input");
    if (flags[2]) return set_err(ctx, SICP_ETIMEOUT, "a grid barrier of the persistent kernel timed out");
    const cudaMemcpyKind k = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    if (particles_out) SICP_CUDA(cudaMemcpyAsync(particles_out, B.theta.p, sizeof(float) * 6 * Ktot, k, s));
    // moments [p][42] -> mean [p][6] and covariance [p][36]
    if (mean6)
        SICP_CUDA(cudaMemcpy2DAsync(mean6, 6 * sizeof(double), B.moments.p, 42 * sizeof(double), 6 * sizeof(double), P,
                                    k, s));
    if (cov36)
        SICP_CUDA(cudaMemcpy2DAsync(cov36, 36 * sizeof(double), (const double*)B.moments.p + 6, 42 * sizeof(double),
                                    36 * sizeof(double), P, k, s));
    SICP_CUDA(cudaStreamSynchronize(s));
    B.grid_ctas = ctas;
    B.smem = smem;
    if (tracing) {
        B.trace_ready = true;
        B.trace_K = Ktot;
        B.trace_m = p.m;
        B.trace_t = -1;   // one run per arming
    }
    return SICP_OK;
}

std::string gpu_name(int dev) {
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, dev) != cudaSuccess) {
        cudaGetLastError();
        return "unknown";
    }
    return prop.name;
}

// Cache file: one line per entry, `"key": [cell_factor, points_per_item, shape],`
// inside a JSON object (shape: index of the CTA shape, 1024 / 512 / 256 threads).
bool cache_lookup(const char* path, const std::string& key, float* f, int* k, int* sh) {
    if (!path) return false;
    FILE* fp = fopen(path, "r");
    if (!fp) return false;
    char line[512];
    bool found = false;
    const std::string needle = "\"" + key + "\"";
    while (fgets(line, sizeof line, fp)) {
        const char* at = strstr(line, needle.c_str());
        if (!at) continue;
        const char* br = strchr(at + needle.size(), '[');
        if (br && sscanf(br, "[%f, %d, %d]", f, k, sh) == 3) found = true;
    }
    fclose(fp);
    return found;
}

void cache_store(const char* path, const std::string& key, float f, int k, int sh) {
    if (!path) return;
    std::vector<std::string> lines;
    FILE* fp = fopen(path, "r");
    const std::string needle = "\"" + key + "\"";
    if (fp) {
        char line[512];
        while (fgets(line, sizeof line, fp)) {
            std::string l(line);
            if (l.find("\"") != std::string::npos && l.find(needle) == std::string::npos && l.find('[') != std::string::npos) {
                while (!l.empty() && (l.back() == '\n' || l.back() == ',')) l.pop_back();
                lines.push_back(l);
            }
        }
        fclose(fp);
    }
    char buf[512];
    snprintf(buf, sizeof buf, "  %s: [%.3f, %d, %d]", needle.c_str(), f, k, sh);
    lines.push_back(buf);
    fp = fopen(path, "w");
    if (!fp) return;
    fprintf(fp, "{\n");
    for (size_t i = 0; i < lines.size(); ++i) fprintf(fp, "%s%s\n", lines[i].c_str(), i + 1 < lines.size() ? "," : "");
    fprintf(fp, "}\n");
    fclose(fp);
}

}  // namespace
}  // namespace sicp

using namespace sicp;

namespace {

struct DeviceScopeB {
    int prev = -1;
    explicit DeviceScopeB(int d) {
        cudaGetDevice(&prev);
        if (prev != d) cudaSetDevice(d);
    }
    ~DeviceScopeB() {
        int cur = -1;
        cudaGetDevice(&cur);
        if (prev >= 0 && cur != prev) cudaSetDevice(prev);
    }
};

sicp_params norm_b(const sicp_params* in) {
    sicp_params p = *in;
    if (p.beta1 == 0.f) p.beta1 = 0.9f;
    if (p.beta2 == 0.f) p.beta2 = 0.999f;
    if (p.eps == 0.f) p.eps = 1e-8f;
    return p;
}

}  // namespace

extern "C" int sicp_register_batched(sicp_ctx* ctx, int32_t P, const int64_t* ref_off, const float* ref_xyz,
                                     const int64_t* src_off, const float* src_xyz, const int32_t* part_off,
                                     const float* particles_in, const sicp_params* p_in, float* particles_out,
                                     double* mean6, double* cov36, int on_device) {
    sicp::NvtxRange nvtx_("batched");
    if (!ctx) return SICP_EINVAL;
    ctx->err.clear();
    if (!p_in) return set_err(ctx, SICP_EINVAL, "null params");
    const sicp_params p = norm_b(p_in);
    BatchInputs in{P, ref_off, ref_xyz, src_off, src_xyz, part_off, particles_in};
    int rc = check_batch(ctx, in, p);
    if (rc) return rc;
    if (!on_device) {
        if (!host_finite_b(ref_xyz, 3 * ref_off[P]) || !host_finite_b(src_xyz, 3 * src_off[P]) ||
            !host_finite_b(particles_in, 6 * (int64_t)part_off[P]))
            return set_err(ctx, SICP_EINVAL, "non-finite input");
    }
    DeviceScopeB ds(ctx->device);
    if (!ctx->batch) ctx->batch = new BatchState();
    const bool graph = getenv("SICP_NO_GRAPH") == nullptr;
    return run_batched(ctx, in, p, on_device, ctx->batch->cell_factor, ctx->batch->kkc, ctx->batch->shape, graph,
                       particles_out, mean6, cov36, nullptr);
}

extern "C" int sicp_autotune_batched(sicp_ctx* ctx, int32_t P, const int64_t* ref_off, const float* ref_xyz,
                                     const int64_t* src_off, const float* src_xyz, const int32_t* part_off,
                                     const float* particles_in, const sicp_params* p_in, int32_t trial_iters,
                                     const char* cache_path, float* out_cell_factor, int32_t* out_points_per_item,
                                     int32_t* out_cta_threads, int on_device) {
    if (!ctx) return SICP_EINVAL;
    ctx->err.clear();
    if (!p_in || trial_iters < 1) return set_err(ctx, SICP_EINVAL, "autotune needs params and trial_iters >= 1");
    sicp_params p = norm_b(p_in);
    BatchInputs in{P, ref_off, ref_xyz, src_off, src_xyz, part_off, particles_in};
    int rc = check_batch(ctx, in, p);
    if (rc) return rc;
    DeviceScopeB ds(ctx->device);
    if (!ctx->batch) ctx->batch = new BatchState();
    BatchState& B = *ctx->batch;
    char keybuf[256];
    const double meanM = (double)ref_off[P] / P;
    snprintf(keybuf, sizeof keybuf, "%s|P=%d|M~2^%d|m=%d", gpu_name(ctx->device).c_str(), P,
             (int)lround(log2(fmax(meanM, 1.0))), p.m);
    const std::string key(keybuf);
    float f = 0.f;
    int k = 0, sh = 0;
    if (cache_lookup(cache_path, key, &f, &k, &sh) && f > 0.f && k > 0 && sh >= 0 && sh < kShapes) {
        B.cell_factor = f;
        B.kkc = k;
        B.shape = sh;
    } else {
        p.T = trial_iters;
        const float factors[] = {0.35f, 0.5f, 0.7f, 1.0f};
        const int items[] = {2, 4, 8};
        float best_ms = FLT_MAX;
        for (int shape = 0; shape < kShapes; ++shape)
            for (float fc : factors)
                for (int kk : items) {
                    float ms = 0.f;
                    rc = run_batched(ctx, in, p, on_device, fc, kk, shape, false, nullptr, nullptr, nullptr, &ms);
                    if (rc) return rc;
                    if (ms < best_ms) {
                        best_ms = ms;
                        B.cell_factor = fc;
                        B.kkc = kk;
                        B.shape = shape;
                    }
                }
        cache_store(cache_path, key, B.cell_factor, B.kkc, B.shape);
    }
    B.graph_valid = false;
    if (out_cell_factor) *out_cell_factor = B.cell_factor;
    if (out_points_per_item) *out_points_per_item = B.kkc;
    if (out_cta_threads) *out_cta_threads = kShapeThreads[B.shape];
    return SICP_OK;
}

extern "C" int sicp_trace_batched(sicp_ctx* ctx, int32_t t) {
    if (!ctx) return SICP_EINVAL;
    ctx->err.clear();
    if (!ctx->batch) ctx->batch = new BatchState();
    ctx->batch->trace_t = t < 0 ? -1 : t;
    return SICP_OK;
}

extern "C" int sicp_read_batched_trace(sicp_ctx* ctx, float* theta, float* adam_m, float* adam_v, int32_t* nn,
                                       float* gbar, float* phi) {
    if (!ctx) return SICP_EINVAL;
    ctx->err.clear();
    if (!ctx->batch || !ctx->batch->trace_ready)
        return set_err(ctx, SICP_EINVAL, "no batched trace recorded since sicp_trace_batched");
    BatchState& B = *ctx->batch;
    DeviceScopeB ds(ctx->device);
    const size_t st = sizeof(float) * 6 * (size_t)B.trace_K;
    const char* t0 = (const char*)B.tr.p;
    float* outs[5] = {theta, adam_m, adam_v, gbar, phi};
    for (int i = 0; i < 5; ++i)
        if (outs[i]) SICP_CUDA(cudaMemcpyAsync(outs[i], t0 + i * st, st, cudaMemcpyDeviceToHost, ctx->stream));
    if (nn)
        SICP_CUDA(cudaMemcpyAsync(nn, t0 + 5 * st, sizeof(int32_t) * (size_t)B.trace_K * B.trace_m,
                                  cudaMemcpyDeviceToHost, ctx->stream));
    SICP_CUDA(cudaStreamSynchronize(ctx->stream));
    return SICP_OK;
}
