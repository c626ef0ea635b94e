// Uniform voxel grid for the exact nearest-neighbour step (Eq. correspondences).
//
// Build, once per reference cloud:
//   bounding box -> cell id of every point -> per-cell counts -> exclusive
//   scan (cell_start) -> scatter into `sorted` (float4, w = original index)
//   -> per row (y, z) the first and last non-empty x -> per brick of 8^3 cells
//   the lowest original index it holds.
// Cells are numbered x fastest, so a run of cells along x is one contiguous
// range of `sorted`: the search reads whole row segments with float4 loads.
//
// Exact search of query q (the same fp32 squared distance and lowest-index
// tie rule as the exhaustive scan, so both give identical answers):
//   1. visit every cell within 1.5 cells of q, row segment by row segment,
//      centre rows first; if a point was found, it is the answer, because all
//      cells closer than it were visited;
//   2. otherwise take the best brick representative in the first two
//      non-empty brick rings as an upper bound, then visit every cell whose box
//      lies within the current best distance (the bound shrinks as points are
//      found; empty rows are skipped through the row spans).
// Pruning is conservative: cell bounds are widened by `tol` and the squared
// bound by a relative 5e-7, so rounding can only add visits, never drop one.
#include <float.h>
#include <math.h>

#include "common.cuh"

namespace sicp {
namespace {

constexpr int kQueryThreads = 128;
constexpr int64_t kMaxCells = 1 << 23;
constexpr float kSlack = 1.0000005f;

__host__ __device__ __forceinline__ int cell_coord(float v, float o, float inv, int n) {
    float f = (v - o) * inv;
    f = fminf(fmaxf(f, 0.f), (float)(n - 1));
    return (int)f;
}

__device__ __forceinline__ int cell_floor_clamped(float v, float o, float inv, int n) {
    float f = (v - o) * inv;
    f = fminf(fmaxf(f, -1.f), (float)n);
    return (int)floorf(f);
}

// Distance from coordinate v to the slab of cell i along one axis, minus tol.
__device__ __forceinline__ float slab(float v, float o, float c, int i, float tol) {
    const float lo = fmaf((float)i, c, o), hi = lo + c;
    const float d = fmaxf(fmaxf(lo - v, v - hi), 0.f);
    return fmaxf(d - tol, 0.f);
}

// Per-query work counters: rows examined, row segments read, candidate points.
struct Work {
    unsigned rows = 0, segs = 0, pts = 0;
};

__device__ __forceinline__ void scan_range(const float4* __restrict__ pts, int b, int e, float3 q, float& best,
                                           int& bi, float3& bp, Work& w) {
    w.segs += 1;
    w.pts += (unsigned)(e - b);
    for (int p = b; p < e; ++p) {
        const float4 r = __ldg(pts + p);
        const float d = dist2(r, q);
        const int id = __float_as_int(r.w);
        if (better(d, id, best, bi)) {
            best = d;
            bi = id;
            bp = make_float3(r.x, r.y, r.z);
        }
    }
}

// Squared pruning radius: min(best, cap2) widened by kSlack, kept finite.
__device__ __forceinline__ float bound2(float best, float cap2) {
    return fminf(fminf(best, cap2) * kSlack, FLT_MAX);
}

// Visit all cells whose box lies within sqrt(min(best, cap2)) of q.
__device__ void ball_rows(const GridView& g, float3 q, int cy, int cz, float cap2, float& best, int& bi,
                          float3& bp, Work& w) {
    for (int oz = 0;; ++oz) {
        bool live_z = false;
        for (int sz = 0; sz < 2; ++sz) {
            if (oz == 0 && sz == 1) break;
            const int z = sz ? cz - oz : cz + oz;
            if (z < 0 || z >= g.dims.z) continue;
            const float dz = slab(q.z, g.origin.z, g.cell, z, g.tol);
            if (bound2(best, cap2) - dz * dz < 0.f) continue;
            live_z = true;
            for (int oy = 0;; ++oy) {
                bool live_y = false;
                for (int sy = 0; sy < 2; ++sy) {
                    if (oy == 0 && sy == 1) break;
                    const int y = sy ? cy - oy : cy + oy;
                    if (y < 0 || y >= g.dims.y) continue;
                    const float dy = slab(q.y, g.origin.y, g.cell, y, g.tol);
                    const float rem = bound2(best, cap2) - dz * dz - dy * dy;
                    if (rem < 0.f) continue;
                    live_y = true;
                    const int rowi = z * g.dims.y + y;
                    w.rows += 1;
                    const int2 span = __ldg(g.row_span + rowi);
                    if (span.x > span.y) continue;
                    const float r = sqrtf(rem) + g.tol;
                    const int x0 = max(cell_floor_clamped(q.x - r, g.origin.x, g.inv_cell, g.dims.x), span.x);
                    const int x1 = min(cell_floor_clamped(q.x + r, g.origin.x, g.inv_cell, g.dims.x), span.y);
                    if (x0 > x1) continue;
                    const int64_t row = (int64_t)rowi * g.dims.x;
                    scan_range(g.sorted, __ldg(g.cell_start + row + x0), __ldg(g.cell_start + row + x1 + 1), q,
                               best, bi, bp, w);
                }
                if (!live_y) break;
            }
        }
        if (!live_z) break;
    }
}

// Upper bound from brick representatives: best over the first non-empty
// Chebyshev ring of bricks around the query's brick and the ring after it.
__device__ void brick_seed(const GridView& g, float3 q, int cx, int cy, int cz, float& best, int& bi, float3& bp,
                           Work& w) {
    const int bx = cx / kBrick, by = cy / kBrick, bz = cz / kBrick;
    const int maxr = max(max(g.bdims.x, g.bdims.y), g.bdims.z);
    int found_at = -1;
    for (int r = 0; r < maxr; ++r) {
        for (int dz = -r; dz <= r; ++dz) {
            const int z = bz + dz;
            if (z < 0 || z >= g.bdims.z) continue;
            for (int dy = -r; dy <= r; ++dy) {
                const int y = by + dy;
                if (y < 0 || y >= g.bdims.y) continue;
                const bool face = (dz == -r || dz == r || dy == -r || dy == r);
                const int step = (face || r == 0) ? 1 : 2 * r;
                for (int dx = -r; dx <= r; dx += step) {
                    const int x = bx + dx;
                    if (x < 0 || x >= g.bdims.x) continue;
                    const int rep = __ldg(g.brick_rep + ((int64_t)z * g.bdims.y + y) * g.bdims.x + x);
                    w.rows += 1;
                    if (rep == kEmpty) continue;
                    w.pts += 1;
                    const float4 p = __ldg(g.ref4 + rep);
                    const float d = dist2(p, q);
                    if (better(d, rep, best, bi)) {
                        best = d;
                        bi = rep;
                        bp = make_float3(p.x, p.y, p.z);
                    }
                    if (found_at < 0) found_at = r;
                }
            }
        }
        if (found_at >= 0 && r >= found_at + 1) break;
    }
}

__device__ __forceinline__ void grid_search(const GridView& g, float3 q, float& best, int& bi, float3& bp,
                                            Work& w) {
    best = FLT_MAX;
    bi = 0x7fffffff;
    bp = make_float3(0.f, 0.f, 0.f);
    const int cx = cell_coord(q.x, g.origin.x, g.inv_cell, g.dims.x);
    const int cy = cell_coord(q.y, g.origin.y, g.inv_cell, g.dims.y);
    const int cz = cell_coord(q.z, g.origin.z, g.inv_cell, g.dims.z);
    const float r0 = 1.5f * g.cell;
    ball_rows(g, q, cy, cz, r0 * r0, best, bi, bp, w);
    if (best <= r0 * r0) return;
    brick_seed(g, q, cx, cy, cz, best, bi, bp, w);
    ball_rows(g, q, cy, cz, FLT_MAX, best, bi, bp, w);
}

// Warp-aggregated accumulation of the work counters (stats: queries, rows, segments, points).
__device__ __forceinline__ void add_stats(unsigned long long* stats, bool active, const Work& w) {
    unsigned long long v[4] = {active ? 1ull : 0ull, w.rows, w.segs, w.pts};
#pragma unroll
    for (int a = 0; a < 4; ++a) {
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) v[a] += __shfl_down_sync(0xffffffffu, v[a], off);
    }
    if ((threadIdx.x & 31) == 0) {
#pragma unroll
        for (int a = 0; a < 4; ++a) atomicAdd(stats + a, v[a]);
    }
}

__global__ void __launch_bounds__(kQueryThreads) k_nn_grid(GridView g, const float* __restrict__ q, int64_t n,
                                                           int32_t* __restrict__ idx, float* __restrict__ d2,
                                                           unsigned long long* __restrict__ stats) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    Work w;
    if (i < n) {
        const float3 qq = make_float3(q[3 * i], q[3 * i + 1], q[3 * i + 2]);
        float best;
        int bi;
        float3 bp;
        grid_search(g, qq, best, bi, bp, w);
        idx[i] = bi != 0x7fffffff ? bi : -1;
        if (d2) d2[i] = best;
    }
    if (stats) add_stats(stats, i < n, w);
}

// Deterministic block sum of 6 values per thread (result in thread 0).
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

// grid (chunks, K); CTA (c, j) handles minibatch entries [c*blockDim, (c+1)*blockDim) of particle j.
__global__ void __launch_bounds__(256) k_grad_grid(GradArgs a, GridView g) {
    __shared__ Pose P;
    __shared__ float red[8][6];
    const int j = blockIdx.y;
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (threadIdx.x == 0) make_pose(a.theta + 6 * j, P);
    __syncthreads();
    float gr[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    Work w;
    if (k < a.m) {
        const float4 s4 = __ldg(a.src + __ldg(a.mb + k));
        const float3 s = make_float3(s4.x, s4.y, s4.z);
        const float3 q = apply_pose(P, s);
        float best;
        int bi;
        float3 bp;
        grid_search(g, q, best, bi, bp, w);
        const bool found = bi != 0x7fffffff;  // false only for a non-finite distance
        if (found) grad_terms(P, s, make_float3(q.x - bp.x, q.y - bp.y, q.z - bp.z), gr);
        if (a.out_nn) a.out_nn[(int64_t)j * a.m + k] = found ? bi : -1;
    }
    if (a.stats) add_stats(a.stats, k < a.m, w);
    block_sum6(gr, red);
    if (threadIdx.x == 0) {
        float* dst = a.partial + ((int64_t)blockIdx.x * a.K + j) * 6;
        for (int c = 0; c < 6; ++c) dst[c] = gr[c];
    }
}

// ---------------------------------------------------------------- build kernels

__global__ void k_cell_assign(const float4* __restrict__ ref, int64_t M, GridView g, int32_t* __restrict__ cell_of,
                              int32_t* __restrict__ counts, int32_t* __restrict__ brick_rep) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < M; i += (int64_t)gridDim.x * blockDim.x) {
        const float4 p = ref[i];
        const int cx = cell_coord(p.x, g.origin.x, g.inv_cell, g.dims.x);
        const int cy = cell_coord(p.y, g.origin.y, g.inv_cell, g.dims.y);
        const int cz = cell_coord(p.z, g.origin.z, g.inv_cell, g.dims.z);
        const int32_t cid = (int32_t)(((int64_t)cz * g.dims.y + cy) * g.dims.x + cx);
        cell_of[i] = cid;
        atomicAdd(counts + cid, 1);
        const int64_t b = ((int64_t)(cz / kBrick) * g.bdims.y + cy / kBrick) * g.bdims.x + cx / kBrick;
        atomicMin(brick_rep + b, (int32_t)i);
    }
}

__global__ void k_scatter(const float4* __restrict__ ref, int64_t M, const int32_t* __restrict__ cell_of,
                          const int32_t* __restrict__ cell_start, int32_t* __restrict__ cursor,
                          float4* __restrict__ sorted) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < M; i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t c = cell_of[i];
        const int pos = cell_start[c] + atomicAdd(cursor + c, 1);
        sorted[pos] = ref[i];
    }
}

// Order each cell's points by original index, so the layout is deterministic.
__global__ void k_sort_cells(const int32_t* __restrict__ cell_start, int64_t ncells, float4* __restrict__ sorted) {
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < ncells; c += (int64_t)gridDim.x * blockDim.x) {
        const int b = cell_start[c], e = cell_start[c + 1];
        for (int i = b + 1; i < e; ++i) {
            const float4 v = sorted[i];
            const int key = __float_as_int(v.w);
            int j = i - 1;
            while (j >= b && __float_as_int(sorted[j].w) > key) {
                sorted[j + 1] = sorted[j];
                --j;
            }
            sorted[j + 1] = v;
        }
    }
}

__global__ void k_row_span(const int32_t* __restrict__ cell_start, GridView g, int2* __restrict__ span) {
    const int64_t rows = (int64_t)g.dims.y * g.dims.z;
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < rows; r += (int64_t)gridDim.x * blockDim.x) {
        const int32_t* cs = cell_start + r * g.dims.x;
        int lo = g.dims.x, hi = -1;
        for (int x = 0; x < g.dims.x; ++x) {
            if (cs[x + 1] > cs[x]) {
                if (lo > x) lo = x;
                hi = x;
            }
        }
        span[r] = make_int2(lo, hi);
    }
}

unsigned blocks_for(int64_t n, int threads, int cap = 8192) {
    int64_t b = (n + threads - 1) / threads;
    return (unsigned)(b < 1 ? 1 : (b > cap ? cap : b));
}

template <typename T>
int grow(sicp_ctx* ctx, T*& p, size_t& cap, size_t n) {
    if (n <= cap && p) return SICP_OK;
    if (p) cudaFree(p);
    p = nullptr;
    cap = 0;
    const size_t want = n + n / 4 + 16;
    if (cudaMalloc(&p, sizeof(T) * want) != cudaSuccess) {
        cudaGetLastError();
        return set_err(ctx, SICP_ENOMEM, "grid allocation of %zu elements failed", want);
    }
    cap = want;
    return SICP_OK;
}

}  // namespace

int grid_build(sicp_ctx* ctx, float cell_size) {
    Grid& G = ctx->grid;
    const int64_t M = ctx->M;
    cudaStream_t s = ctx->stream;
    int rc = ensure(ctx, ctx->bbox, 8 * sizeof(unsigned));
    if (rc) return rc;
    unsigned* lohi = (unsigned*)ctx->bbox.p;
    SICP_CUDA(cudaMemsetAsync(lohi, 0xff, 3 * sizeof(unsigned), s));
    SICP_CUDA(cudaMemsetAsync(lohi + 3, 0x00, 3 * sizeof(unsigned), s));
    SICP_CUDA(launch_bbox(ctx->ref4, M, lohi, s));
    unsigned h[6];
    SICP_CUDA(cudaMemcpyAsync(h, lohi, sizeof h, cudaMemcpyDeviceToHost, s));
    SICP_CUDA(cudaStreamSynchronize(s));
    float lo[3], hi[3], ext[3];
    double X = 0.0;
    for (int a = 0; a < 3; ++a) {
        lo[a] = ordered_to_float(h[a]);
        hi[a] = ordered_to_float(h[3 + a]);
        ext[a] = hi[a] - lo[a];
        X = fmax(X, fmax(fabs((double)lo[a]), fabs((double)hi[a])));
    }
    ctx->ref_lo = make_float3(lo[0], lo[1], lo[2]);
    ctx->ref_hi = make_float3(hi[0], hi[1], hi[2]);
    double maxext = fmax(ext[0], fmax(ext[1], ext[2]));
    double c = cell_size;
    if (!(c > 0.0)) {
        if (maxext <= 0.0) {
            c = 1.0;
        } else {
            // half the volumetric spacing of the (degenerate axes padded) box
            const double floor_ext = maxext * 1e-3;
            const double V = fmax(ext[0], floor_ext) * fmax(ext[1], floor_ext) * fmax(ext[2], floor_ext);
            c = 0.5 * cbrt(V / (double)M);
        }
    }
    int3 dims;
    for (;;) {
        dims.x = (int)fmin(floor(ext[0] / c) + 1.0, 1 << 20);
        dims.y = (int)fmin(floor(ext[1] / c) + 1.0, 1 << 20);
        dims.z = (int)fmin(floor(ext[2] / c) + 1.0, 1 << 20);
        const double n = (double)dims.x * dims.y * dims.z;
        if (n <= (double)kMaxCells) break;
        c *= cbrt(n / (double)kMaxCells) * 1.01;
    }
    const int64_t ncells = (int64_t)dims.x * dims.y * dims.z;
    const int3 bd = make_int3((dims.x + kBrick - 1) / kBrick, (dims.y + kBrick - 1) / kBrick,
                              (dims.z + kBrick - 1) / kBrick);
    const int64_t nbricks = (int64_t)bd.x * bd.y * bd.z;
    const int64_t rows = (int64_t)dims.y * dims.z;
    if ((rc = grow(ctx, G.sorted, G.cap_points, (size_t)M))) return rc;
    if ((rc = grow(ctx, G.cell_of, G.cap_cellof, (size_t)M))) return rc;
    if ((rc = grow(ctx, G.cell_start, G.cap_cells, (size_t)ncells + 1))) return rc;
    if ((rc = grow(ctx, G.counts, G.cap_counts, (size_t)ncells + 1))) return rc;
    if ((rc = grow(ctx, G.row_span, G.cap_rows, (size_t)rows))) return rc;
    if ((rc = grow(ctx, G.brick_rep, G.cap_bricks, (size_t)nbricks))) return rc;
    if ((rc = grow(ctx, G.scan_sums, G.cap_sums, scan_sums_size(ncells)))) return rc;

    GridView& v = G.v;
    v.origin = make_float3(lo[0], lo[1], lo[2]);
    v.cell = (float)c;
    v.inv_cell = (float)(1.0 / c);
    v.tol = (float)(1e-6 * (X + c));
    v.dims = dims;
    v.bdims = bd;
    v.sorted = G.sorted;
    v.cell_start = G.cell_start;
    v.row_span = G.row_span;
    v.brick_rep = G.brick_rep;
    v.ref4 = ctx->ref4;
    G.ncells = ncells;
    G.nbricks = nbricks;

    SICP_CUDA(cudaMemsetAsync(G.counts, 0, sizeof(int32_t) * ncells, s));
    SICP_CUDA(cudaMemsetAsync(G.brick_rep, 0x7f, sizeof(int32_t) * nbricks, s));
    k_cell_assign<<<blocks_for(M, 256), 256, 0, s>>>(ctx->ref4, M, v, G.cell_of, G.counts, G.brick_rep);
    SICP_CUDA(cudaGetLastError());
    SICP_CUDA(launch_exclusive_scan(G.counts, ncells, G.cell_start, G.scan_sums, s));
    SICP_CUDA(cudaMemsetAsync(G.counts, 0, sizeof(int32_t) * ncells, s));
    k_scatter<<<blocks_for(M, 256), 256, 0, s>>>(ctx->ref4, M, G.cell_of, G.cell_start, G.counts, G.sorted);
    SICP_CUDA(cudaGetLastError());
    k_sort_cells<<<blocks_for(ncells, 256), 256, 0, s>>>(G.cell_start, ncells, G.sorted);
    SICP_CUDA(cudaGetLastError());
    k_row_span<<<blocks_for(rows, 128), 128, 0, s>>>(G.cell_start, v, G.row_span);
    SICP_CUDA(cudaGetLastError());
    return SICP_OK;
}

cudaError_t launch_nn_grid(const GridView& g, const float* q, int64_t n, int32_t* idx, float* d2,
                           unsigned long long* stats, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    k_nn_grid<<<(unsigned)((n + kQueryThreads - 1) / kQueryThreads), kQueryThreads, 0, s>>>(g, q, n, idx, d2, stats);
    return cudaGetLastError();
}

cudaError_t launch_grad_grid(const GradArgs& a, const GridView& g, cudaStream_t s) {
    const GradLayout L = grad_layout(a.m);
    dim3 grid(L.chunks, a.K);
    k_grad_grid<<<grid, L.threads, 0, s>>>(a, g);
    return cudaGetLastError();
}

}  // namespace sicp
