// Uniform voxel grid for the exact nearest-neighbour step (Eq. correspondences).
//
// Build, once per reference cloud, for a fine level (cell c) and a coarse
// level (cell 4c) over the same points:
//   cell id of every point -> per-cell counts -> exclusive scan (cell_start)
//   -> scatter into `sorted` (float4, w = original index) -> order each cell
//   by index.
// The fine level also gets a seed map: for every cell, a point close to the
// cell centre, found by jump flooding (each cell repeatedly adopts the
// closest seed among its neighbours at offsets n/2, n/4, ..., 1, 1).
// Cells are numbered x fastest, so a run of cells along x is one contiguous
// range of `sorted`: the search reads whole row segments with float4 loads.
//
// Exact search of one query by one warp.  A host-built table lists row
// offsets (dy, dz) in increasing order of a lower bound on the distance from
// the query to the row (offsets mirrored into the half of the cell the query
// lies in).  A round gives each lane one row; the lane clips the row to the
// ball of the current bound (skipping out-of-reach rows) and publishes the
// row segment (two cell_start loads); the warp flattens the round's segments and
// evaluates their points 32 at a time, so all lanes do the same work; a warp
// minimum (squared distance, then lowest index) closes the round.
// The seed of the query's cell gives a first point and bound; then the table
// is walked from the start, 32 rows a round, with that bound on the fine level
// (bound under 6 cells) or the coarse level, until the next row is out of
// reach.  (A first round over the 3 x 3 x 3 cells around the seed, to tighten
// the bound before the walk, cost more than it saved: the walk's first 32 rows
// already hold them.)  A query the table cannot settle scans all points.  In the
// gradient kernel a query whose neighbouring particle's answer lies within
// two fine cells starts the walk from that answer instead.  The same search
// also runs on a half-warp (16 lanes, 16 rows a round), two queries per warp:
// the gradient kernel of independent runs uses it.
// Every search uses the same fp32 squared distance and tie rule as the
// exhaustive scan, so both give the same answer.
//
// Pruning is conservative: cell bounds are widened by `tol` and the squared
// bound by a relative 5e-7, so rounding can only add visits, never drop one.
#include <float.h>
#include <math.h>

#include <algorithm>
#include <cmath>
#include <mutex>
#include <vector>

#include "common.cuh"
#include "grid_search.cuh"

namespace sicp {
namespace {

// Search descriptions in constant memory, one slot per context (uniform reads
// through the constant cache, as fast as kernel parameters).  A reference
// build rewrites its context's slot in stream order, so a captured loop stays
// valid when the reference changes.  Contexts beyond kSearchSlots read the
// device-memory copy instead.
constexpr int kSearchSlots = 32;
__constant__ GridSearch c_search[kSearchSlots];
std::mutex g_slot_mu;
bool g_slot_used[kSearchSlots];

using namespace gs;


__global__ void __launch_bounds__(kThreads) k_nn_grid(GridSearch S, const float* __restrict__ q, int64_t n,
                                                      int32_t* __restrict__ idx, float* __restrict__ d2,
                                                      unsigned long long* __restrict__ stats) {
    const int lane = threadIdx.x & 31;
    const int64_t i = (int64_t)blockIdx.x * kWarps + (threadIdx.x >> 5);
    Work w;
    if (i < n) {
        const float3 qq = make_float3(q[3 * i], q[3 * i + 1], q[3 * i + 2]);
        Best B;
        grid_search(S, qq, B, w);
        if (lane == 0) {
            idx[i] = B.i != kNone ? B.i : -1;
            if (d2) d2[i] = B.d;
        }
    }
    if (stats) add_stats(stats, w);
}

// grid (minibatch entries, blocks of part<G>() particles).  Each group of G
// lanes (a warp, G = 32, or a half-warp, G = 16) of CTA (k, b) handles
// minibatch entry k for the kSeq particles b*part + group*kSeq ...: the first
// query runs the whole search; each next one is the same source point under a
// neighbouring particle, so the previous answer is a starting bound (kept
// when it lies within kReuse cells, else the seed map is used).  Lane 0 of
// the group writes the query's gradient terms to qterms[j][k]; a fixed-order
// reduction over k follows (launch_qterms_to_gbar).  One particle per group
// is fastest on the kinect scene: the seed map gives a tighter start than a
// neighbouring particle's answer (45.2 against 46.6 candidates per query),
// and 128-thread CTAs at 40 registers hold 48 warps per SM.
constexpr int kSeq = 1;                                   // particles per group
constexpr float kReuse = 2.f;
template <int G>
__host__ __device__ constexpr int part() {                // particles per CTA
    return kSeq * (kGradThreads / G);
}

// The search description is read from memory that the reference build
// rewrites, so a captured graph of these launches stays valid when the
// reference changes: kConst, the context's constant-memory slot c_search[slot];
// else the device copy Sd.  (Staging it in shared memory was slower.)
// kStats: the work counters are kept (sicp_stats on); otherwise they are dead
// code and the compiler drops them.
template <int G, bool kStats, bool kConst>
__global__ void __launch_bounds__(kGradThreads, 12) k_grad_grid(GradArgs a, const GridSearch* __restrict__ Sd,
                                                                int slot) {
    constexpr int kPart = part<G>();
    __shared__ Pose P[kPart];
    const int grp = threadIdx.x / G, lane = threadIdx.x & (G - 1);
    const int k = blockIdx.x;
    const int j0 = blockIdx.y * kPart;
    // the minibatch entry and its source point were written before the chain of
    // launches (see pdl_wait), so they are read before the wait
    const float4 s4 = __ldg(a.src + SICP_IDX(__ldg(a.mb + k), a.n_src, kChkSrc));
    pdl_wait();      // the particles of the previous Stein step
    pdl_trigger();   // only after the wait: see pdl_wait
    for (int i = threadIdx.x; i < kPart; i += blockDim.x)
        if (j0 + i < a.K) make_pose(a.theta + 6 * (j0 + i), P[i]);
    __syncthreads();
    const GridSearch& S = kConst ? c_search[slot] : *Sd;
    float3 s = make_float3(s4.x, s4.y, s4.z);
    const float reuse2 = (kReuse * S.fine.cell) * (kReuse * S.fine.cell);
    Work w;
    Best B;
    B.i = kNone;
    for (int i = 0; i < kSeq; ++i) {
        const int jl = grp * kSeq + i, j = j0 + jl;
        if (j >= a.K) break;                        // uniform over the group
        if (a.mb_stride) {                          // independent runs: particle j's own minibatch
            const float4 sj = __ldg(a.src + SICP_IDX(__ldg(a.mb + (int64_t)j * a.mb_stride + k), a.n_src, kChkSrc));
            s = make_float3(sj.x, sj.y, sj.z);
        }
        const float3 q = apply_pose(P[jl], s);
        bool seeded = false;
        if (B.i != kNone) {
            const float d = dist2(make_float4(B.p.x, B.p.y, B.p.z, 0.f), q);
            if (d <= reuse2) {
                B.d = d;
                seeded = true;
                w.queries += lane == 0;
                prove<G>(S, q, B, w);
            }
        }
        if (!seeded) grid_search<G>(S, q, B, w);
        // the six gradient terms, one per lane (B, q and s are the same in every lane of the group)
        const bool found = B.i != kNone;   // false only for a non-finite distance
        float3 d = make_float3(q.x - B.p.x, q.y - B.p.y, q.z - B.p.z);
        if (found && a.normals) d = plane_residual(__ldg(a.normals + SICP_IDX(B.i, a.n_ref, kChkRef)), d);
        if (lane < 6) a.partial[((int64_t)j * a.m + k) * 6 + lane] = found ? grad_term(P[jl], s, d, lane) : 0.f;
        if (lane == 0 && a.out_nn) a.out_nn[(int64_t)j * a.m + k] = found ? B.i : -1;
    }
    if (kStats) add_stats(a.stats, w);
}

// ---------------------------------------------------------------- build kernels

__global__ void k_cell_assign(const float4* __restrict__ ref, int64_t M, GridView g, int32_t* __restrict__ cell_of,
                              int32_t* __restrict__ counts) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < M; i += (int64_t)gridDim.x * blockDim.x) {
        const float4 p = ref[i];
        const int cx = cell_coord(p.x, g.origin.x, g.inv_cell, g.dims.x);
        const int cy = cell_coord(p.y, g.origin.y, g.inv_cell, g.dims.y);
        const int cz = cell_coord(p.z, g.origin.z, g.inv_cell, g.dims.z);
        const int32_t cid = (int32_t)(((int64_t)cz * g.dims.y + cy) * g.dims.x + cx);
        cell_of[i] = cid;
        atomicAdd(counts + cid, 1);
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
// One thread per point (most cells are empty; every point has a cell): its
// rank in its cell is the number of the cell's points with a smaller index,
// counted over the cell's unordered copy in `staging`.
__global__ void k_sort_points(const float4* __restrict__ ref, int64_t M, const int32_t* __restrict__ cell_of,
                              const int32_t* __restrict__ cell_start, const float4* __restrict__ staging,
                              float4* __restrict__ out) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < M; i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t c = cell_of[i];
        const int b = cell_start[c], e = cell_start[c + 1];
        int rank = 0;
        for (int k = b; k < e; ++k) rank += __float_as_int(staging[k].w) < (int)i;
        out[b + rank] = ref[i];
    }
}

// Cell coordinates of cell id c (x fastest).  Grids hold at most kMaxCells
// (2^23) cells, so the decode runs in 32-bit integer arithmetic.
__device__ __forceinline__ void cell_xyz(const GridView& g, int64_t c, int& x, int& y, int& z) {
    const int ci = (int)c, t = ci / g.dims.x;
    x = ci - t * g.dims.x;
    z = t / g.dims.y;
    y = t - z * g.dims.y;
}

__device__ __forceinline__ float3 cell_centre(const GridView& g, int x, int y, int z) {
    return make_float3(g.origin.x + ((float)x + 0.5f) * g.cell, g.origin.y + ((float)y + 0.5f) * g.cell,
                       g.origin.z + ((float)z + 0.5f) * g.cell);
}

// Seed of a non-empty cell: its point closest to the cell centre; -1 otherwise.
__global__ void k_seed_init(GridView g, int64_t ncells, int32_t* __restrict__ seed) {
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < ncells; c += (int64_t)gridDim.x * blockDim.x) {
        const int b = g.cell_start[c], e = g.cell_start[c + 1];
        int best = -1;
        if (e > b) {
            int x, y, z;
            cell_xyz(g, c, x, y, z);
            const float3 ct = cell_centre(g, x, y, z);
            float bd = FLT_MAX;
            for (int p = b; p < e; ++p) {
                const float d = dist2(g.sorted[p], ct);
                if (d < bd) {
                    bd = d;
                    best = p;
                }
            }
        }
        seed[c] = best;
    }
}

// One jump-flooding step at offset k: adopt the closest seed among the 27 cells at offsets {-k, 0, k}^3.
__global__ void k_seed_step(GridView g, int64_t ncells, int k, const int32_t* __restrict__ in,
                            int32_t* __restrict__ out) {
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < ncells; c += (int64_t)gridDim.x * blockDim.x) {
        int x, y, z;
        cell_xyz(g, c, x, y, z);
        const float3 ct = cell_centre(g, x, y, z);
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
                    const int s = in[((int64_t)zz * g.dims.y + yy) * g.dims.x + xx];
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

// The seed points themselves, so that a query's first candidate is one load
// (none: an infinitely far point, never taken).
__global__ void k_seed_points(const float4* __restrict__ sorted, const int32_t* __restrict__ seed, int64_t ncells,
                              float4* __restrict__ seed4) {
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < ncells; c += (int64_t)gridDim.x * blockDim.x) {
        const int32_t s = seed[c];
        seed4[c] = s >= 0 ? sorted[s] : make_float4(INFINITY, INFINITY, INFINITY, __int_as_float(-1));
    }
}

unsigned blocks_for(int64_t n, int threads, int cap = 8192) {
    int64_t b = (n + threads - 1) / threads;
    return (unsigned)(b < 1 ? 1 : (b > cap ? cap : b));
}

template <typename T>
int grow(sicp_ctx* ctx, T*& p, size_t& cap, size_t n) {
    if (n <= cap && p) return SICP_OK;
    const size_t held = sizeof(T) * cap;
    if (p) cudaFree(p);
    p = nullptr;
    cap = 0;
    const size_t want = n + n / 4 + 16;
    void* q = nullptr;
    int rc = budget_malloc(ctx, &q, sizeof(T) * want, held);
    if (rc) return rc;
    p = (T*)q;
    cap = want;
    return SICP_OK;
}

int3 dims_for(const float ext[3], double& c) {
    int3 d;
    for (;;) {
        d.x = (int)fmin(floor(ext[0] / c) + 1.0, 1 << 20);
        d.y = (int)fmin(floor(ext[1] / c) + 1.0, 1 << 20);
        d.z = (int)fmin(floor(ext[2] / c) + 1.0, 1 << 20);
        const double n = (double)d.x * d.y * d.z;
        if (n <= (double)kMaxCells) return d;
        c *= cbrt(n / (double)kMaxCells) * 1.01;
    }
}

// Build one level with cell edge c over the context's reference points; the
// seed map only when `seeds`.
int build_level(sicp_ctx* ctx, Grid& G, const float lo[3], const float ext[3], double X, double c, bool seeds) {
    const int64_t M = ctx->M;
    cudaStream_t s = ctx->stream;
    const int3 dims = dims_for(ext, c);
    const int64_t ncells = (int64_t)dims.x * dims.y * dims.z;
    int rc;
    if ((rc = grow(ctx, G.sorted, G.cap_points, (size_t)M))) return rc;
    if ((rc = grow(ctx, G.cell_of, G.cap_cellof, (size_t)M))) return rc;
    if ((rc = grow(ctx, G.cell_start, G.cap_cells, (size_t)ncells + 1))) return rc;
    if ((rc = grow(ctx, G.counts, G.cap_counts, (size_t)ncells + 1))) return rc;
    if ((rc = grow(ctx, G.scan_sums, G.cap_sums, scan_sums_size(ncells)))) return rc;
    if (seeds) {
        if ((rc = grow(ctx, G.seed, G.cap_seed, (size_t)ncells))) return rc;
        if ((rc = grow(ctx, G.seed_tmp, G.cap_seed_tmp, (size_t)ncells))) return rc;
        if ((rc = grow(ctx, G.seed4, G.cap_seed4, (size_t)ncells))) return rc;
    }
    // the scatter target doubles as the unsorted staging area of the per-cell sort
    float4* staging = (float4*)ctx->tmp_aux.p;
    if ((rc = ensure(ctx, ctx->tmp_aux, sizeof(float4) * (size_t)M))) return rc;
    staging = (float4*)ctx->tmp_aux.p;
    GridView& v = G.v;
    v.origin = make_float3(lo[0], lo[1], lo[2]);
    v.cell = (float)c;
    v.inv_cell = (float)(1.0 / c);
    v.tol = (float)(1e-6 * (X + c));
    v.dims = dims;
    v.sorted = G.sorted;
    v.nsorted = (int32_t)M;
    v.cell_start = G.cell_start;
    v.seed = seeds ? G.seed : nullptr;
    v.seed4 = seeds ? G.seed4 : nullptr;
    G.ncells = ncells;
    SICP_CUDA(cudaMemsetAsync(G.counts, 0, sizeof(int32_t) * ncells, s));
    k_cell_assign<<<blocks_for(M, 256), 256, 0, s>>>(ctx->ref4, M, v, G.cell_of, G.counts);
    SICP_CUDA(cudaGetLastError());
    SICP_CUDA(launch_exclusive_scan(G.counts, ncells, G.cell_start, G.scan_sums, s));
    SICP_CUDA(cudaMemsetAsync(G.counts, 0, sizeof(int32_t) * ncells, s));
    k_scatter<<<blocks_for(M, 256), 256, 0, s>>>(ctx->ref4, M, G.cell_of, G.cell_start, G.counts, staging);
    SICP_CUDA(cudaGetLastError());
    k_sort_points<<<blocks_for(M, 256), 256, 0, s>>>(ctx->ref4, M, G.cell_of, G.cell_start, staging, G.sorted);
    SICP_CUDA(cudaGetLastError());
    if (seeds) {
        int32_t* a = G.seed;
        int32_t* b = G.seed_tmp;
        k_seed_init<<<blocks_for(ncells, 256), 256, 0, s>>>(v, ncells, a);
        SICP_CUDA(cudaGetLastError());
        int k = 1;
        while (k * 2 <= std::max(dims.x, std::max(dims.y, dims.z)) / 2) k *= 2;
        std::vector<int> steps;
        for (; k >= 1; k /= 2) steps.push_back(k);
        steps.push_back(1);
        for (int st : steps) {
            k_seed_step<<<blocks_for(ncells, 256), 256, 0, s>>>(v, ncells, st, a, b);
            SICP_CUDA(cudaGetLastError());
            std::swap(a, b);
        }
        if (a != G.seed) SICP_CUDA(cudaMemcpyAsync(G.seed, a, sizeof(int32_t) * ncells, cudaMemcpyDeviceToDevice, s));
        k_seed_points<<<blocks_for(ncells, 256), 256, 0, s>>>(G.sorted, G.seed, ncells, G.seed4);
        SICP_CUDA(cudaGetLastError());
    }
    return SICP_OK;
}

}  // namespace

int search_table_init(sicp_ctx* ctx) {
    struct E {
        short dy, dz;
        float lb2;
    };
    std::vector<E> es;
    const int R = kTableRadius;
    for (int dz = -R; dz <= R; ++dz)
        for (int dy = -R; dy <= R; ++dy) {
            // lower bound (cell units) on the distance from a query in the upper half of its cell
            const float lz = dz == 0 ? 0.f : (dz > 0 ? (float)(dz - 1) : (float)(-dz) - 0.5f);
            const float ly = dy == 0 ? 0.f : (dy > 0 ? (float)(dy - 1) : (float)(-dy) - 0.5f);
            const float lb2 = lz * lz + ly * ly;
            if (lb2 <= (float)((R - 1) * (R - 1))) es.push_back({(short)dy, (short)dz, lb2});
        }
    std::stable_sort(es.begin(), es.end(), [](const E& a, const E& b) {
        if (a.lb2 != b.lb2) return a.lb2 < b.lb2;
        return abs(a.dy) + abs(a.dz) < abs(b.dy) + abs(b.dz);
    });
    std::vector<short2> off(es.size());
    std::vector<float> lb2(es.size()), lb(es.size());
    for (size_t i = 0; i < es.size(); ++i) {
        off[i] = make_short2(es[i].dy, es[i].dz);
        lb2[i] = es[i].lb2;
        lb[i] = std::sqrt(es[i].lb2);   // correctly rounded, as sqrtf on the device
    }
    if (cudaMalloc(&ctx->tab_off, sizeof(short2) * off.size()) != cudaSuccess ||
        cudaMalloc(&ctx->tab_lb, sizeof(float) * lb.size()) != cudaSuccess) {
        cudaGetLastError();
        return set_err(ctx, SICP_ENOMEM, "search table allocation failed");
    }
    SICP_CUDA(cudaMemcpy(ctx->tab_off, off.data(), sizeof(short2) * off.size(), cudaMemcpyHostToDevice));
    SICP_CUDA(cudaMemcpy(ctx->tab_lb, lb.data(), sizeof(float) * lb.size(), cudaMemcpyHostToDevice));
    SearchTable& t = ctx->search.tab;
    t.off = ctx->tab_off;
    t.lb = ctx->tab_lb;
    t.n = (int)off.size();
    for (int k = 0; k < 8; ++k) {
        const float cap = 1.5f * (float)(1 << k);
        t.upto[k] = (int)(std::upper_bound(lb2.begin(), lb2.end(), cap * cap) - lb2.begin());
    }
    return SICP_OK;
}

int grid_build(sicp_ctx* ctx, float cell_size) {
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
    const double maxext = fmax(ext[0], fmax(ext[1], ext[2]));
    double c = cell_size;
    if (!(c > 0.0)) {
        if (maxext <= 0.0) {
            c = 1.0;
        } else {
            // half the volumetric spacing of the box (degenerate axes padded)
            const double floor_ext = maxext * 1e-3;
            const double V = fmax(ext[0], floor_ext) * fmax(ext[1], floor_ext) * fmax(ext[2], floor_ext);
            c = 0.5 * cbrt(V / (double)M);
        }
    }
    if ((rc = build_level(ctx, ctx->grid, lo, ext, X, c, true))) return rc;
    const double c2 = (double)ctx->grid.v.cell * kCoarseFactor;
    if ((rc = build_level(ctx, ctx->grid2, lo, ext, X, c2, false))) return rc;
    ctx->search.fine = ctx->grid.v;
    ctx->search.coarse = ctx->grid2.v;
    ctx->search.ref4 = ctx->ref4;
    ctx->search.M = (int)M;
    ctx->search.reach = kFineReach;
    // the device copy the captured gradient launches read
    if ((rc = ensure(ctx, ctx->search_dev, sizeof(GridSearch)))) return rc;
    SICP_CUDA(cudaMemcpyAsync(ctx->search_dev.p, &ctx->search, sizeof(GridSearch), cudaMemcpyHostToDevice, s));
    if (ctx->search_slot == -2) ctx->search_slot = search_slot_acquire();
    if (ctx->search_slot >= 0)
        SICP_CUDA(cudaMemcpyToSymbolAsync(c_search, &ctx->search, sizeof(GridSearch),
                                          sizeof(GridSearch) * (size_t)ctx->search_slot, cudaMemcpyHostToDevice, s));
    return SICP_OK;
}

GradLayout grad_layout_grid(int32_t m) {
    GradLayout L;
    L.chunks = m;   // per-query terms, [K][m][6]
    L.threads = kGradThreads;
    return L;
}

cudaError_t launch_nn_grid(const GridSearch& g, const float* q, int64_t n, int32_t* idx, float* d2,
                           unsigned long long* stats, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    k_nn_grid<<<(unsigned)((n + kWarps - 1) / kWarps), kThreads, 0, s>>>(g, q, n, idx, d2, stats);
    return cudaGetLastError();
}

int search_slot_acquire() {
    std::lock_guard<std::mutex> lk(g_slot_mu);
    for (int i = 0; i < kSearchSlots; ++i)
        if (!g_slot_used[i]) {
            g_slot_used[i] = true;
            return i;
        }
    return -1;
}

void search_slot_release(int slot) {
    if (slot < 0 || slot >= kSearchSlots) return;
    std::lock_guard<std::mutex> lk(g_slot_mu);
    g_slot_used[slot] = false;
}

template <int G>
cudaError_t launch_grad_grid_g(const GradArgs& a, const GridSearch* d_search, int slot, cudaStream_t s) {
    const dim3 grid((unsigned)a.m, (unsigned)((a.K + part<G>() - 1) / part<G>()));
    const dim3 blk(kGradThreads);
    if (slot >= 0)
        return a.stats ? launch_pdl(k_grad_grid<G, true, true>, grid, blk, 0, s, a, d_search, slot)
                       : launch_pdl(k_grad_grid<G, false, true>, grid, blk, 0, s, a, d_search, slot);
    return a.stats ? launch_pdl(k_grad_grid<G, true, false>, grid, blk, 0, s, a, d_search, slot)
                   : launch_pdl(k_grad_grid<G, false, false>, grid, blk, 0, s, a, d_search, slot);
}

// Independent runs (each particle its own minibatch) search with half-warps,
// Stein runs with whole warps.  Measured on the kinect scene (the gradient
// launch, warp against half-warp): 1000 independent runs, 198 against 165 us;
// 100 Stein particles, 34.4 against 40.5 us, and the warp kept ahead at every
// size tried up to 1000 particles x 300 minibatch entries.  Converged
// independent runs give every query a small, even amount of work that 16
// lanes cover in one round; the Stein particles' spread gives more rows and
// candidates per query, and a half-warp then needs extra rounds.
cudaError_t launch_grad_grid(const GradArgs& a, const GridSearch* d_search, int slot, cudaStream_t s) {
    const cudaError_t e = a.mb_stride ? launch_grad_grid_g<16>(a, d_search, slot, s)
                                      : launch_grad_grid_g<32>(a, d_search, slot, s);
    if (e != cudaSuccess) return e;
    return launch_qterms_to_gbar(a.partial, a.K, a.m, a.inv_m, a.gbar, nullptr, s);
}

}  // namespace sicp
