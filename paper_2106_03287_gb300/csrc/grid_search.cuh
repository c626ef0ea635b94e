// Exact grid search device code shared by the single-problem and batched
// kernels: constants, the per-query work counters, one table-driven round of
// row segments, the table walk and the full search of one query by one warp.
// See k_grid.cu for the description of the structure and the algorithm.
#pragma once

#include <float.h>
#include <math.h>

#include "common.cuh"

namespace sicp {
namespace gs {
namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;  // queries in flight per CTA, one warp each
constexpr int kGradThreads = 128;      // gradient kernel CTA: one warp per particle
constexpr int kCoarseFactor = 4;
// The far phase proves on the fine level while the bound is under this many fine
// cells, else on the coarse level (GridSearch::reach).  Measured (M particle-point
// evaluations per second): the kinect run 788 / 793 / 794 / 794 / 792 / 739 at 3 / 4 /
// 5 / 6 / 10 / 16 cells; the 256 batched problems, each reach with its own autotuned
// cell size, 767.6 at 3 against 753.1 at 6.
constexpr float kFineReach = 6.f;          // single problems
constexpr float kBatchedFineReach = 3.f;   // the persistent batched kernel
constexpr int kTableRadius = 48;
constexpr int64_t kMaxCells = 1 << 23;
constexpr float kSlack = 1.0000005f;
constexpr int kNone = 0x7fffffff;
constexpr unsigned kFull = 0xffffffffu;

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

// At least sqrt(x), for x >= 0: the hardware approximation widened by 1e-5
// relative, far above its error.  Used for a search range, where a wider
// range only adds candidates.
__device__ __forceinline__ float sqrt_up(float x) {
    float r;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r * 1.00001f;
}

// Squared pruning radius: best widened by kSlack, kept finite.
__device__ __forceinline__ float bound2(float best) { return fminf(best * kSlack, FLT_MAX); }

// Per-lane work counters: rows examined, row segments read, candidate points;
// lane 0 also counts queries, queries that reached the far phase and queries
// that reached the exhaustive scan.
struct Work {
    unsigned rows = 0, segs = 0, pts = 0, queries = 0, far = 0, exh = 0;
};

struct Best {
    float d;
    int i;
    float3 p;
};

__device__ __forceinline__ void take(Best& B, float4 r, float3 q, int id) {
    const float d = dist2(r, q);
    if (better(d, id, B.d, B.i)) {
        B.d = d;
        B.i = id;
        B.p = make_float3(r.x, r.y, r.z);
    }
}

// A query is searched by a group of G lanes (G = 32: the whole warp; G = 16:
// each half-warp runs its own query).  The group's lanes and its lane index.
template <int G>
__device__ __forceinline__ unsigned group_mask() {
    static_assert(G == 16 || G == 32, "group of 16 or 32 lanes");
    return G == 32 ? kFull : (0xffffu << (threadIdx.x & 16));
}
template <int G>
__device__ __forceinline__ int group_lane() {
    return threadIdx.x & (G - 1);
}

// Group minimum (distance, then lowest index); every lane of the group ends
// with the result.  Distances are non-negative, so their bit patterns order
// like unsigned ints.
template <int G = 32>
__device__ __forceinline__ void warp_min(Best& B) {
    const unsigned gm = group_mask<G>();
    const unsigned db = __float_as_uint(B.d);
    const unsigned md = __reduce_min_sync(gm, db);
    const unsigned mi = __reduce_min_sync(gm, db == md ? (unsigned)B.i : 0xffffffffu);
    const unsigned who = __ballot_sync(gm, db == md && (unsigned)B.i == mi) & gm;
    const int src = __ffs(who) - 1;   // a lane of this group
    B.d = __uint_as_float(md);
    B.i = (int)mi;
    B.p.x = __shfl_sync(gm, B.p.x, src);
    B.p.y = __shfl_sync(gm, B.p.y, src);
    B.p.z = __shfl_sync(gm, B.p.z, src);
}

// Every row from table entry e on is farther than the current best.
__device__ __forceinline__ bool cleared(const GridView& g, const SearchTable& tab, int e, float best) {
    const float lbd = __ldg(tab.lb + SICP_IDX(e, tab.n, kChkTable)) * g.cell - g.tol;
    return lbd > 0.f && lbd * lbd > bound2(best);
}

// One round: lane l of the group contributes row (y, z) if `has`, limited to
// cells [xlo, xhi] along x and clipped to the ball of squared radius clip2.
template <int G = 32>
__device__ void round_rows(const GridView& g, float3 q, bool has, int y, int z, int xlo, int xhi, float clip2,
                           Best& B, Work& w) {
    const int lane = group_lane<G>();
    const unsigned gm = group_mask<G>();
    int b = 0, len = 0;
    if (has && y >= 0 && y < g.dims.y && z >= 0 && z < g.dims.z) {
        const float dz = slab(q.z, g.origin.z, g.cell, z, g.tol);
        const float dy = slab(q.y, g.origin.y, g.cell, y, g.tol);
        const float rem = clip2 - dz * dz - dy * dy;
        if (rem >= 0.f) {
            w.rows += 1;
            // the row's cells within reach along x; cell_start bounds their points (empty cells add none)
            const int rowi = z * g.dims.y + y;
            const float r = sqrt_up(rem) + g.tol;
            const int x0 = max(max(cell_floor_clamped(q.x - r, g.origin.x, g.inv_cell, g.dims.x), 0), xlo);
            const int x1 = min(min(cell_floor_clamped(q.x + r, g.origin.x, g.inv_cell, g.dims.x), g.dims.x - 1), xhi);
            if (x0 <= x1) {
                const int64_t row = (int64_t)rowi * g.dims.x;
                const int64_t nc1 = (int64_t)g.dims.x * g.dims.y * g.dims.z + 1;   // (bounds checks)
                b = __ldg(g.cell_start + SICP_IDX(row + x0, nc1, kChkCellStart));
                len = __ldg(g.cell_start + SICP_IDX(row + x1 + 1, nc1, kChkCellStart)) - b;
                w.segs += len > 0;
            }
        }
    }
    // flatten the round's segments: exclusive offsets and total
    int incl = len;
#pragma unroll
    for (int off = 1; off < G; off <<= 1) {
        const int v = __shfl_up_sync(gm, incl, off, G);
        if (lane >= off) incl += v;
    }
    const int total = __shfl_sync(gm, incl, G - 1, G);
    if (total == 0) return;
    const int excl = incl - len;
    // flattened point t belongs to the last lane whose offset is <= t
    Best L = B;
    for (int t0 = 0; t0 < total; t0 += G) {
        const int t = t0 + lane;
        int o = 0;
#pragma unroll
        for (int step = G / 2; step > 0; step >>= 1) {
            const int ex = __shfl_sync(gm, excl, o + step, G);
            if (ex <= t) o += step;
        }
        const int ob = __shfl_sync(gm, b, o, G);
        const int oe = __shfl_sync(gm, excl, o, G);
        if (t < total) {
            const float4 r = __ldg(g.sorted + SICP_IDX(ob + (t - oe), g.nsorted, kChkSorted));
            take(L, r, q, __float_as_int(r.w));
        }
    }
    if (lane == 0) w.pts += (unsigned)total;
    warp_min<G>(L);
    B = L;
}

struct QueryCell {
    int cy, cz, sy, sz;
};

__device__ __forceinline__ QueryCell query_cell(const GridView& g, float3 q) {
    QueryCell c;
    c.cy = cell_coord(q.y, g.origin.y, g.inv_cell, g.dims.y);
    c.cz = cell_coord(q.z, g.origin.z, g.inv_cell, g.dims.z);
    const float fy = fminf(fmaxf((q.y - g.origin.y) * g.inv_cell - (float)c.cy, 0.f), 1.f);
    const float fz = fminf(fmaxf((q.z - g.origin.z) * g.inv_cell - (float)c.cz, 0.f), 1.f);
    c.sy = fy >= 0.5f ? 1 : -1;
    c.sz = fz >= 0.5f ? 1 : -1;
    return c;
}

// Walk table entries [0, n) with rows clipped at min(bound, cap2).  Stops at
// the first entry out of reach of the best; the answer is exact then if the
// clipping never cut below the best (best within cap2).
template <int G = 32>
__device__ bool walk(const GridView& g, const SearchTable& tab, int n, float cap2, float3 q, Best& B, Work& w) {
    const int lane = group_lane<G>();
    const QueryCell c = query_cell(g, q);
    for (int base = 0; base < n;) {
        // (entry 0 is the query's own row, bound 0: never cleared)
        if (base > 0 && cleared(g, tab, base, B.d)) return bound2(B.d) <= cap2;
        const int e = base + lane;
        const bool has = e < n;
        int y = 0, z = 0;
        if (has) {
            const short2 o = __ldg(tab.off + SICP_IDX(e, tab.n, kChkTable));
            y = c.cy + c.sy * o.x;
            z = c.cz + c.sz * o.y;
        }
        round_rows<G>(g, q, has, y, z, 0, g.dims.x - 1, fminf(bound2(B.d), cap2), B, w);
        base += G;
    }
    return false;
}

template <int G = 32>
__device__ __forceinline__ void prove(const GridSearch& S, float3 q, Best& B, Work& w);

template <int G = 32>
__device__ __forceinline__ void grid_search(const GridSearch& S, float3 q, Best& B, Work& w) {
    const int lane = group_lane<G>();
    const GridView& F = S.fine;
    B.d = FLT_MAX;
    B.i = kNone;
    B.p = make_float3(0.f, 0.f, 0.f);
    w.queries += lane == 0;
    // the seed of the query's cell is the starting answer (every lane loads it)
    const int cx = cell_coord(q.x, F.origin.x, F.inv_cell, F.dims.x);
    const int cy = cell_coord(q.y, F.origin.y, F.inv_cell, F.dims.y);
    const int cz = cell_coord(q.z, F.origin.z, F.inv_cell, F.dims.z);
    const int64_t cell = SICP_IDX(((int64_t)cz * F.dims.y + cy) * F.dims.x + cx,
                                  (int64_t)F.dims.x * F.dims.y * F.dims.z, kChkSeedCell);
    if (F.seed4) {   // the seed point itself: one load
        const float4 r = __ldg(F.seed4 + cell);
        take(B, r, q, __float_as_int(r.w));
    } else {
        const int s = __ldg(F.seed + cell);
        if (s >= 0) {
            const float4 r = __ldg(F.sorted + SICP_IDX(s, F.nsorted, kChkSeedPoint));
            take(B, r, q, __float_as_int(r.w));
        }
    }
    prove<G>(S, q, B, w);
}

// The exact nearest point of q given a starting answer B (any reference
// point, or none): walk the table with the shrinking bound on the fine level
// (bound under S.reach cells) or the coarse level, and scan everything if
// the table cannot settle it.
template <int G>
__device__ __forceinline__ void prove(const GridSearch& S, float3 q, Best& B, Work& w) {
    const int lane = group_lane<G>();
    const GridView& F = S.fine;
    const float reach = S.reach * F.cell;
    const bool fine = B.d <= reach * reach;
    w.far += (lane == 0 && !fine);
    const GridView& L = fine ? S.fine : S.coarse;
    if (walk<G>(L, S.tab, S.tab.n, FLT_MAX, q, B, w)) return;
    if (cleared(L, S.tab, S.tab.n - 1, B.d)) return;
    // the table cannot settle it: scan every point
    w.exh += lane == 0;
    Best E = B;
    for (int p = lane; p < S.M; p += G) take(E, __ldg(S.ref4 + p), q, p);
    if (lane == 0) {
        w.segs += 1;
        w.pts += (unsigned)S.M;
    }
    warp_min<G>(E);
    B = E;
}

// Warp-aggregated accumulation of the work counters: queries, rows, segments,
// points, queries that reached the far phase, queries that reached the
// exhaustive scan.
__device__ __forceinline__ void add_stats(unsigned long long* stats, const Work& w) {
    unsigned long long v[6] = {w.queries, w.rows, w.segs, w.pts, w.far, w.exh};
#pragma unroll
    for (int a = 0; a < 6; ++a) {
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) v[a] += __shfl_down_sync(kFull, v[a], off);
    }
    if ((threadIdx.x & 31) == 0) {
#pragma unroll
        for (int a = 0; a < 6; ++a) atomicAdd(stats + a, v[a]);
    }
}

}  // namespace
}  // namespace gs
}  // namespace sicp
