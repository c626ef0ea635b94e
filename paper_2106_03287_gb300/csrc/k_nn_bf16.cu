// Exhaustive nearest-neighbour search with the distance tiles on the
// fifth-generation tensor cores (bf16 operands, fp32 accumulation in tensor
// memory) and an exact fp32 re-check of the few candidates they cannot rule
// out.  The result is the same (index, squared distance) as the fp32
// exhaustive search: the lowest-index minimiser of the fp32 squared distance.
//
// Distances.  With c the centre of the reference bounding box, q' = q - c and
// r' = r - c, the squared distance is |q'|^2 + d~(q, r) with
//   d~(q, r) = |r'|^2 - 2 q'.r'.
// |q'|^2 does not depend on r, so the nearest r minimises d~.  Each fp32
// coordinate is split into two bf16 parts, x = x_h + x_l + O(2^-16 |x|); the
// product q'.r' is taken as q_h.r_h + q_l.r_h + q_h.r_l (the dropped q_l.r_l
// is O(2^-16)).  The 9 products and the two bf16 parts of |r'|^2 fill 11 of
// the 16 K slots of one MMA, so one M = 128 x N = 256 x K = 16 MMA gives, for
// 128 queries and 256 reference points, v ~ d~(q, r) with
//   |v - d~(q, r)| <= E(q, t) = a |q'| N_t + b N_t^2 + e |q'|^2,
// N_t the largest |r'| of reference tile t.  E bounds, with a factor of two to
// spare, every rounding between the bf16 products and the exact fp32 squared
// distance that the fp32 search compares: the splits (2^-16 per product), the
// fp32 accumulation, and the fp32 evaluation of |q - r|^2.
//
// Search (one sweep).  Per query, u = the smallest upper bound v + E seen so
// far bounds the minimum of d~ from above at every moment, so a point whose
// lower bound v - E exceeds the current u cannot be the fp32 minimiser (nor
// tie with it); every other point is a candidate and gets its exact fp32
// squared distance; the best candidate under the (distance, index) order is
// the answer.  Per element of a tile the work is one min; the candidates
// (points within a few bound widths of the best so far) are rare once u has
// come down.
//
// Tiles that cannot hold an answer are skipped.  Before its sweep a query tile
// takes, for every query, the fp32 squared distance U_q to the seed point of
// its grid cell (a reference point near the cell centre): the query's answer
// is at most that far.  A reference tile whose bounding box lies farther from
// the query tile's bounding box than max_q U_q, with margins for fp32
// rounding, holds no point that can be the answer or tie with it, and is
// left out of the sweep with its MMA and its accumulator readback.  The kept
// tiles (all of them when R exceeds the list's capacity) are swept in the
// same order as before.
//
// Pipeline per CTA (one 128-query tile at a time, persistent over tiles, one
// CTA per SM, query tiles taken from a counter; the queries in key order and the reference points
// in brick order, both described below; the sweep starts at the reference tile holding the
// grid cell of the tile's first query and wraps around): the 16 warps copy each reference tile (8 KB, precomputed per
// reference cloud) and its 256
// fp32 points into a shared-memory ring with asynchronous 16-byte copies,
// three tiles ahead; thread 0 issues a landed tile's MMA into one of two
// 256-column tensor-memory buffers while the warps read the other (four warps
// per 32 rows, one per column quarter).  The only wait, on MMA completion, is
// bounded.
#include <cuda_bf16.h>
#include <float.h>

#include "common.cuh"
#include "grid_search.cuh"
#include "tc.cuh"

namespace sicp {
namespace {

using gs::cell_coord;

constexpr int kQRows = 128;
constexpr int kRCols = 256;
constexpr int kKDim = 16;
constexpr int kTileBytes = kRCols * kKDim * 2;        // one reference tile
constexpr int kSlotBytes = kTileBytes + kRCols * 16;  // a tile and its 256 fp32 points
constexpr int kSlots = 5;                             // tile t in slot t % kSlots
constexpr int kAhead = 3;                             // tiles whose copies are in flight ahead of the MMA
constexpr int kWarps = 16;                            // 4 row groups x 4 column quarters
constexpr int kQuarter = kRCols / 4;
constexpr int kBfThreads = kWarps * 32;
constexpr long long kPolls = 1ll << 24;
// error-bound coefficients (see the header comment): a, b, e
constexpr float kEpsQR = 2.2e-4f, kEpsRR = 3.6e-5f, kEpsQQ = 1.2e-6f;
constexpr float kPadW = 1e30f;                        // |r'|^2 of the padding columns of the last tile
constexpr unsigned kNoIdx = 0x7fffffffu;

constexpr int sA = 0;                                 // 128 x 16 bf16, K-major
constexpr int sRing = sA + kQRows * kKDim * 2;        // kSlots x kSlotBytes
constexpr int sQ = sRing + kSlots * kSlotBytes;       // float4 per row
constexpr int sXD = sQ + kQRows * 16;                 // quarters 1..3: best distance, index, point
constexpr int sXI = sXD + 3 * kQRows * 4;
constexpr int sXP = sXI + 3 * kQRows * 4;
constexpr int kMaxList = 8192;                        // reference tiles a sweep list holds (2M points)
constexpr int sList = sXP + 3 * kQRows * 16;          // uint16 [kMaxList]: the kept tiles in sweep order
constexpr int kBfSmemUsed = sList + kMaxList * 2;
constexpr float kBoxRel = 1e-6f;                      // box gaps shrink by this x the coordinate magnitudes
constexpr float kSkipRel = 1e-5f;                     // a tile is skipped only if its bound beats U by this
constexpr int kBrick = 8;                             // fine cells per brick edge (reference order)
constexpr int kQCell = 4;                             // fine cells per query-key cell edge
constexpr int kOrderMinTiles = 32;                    // queries put in key order from this many reference tiles
// Launched with more shared memory than it uses so that no two CTAs share an
// SM: each holds all 512 tensor-memory columns for its whole life.
constexpr int kBfSmem = 120 * 1024;
static_assert(kBfSmemUsed <= kBfSmem, "layout exceeds the launch size");
static_assert(kTileBytes == 16 * kBfThreads && kRCols <= kBfThreads, "one 16-byte copy per thread and tile");

__device__ __forceinline__ void split_bf16(float x, __nv_bfloat16& h, __nv_bfloat16& l) {
    h = __float2bfloat16_rn(x);
    l = __float2bfloat16_rn(x - __bfloat162float(h));
}

__device__ __forceinline__ void store_row16(unsigned char* tile, int row, const __nv_bfloat16 v[16]) {
    uint4 lo, hi;
    const uint32_t* p = reinterpret_cast<const uint32_t*>(v);
    lo.x = p[0]; lo.y = p[1]; lo.z = p[2]; lo.w = p[3];
    hi.x = p[4]; hi.y = p[5]; hi.z = p[6]; hi.w = p[7];
    *reinterpret_cast<uint4*>(tile + tc::kmajor_offset(row, 0, kKDim)) = lo;
    *reinterpret_cast<uint4*>(tile + tc::kmajor_offset(row, 8, kKDim)) = hi;
}

// The B operand of every reference tile (tile t at out + t * kTileBytes) from
// the points in brick order, and N_t = the largest |r'| of each tile (nmax,
// zeroed beforehand; non-negative floats order like their bit patterns).
__global__ void k_bf16_btiles(const float4* __restrict__ sorted, int M, float3 c, int R,
                              unsigned char* __restrict__ out, unsigned* __restrict__ nmax) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)R * kRCols) return;
    const int tile = (int)(i / kRCols), row = (int)(i % kRCols);
    __nv_bfloat16 v[16];
    const __nv_bfloat16 z = __float2bfloat16_rn(0.f);
    for (int k = 0; k < 16; ++k) v[k] = z;
    if (i < M) {
        const float4 r = sorted[i];
        const float p[3] = {r.x - c.x, r.y - c.y, r.z - c.z};
        const float n2 = fmaf(p[0], p[0], fmaf(p[1], p[1], p[2] * p[2]));
        for (int a = 0; a < 3; ++a) {
            __nv_bfloat16 h, l;
            split_bf16(p[a], h, l);
            v[a] = h;
            v[3 + a] = h;
            v[6 + a] = l;
        }
        split_bf16(n2, v[9], v[10]);
        atomicMax(nmax + tile, __float_as_uint(sqrtf(n2)));
    } else {
        v[9] = __float2bfloat16_rn(kPadW);
    }
    store_row16(out + (size_t)tile * kTileBytes, row, v);
}

// Bounding box of each reference tile's points (tbox[2 t] = lo, tbox[2 t + 1] =
// hi) and the largest coordinate magnitude of the cloud (amax, zeroed
// beforehand); one warp per tile.
__global__ void k_bf16_tbox(const float4* __restrict__ sorted, int M, int R, float4* __restrict__ tbox,
                            unsigned* __restrict__ amax) {
    const int warp = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
    if (warp >= R) return;
    float lo[3] = {FLT_MAX, FLT_MAX, FLT_MAX}, hi[3] = {-FLT_MAX, -FLT_MAX, -FLT_MAX};
    for (int k = lane; k < kRCols; k += 32) {
        const int64_t i = (int64_t)warp * kRCols + k;
        if (i < M) {
            const float4 r = sorted[i];
            lo[0] = fminf(lo[0], r.x); lo[1] = fminf(lo[1], r.y); lo[2] = fminf(lo[2], r.z);
            hi[0] = fmaxf(hi[0], r.x); hi[1] = fmaxf(hi[1], r.y); hi[2] = fmaxf(hi[2], r.z);
        }
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        for (int off = 16; off > 0; off >>= 1) {
            lo[a] = fminf(lo[a], __shfl_xor_sync(0xffffffffu, lo[a], off));
            hi[a] = fmaxf(hi[a], __shfl_xor_sync(0xffffffffu, hi[a], off));
        }
    }
    if (lane == 0) {
        tbox[2 * warp] = make_float4(lo[0], lo[1], lo[2], 0.f);
        tbox[2 * warp + 1] = make_float4(hi[0], hi[1], hi[2], 0.f);
        const float m = fmaxf(fmaxf(fmaxf(fabsf(lo[0]), fabsf(lo[1])), fmaxf(fabsf(lo[2]), fabsf(hi[0]))),
                              fmaxf(fabsf(hi[1]), fabsf(hi[2])));
        atomicMax(amax, __float_as_uint(m));
    }
}

// What the search reads of the current reference, kept in device memory and
// rewritten by every tile build (bf16_prepare), so a captured graph of the
// search stays valid when the reference changes.
struct BfRef {
    float3 c;                  // centre of the bounding box, subtracted before the split
    int M, R;                  // points, tiles of 256
    const unsigned char* btiles;
    const float* nmax;         // [R]
    GridView grid;             // the fine grid: its seed map and the cells of the queries
    const float4* tbox;        // [R][2]: each tile's bounding box (lo, hi)
    const float* amax;         // largest coordinate magnitude of the cloud
    // brick order: the fine cells in bricks of kBrick^3 (bricks x fastest, then the cells of a brick
    // x fastest); the reference tiles hold the points in this order
    const float4* bsorted;     // [M] the points in brick order (w = original index)
    const int32_t* bbase;      // [bricks + 1] first position of each brick in bsorted
    const int32_t* loc_off;    // [cells] position of each cell's first point within its brick
    int3 nb;                   // bricks per axis
    // query keys: cells of kQCell^3 fine cells in bricks of 2^3, ordered like the reference
    int3 qd, qnb;              // key cells and key bricks per axis
    int nqkeys;
    int32_t* qcnt;             // [nqkeys] queries per key (zero between launches)
    int32_t* qstart;           // [nqkeys] first position of each key in key order
    // query-tile scheduling of a launch: next tile, CTAs done (zero between launches: written as
    // zeros with the description, and the last CTA of every launch zeroes them again)
    unsigned long long sched[2];
};

struct BfArgs {
    const BfRef* ref;          // the reference description (device memory); fills the fields below
    int grad;                  // 0: queries given; 1: queries R_j s_k + u_j of a registration iteration
    const float* q;            // grad = 0: [n][3]
    int64_t n;
    const float4* src;         // grad = 1
    int64_t n_src;             // its points (bounds checks)
    const int32_t* mb;
    int m;
    const float* theta;
    int K;
    float3 c;
    const unsigned char* btiles;
    const float* nmax;         // [R]
    const float4* sorted;      // the points in brick order (the tiles' fp32 points)
    GridView grid;             // the fine grid: its seed map and the cells of the queries
    const float4* tbox;
    float amax;
    int M, R;
    int32_t* out_idx;          // grad = 0: [n]; grad = 1: [K][m] or null
    float* out_d2;             // grad = 0
    float* qterms;             // grad = 1: [K][m][6]
    int* err;
    const float4* normals;     // grad = 1, point-to-plane: unit normals by original index; null: point-to-point
    int64_t mb_stride;         // grad = 1: minibatch entries between particles' rows (0: one shared row)
    unsigned long long* stats; // work counters or null: [8] query tiles, [9] reference tiles swept
    long long polls;           // polls of an mbarrier wait before it gives up (0: kPolls)
    int never;                 // failure-detection check: first wait on an mbarrier nothing arrives on
    // the launch's queries in key order: qtmp / qkr by query index (the query; its key and its
    // rank among the queries of that key), qs by position in key order (w = query index); qs null:
    // the queries in their own order, computed by the search
    float4* qtmp;
    int2* qkr;
    float4* qs;
};

// Wait for phase `parity` of the mbarrier; false (and the error flag set)
// after `polls` polls (0: kPolls).
__device__ __forceinline__ bool bwait(uint64_t* mb, uint32_t parity, int* err, long long polls) {
    if (tc::mbar_wait(mb, parity, polls > 0 ? polls : kPolls)) return true;
    atomicOr(err, 1);
    return false;
}

__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(tc::smem_u32(dst)), "l"(src) : "memory");
}

__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// 16 columns of the thread's TMEM lane and their minimum, reduced by the load
// itself (tcgen05.ld.red, .min over the loaded elements: sm_103a).  Like the
// values, the minimum is valid after tmem_wait_ld().
__device__ __forceinline__ void tmem_ld16_min(uint32_t taddr, float r[16], float& mn) {
    asm volatile(
        "tcgen05.ld.red.sync.aligned.32x32b.x16.min.f32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, "
        "%16, [%17];"
        : "=f"(r[0]), "=f"(r[1]), "=f"(r[2]), "=f"(r[3]), "=f"(r[4]), "=f"(r[5]), "=f"(r[6]), "=f"(r[7]),
          "=f"(r[8]), "=f"(r[9]), "=f"(r[10]), "=f"(r[11]), "=f"(r[12]), "=f"(r[13]), "=f"(r[14]), "=f"(r[15]),
          "=f"(mn)
        : "r"(taddr)
        : "memory");
}

// min(a, b, c) in one instruction (three-input min.f32 of sm_100 and later).
__device__ __forceinline__ float min3f(float a, float b, float c) {
    float r;
    asm("min.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
    return r;
}

// Reference tile swept at step t (all R tiles, from `rot` on).
__device__ __forceinline__ int ref_tile(int t, int R, int rot) {
    const int r = t + rot;
    return r >= R ? r - R : r;
}

__device__ __forceinline__ bool better_u(float d, unsigned i, float bd, unsigned bi) {
    return d < bd || (d == bd && i < bi);
}

// ---------------------------------------------------------------- brick order
// The reference tiles take the points in brick order: the fine grid's cells
// grouped in bricks of kBrick^3 cells, bricks x fastest, then the cells of a
// brick x fastest, each cell's points in the grid's order.  256 consecutive
// points then fill a compact region, so a query tile's sweep reaches fewer
// reference tiles than in the grid's row order.  The queries of a launch are
// ordered the same way at a coarser key (bricks of 2^3 key cells of kQCell^3
// fine cells), so a query tile is compact too.  Neither order changes any
// result: the answer is the lowest-index minimiser whatever the tiles hold.

__device__ __forceinline__ int brick_of(int x, int y, int z, int3 nb) {
    return ((z / kBrick) * nb.y + y / kBrick) * nb.x + x / kBrick;
}

// One CTA of kBrick^3 threads per brick: each cell's offset within its brick
// (exclusive sum of the point counts of the brick's cells before it) and the
// brick's point count.
__global__ void __launch_bounds__(kBrick* kBrick* kBrick) k_bf16_brick_local(GridView g, int3 nb,
                                                                              int32_t* __restrict__ loc_off,
                                                                              int32_t* __restrict__ bsum) {
    constexpr int kN = kBrick * kBrick * kBrick;
    __shared__ int wsum[kN / 32];
    const int b = blockIdx.x, l = threadIdx.x, lane = l & 31, w = l >> 5;
    const int x = (b % nb.x) * kBrick + l % kBrick;
    const int y = (b / nb.x % nb.y) * kBrick + l / kBrick % kBrick;
    const int z = (b / nb.x / nb.y) * kBrick + l / (kBrick * kBrick);
    const bool in = x < g.dims.x && y < g.dims.y && z < g.dims.z;
    const int64_t c = in ? ((int64_t)z * g.dims.y + y) * g.dims.x + x : 0;
    const int cnt = in ? g.cell_start[c + 1] - g.cell_start[c] : 0;
    int incl = cnt;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const int v = __shfl_up_sync(0xffffffffu, incl, off);
        if (lane >= off) incl += v;
    }
    if (lane == 31) wsum[w] = incl;
    __syncthreads();
    int base = 0;
    for (int k = 0; k < w; ++k) base += wsum[k];
    if (in) loc_off[c] = base + incl - cnt;
    if (l == kN - 1) bsum[b] = base + incl;
}

// Each point of the grid's order to its place in brick order.
__global__ void k_bf16_brick_scatter(GridView g, const int32_t* __restrict__ cell_of, int3 nb,
                                     const int32_t* __restrict__ bbase, const int32_t* __restrict__ loc_off, int M,
                                     float4* __restrict__ bsorted) {
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < M; p += (int64_t)gridDim.x * blockDim.x) {
        const float4 r = g.sorted[p];
        const int c = cell_of[SICP_IDX(__float_as_int(r.w), M, kChkRef)];
        const int x = c % g.dims.x, y = c / g.dims.x % g.dims.y, z = c / g.dims.x / g.dims.y;
        const int64_t pos = (int64_t)bbase[brick_of(x, y, z, nb)] + loc_off[c] + (p - g.cell_start[c]);
        if (pos >= 0 && pos < M) bsorted[SICP_IDX(pos, M, kChkSorted)] = r;
    }
}

// Query g of a launch: R_j s_k + u_j for (k, j) = (g / K, g % K) in a
// registration iteration, else the given point.
__device__ __forceinline__ float3 bf_query(const BfArgs& a, int64_t g) {
    if (a.grad) {
        const int k = (int)(g / a.K), j = (int)(g % a.K);
        Pose P;
        make_pose(a.theta + 6 * j, P);
        const float4 s4 = __ldg(a.src + SICP_IDX(__ldg(a.mb + (int64_t)j * a.mb_stride + k), a.n_src, kChkSrc));
        return apply_pose(P, make_float3(s4.x, s4.y, s4.z));
    }
    return make_float3(a.q[3 * g], a.q[3 * g + 1], a.q[3 * g + 2]);
}

__device__ __forceinline__ int query_key(const GridView& g, int3 qnb, float3 q) {
    const int x = cell_coord(q.x, g.origin.x, g.inv_cell, g.dims.x) / kQCell;
    const int y = cell_coord(q.y, g.origin.y, g.inv_cell, g.dims.y) / kQCell;
    const int z = cell_coord(q.z, g.origin.z, g.inv_cell, g.dims.z) / kQCell;
    return (((z >> 1) * qnb.y + (y >> 1)) * qnb.x + (x >> 1)) * 8 + (z & 1) * 4 + (y & 1) * 2 + (x & 1);
}

// The launch's queries, their keys, and their ranks among the queries of a key.
__global__ void __launch_bounds__(256) k_bf16_qkey(BfArgs a, int64_t Q) {
    const BfRef* r = a.ref;
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= Q) return;
    const float3 q = bf_query(a, g);
    const int key = query_key(r->grid, r->qnb, q);
    a.qtmp[g] = make_float4(q.x, q.y, q.z, 0.f);
    a.qkr[g] = make_int2(key, atomicAdd(r->qcnt + key, 1));
}

// One CTA: qstart = exclusive sums of qcnt, and qcnt back to zero.
__global__ void __launch_bounds__(1024) k_bf16_qscan(const BfRef* __restrict__ r) {
    __shared__ int wsum[32];
    const int n = r->nqkeys, t = threadIdx.x, lane = t & 31, w = t >> 5;
    const int per = (n + 1023) / 1024;
    const int b = min(n, t * per), e = min(n, b + per);
    int32_t* cnt = r->qcnt;
    int s = 0;
    for (int i = b; i < e; ++i) s += cnt[i];
    int incl = s;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const int v = __shfl_up_sync(0xffffffffu, incl, off);
        if (lane >= off) incl += v;
    }
    if (lane == 31) wsum[w] = incl;
    __syncthreads();
    int run = incl - s;
    for (int k = 0; k < w; ++k) run += wsum[k];
    for (int i = b; i < e; ++i) {
        const int c = cnt[i];
        r->qstart[i] = run;
        run += c;
        cnt[i] = 0;
    }
}

// Query g to its position in key order (qs[pos].w = g).
__global__ void __launch_bounds__(256) k_bf16_qscatter(BfArgs a, int64_t Q) {
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= Q) return;
    const int2 kr = a.qkr[g];
    const int64_t pos = (int64_t)a.ref->qstart[kr.x] + kr.y;
    const float4 q = a.qtmp[g];
    // (always in range: the counts start at zero and each query took one rank of its key)
    if (pos >= 0 && pos < Q) a.qs[SICP_IDX(pos, Q, kChkSorted)] = make_float4(q.x, q.y, q.z, __int_as_float((int)g));
}

__global__ void __launch_bounds__(kBfThreads, 1) k_nn_bf16(BfArgs args) {
    pdl_wait();      // the particles of the previous Stein step (and the reference description)
    pdl_trigger();   // only after the wait: see pdl_wait
    BfArgs a = args;
    {
        const BfRef* r = args.ref;
        a.c = r->c;
        a.M = r->M;
        a.R = r->R;
        a.btiles = r->btiles;
        a.nmax = r->nmax;
        a.grid = r->grid;
        a.sorted = r->bsorted;
        a.tbox = r->tbox;
        a.amax = *r->amax;
    }
    extern __shared__ __align__(1024) unsigned char sm[];
    __shared__ uint64_t tfull[2], tnever;
    __shared__ uint32_t tbase;
    __shared__ int s_fail, s_rot, s_T;
    __shared__ long long s_tile;
    __shared__ float s_red[4][8];
    __shared__ int s_cnt[kWarps];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, tid = threadIdx.x;
    const int64_t Q = a.grad ? (int64_t)a.K * a.m : a.n;
    const int64_t ntiles = (Q + kQRows - 1) / kQRows;
    float4* qrow = reinterpret_cast<float4*>(sm + sQ);
    uint16_t* list = reinterpret_cast<uint16_t*>(sm + sList);
    const bool use_list = a.R <= kMaxList;
    float* xd = reinterpret_cast<float*>(sm + sXD);
    unsigned* xi = reinterpret_cast<unsigned*>(sm + sXI);
    float4* xp = reinterpret_cast<float4*>(sm + sXP);

    if (warp == 0) tc::tmem_alloc(&tbase, 512);
    if (tid == 0) {
        tc::mbar_init(&tfull[0], 1);
        tc::mbar_init(&tfull[1], 1);
        tc::mbar_init(&tnever, 1);
        s_fail = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    // Failure-detection check: a wait on an mbarrier that nothing arrives on, before any copy or
    // MMA is issued.  It gives up after a.polls polls, sets the error flag, and the CTA then skips
    // all work (nothing in flight), frees its tensor memory and returns.
    if (a.never) {
        if (tid == 0 && !bwait(&tnever, 0u, a.err, a.polls)) s_fail = 1;
        __syncthreads();
    }
    const bool skip = s_fail != 0;
    const uint32_t tmem = tbase;
    const uint32_t idesc = tc::idesc_bf16(kQRows, kRCols);
    const uint64_t adesc = tc::smem_desc(tc::smem_u32(sm + sA), 128, kKDim * 16, false);
    int rot = 0, T = a.R;
    const int qtr = warp >> 2, rq = warp & 3, row = 32 * rq + lane;
    int64_t N0 = 0;   // MMAs issued by this CTA before the current query tile
    // reference tile swept at step t of the current query tile
    auto tile_at = [&](int t) -> int { return use_list ? (int)list[t] : ref_tile(t, a.R, rot); };

    // asynchronous copy (no registers) of this thread's 16 bytes of tile t
    // and of its points; one commit group per tile
    auto fetch = [&](int t) {
        if (t < T) {
            const int rt = tile_at(t);
            unsigned char* slot = sm + sRing + (t % kSlots) * kSlotBytes;
            cp_async16(slot + 16 * tid, a.btiles + (size_t)rt * kTileBytes + 16 * tid);
            if (tid < kRCols && rt * kRCols + tid < a.M)
                cp_async16(slot + kTileBytes + 16 * tid, a.sorted + (size_t)rt * kRCols + tid);
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
    };
    // publish tile t's slot and, from thread 0, issue its MMA.  With wait_prev, thread 0 first waits
    // for the MMA of tile t - 1, so that after the barrier every warp may read its accumulators.
    auto issue_mma = [&](int t, bool wait_prev) {
        tc::fence_async_shared();
        if (wait_prev && tid == 0 && !s_fail) {
            const int64_t Np = N0 + t - 1;
            if (!bwait(&tfull[Np & 1], (uint32_t)((Np >> 1) & 1), a.err, a.polls)) s_fail = 1;
        }
        tc::fence_before_sync();
        __syncthreads();
        tc::fence_after_sync();
        if (tid == 0 && !s_fail) {
            const int64_t N = N0 + t;
            const uint64_t bdesc =
                tc::smem_desc(tc::smem_u32(sm + sRing + (t % kSlots) * kSlotBytes), 128, kKDim * 16, false);
            tc::mma_bf16(tmem + (uint32_t)((N & 1) * kRCols), adesc, bdesc, idesc, false);
            tc::mma_commit(&tfull[N & 1]);
        }
    };

    // query tiles are taken from a counter, so that CTAs that drew cheap tiles (few reference tiles
    // within reach) take more of them; with no more tiles than CTAs, CTA b takes tile b alone
    unsigned long long* sched = const_cast<unsigned long long*>(args.ref->sched);
    const bool dyn = ntiles > (int64_t)gridDim.x;
    if (tid == 0) s_tile = skip ? ntiles : dyn ? (long long)atomicAdd(sched, 1ull) : (long long)blockIdx.x;
    __syncthreads();
    int64_t g_row = Q;   // query index of row tid (tid < kQRows) of the current query tile
    for (int64_t tile = s_tile; tile < ntiles && !skip; tile = s_tile) {
        // ---- A operand and the fp32 queries of this tile: the rows in key order, each with its
        // query index g (padding rows: g = Q), kept by the thread that writes the row's result
        if (tid < kQRows) {
            const int64_t gp = tile * kQRows + tid;
            float3 q = make_float3(0.f, 0.f, 0.f);
            int64_t g = Q;
            if (gp < Q) {
                if (a.qs) {
                    const float4 e = a.qs[gp];
                    q = make_float3(e.x, e.y, e.z);
                    g = __float_as_int(e.w);
                    if (g < 0 || g >= Q) g = Q;
                } else {   // a small reference: the queries in their own order
                    q = bf_query(a, gp);
                    g = gp;
                }
            }
            g_row = g;
            const float p[3] = {q.x - a.c.x, q.y - a.c.y, q.z - a.c.z};
            const float n2 = fmaf(p[0], p[0], fmaf(p[1], p[1], p[2] * p[2]));
            qrow[tid] = make_float4(q.x, q.y, q.z, sqrtf(n2));
            if (use_list) {
                // U_q: the fp32 squared distance to the seed point of the query's grid cell (an
                // actual reference point, so the answer is at most that far); the query tile's
                // box; padding rows (g >= Q) take no part
                const GridView& G = a.grid;
                float U = g < Q ? FLT_MAX : 0.f;
                if (g < Q && G.seed4) {
                    const int cx = cell_coord(q.x, G.origin.x, G.inv_cell, G.dims.x);
                    const int cy = cell_coord(q.y, G.origin.y, G.inv_cell, G.dims.y);
                    const int cz = cell_coord(q.z, G.origin.z, G.inv_cell, G.dims.z);
                    const float4 sp = __ldg(G.seed4 + ((int64_t)cz * G.dims.y + cy) * G.dims.x + cx);
                    if (__float_as_int(sp.w) >= 0) U = dist2(sp, q);
                }
                float v[8] = {U, g < Q ? -q.x : -FLT_MAX, g < Q ? -q.y : -FLT_MAX, g < Q ? -q.z : -FLT_MAX,
                              g < Q ? q.x : -FLT_MAX, g < Q ? q.y : -FLT_MAX, g < Q ? q.z : -FLT_MAX,
                              g < Q ? fmaxf(fmaxf(fabsf(q.x), fabsf(q.y)), fabsf(q.z)) : 0.f};
#pragma unroll
                for (int k = 0; k < 8; ++k)
                    for (int off = 16; off > 0; off >>= 1) v[k] = fmaxf(v[k], __shfl_xor_sync(0xffffffffu, v[k], off));
                if (lane == 0)
                    for (int k = 0; k < 8; ++k) s_red[warp][k] = v[k];
            }
            __nv_bfloat16 v[16];
            const __nv_bfloat16 z = __float2bfloat16_rn(0.f);
            for (int k = 0; k < 16; ++k) v[k] = z;
            for (int d = 0; d < 3; ++d) {
                __nv_bfloat16 h, l;
                split_bf16(-2.f * p[d], h, l);     // exact scaling by -2
                v[d] = h;
                v[3 + d] = l;
                v[6 + d] = h;
            }
            v[9] = v[10] = __float2bfloat16_rn(1.f);
            store_row16(sm + sA, tid, v);
            if (tid == 0) {
                // the sweep starts at the reference tile that holds the grid cell of the
                // tile's first query (the points around it come early and bring u down)
                const GridView& G = a.grid;
                const int cx = cell_coord(q.x, G.origin.x, G.inv_cell, G.dims.x);
                const int cy = cell_coord(q.y, G.origin.y, G.inv_cell, G.dims.y);
                const int cz = cell_coord(q.z, G.origin.z, G.inv_cell, G.dims.z);
                const BfRef* r = args.ref;
                const int32_t start = __ldg(r->bbase + brick_of(cx, cy, cz, r->nb)) +
                                      __ldg(r->loc_off + ((int64_t)cz * G.dims.y + cy) * G.dims.x + cx);
                s_rot = max(0, min(start / kRCols, a.R - 1));
            }
        }
        __syncthreads();
        rot = s_rot;
        if (use_list) {
            // the query tile's bound and box (max over the four row warps)
            float v[8];
#pragma unroll
            for (int k = 0; k < 8; ++k) v[k] = fmaxf(fmaxf(s_red[0][k], s_red[1][k]), fmaxf(s_red[2][k], s_red[3][k]));
            const float U = v[0];
            const float qlo[3] = {-v[1], -v[2], -v[3]}, qhi[3] = {v[4], v[5], v[6]};
            const float tol = kBoxRel * (v[7] + a.amax);   // covers the fp32 rounding of the box gaps
            // this thread's run of tiles in sweep order: keep those whose box can hold an answer
            const int per = (a.R + kBfThreads - 1) / kBfThreads;
            const int t0 = min(a.R, tid * per), t1 = min(a.R, t0 + per);
            uint32_t keep = 0;   // per <= kMaxList / kBfThreads = 16 tiles
            int cnt = 0;
            for (int t = t0; t < t1; ++t) {
                const int rt = ref_tile(t, a.R, rot);
                const float4 lo = __ldg(a.tbox + 2 * rt), hi = __ldg(a.tbox + 2 * rt + 1);
                const float gx = fmaxf(fmaxf(lo.x - qhi[0], qlo[0] - hi.x) - tol, 0.f);
                const float gy = fmaxf(fmaxf(lo.y - qhi[1], qlo[1] - hi.y) - tol, 0.f);
                const float gz = fmaxf(fmaxf(lo.z - qhi[2], qlo[2] - hi.z) - tol, 0.f);
                const float lb2 = fmaf(gx, gx, fmaf(gy, gy, gz * gz));
                if (!(lb2 * (1.f - kSkipRel) > U)) {
                    keep |= 1u << (t - t0);
                    ++cnt;
                }
            }
            // exclusive prefix of the counts over the CTA, then the kept tiles in order
            int incl = cnt;
#pragma unroll
            for (int off = 1; off < 32; off <<= 1) {
                const int x = __shfl_up_sync(0xffffffffu, incl, off);
                if (lane >= off) incl += x;
            }
            if (lane == 31) s_cnt[warp] = incl;
            __syncthreads();
            int base = incl - cnt;
            for (int w = 0; w < warp; ++w) base += s_cnt[w];
            for (int t = t0; t < t1; ++t)
                if (keep >> (t - t0) & 1u) list[base++] = (uint16_t)ref_tile(t, a.R, rot);
            if (tid == kBfThreads - 1) s_T = base;
            __syncthreads();
            if (s_T == 0) {   // (not reached: the tile of row 0's seed point is always kept)
                if (tid == 0) {
                    list[0] = (uint16_t)rot;
                    s_T = 1;
                }
                __syncthreads();
            }
            T = s_T;
        }
        if (tid == 0 && a.stats) {
            atomicAdd(a.stats + 8, 1ull);
            atomicAdd(a.stats + 9, (unsigned long long)T);
        }
        // ---- prologue: tiles 0 .. kAhead in flight, tile 0 landed and its MMA issued
        for (int t = 0; t <= kAhead; ++t) fetch(t);
        asm volatile("cp.async.wait_group %0;" ::"n"(kAhead) : "memory");
        issue_mma(0, false);
        const float4 q4 = qrow[row];
        const float3 q = make_float3(q4.x, q4.y, q4.z);
        const float qn = q4.w;
        // the per-row part of the bound: E = aq N + b N^2 + eq
        const float aq = kEpsQR * qn, eq = kEpsQQ * qn * qn;
        float u = FLT_MAX, bd = FLT_MAX;
        unsigned bi = kNoIdx;
        float4 bp = make_float4(0.f, 0.f, 0.f, 0.f);

        // the radius N_t of the next tile is loaded one step ahead, so that its
        // round trip overlaps the barrier and the MMA wait of the current step
        float nt_next = T > 0 ? __ldg(a.nmax + tile_at(0)) : 0.f;
        for (int t = 0; t < T; ++t) {
            const float nt = nt_next;
            if (t + 1 < T) nt_next = __ldg(a.nmax + tile_at(t + 1));
            // tile t + 1 has landed (the kAhead - 1 newer groups may still be in
            // flight); its slot is published and its MMA issued, and the MMA of
            // tile t is complete (thread 0 waited for it before the barrier)
            const bool last = t + 1 >= T;
            if (!last) {
                asm volatile("cp.async.wait_group %0;" ::"n"(kAhead - 1) : "memory");
                issue_mma(t + 1, true);
            }
            // the slot of tile t + 1 + kAhead last held tile t + 1 + kAhead - kSlots = t - 1,
            // consumed before the barrier above
            fetch(t + 1 + kAhead);

            // ---- accumulators of tile t: warp w reads rows 32 (w % 4) .. + 31, columns of quarter w / 4
            const int64_t N = N0 + t;
            const int b = (int)(N & 1);
            if (last) {   // no barrier in this step: each warp waits for the MMA itself
                int ok = 1;
                if (lane == 0) ok = s_fail ? 0 : bwait(&tfull[b], (uint32_t)((N >> 1) & 1), a.err, a.polls);
                ok = __shfl_sync(0xffffffffu, ok, 0);
                tc::fence_after_sync();
                if (!ok) {
                    if (lane == 0) s_fail = 1;
                    continue;
                }
            } else if (s_fail) {
                continue;
            }
            const uint32_t tb = tmem + (uint32_t)(b * kRCols + qtr * kQuarter) + ((uint32_t)(32 * rq) << 16);
            // the 64 values and the minimum of each run of 16, reduced by the loads
            float r[64], g[4];
            tmem_ld16_min(tb, r, g[0]);
            tmem_ld16_min(tb + 16, r + 16, g[1]);
            tmem_ld16_min(tb + 32, r + 32, g[2]);
            tmem_ld16_min(tb + 48, r + 48, g[3]);
            tmem_wait_ld();
            const int rt = tile_at(t);
            const float E = fmaf(aq, nt, fmaf(kEpsRR * nt, nt, eq));
            const float cm = min3f(g[0], g[1], fminf(g[2], g[3]));
            u = fminf(u, cm + E);
            const float thr = u + E;   // lower bound v - E <= u
            if (cm <= thr) {
                const int col0 = qtr * kQuarter;
                const int lim = a.M - rt * kRCols - col0;   // columns from lim on are padding
                const float4* pts =
                    reinterpret_cast<const float4*>(sm + sRing + (t % kSlots) * kSlotBytes + kTileBytes);
                // the lane's candidates as a bit mask first, then one exact check per
                // set bit: a warp runs as many checks as its busiest lane has
                // candidates, not one per column that any lane flags
                unsigned long long cmask = 0ull;
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    if (g[i] > thr) continue;   // no candidate in this run
#pragma unroll
                    for (int jj = 0; jj < 16; ++jj)
                        if (r[16 * i + jj] <= thr) cmask |= 1ull << (16 * i + jj);
                }
                if (lim < 64) cmask &= lim > 0 ? (1ull << lim) - 1ull : 0ull;
                while (cmask) {
                    const int j = __ffsll((long long)cmask) - 1;
                    cmask &= cmask - 1ull;
                    const float4 r4 = pts[col0 + j];
                    const float d = dist2(r4, q);
                    const unsigned id = __float_as_uint(r4.w);
                    if (better_u(d, id, bd, bi)) {
                        bd = d;
                        bi = id;
                        bp = r4;
                    }
                }
            }
        }
        asm volatile("cp.async.wait_group 0;" ::: "memory");

        // the four column quarters of each row: the best answer wins
        if (qtr > 0) {
            xd[(qtr - 1) * kQRows + row] = bd;
            xi[(qtr - 1) * kQRows + row] = bi;
            xp[(qtr - 1) * kQRows + row] = bp;
        }
        tc::fence_before_sync();
        __syncthreads();
        tc::fence_after_sync();
        if (qtr == 0) {
            for (int o = 0; o < 3; ++o) {
                if (better_u(xd[o * kQRows + row], xi[o * kQRows + row], bd, bi)) {
                    bd = xd[o * kQRows + row];
                    bi = xi[o * kQRows + row];
                    bp = xp[o * kQRows + row];
                }
            }
            const int64_t g = g_row;   // this thread set up the row (row == tid for qtr == 0)
            const bool found = !s_fail && bi != kNoIdx;
            if (g < Q) {
                if (a.grad) {
                    const int k = (int)(g / a.K), j = (int)(g % a.K);
                    const int64_t o = (int64_t)j * a.m + k;      // [K][m] layout of the outputs
                    float t6[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
                    if (found) {
                        Pose P;
                        make_pose(a.theta + 6 * j, P);
                        const float4 s4 =
                            __ldg(a.src + SICP_IDX(__ldg(a.mb + (int64_t)j * a.mb_stride + k), a.n_src, kChkSrc));
                        float3 dv = make_float3(q.x - bp.x, q.y - bp.y, q.z - bp.z);
                        if (a.normals) dv = plane_residual(__ldg(a.normals + SICP_IDX(bi, a.M, kChkRef)), dv);
                        grad_terms(P, make_float3(s4.x, s4.y, s4.z), dv, t6);
                    }
#pragma unroll
                    for (int cc = 0; cc < 6; ++cc) a.qterms[o * 6 + cc] = t6[cc];
                    if (a.out_idx) a.out_idx[o] = found ? (int32_t)bi : -1;
                } else {
                    a.out_idx[g] = found ? (int32_t)bi : -1;
                    if (a.out_d2) a.out_d2[g] = found ? bd : FLT_MAX;
                }
            }
        }
        N0 += T;
        if (tid == 0) s_tile = dyn ? (long long)atomicAdd(sched, 1ull) : ntiles;
        __syncthreads();
        if (s_fail) break;
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, 512);
    // the last CTA to leave zeroes the counters for the next launch (every CTA's last take of a
    // tile happened before its own arrival here)
    if (tid == 0 && dyn) {
        __threadfence();
        if (atomicAdd(sched + 1, 1ull) + 1ull == (unsigned long long)gridDim.x) {
            sched[0] = 0ull;
            sched[1] = 0ull;
            __threadfence();
        }
    }
}

}  // namespace

cudaError_t bf16_kernel_attrs() {
    return cudaFuncSetAttribute(k_nn_bf16, cudaFuncAttributeMaxDynamicSharedMemorySize, kBfSmem);
}

// The reference tiles of the current reference cloud (built on first use):
// R tiles of kTileBytes, then the R tile radii N_t.
int bf16_prepare(sicp_ctx* ctx) {
    if (ctx->bf16_ready) return SICP_OK;
    const int R = (int)((ctx->M + kRCols - 1) / kRCols);
    const size_t tiles_bytes = (size_t)R * kTileBytes;
    // tiles, then N_t [R], the largest coordinate magnitude, and the tile boxes [R][2] (16-byte aligned)
    const size_t box_off = (tiles_bytes + sizeof(float) * ((size_t)R + 1) + 15) / 16 * 16;
    int rc = ensure(ctx, ctx->bf16_tiles, box_off + sizeof(float4) * 2 * (size_t)R);
    if (rc) return rc;
    const float3 c = make_float3(0.5f * (ctx->ref_lo.x + ctx->ref_hi.x), 0.5f * (ctx->ref_lo.y + ctx->ref_hi.y),
                                 0.5f * (ctx->ref_lo.z + ctx->ref_hi.z));
    unsigned* nmax = (unsigned*)((char*)ctx->bf16_tiles.p + tiles_bytes);
    unsigned* amax = nmax + R;
    float4* tbox = (float4*)((char*)ctx->bf16_tiles.p + box_off);

    // brick order of the fine grid's cells, and the query keys
    const GridView& gv = ctx->grid.v;
    const int3 d = gv.dims;
    const int3 nb = make_int3((d.x + kBrick - 1) / kBrick, (d.y + kBrick - 1) / kBrick, (d.z + kBrick - 1) / kBrick);
    const int64_t nbricks = (int64_t)nb.x * nb.y * nb.z;
    const int64_t ncells = (int64_t)d.x * d.y * d.z;
    const int3 qd = make_int3((d.x + kQCell - 1) / kQCell, (d.y + kQCell - 1) / kQCell, (d.z + kQCell - 1) / kQCell);
    const int3 qnb = make_int3((qd.x + 1) / 2, (qd.y + 1) / 2, (qd.z + 1) / 2);
    const int64_t nqkeys = (int64_t)qnb.x * qnb.y * qnb.z * 8;
    // bf16_order: bsorted [M], loc_off [cells], bsum [bricks], bbase [bricks + 1], scan scratch,
    // qcnt [keys], qstart [keys] (each part 16-byte aligned)
    auto al = [](size_t b) { return (b + 15) / 16 * 16; };
    const size_t o_loc = al(sizeof(float4) * (size_t)ctx->M);
    const size_t o_bsum = o_loc + al(sizeof(int32_t) * (size_t)ncells);
    const size_t o_bbase = o_bsum + al(sizeof(int32_t) * (size_t)nbricks);
    const size_t o_sums = o_bbase + al(sizeof(int32_t) * ((size_t)nbricks + 1));
    const size_t o_qcnt = o_sums + al(sizeof(int32_t) * scan_sums_size(nbricks));
    const size_t o_qstart = o_qcnt + al(sizeof(int32_t) * (size_t)nqkeys);
    if ((rc = ensure(ctx, ctx->bf16_order, o_qstart + al(sizeof(int32_t) * (size_t)nqkeys)))) return rc;
    char* ob = (char*)ctx->bf16_order.p;
    float4* bsorted = (float4*)ob;
    int32_t* loc_off = (int32_t*)(ob + o_loc);
    int32_t* bsum = (int32_t*)(ob + o_bsum);
    int32_t* bbase = (int32_t*)(ob + o_bbase);
    int32_t* sums = (int32_t*)(ob + o_sums);
    int32_t* qcnt = (int32_t*)(ob + o_qcnt);
    int32_t* qstart = (int32_t*)(ob + o_qstart);
    SICP_CUDA(cudaMemsetAsync(qcnt, 0, sizeof(int32_t) * (size_t)nqkeys, ctx->stream));
    k_bf16_brick_local<<<(unsigned)nbricks, kBrick * kBrick * kBrick, 0, ctx->stream>>>(gv, nb, loc_off, bsum);
    SICP_CUDA(cudaGetLastError());
    SICP_CUDA(launch_exclusive_scan(bsum, nbricks, bbase, sums, ctx->stream));
    k_bf16_brick_scatter<<<(unsigned)((ctx->M + 255) / 256), 256, 0, ctx->stream>>>(
        gv, ctx->grid.cell_of, nb, bbase, loc_off, (int)ctx->M, bsorted);
    SICP_CUDA(cudaGetLastError());

    SICP_CUDA(cudaMemsetAsync(nmax, 0, sizeof(float) * ((size_t)R + 1), ctx->stream));
    const int64_t rows = (int64_t)R * kRCols;
    k_bf16_btiles<<<(unsigned)((rows + 255) / 256), 256, 0, ctx->stream>>>(
        bsorted, (int)ctx->M, c, R, (unsigned char*)ctx->bf16_tiles.p, nmax);
    SICP_CUDA(cudaGetLastError());
    k_bf16_tbox<<<(unsigned)(((int64_t)R * 32 + 255) / 256), 256, 0, ctx->stream>>>(bsorted, (int)ctx->M, R, tbox,
                                                                                  amax);
    SICP_CUDA(cudaGetLastError());
    ctx->bf16_centre = c;
    ctx->bf16_R = R;
    BfRef h;
    h.c = c;
    h.M = (int)ctx->M;
    h.R = R;
    h.btiles = (const unsigned char*)ctx->bf16_tiles.p;
    h.nmax = (const float*)nmax;
    h.grid = ctx->grid.v;
    h.tbox = tbox;
    h.amax = (const float*)amax;
    h.bsorted = bsorted;
    h.bbase = bbase;
    h.loc_off = loc_off;
    h.nb = nb;
    h.qd = qd;
    h.qnb = qnb;
    h.nqkeys = (int)nqkeys;
    h.qcnt = qcnt;
    h.qstart = qstart;
    h.sched[0] = h.sched[1] = 0ull;
    if ((rc = ensure(ctx, ctx->bf16_ref, sizeof(BfRef)))) return rc;
    SICP_CUDA(cudaMemcpyAsync(ctx->bf16_ref.p, &h, sizeof(BfRef), cudaMemcpyHostToDevice, ctx->stream));
    ctx->bf16_ready = true;
    return SICP_OK;
}

static BfArgs bf_args(sicp_ctx* ctx, int* err) {
    BfArgs a{};
    a.ref = (const BfRef*)ctx->bf16_ref.p;   // the kernel fills the reference fields from it
    a.err = err;
    a.polls = ctx->wait_polls;
    a.never = ctx->wait_never;
    a.stats = ctx->stats_on ? (unsigned long long*)ctx->stats.p : nullptr;
    return a;
}

// The Q queries of a launch: qtmp [Q] float4, qs [Q] float4, qkr [Q] int2.
int bf16_queries(sicp_ctx* ctx, int64_t Q) {
    return ensure(ctx, ctx->bf16_q, (size_t)(Q > 0 ? Q : 1) * (2 * sizeof(float4) + sizeof(int2)));
}

// Put the launch's queries in key order (three launches; the buffers come from bf16_queries).
// Below kOrderMinTiles reference tiles a query tile sweeps nearly all of them whatever its
// queries, so the search takes the queries in their own order (qs null).
static cudaError_t bf_order_queries(sicp_ctx* ctx, BfArgs& a, int64_t Q) {
    float4* base = (float4*)ctx->bf16_q.p;
    a.qtmp = base;
    a.qs = nullptr;
    a.qkr = (int2*)(base + 2 * Q);
    if (Q <= 0 || ctx->bf16_R < kOrderMinTiles) return cudaSuccess;
    a.qs = base + Q;
    const unsigned blocks = (unsigned)((Q + 255) / 256);
    k_bf16_qkey<<<blocks, 256, 0, ctx->stream>>>(a, Q);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_bf16_qscan<<<1, 1024, 0, ctx->stream>>>(a.ref);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    k_bf16_qscatter<<<blocks, 256, 0, ctx->stream>>>(a, Q);
    return cudaGetLastError();
}

static unsigned bf_grid(sicp_ctx* ctx, int64_t Q) {
    const int64_t tiles = (Q + kQRows - 1) / kQRows;
    return (unsigned)(tiles < ctx->num_sms ? tiles : ctx->num_sms);
}

cudaError_t launch_nn_bf16(sicp_ctx* ctx, const float* q, int64_t n, int32_t* idx, float* d2, int* err) {
    BfArgs a = bf_args(ctx, err);
    a.grad = 0;
    a.q = q;
    a.n = n;
    a.out_idx = idx;
    a.out_d2 = d2;
    const cudaError_t e = bf_order_queries(ctx, a, n);
    if (e != cudaSuccess) return e;
    return launch_pdl(k_nn_bf16, dim3(bf_grid(ctx, n)), dim3(kBfThreads), kBfSmem, ctx->stream, a);
}

cudaError_t launch_grad_bf16(sicp_ctx* ctx, const float4* src, const int32_t* mb, int m, const float* theta, int K,
                             float* qterms, float* gbar, int32_t* out_nn, int* err, const float4* normals,
                             int64_t mb_stride) {
    BfArgs a = bf_args(ctx, err);
    a.normals = normals;
    a.mb_stride = mb_stride;
    a.grad = 1;
    a.src = src;
    a.n_src = ctx->src_n;
    a.mb = mb;
    a.m = m;
    a.theta = theta;
    a.K = K;
    a.qterms = qterms;
    a.out_idx = out_nn;
    cudaError_t e = bf_order_queries(ctx, a, (int64_t)K * m);
    if (e != cudaSuccess) return e;
    e = launch_pdl(k_nn_bf16, dim3(bf_grid(ctx, (int64_t)K * m)), dim3(kBfThreads), kBfSmem, ctx->stream, a);
    if (e != cudaSuccess) return e;
    return launch_qterms_to_gbar(qterms, K, m, 1.f / (float)m, gbar, nullptr, ctx->stream);
}

}  // namespace sicp
