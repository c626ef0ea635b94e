// Internal declarations shared by the CUDA translation units of libsteinicp.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "../../include/steinicp.h"

namespace sicp {

// ---------------------------------------------------------------- bounds-checked build
// A build with -DSICP_CHECKED checks every index that comes from data (cell
// coordinates, the seed map, cell_start, the row table, minibatch entries,
// search results, fallback lists, work items) before the access:
// SICP_IDX(i, n, site) is i when 0 <= i < n; otherwise the first such failure
// of the translation unit is recorded (site and index) and counted, and index
// 0 is used instead, so the access stays inside the buffer.  In the normal
// build SICP_IDX(i, n, site) is i.  sicp_check_status reads and clears the
// records of every translation unit.
enum CheckSite : int {
    kChkSeedCell = 1,   // fine-level cell of a query (seed map)
    kChkSeedPoint,      // seed map entry -> sorted points
    kChkCellStart,      // row segment bounds -> cell_start
    kChkSorted,         // candidate -> sorted points
    kChkTable,          // row table entry
    kChkSrc,            // minibatch entry -> source points
    kChkRef,            // search result -> reference points or normals
    kChkFallback,       // fallback list entry -> queries
    kChkProblem,        // batched work item -> problem
};
using CheckReader = void (*)(unsigned long long* first, unsigned long long* count);
void check_register(CheckReader r);   // each translation unit's reader (checked build)

#ifdef SICP_CHECKED
namespace {
__device__ unsigned long long g_check_first, g_check_count;

__device__ __noinline__ int64_t check_fail(int64_t i, int site) {
    const unsigned long long code =
        (1ull << 63) | ((unsigned long long)(site & 0x7fffff) << 40) | ((unsigned long long)i & ((1ull << 40) - 1));
    atomicCAS(&g_check_first, 0ull, code);
    atomicAdd(&g_check_count, 1ull);
    return 0;
}
__device__ __forceinline__ int64_t check_idx(int64_t i, int64_t n, int site) {
    return (uint64_t)i < (uint64_t)n ? i : check_fail(i, site);
}
void check_read(unsigned long long* first, unsigned long long* count) {
    unsigned long long f = 0, c = 0;
    const unsigned long long z = 0;
    cudaMemcpyFromSymbol(&f, g_check_first, sizeof f);
    cudaMemcpyFromSymbol(&c, g_check_count, sizeof c);
    cudaMemcpyToSymbol(g_check_first, &z, sizeof z);
    cudaMemcpyToSymbol(g_check_count, &z, sizeof z);
    if (f && !*first) *first = f;
    *count += c;
}
struct CheckRegistration {
    CheckRegistration() { check_register(&check_read); }
};
CheckRegistration g_check_registration;
}  // namespace
#define SICP_IDX(i, n, site) (::sicp::check_idx((int64_t)(i), (int64_t)(n), (site)))
#else
#define SICP_IDX(i, n, site) (i)
#endif

// ---------------------------------------------------------------- device helpers

// splitmix64 (Steele, Lea, Flood 2014): output k >= 1 of the generator
// started at state s is mix(s + k * 0x9e3779b97f4a7c15).
__host__ __device__ __forceinline__ uint64_t sm64_mix(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    return z ^ (z >> 31);
}
__host__ __device__ __forceinline__ uint64_t sm64_at(uint64_t s, uint64_t k) {
    return sm64_mix(s + k * 0x9e3779b97f4a7c15ULL);
}

// Programmatic dependent launch.  A kernel launched with launch_pdl may be
// scheduled while its predecessor in the stream still runs: pdl_wait() blocks
// until the predecessor grid has completed and its writes are visible (at once
// when there is no programmatic predecessor), and pdl_trigger() lets the
// successor be scheduled once every CTA of this grid has called it or exited.
// The registration loop chains gradient -> reduction -> Stein step -> next
// gradient this way.  The gradient kernels trigger only after their own wait,
// so a Stein step is never scheduled before the previous Stein step has
// completed, which lets it read the particles before its own wait.  Only the
// reduction triggers before its wait; every other kernel triggers after it, so
// when a kernel starts, every kernel at least three launches earlier in the
// stream has completed.  The minibatch rows and the packed source points are
// written before the chain starts (and never inside it), so the grid gradient
// kernel reads them before its wait.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// Rotation R = Rz(yaw) Ry(pitch) Rx(roll) and its partials with respect to
// roll, pitch and yaw: 36 floats, R row-major then dR_roll, dR_pitch, dR_yaw.
struct Pose {
    float R[9];
    float dR[27];
    float u[3];
};

__device__ __forceinline__ void make_pose(const float* th, Pose& P) {
    float sr, cr, sp, cp, sy, cy;
    sincosf(th[3], &sr, &cr);
    sincosf(th[4], &sp, &cp);
    sincosf(th[5], &sy, &cy);
    // R = Rz Ry Rx
    P.R[0] = cy * cp; P.R[1] = cy * sp * sr - sy * cr; P.R[2] = cy * sp * cr + sy * sr;
    P.R[3] = sy * cp; P.R[4] = sy * sp * sr + cy * cr; P.R[5] = sy * sp * cr - cy * sr;
    P.R[6] = -sp;     P.R[7] = cp * sr;                P.R[8] = cp * cr;
    // d/droll: Rz Ry dRx
    P.dR[0] = 0.f; P.dR[1] = cy * sp * cr + sy * sr;  P.dR[2] = -cy * sp * sr + sy * cr;
    P.dR[3] = 0.f; P.dR[4] = sy * sp * cr - cy * sr;  P.dR[5] = -sy * sp * sr - cy * cr;
    P.dR[6] = 0.f; P.dR[7] = cp * cr;                 P.dR[8] = -cp * sr;
    // d/dpitch: Rz dRy Rx
    P.dR[9] = -cy * sp;  P.dR[10] = cy * cp * sr; P.dR[11] = cy * cp * cr;
    P.dR[12] = -sy * sp; P.dR[13] = sy * cp * sr; P.dR[14] = sy * cp * cr;
    P.dR[15] = -cp;      P.dR[16] = -sp * sr;     P.dR[17] = -sp * cr;
    // d/dyaw: dRz Ry Rx
    P.dR[18] = -sy * cp; P.dR[19] = -sy * sp * sr - cy * cr; P.dR[20] = -sy * sp * cr + cy * sr;
    P.dR[21] = cy * cp;  P.dR[22] = cy * sp * sr - sy * cr;  P.dR[23] = cy * sp * cr + sy * sr;
    P.dR[24] = 0.f;      P.dR[25] = 0.f;                     P.dR[26] = 0.f;
    P.u[0] = th[0]; P.u[1] = th[1]; P.u[2] = th[2];
}

__device__ __forceinline__ float3 apply_pose(const Pose& P, float3 s) {
    return make_float3(fmaf(P.R[0], s.x, fmaf(P.R[1], s.y, fmaf(P.R[2], s.z, P.u[0]))),
                       fmaf(P.R[3], s.x, fmaf(P.R[4], s.y, fmaf(P.R[5], s.z, P.u[1]))),
                       fmaf(P.R[6], s.x, fmaf(P.R[7], s.y, fmaf(P.R[8], s.z, P.u[2]))));
}

// Contribution of one correspondence to the gradient of L/2:
// [e ; e . (dR_a s)] with e = s' - r.
__device__ __forceinline__ void grad_terms(const Pose& P, float3 s, float3 e, float g[6]) {
    g[0] = e.x; g[1] = e.y; g[2] = e.z;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const float* D = P.dR + 9 * a;
        float jx = fmaf(D[0], s.x, fmaf(D[1], s.y, D[2] * s.z));
        float jy = fmaf(D[3], s.x, fmaf(D[4], s.y, D[5] * s.z));
        float jz = fmaf(D[6], s.x, fmaf(D[7], s.y, D[8] * s.z));
        g[3 + a] = fmaf(e.x, jx, fmaf(e.y, jy, e.z * jz));
    }
}

// Term c (0..5) of grad_terms, by the same arithmetic, for a lane of its own.
__device__ __forceinline__ float grad_term(const Pose& P, float3 s, float3 e, int c) {
    if (c < 3) return c == 0 ? e.x : (c == 1 ? e.y : e.z);
    const float* D = P.dR + 9 * (c - 3);
    const float jx = fmaf(D[0], s.x, fmaf(D[1], s.y, D[2] * s.z));
    const float jy = fmaf(D[3], s.x, fmaf(D[4], s.y, D[5] * s.z));
    const float jz = fmaf(D[6], s.x, fmaf(D[7], s.y, D[8] * s.z));
    return fmaf(e.x, jx, fmaf(e.y, jy, e.z * jz));
}

// Point-to-plane: the residual vector d = s' - r replaced by (n . d) n, n the
// unit normal at r (xyz of n4), so that grad_terms gives the gradient of
// (n . d)^2 / 2.
__device__ __forceinline__ float3 plane_residual(float4 n4, float3 d) {
    const float e = fmaf(n4.x, d.x, fmaf(n4.y, d.y, n4.z * d.z));
    return make_float3(e * n4.x, e * n4.y, e * n4.z);
}

// Exact squared distance, the comparison every search mode uses.
__device__ __forceinline__ float dist2(float4 r, float3 q) {
    float dx = r.x - q.x, dy = r.y - q.y, dz = r.z - q.z;
    return fmaf(dx, dx, fmaf(dy, dy, dz * dz));
}

// Candidate (d2, idx) is better than (bd, bi): smaller distance, ties to the lower index.
__device__ __forceinline__ bool better(float d2, int idx, float bd, int bi) {
    return d2 < bd || (d2 == bd && idx < bi);
}

// ---------------------------------------------------------------- host context

// Uniform voxel grid over the reference bounding box.  Points are stored
// sorted by linear cell id (x fastest), so every run of consecutive cells along
// x is one contiguous range of `sorted`.
struct GridView {
    float3 origin;
    float cell, inv_cell, tol;      // tol: absolute slack covering rounding of cell bounds
    int3 dims;                      // cells per axis
    const float4* sorted;           // M, w = original index bits
    const int32_t* cell_start;      // ncells + 1
    const int32_t* seed;            // ncells: position in `sorted` of a point near the cell centre (fine level)
    const float4* seed4;            // ncells: that point itself (single-problem fine level; null elsewhere)
    int32_t nsorted;                // entries of `sorted` (bounds checks)
};

struct Grid {
    GridView v{};
    int64_t ncells = 0;
    float4* sorted = nullptr;
    int32_t* cell_start = nullptr;
    int32_t* cell_of = nullptr;     // M: cell id of each reference point (build scratch)
    int32_t* counts = nullptr;      // ncells + 1 (build scratch)
    int32_t* scan_sums = nullptr;   // build scratch
    int32_t* seed = nullptr;        // ncells (fine level only)
    int32_t* seed_tmp = nullptr;    // ncells (build scratch)
    float4* seed4 = nullptr;        // ncells (fine level only)
    size_t cap_seed4 = 0;
    size_t cap_points = 0, cap_cellof = 0, cap_cells = 0, cap_counts = 0, cap_sums = 0,
           cap_seed = 0, cap_seed_tmp = 0;
};

// Row offsets (dy, dz) in cell units, in increasing order of a lower bound on
// the distance from a query (mirrored into the upper half of its cell) to the
// row; lb holds that bound, in cell units.
struct SearchTable {
    const short2* off;
    const float* lb;
    int n;
    int upto[8];   // upto[k]: number of entries with lb <= 1.5 * 2^k
};

// Everything an exact grid search reads: a fine and a coarse level over the
// same points, the row table, and the points in original order for the
// exhaustive fallback.
struct GridSearch {
    GridView fine, coarse;
    SearchTable tab;
    const float4* ref4;
    int M;
    float reach;   // fine-level reach of the far phase, in fine cells
};

bool pdl_enabled();   // false when the environment sets SICP_NO_PDL

struct Buf {
    void* p = nullptr;
    size_t cap = 0;
};

// Launch `k` with programmatic stream serialisation (see pdl_wait); plain
// stream order when SICP_NO_PDL is set.
template <typename... P, typename... A>
cudaError_t launch_pdl(void (*k)(P...), dim3 grid, dim3 block, size_t smem, cudaStream_t s, A&&... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = pdl_enabled() ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, k, static_cast<A&&>(args)...);
}

struct GraphCache;
struct BatchState;
void batch_destroy(BatchState* b);
struct Surrogate;
void surrogate_destroy(Surrogate* s);

}  // namespace sicp

struct sicp_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    std::string err;
    int num_sms = 0;

    // reference cloud
    int64_t M = 0;
    float4* ref4 = nullptr;   // original order, w = index bits
    size_t ref_cap = 0;
    sicp::Grid grid, grid2;           // fine and coarse levels
    sicp::GridSearch search{};
    short2* tab_off = nullptr;
    float* tab_lb = nullptr;
    float3 ref_lo = {0, 0, 0}, ref_hi = {0, 0, 0};

    // per-problem and scratch buffers (grow-only)
    sicp::Buf src4, mb, theta, adam_m, adam_v, partial, moments, flags, tmp_in, tmp_out, tmp_aux;
    sicp::Buf bbox, stats, gbar;
    bool stats_on = false;
    int prof_stride = 0;
    double prof[4] = {0, 0, 0, 0};   // gradient ms, gradient launches, Stein ms, Stein launches
    sicp::GraphCache* graphs = nullptr;
    sicp::BatchState* batch = nullptr;   // state of the batched path, created on first use
    sicp::Buf bf16_tiles;                // reference tiles of the tensor-core exhaustive search
    bool bf16_ready = false;             // bf16_tiles hold the current reference
    float3 bf16_centre = {0, 0, 0};
    int bf16_R = 0;                      // reference tiles of 256 points
    sicp::Buf bf16_ref;                  // device copy of what the tensor-core search reads of the reference
    sicp::Buf bf16_order;                // the reference in brick order, its offsets and the query-key counters
    sicp::Buf bf16_q;                    // a launch's queries, keyed and in key order
    sicp::Surrogate* surr = nullptr;     // learned closest-point field, created on first use
    uint64_t surr_gen = 0;               // bumped whenever the surrogate's weights or normalisation change
    sicp::Buf search_dev;                // device copy of `search`, rewritten by every reference build
    int search_slot = -2;                // constant-memory copy of `search` (-2: none yet, -1: none free)
    // the last registration run: its particles and Adam moments stay in theta,
    // adam_m, adam_v (sicp_export_state, sicp_import_state, sicp_resume)
    bool run_valid = false;
    int32_t run_K = 0;
    int64_t run_t = 0;                   // iterations done
    uint64_t run_seed = 0;               // its minibatch stream
    sicp::Buf resume;                    // device staging of that state for sicp_resume
    sicp::Buf normals;                   // point-to-plane: float4 [M] unit normals by original index
    int normals_k = 0;                   // neighbours they were computed from; 0: none for this reference
    // failure-detection check (sicp_set_wait_check): when set, every bounded device wait of the
    // context's kernels waits for an event that never comes, polling at most wait_polls times
    // (0: each wait's default limit)
    int wait_never = 0;
    long long wait_polls = 0;
    // device memory budget (sicp_set_memory_limit; 0: none) and the bytes the context holds in
    // buffers that can grow (references, grids, run state, scratch)
    size_t mem_limit = 0, mem_used = 0;
    // per-iteration telemetry of registration runs (sicp_set_telemetry): rows [T][16] of the last
    // run, the correspondences of one iteration, per-particle distance sums and the fallback count
    bool telemetry = false;
    sicp::Buf tel, tel_nn, tel_part;
    int32_t tel_rows = 0;
    int64_t src_n = 0;   // points packed into src4 (bounds checks)
};

namespace sicp {

int set_err(sicp_ctx* c, int code, const char* fmt, ...);
int cuda_err(sicp_ctx* c, cudaError_t e, const char* what);
int ensure(sicp_ctx* c, Buf& b, size_t bytes);
// cudaMalloc of `bytes` counted against the context's budget (SICP_ENOMEM past it);
// `held` bytes are freed by the caller first and no longer count
int budget_malloc(sicp_ctx* c, void** p, size_t bytes, size_t held);

#define SICP_CUDA(call)                                     \
    do {                                                    \
        cudaError_t e_ = (call);                            \
        if (e_ != cudaSuccess) return cuda_err(ctx, e_, #call); \
    } while (0)

// ---- kernel launchers (each returns the launch status) ----


// points [n][3] -> float4 (w = index bits); flags[0] |= 1 on a non-finite value
cudaError_t launch_pack_points(const float* xyz, int64_t n, float4* out, int* flags, cudaStream_t s);
cudaError_t launch_check_finite(const float* x, int64_t n, int* flags, cudaStream_t s);
// flags[0] |= 1 on a non-finite or negative value (Adam second moments)
cudaError_t launch_check_nonneg(const float* x, int64_t n, int* flags, cudaStream_t s);
// flags[1] |= 1 if any index is outside [0, N)
cudaError_t launch_check_index(const int32_t* idx, int64_t n, int64_t N, int* flags, cudaStream_t s);
// gbar[j][c] = inv_m * sum over chunks of partial[chunk][j][c]
cudaError_t launch_partial_to_gbar(const float* partial, int chunks, int32_t K, float inv_m, float* gbar,
                                   cudaStream_t s);
// gbar[j][c] = inv_m * sum over k of qterms[j][k][c] ([K][m][6], fixed order); also zeroes
// *fb_count when it is not null, after copying it to *fb_keep when that is not null
cudaError_t launch_qterms_to_gbar(const float* qterms, int32_t K, int32_t m, float inv_m, float* gbar, int* fb_count,
                                  cudaStream_t s, int* fb_keep = nullptr);
// ordered-uint bounding box of float4 points into lohi[6] (min xyz, max xyz), pre-initialised
cudaError_t launch_bbox(const float4* p, int64_t n, unsigned* lohi, cudaStream_t s);
float ordered_to_float(unsigned u);
// exclusive scan of n int32 counts into out[0..n] (out[n] = total); sums: scratch of scan_sums_size(n)
size_t scan_sums_size(int64_t n);
cudaError_t launch_exclusive_scan(const int32_t* in, int64_t n, int32_t* out, int32_t* sums, cudaStream_t s);
// one-time kernel attributes (dynamic shared memory opt-in)
cudaError_t kernel_attrs_init();
cudaError_t minibatch_kernel_attrs();   // dynamic shared memory of the minibatch kernels

cudaError_t launch_minibatch(uint64_t seed, int64_t t0, int32_t T, int64_t N, int32_t m,
                             int32_t* out, cudaStream_t s);
// Independent runs: run j draws the stream of seed + j; out [R][T][m].
cudaError_t launch_minibatch_runs(uint64_t seed, int64_t t0, int32_t T, int64_t N, int32_t m, int32_t R,
                                  int32_t* out, cudaStream_t s);

// Per-query search of the whole reference (fp32 exhaustive).
cudaError_t launch_nn_brute(const float4* ref, int64_t M, const float* q, int64_t n,
                            int32_t* idx, float* d2, cudaStream_t s);

// The fused gradient kernels write one partial sum per (chunk of minibatch
// entries, particle); `chunks` is how many chunks a launch uses.
struct GradLayout {
    int chunks, threads;
};
GradLayout grad_layout(int32_t m);            // exhaustive search: threads per CTA, one query each
GradLayout grad_layout_grid(int32_t m);       // grid search: a lane group per query

struct GradArgs {
    const float4* src;     // N
    const int32_t* mb;     // m indices of this iteration
    int32_t m;
    const float* theta;    // K x 6
    int32_t K;
    float* partial;        // exhaustive search: [chunks][K][6] sums of gradient terms (not divided by m);
                           // grid search: [K][m][6] terms of each query
    int32_t* out_nn;       // K x m or null
    unsigned long long* stats;  // search work counters or null
    // grid search only: gbar = inv_m * (sum over the minibatch of the terms),
    // reduced in a fixed order after the search kernel.
    float* gbar;           // K x 6
    float inv_m;
    // point-to-plane metric: unit normals by original reference index (w
    // unused); null: point-to-point
    const float4* normals;
    // minibatch entries between consecutive particles' rows: 0, one row
    // shared by all particles; else particle j reads mb[j * mb_stride + k]
    int64_t mb_stride;
    int64_t n_src;         // source points (bounds checks)
    int64_t n_ref;         // reference points (bounds checks)
};
cudaError_t launch_grad_brute(const GradArgs& a, const float4* ref, int64_t M, cudaStream_t s);

struct SteinArgs {
    float* theta;          // K x 6 in/out
    float* adam_m;         // K x 6
    float* adam_v;         // K x 6
    const float* partial;  // [chunks][K][6]
    int32_t chunks;
    float inv_m;           // 1/m: gbar = inv_m * sum over chunks
    int32_t K;
    float N;
    int64_t t;             // 1-based Adam step
    float lr, beta1, beta2, eps;
    int32_t prior;
    float mu[6], sigma[3], kappa[3];
    float* out_phi;        // K x 6 or null
    float* out_gbar;       // K x 6 or null: the mean gradients the update used (single-CTA form only)
    float* out_h;          // 2 or null
    // the two blocks' medians of the previous iteration (in/out; 0: none) or
    // null: starts the median selection next to the previous median
    float* med_state;
    // two arrival counters (one per block) and an error flag, or null: with
    // them the update of each block is split over several CTAs (particles).
    // gen: 1-based count of such updates since the counters were zeroed.
    unsigned* arrive;
    int* err;
    uint32_t gen;
    // the arrival wait: at most max_spins polls (0: the default), for gen * P + extra arrivals
    // (extra = 1 only in the failure-detection check, where the wait must give up)
    long long max_spins;
    uint32_t extra;
    // single-CTA form: keep the pair distances in shared memory when they fit (1) or never (0)
    int32_t cache;
};
cudaError_t launch_stein_adam(const SteinArgs& a, cudaStream_t s);
// Independent runs (no Stein coupling): Adam on g = -G_j for every particle j,
// the K = 1 update of the same kernel for each particle.
cudaError_t launch_adam_independent(const SteinArgs& a, cudaStream_t s);
cudaError_t launch_moments(const float* theta, int32_t K, double* out42, cudaStream_t s);
cudaError_t launch_moments_circular(const float* theta, int32_t K, double* out42, cudaStream_t s);

// Learned closest-point field (k_mlp.cu)
cudaError_t surrogate_kernel_attrs();
bool surrogate_ready(const sicp_ctx* ctx);
void surrogate_invalidate(sicp_ctx* ctx);
// One iteration's gradient with the surrogate: per-query terms into qterms
// [K][m][6] (the exact grid search, in a second kernel, for queries whose
// confidence is below min_conf or that leave the trained cube), then gbar
// [K][6] = their mean per particle.
// stats (8 counters or null): slots 0..5 as the grid search, 6 surrogate
// tiles' queries, 7 queries sent to the exact search.  err: set on a
// tensor-core wait that gave up.
// Size the surrogate path's fallback list for `queries` per iteration and
// clear its count (before capturing a loop that calls surrogate_launch_grad).
int surrogate_prepare(sicp_ctx* ctx, int64_t queries);
// fb_keep (or null): receives the number of queries sent to the exact search.
cudaError_t surrogate_launch_grad(sicp_ctx* ctx, const float4* src, const int32_t* mb, int m, const float* theta,
                                  int K, float min_conf, float* qterms, float* gbar, unsigned long long* stats,
                                  int* err, int* fb_keep = nullptr);

// Exhaustive search with tensor-core distance tiles and an exact fp32 re-check
// (k_nn_bf16.cu); same results as launch_nn_brute / the fp32 gradient.
cudaError_t bf16_kernel_attrs();
int bf16_prepare(sicp_ctx* ctx);   // reference tiles of the current reference (needs the grid)
int bf16_queries(sicp_ctx* ctx, int64_t Q);   // a launch's query buffers (before any capture)
// err: set when a bounded wait gave up
cudaError_t launch_nn_bf16(sicp_ctx* ctx, const float* q, int64_t n, int32_t* idx, float* d2, int* err);
// per-query gradient terms into qterms [K][m][6], then gbar [K][6]; out_nn [K][m] or null;
// normals (unit, by original index) select the point-to-plane metric, null point-to-point
cudaError_t launch_grad_bf16(sicp_ctx* ctx, const float4* src, const int32_t* mb, int m, const float* theta, int K,
                             float* qterms, float* gbar, int32_t* out_nn, int* err, const float4* normals,
                             int64_t mb_stride);

// One telemetry row of a registration iteration (k_telemetry.cu): the particles it starts from,
// the mean distance from its queries to their correspondences, the share the learned field served.
struct TelArgs {
    const float* theta;        // [K][6] particles at the start of the iteration
    int32_t K, m;
    const float4* src;         // packed source
    int64_t n_src;             // its points (bounds checks)
    const int32_t* mb;         // the iteration's minibatch row (independent runs: row of run 0)
    int64_t mb_stride;         // run j's row at mb + j * mb_stride (0: one shared row)
    const int32_t* nn;         // exact iterations: correspondences [K][m] (-1: none); else null
    const float4* ref4;        // reference points by original index
    int64_t n_ref;             // their number (bounds checks)
    const float* qterms;       // learned iterations: per-query terms [K][m][6]; else null
    const int* fb;             // learned iterations: queries sent to the exact search
    float* part;               // [K] scratch: per-particle distance sums and counts ([2K])
    float* row;                // [16] the row
    double t_abs;              // the iteration's absolute index
};
cudaError_t launch_telemetry(const TelArgs& a, cudaStream_t s);

// Grid (uniform voxel) search structure
int grid_build(sicp_ctx* ctx, float cell_size);
int search_table_init(sicp_ctx* ctx);
cudaError_t launch_nn_grid(const GridSearch& g, const float* q, int64_t n, int32_t* idx, float* d2,
                           unsigned long long* stats, cudaStream_t s);
// d_search: the device copy of the context's GridSearch (sicp_ctx::search_dev);
// slot: the context's constant-memory copy (sicp_ctx::search_slot), or < 0
cudaError_t launch_grad_grid(const GradArgs& a, const GridSearch* d_search, int slot, cudaStream_t s);
int search_slot_acquire();   // a free constant-memory slot, or -1
void search_slot_release(int slot);

}  // namespace sicp
