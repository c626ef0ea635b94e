// Reference normals for the point-to-plane metric.  The paper compares methods
// with the point-to-plane error metric (its comparison table and trajectory
// errors) without printing it; the metric used here takes the residual of a
// correspondence along the unit normal at the reference point.
//
// Normal of reference point i: the unit eigenvector of the smallest
// eigenvalue of the covariance (float64, divisor k) of its k nearest reference
// points, itself included.  Neighbours are ranked by the fp32 squared distance
// of every search in this library (dist2) with ties to the lower index, so the
// neighbour set is a fixed function of the input.
//
// One thread per reference point walks the fine grid in cubic shells of cells
// around its own cell (Chebyshev radius 0, 1, 2, ...), keeping the k best in
// order, and stops once the k-th best is closer than every cell outside the
// scanned cube (cell bounds widened by the grid's tolerance, the squared bound
// by a relative 5e-7, as in the nearest-neighbour search).  The 3 x 3
// eigenproblem is solved by cyclic Jacobi rotations in float64.
#include <float.h>
#include <math.h>

#include "common.cuh"
#include "grid_search.cuh"

namespace sicp {
namespace {

constexpr int kNormalThreads = 128;
constexpr int kNormalMaxK = 32;
constexpr int kJacobiSweeps = 32;

// A <- J^T A J and V <- V J for the plane rotation J in (p, q) that zeroes A[p][q].
__device__ void jacobi_rotate(double A[3][3], double V[3][3], int p, int q) {
    const double apq = A[p][q];
    if (apq == 0.0) return;
    const double theta = (A[q][q] - A[p][p]) / (2.0 * apq);
    const double t = fabs(theta) > 1e150 ? 0.5 / theta
                                         : (theta >= 0.0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
    const double c = 1.0 / sqrt(t * t + 1.0), s = t * c;
    double J[3][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
    J[p][p] = c;
    J[q][q] = c;
    J[p][q] = s;
    J[q][p] = -s;
    double T[3][3], N[3][3];
    for (int r = 0; r < 3; ++r)
        for (int col = 0; col < 3; ++col) T[r][col] = A[r][0] * J[0][col] + A[r][1] * J[1][col] + A[r][2] * J[2][col];
    for (int r = 0; r < 3; ++r)
        for (int col = 0; col < 3; ++col) N[r][col] = J[0][r] * T[0][col] + J[1][r] * T[1][col] + J[2][r] * T[2][col];
    for (int r = 0; r < 3; ++r)
        for (int col = 0; col < 3; ++col) A[r][col] = N[r][col];
    A[p][q] = A[q][p] = 0.0;
    for (int r = 0; r < 3; ++r)
        for (int col = 0; col < 3; ++col) T[r][col] = V[r][0] * J[0][col] + V[r][1] * J[1][col] + V[r][2] * J[2][col];
    for (int r = 0; r < 3; ++r)
        for (int col = 0; col < 3; ++col) V[r][col] = T[r][col];
}

// Unit eigenvector of the smallest eigenvalue of the symmetric A; *lmin and
// *lsum receive that eigenvalue and the sum of all three.
__device__ void smallest_eigvec(double A[3][3], double n[3], double* lmin, double* lsum) {
    double V[3][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
    for (int sweep = 0; sweep < kJacobiSweeps; ++sweep) {
        const double off = A[0][1] * A[0][1] + A[0][2] * A[0][2] + A[1][2] * A[1][2];
        const double diag = A[0][0] * A[0][0] + A[1][1] * A[1][1] + A[2][2] * A[2][2];
        if (!(off > 1e-32 * diag) || off == 0.0) break;
        jacobi_rotate(A, V, 0, 1);
        jacobi_rotate(A, V, 0, 2);
        jacobi_rotate(A, V, 1, 2);
    }
    int j = 0;
    if (A[1][1] < A[j][j]) j = 1;
    if (A[2][2] < A[j][j]) j = 2;
    const double len = sqrt(V[0][j] * V[0][j] + V[1][j] * V[1][j] + V[2][j] * V[2][j]);
    for (int a = 0; a < 3; ++a) n[a] = V[a][j] / len;
    *lmin = A[j][j];
    *lsum = A[0][0] + A[1][1] + A[2][2];
}

struct TopK {
    float d[kNormalMaxK];
    int id[kNormalMaxK];
    int n = 0;
};

// Insert (d2, id) into the ordered list of the k best (distance, then index).
__device__ __forceinline__ void topk_insert(TopK& L, int k, float d2, int id) {
    if (L.n == k && !(d2 < L.d[k - 1] || (d2 == L.d[k - 1] && id < L.id[k - 1]))) return;
    int p = L.n < k ? L.n++ : k - 1;
    while (p > 0 && (d2 < L.d[p - 1] || (d2 == L.d[p - 1] && id < L.id[p - 1]))) {
        L.d[p] = L.d[p - 1];
        L.id[p] = L.id[p - 1];
        --p;
    }
    L.d[p] = d2;
    L.id[p] = id;
}

__device__ __forceinline__ void scan_cells(const GridView& g, int64_t row, int x0, int x1, float3 q, TopK& L, int k) {
    const int b = __ldg(g.cell_start + row + x0), e = __ldg(g.cell_start + row + x1 + 1);
    for (int p = b; p < e; ++p) {
        const float4 r = __ldg(g.sorted + p);
        topk_insert(L, k, dist2(r, q), __float_as_int(r.w));
    }
}

// out[i] = (normal, surface variation lmin / lsum) of reference point i (original order).
__global__ void __launch_bounds__(kNormalThreads) k_normals(GridView g, const float4* __restrict__ ref, int64_t M,
                                                            int k, float4* __restrict__ out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= M) return;
    const float4 q4 = ref[i];
    const float3 q = make_float3(q4.x, q4.y, q4.z);
    const int cx = gs::cell_coord(q.x, g.origin.x, g.inv_cell, g.dims.x);
    const int cy = gs::cell_coord(q.y, g.origin.y, g.inv_cell, g.dims.y);
    const int cz = gs::cell_coord(q.z, g.origin.z, g.inv_cell, g.dims.z);
    TopK L;
    const int rmax = max(g.dims.x, max(g.dims.y, g.dims.z));
    for (int r = 0; r <= rmax; ++r) {
        // shell r: the cells at Chebyshev distance r from (cx, cy, cz)
        for (int z = max(cz - r, 0); z <= min(cz + r, g.dims.z - 1); ++z)
            for (int y = max(cy - r, 0); y <= min(cy + r, g.dims.y - 1); ++y) {
                const int64_t row = ((int64_t)z * g.dims.y + y) * g.dims.x;
                if (abs(z - cz) == r || abs(y - cy) == r) {
                    scan_cells(g, row, max(cx - r, 0), min(cx + r, g.dims.x - 1), q, L, k);
                } else {
                    if (cx - r >= 0) scan_cells(g, row, cx - r, cx - r, q, L, k);
                    if (cx + r < g.dims.x) scan_cells(g, row, cx + r, cx + r, q, L, k);
                }
            }
        // the cube [c - r, c + r] holds the whole grid: nothing is left
        const bool lo_x = cx - r > 0, hi_x = cx + r < g.dims.x - 1;
        const bool lo_y = cy - r > 0, hi_y = cy + r < g.dims.y - 1;
        const bool lo_z = cz - r > 0, hi_z = cz + r < g.dims.z - 1;
        if (!(lo_x || hi_x || lo_y || hi_y || lo_z || hi_z)) break;
        if (L.n == k) {
            // distance from q to the nearest face of the scanned cube that has cells beyond it
            float lb = FLT_MAX;
            if (lo_x) lb = fminf(lb, q.x - fmaf((float)(cx - r), g.cell, g.origin.x));
            if (hi_x) lb = fminf(lb, fmaf((float)(cx + r + 1), g.cell, g.origin.x) - q.x);
            if (lo_y) lb = fminf(lb, q.y - fmaf((float)(cy - r), g.cell, g.origin.y));
            if (hi_y) lb = fminf(lb, fmaf((float)(cy + r + 1), g.cell, g.origin.y) - q.y);
            if (lo_z) lb = fminf(lb, q.z - fmaf((float)(cz - r), g.cell, g.origin.z));
            if (hi_z) lb = fminf(lb, fmaf((float)(cz + r + 1), g.cell, g.origin.z) - q.z);
            lb -= g.tol;
            if (lb > 0.f && L.d[k - 1] * gs::kSlack < lb * lb) break;
        }
    }
    // covariance of the neighbourhood (float64, divisor k)
    double mu[3] = {0.0, 0.0, 0.0};
    for (int c = 0; c < L.n; ++c) {
        const float4 p = __ldg(ref + L.id[c]);
        mu[0] += (double)p.x;
        mu[1] += (double)p.y;
        mu[2] += (double)p.z;
    }
    for (int a = 0; a < 3; ++a) mu[a] /= (double)L.n;
    double C[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
    for (int c = 0; c < L.n; ++c) {
        const float4 p = __ldg(ref + L.id[c]);
        const double d[3] = {(double)p.x - mu[0], (double)p.y - mu[1], (double)p.z - mu[2]};
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) C[a][b] += d[a] * d[b];
    }
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) C[a][b] /= (double)L.n;
    double n[3], lmin, lsum;
    smallest_eigvec(C, n, &lmin, &lsum);
    out[i] = make_float4((float)n[0], (float)n[1], (float)n[2], lsum > 0.0 ? (float)(lmin / lsum) : 0.f);
}

struct DevScope {
    int prev = -1;
    explicit DevScope(int d) {
        cudaGetDevice(&prev);
        if (prev != d) cudaSetDevice(d);
    }
    ~DevScope() {
        int cur = -1;
        cudaGetDevice(&cur);
        if (prev >= 0 && cur != prev) cudaSetDevice(prev);
    }
};

}  // namespace
}  // namespace sicp

using namespace sicp;

extern "C" int sicp_reference_normals(sicp_ctx* ctx, int32_t k, float* out_normals, int on_device) {
    if (!ctx) return SICP_EINVAL;
    ctx->err.clear();
    if (ctx->M < 1) return set_err(ctx, SICP_ENOREF, "no reference cloud set");
    if (k < 3 || k > kNormalMaxK || k > ctx->M)
        return set_err(ctx, SICP_EINVAL, "normals need 3 <= k <= min(%d, M)", kNormalMaxK);
    DevScope ds(ctx->device);
    cudaStream_t s = ctx->stream;
    const int64_t M = ctx->M;
    int rc = ensure(ctx, ctx->normals, sizeof(float4) * (size_t)M);
    if (rc) return rc;
    ctx->normals_k = 0;
    k_normals<<<(unsigned)((M + kNormalThreads - 1) / kNormalThreads), kNormalThreads, 0, s>>>(
        ctx->grid.v, ctx->ref4, M, k, (float4*)ctx->normals.p);
    SICP_CUDA(cudaGetLastError());
    if (out_normals)
        SICP_CUDA(cudaMemcpy2DAsync(out_normals, 3 * sizeof(float), ctx->normals.p, sizeof(float4), 3 * sizeof(float),
                                    (size_t)M, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s));
    SICP_CUDA(cudaStreamSynchronize(s));
    ctx->normals_k = k;
    return SICP_OK;
}
