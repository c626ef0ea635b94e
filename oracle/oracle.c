/*
 * Stein ICP -- plain FP64 CPU oracle.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously correct
 * statement of what one Stein ICP run computes, written from the paper
 * ("Stein ICP for Uncertainty Estimation in Point Cloud Matching",
 * Afzal Maken, Ramos, Ott).  Only the tests, the smoke check and the
 * benchmark's CPU-baseline leg may load it.  It shares no code, header,
 * table or constant with the CUDA library: the two meet only through the
 * seeded synthetic inputs.
 *
 * Every floating-point operation is in double precision.  Inputs arrive as
 * float32 clouds (the library's input type) and are widened exactly.
 * Loops over independent queries or particles carry an OpenMP pragma; the
 * result does not depend on the thread count.
 *
 * Readings of the paper where it is silent or garbled (each used below):
 *  R1  rotation: R = Rz(yaw) Ry(pitch) Rx(roll), angles theta[3..5] in rad.
 *  R2  s' = R s + u maps the source into the reference frame (Sec. III-A).
 *  R3  the mean gradients of Eqs. (trans/rotation gradient) are the exact
 *      gradient of L/2 with the correspondences held fixed (no factor 2).
 *  R4  log-posterior gradient G = -N gbar + grad log prior (the printed
 *      bracket in Eq. (stein_icp_phi) would flip the prior's sign).
 *  R5  the Stein sum carries a 1/K factor (expectation form of phi*).
 *  R6  the Gaussian prior divides by sigma as printed (sigma = variance).
 *  R7  translation and rotation blocks use separate kernels and bandwidths.
 *  R8  the rotation kernel squares and sums the three wrapped differences,
 *      wrap(x) = atan2(sin x, cos x); d wrap / dx = 1 everywhere.
 *  R9  median heuristic: h = med / ln(K+1), med = median of the K*K squared
 *      pairwise distances including the diagonal (mean of the two middle
 *      values for an even count); h = 1 if med = 0.
 *  R10 Adam: beta1 = 0.9, beta2 = 0.999, eps = 1e-8 outside the root, bias
 *      correction from t = 1, gradient fed to Adam is -phi.
 *  R11 one minibatch per iteration, shared by all particles: the m source
 *      indices with the smallest splitmix64 keys (see or_mb_key), returned
 *      in ascending index order.
 *  R12 correspondence ties go to the lowest reference index; distances are
 *      the exact sum of squared differences.
 *  R16 point-to-plane metric (named, not printed: the paper's comparison
 *      table and trajectory errors use it): correspondences as R12; residual
 *      e = n . (R s + u - r) with n the unit normal at r; the gradient is
 *      that of (1/2m) sum e^2 with r and n held fixed, i.e. the point-to-point
 *      terms with the residual vector replaced by e n.  The normal at a
 *      reference point is the eigenvector of the smallest eigenvalue of the
 *      covariance of its k nearest reference points (itself included), the
 *      neighbours ranked by their exact fp64 squared distance, ties to the
 *      lower index; the covariance in fp64.  Where the k-th and (k+1)-th
 *      distances tie to within fp32 rounding the neighbourhood, and so the
 *      normal, is not unique, and a float32 ranking may pick either set.
 *  R17 Monte Carlo ground truth (the experiments' reference distribution:
 *      many SGD-ICP runs from spread initial poses): with `independent` set,
 *      every particle j is its own SGD-ICP run (Sec. III-B): its own
 *      minibatch stream (R11 with seed + j), Adam on its own log-posterior
 *      gradient, phi_j = G_j -- exactly the K = 1 run with seed + j.
 *  R15 circular moments (for rotation blocks whose particles straddle +-pi):
 *      each angle's mean is the circular mean atan2(sum sin, sum cos) (0 if
 *      both sums vanish); the covariance is that of the deviations
 *      [theta_t - mean_t ; wrap(theta_r - mean_r)], divisor K-1 (0 for K = 1).
 *      Translations keep the arithmetic mean.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_EXPORT __attribute__((visibility("default")))

/* ------------------------------------------------------------------------ */
/* splitmix64 (Steele, Lea, Flood 2014; Vigna's public-domain reference):    */
/* state += 0x9e3779b97f4a7c15, then the output mix of the state.            */
/* ------------------------------------------------------------------------ */

static uint64_t or_mix(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    return z ^ (z >> 31);
}

/* Output number k (k >= 1) of splitmix64 started from state s. */
OR_EXPORT uint64_t or_splitmix64_at(uint64_t s, uint64_t k) {
    return or_mix(s + k * 0x9e3779b97f4a7c15ULL);
}

/* Minibatch key of source point i at iteration t (R11): the (i+1)-th output of
 * a splitmix64 stream whose state is the (t+1)-th output of one seeded with
 * `seed`.  The keys of one iteration are pairwise distinct (the output mix is a
 * bijection and the states differ), so "the m smallest" is unique. */
OR_EXPORT uint64_t or_mb_key(uint64_t seed, int64_t t, int64_t i) {
    uint64_t base = or_splitmix64_at(seed, (uint64_t)t + 1);
    return or_splitmix64_at(base, (uint64_t)i + 1);
}

typedef struct { uint64_t key; int64_t idx; } or_keyed;

static int or_cmp_keyed(const void* a, const void* b) {
    const or_keyed* x = (const or_keyed*)a;
    const or_keyed* y = (const or_keyed*)b;
    if (x->key < y->key) return -1;
    if (x->key > y->key) return 1;
    return (x->idx > y->idx) - (x->idx < y->idx);
}

static int or_cmp_i32(const void* a, const void* b) {
    int32_t x = *(const int32_t*)a, y = *(const int32_t*)b;
    return (x > y) - (x < y);
}

/* Sec. III-B: SGD-ICP samples a minibatch of m source points per iteration.
 * Reading R11: sort all N keys, keep the m smallest, return them by index. */
OR_EXPORT int or_minibatch(uint64_t seed, int64_t t, int64_t N, int32_t m, int32_t* out) {
    if (N < 1 || m < 1 || m > N) return -1;
    or_keyed* kv = (or_keyed*)malloc(sizeof(or_keyed) * (size_t)N);
    if (!kv) return -2;
    for (int64_t i = 0; i < N; ++i) { kv[i].key = or_mb_key(seed, t, i); kv[i].idx = i; }
    qsort(kv, (size_t)N, sizeof(or_keyed), or_cmp_keyed);
    for (int32_t k = 0; k < m; ++k) out[k] = (int32_t)kv[k].idx;
    qsort(out, (size_t)m, sizeof(int32_t), or_cmp_i32);
    free(kv);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Rotation (Sec. III-A, R1) and its partial derivatives                     */
/* ------------------------------------------------------------------------ */

static void or_mat3_mul(const double A[9], const double B[9], double C[9]) {
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) {
            double s = 0.0;
            for (int k = 0; k < 3; ++k) s += A[3 * r + k] * B[3 * k + c];
            C[3 * r + c] = s;
        }
}

/* Elementary rotations and their derivatives with respect to their angle. */
static void or_rx(double a, double M[9], double D[9]) {
    double c = cos(a), s = sin(a);
    double m[9] = {1, 0, 0, 0, c, -s, 0, s, c};
    double d[9] = {0, 0, 0, 0, -s, -c, 0, c, -s};
    memcpy(M, m, sizeof m); memcpy(D, d, sizeof d);
}
static void or_ry(double a, double M[9], double D[9]) {
    double c = cos(a), s = sin(a);
    double m[9] = {c, 0, s, 0, 1, 0, -s, 0, c};
    double d[9] = {-s, 0, c, 0, 0, 0, -c, 0, -s};
    memcpy(M, m, sizeof m); memcpy(D, d, sizeof d);
}
static void or_rz(double a, double M[9], double D[9]) {
    double c = cos(a), s = sin(a);
    double m[9] = {c, -s, 0, s, c, 0, 0, 0, 1};
    double d[9] = {-s, -c, 0, c, -s, 0, 0, 0, 0};
    memcpy(M, m, sizeof m); memcpy(D, d, sizeof d);
}

/* R (row-major 3x3) and dR[a] = dR / d theta[3+a], a = roll, pitch, yaw. */
OR_EXPORT void or_rotation(const double th[6], double R[9], double dR[27]) {
    double X[9], dX[9], Y[9], dY[9], Z[9], dZ[9], ZY[9], T[9];
    or_rx(th[3], X, dX);
    or_ry(th[4], Y, dY);
    or_rz(th[5], Z, dZ);
    or_mat3_mul(Z, Y, ZY);
    or_mat3_mul(ZY, X, R);
    if (!dR) return;
    or_mat3_mul(ZY, dX, dR + 0);           /* Rz Ry dRx */
    or_mat3_mul(Z, dY, T);
    or_mat3_mul(T, X, dR + 9);             /* Rz dRy Rx */
    or_mat3_mul(dZ, Y, T);
    or_mat3_mul(T, X, dR + 18);            /* dRz Ry Rx */
}

/* ------------------------------------------------------------------------ */
/* Point-to-point correspondence, Eq. (correspondences): exhaustive argmin   */
/* ------------------------------------------------------------------------ */

static int64_t or_nn_one(const float* ref, int64_t M, const double q[3], double* d2_out) {
    int64_t best = -1;
    double bd = INFINITY;
    for (int64_t r = 0; r < M; ++r) {
        double dx = (double)ref[3 * r] - q[0];
        double dy = (double)ref[3 * r + 1] - q[1];
        double dz = (double)ref[3 * r + 2] - q[2];
        double d2 = dx * dx + dy * dy + dz * dz;
        if (d2 < bd) { bd = d2; best = r; }      /* strict: lowest index wins ties (R12) */
    }
    *d2_out = bd;
    return best;
}

/* Nearest reference point of each query; q is nq x 3 doubles. */
OR_EXPORT void or_nn(const float* ref, int64_t M, const double* q, int64_t nq,
                     int64_t* idx, double* d2) {
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t i = 0; i < nq; ++i) idx[i] = or_nn_one(ref, M, q + 3 * i, d2 + i);
}

/* Second-nearest distance of each query as well (used to flag near-ties). */
OR_EXPORT void or_nn2(const float* ref, int64_t M, const double* q, int64_t nq,
                      int64_t* idx, double* d2, double* d2_second) {
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t i = 0; i < nq; ++i) {
        int64_t best = -1;
        double b1 = INFINITY, b2 = INFINITY;
        const double* qq = q + 3 * i;
        for (int64_t r = 0; r < M; ++r) {
            double dx = (double)ref[3 * r] - qq[0];
            double dy = (double)ref[3 * r + 1] - qq[1];
            double dz = (double)ref[3 * r + 2] - qq[2];
            double dd = dx * dx + dy * dy + dz * dz;
            if (dd < b1) { b2 = b1; b1 = dd; best = r; }
            else if (dd < b2) { b2 = dd; }
        }
        idx[i] = best; d2[i] = b1; d2_second[i] = b2;
    }
}

/* ------------------------------------------------------------------------ */
/* The same argmin through a k-d tree (a faster route to or_nn's answer)     */
/* ------------------------------------------------------------------------ */
/*
 * A k-d tree over the reference points: each node holds a contiguous range
 * of a permutation of the point indices and the tight bounding box of its
 * points; an inner node splits its range at the median of the box's longest
 * axis.  A query walks the tree depth first, nearer child first, and skips a
 * node only when the squared distance from the query to the node's box is
 * strictly larger than the best squared distance found so far.  The box
 * distance is summed over the axes in the same order (x, y, z) as a point's
 * squared distance, and floating-point subtraction, squaring and addition are
 * monotone, so no point of a skipped box can be nearer than or tie with the
 * best: the walk returns exactly or_nn's answer, lowest index on ties (R12).
 */
#define OR_KD_LEAF 8

typedef struct {
    int64_t lo, hi;          /* range [lo, hi) of perm */
    int64_t left, right;     /* children (-1 for a leaf) */
    double bmin[3], bmax[3]; /* bounding box of the node's points */
} or_kdnode;

typedef struct or_kdtree {
    const float* ref;
    int64_t M;
    int64_t* perm;
    or_kdnode* node;
    int64_t n_nodes, cap;
} or_kdtree;

static double or_kd_coord(const or_kdtree* t, int64_t i, int a) { return (double)t->ref[3 * t->perm[i] + a]; }

static void or_kd_swap(int64_t* p, int64_t a, int64_t b) { int64_t x = p[a]; p[a] = p[b]; p[b] = x; }

/* Reorder perm[lo, hi) so that perm[k] holds the point of rank k - lo along
 * axis a (ties by index), smaller ranks before it, larger after (quickselect). */
static void or_kd_select(or_kdtree* t, int64_t lo, int64_t hi, int64_t k, int a) {
    while (hi - lo > 1) {
        int64_t mid = lo + (hi - lo) / 2;
        or_kd_swap(t->perm, mid, hi - 1);
        const double pv = or_kd_coord(t, hi - 1, a);
        const int64_t pi = t->perm[hi - 1];
        int64_t store = lo;
        for (int64_t i = lo; i < hi - 1; ++i) {
            const double v = or_kd_coord(t, i, a);
            if (v < pv || (v == pv && t->perm[i] < pi)) or_kd_swap(t->perm, i, store++);
        }
        or_kd_swap(t->perm, store, hi - 1);
        if (store == k) return;
        if (k < store) hi = store; else lo = store + 1;
    }
}

static int64_t or_kd_new_node(or_kdtree* t, int64_t lo, int64_t hi) {
    if (t->n_nodes == t->cap) {
        t->cap = t->cap ? 2 * t->cap : 64;
        t->node = (or_kdnode*)realloc(t->node, sizeof(or_kdnode) * (size_t)t->cap);
    }
    or_kdnode* n = &t->node[t->n_nodes];
    n->lo = lo; n->hi = hi; n->left = n->right = -1;
    for (int a = 0; a < 3; ++a) { n->bmin[a] = INFINITY; n->bmax[a] = -INFINITY; }
    for (int64_t i = lo; i < hi; ++i)
        for (int a = 0; a < 3; ++a) {
            const double v = or_kd_coord(t, i, a);
            if (v < n->bmin[a]) n->bmin[a] = v;
            if (v > n->bmax[a]) n->bmax[a] = v;
        }
    return t->n_nodes++;
}

static int64_t or_kd_build_node(or_kdtree* t, int64_t lo, int64_t hi) {
    const int64_t id = or_kd_new_node(t, lo, hi);
    if (hi - lo <= OR_KD_LEAF) return id;
    int axis = 0;
    double best = -1.0;
    for (int a = 0; a < 3; ++a) {
        const double ext = t->node[id].bmax[a] - t->node[id].bmin[a];
        if (ext > best) { best = ext; axis = a; }
    }
    const int64_t mid = lo + (hi - lo) / 2;
    or_kd_select(t, lo, hi, mid, axis);
    const int64_t l = or_kd_build_node(t, lo, mid);
    const int64_t r = or_kd_build_node(t, mid, hi);
    t->node[id].left = l;       /* (t->node may have moved while the children were built) */
    t->node[id].right = r;
    return id;
}

/* Build a tree over ref (M x 3 floats; the caller keeps ref alive while the
 * tree is used).  NULL on bad arguments or when memory runs out. */
OR_EXPORT or_kdtree* or_kd_build(const float* ref, int64_t M) {
    if (!ref || M < 1) return NULL;
    or_kdtree* t = (or_kdtree*)calloc(1, sizeof(or_kdtree));
    if (!t) return NULL;
    t->ref = ref;
    t->M = M;
    t->perm = (int64_t*)malloc(sizeof(int64_t) * (size_t)M);
    if (!t->perm) { free(t); return NULL; }
    for (int64_t i = 0; i < M; ++i) t->perm[i] = i;
    or_kd_build_node(t, 0, M);
    return t;
}

OR_EXPORT void or_kd_free(or_kdtree* t) {
    if (!t) return;
    free(t->perm);
    free(t->node);
    free(t);
}

/* Squared distance from q to a node's box, summed in the order of a point's. */
static double or_kd_box_d2(const or_kdnode* n, const double q[3]) {
    double g[3];
    for (int a = 0; a < 3; ++a) {
        if (q[a] < n->bmin[a]) g[a] = n->bmin[a] - q[a];
        else if (q[a] > n->bmax[a]) g[a] = q[a] - n->bmax[a];
        else g[a] = 0.0;
    }
    return g[0] * g[0] + g[1] * g[1] + g[2] * g[2];
}

static int64_t or_kd_nn_one(const or_kdtree* t, const double q[3], double* d2_out) {
    int64_t stack[128];
    int sp = 0;
    int64_t best = -1;
    double bd = INFINITY;
    stack[sp++] = 0;
    while (sp > 0) {
        const or_kdnode* n = &t->node[stack[--sp]];
        if (or_kd_box_d2(n, q) > bd) continue;
        if (n->left < 0) {
            for (int64_t i = n->lo; i < n->hi; ++i) {
                const int64_t r = t->perm[i];
                const double dx = (double)t->ref[3 * r] - q[0];
                const double dy = (double)t->ref[3 * r + 1] - q[1];
                const double dz = (double)t->ref[3 * r + 2] - q[2];
                const double d2 = dx * dx + dy * dy + dz * dz;
                if (d2 < bd || (d2 == bd && r < best)) { bd = d2; best = r; }
            }
            continue;
        }
        const double dl = or_kd_box_d2(&t->node[n->left], q);
        const double dr = or_kd_box_d2(&t->node[n->right], q);
        /* push the farther child first so that the nearer one is walked first */
        if (dl <= dr) { stack[sp++] = n->right; stack[sp++] = n->left; }
        else { stack[sp++] = n->left; stack[sp++] = n->right; }
    }
    *d2_out = bd;
    return best;
}

/* or_nn through the tree: the same indices and distances. */
OR_EXPORT void or_kd_nn(const or_kdtree* t, const double* q, int64_t nq, int64_t* idx, double* d2) {
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t i = 0; i < nq; ++i) idx[i] = or_kd_nn_one(t, q + 3 * i, d2 + i);
}

/* ------------------------------------------------------------------------ */
/* Mean ICP gradient, Eqs. (trans_gradient) and (rotation_gradient), R3      */
/* ------------------------------------------------------------------------ */

/* Transform source point s by particle th: out = R s + u. */
static void or_transform(const double R[9], const double th[6], const float* s, double out[3]) {
    for (int r = 0; r < 3; ++r)
        out[r] = R[3 * r] * (double)s[0] + R[3 * r + 1] * (double)s[1] + R[3 * r + 2] * (double)s[2] + th[r];
}

/* gbar for one particle given its correspondences nn[0..m-1] (reference
 * indices of the minibatch points mb[0..m-1]).  Also returns L/2 over the
 * minibatch, (1/2m) sum ||R s + u - r||^2. */
static double or_grad_given_nn_one(const float* ref, const float* src, const int32_t* mb,
                                   int32_t m, const double th[6], const int64_t* nn,
                                   const double* normals, double g[6]) {
    double R[9], dR[27];
    or_rotation(th, R, dR);
    double acc[6] = {0, 0, 0, 0, 0, 0}, loss = 0.0;
    for (int32_t k = 0; k < m; ++k) {
        const float* s = src + 3 * (int64_t)mb[k];
        double sp[3], e[3];
        or_transform(R, th, s, sp);
        const float* r = ref + 3 * nn[k];
        for (int a = 0; a < 3; ++a) e[a] = sp[a] - (double)r[a];
        if (normals) {
            /* point-to-plane (R16): the residual vector becomes (n . e) n */
            const double* n = normals + 3 * nn[k];
            const double en = n[0] * e[0] + n[1] * e[1] + n[2] * e[2];
            for (int a = 0; a < 3; ++a) e[a] = en * n[a];
        }
        /* d s'/d u = I */
        for (int a = 0; a < 3; ++a) acc[a] += e[a];
        /* d s'/d theta_{3+a} = dR_a s */
        for (int a = 0; a < 3; ++a) {
            const double* D = dR + 9 * a;
            double js[3];
            for (int r2 = 0; r2 < 3; ++r2)
                js[r2] = D[3 * r2] * (double)s[0] + D[3 * r2 + 1] * (double)s[1] + D[3 * r2 + 2] * (double)s[2];
            acc[3 + a] += e[0] * js[0] + e[1] * js[1] + e[2] * js[2];
        }
        loss += e[0] * e[0] + e[1] * e[1] + e[2] * e[2];
    }
    for (int a = 0; a < 6; ++a) g[a] = acc[a] / (double)m;
    return loss / (2.0 * (double)m);
}

/* For each of K particles (th: K x 6): correspondences of the transformed
 * minibatch (nn_out: K x m, may be NULL) and gbar (K x 6).  loss_out (K, may be
 * NULL) receives L/2 over the minibatch.  normals (M x 3, may be NULL): the
 * point-to-plane metric (R16). */
static void or_icp_grad_tree(const float* ref, int64_t M, const or_kdtree* tree, const float* src,
                             const int32_t* mb, int32_t m, const double* th, int32_t K, const double* normals,
                             double* gbar, int64_t* nn_out, double* loss_out) {
    int64_t* nn = (int64_t*)malloc(sizeof(int64_t) * (size_t)K * (size_t)m);
    double* qs = (double*)malloc(sizeof(double) * 3 * (size_t)K * (size_t)m);
    for (int32_t j = 0; j < K; ++j) {
        double R[9];
        or_rotation(th + 6 * j, R, NULL);
        for (int32_t k = 0; k < m; ++k)
            or_transform(R, th + 6 * j, src + 3 * (int64_t)mb[k], qs + 3 * ((int64_t)j * m + k));
    }
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t q = 0; q < (int64_t)K * m; ++q) {
        double d2;
        nn[q] = tree ? or_kd_nn_one(tree, qs + 3 * q, &d2) : or_nn_one(ref, M, qs + 3 * q, &d2);
    }
    for (int32_t j = 0; j < K; ++j) {
        double l = or_grad_given_nn_one(ref, src, mb, m, th + 6 * j, nn + (int64_t)j * m, normals, gbar + 6 * j);
        if (loss_out) loss_out[j] = l;
    }
    if (nn_out) memcpy(nn_out, nn, sizeof(int64_t) * (size_t)K * (size_t)m);
    free(nn);
    free(qs);
}

OR_EXPORT void or_icp_grad(const float* ref, int64_t M, const float* src, const int32_t* mb,
                           int32_t m, const double* th, int32_t K, const double* normals, double* gbar,
                           int64_t* nn_out, double* loss_out) {
    or_icp_grad_tree(ref, M, NULL, src, mb, m, th, K, normals, gbar, nn_out, loss_out);
}

/* The same through a k-d tree of ref (or_kd_build): identical results. */
OR_EXPORT void or_icp_grad_kd(const or_kdtree* tree, const float* src, const int32_t* mb, int32_t m,
                              const double* th, int32_t K, const double* normals, double* gbar,
                              int64_t* nn_out, double* loss_out) {
    or_icp_grad_tree(tree->ref, tree->M, tree, src, mb, m, th, K, normals, gbar, nn_out, loss_out);
}

/* Same gradient with the correspondences given (K x m reference indices). */
OR_EXPORT void or_icp_grad_given_nn(const float* ref, const float* src, const int32_t* mb,
                                    int32_t m, const double* th, int32_t K, const int64_t* nn,
                                    const double* normals, double* gbar) {
    for (int32_t j = 0; j < K; ++j)
        or_grad_given_nn_one(ref, src, mb, m, th + 6 * j, nn + (int64_t)j * m, normals, gbar + 6 * j);
}

/* ------------------------------------------------------------------------ */
/* Reference normals for the point-to-plane metric (R16)                     */
/* ------------------------------------------------------------------------ */

/* The k nearest reference points of every reference point (itself included),
 * nearest first: exhaustive, exact fp64 squared distances, ties to the lower
 * index.  idx: M x k; d2 (M x k, may be NULL) the squared distances. */
OR_EXPORT void or_knn(const float* ref, int64_t M, int32_t k, int64_t* idx, double* d2_out) {
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t i = 0; i < M; ++i) {
        double bd[64];
        int64_t bi[64];
        int32_t n = 0;
        const double qx = ref[3 * i], qy = ref[3 * i + 1], qz = ref[3 * i + 2];
        for (int64_t r = 0; r < M; ++r) {
            const double dx = (double)ref[3 * r] - qx, dy = (double)ref[3 * r + 1] - qy, dz = (double)ref[3 * r + 2] - qz;
            const double d2 = dx * dx + dy * dy + dz * dz;
            if (n == k && !(d2 < bd[k - 1])) continue;      /* r > every kept index: equal loses */
            int32_t p = n < k ? n++ : k - 1;                /* insertion position from the end */
            while (p > 0 && d2 < bd[p - 1]) {
                bd[p] = bd[p - 1];
                bi[p] = bi[p - 1];
                --p;
            }
            bd[p] = d2;
            bi[p] = r;
        }
        for (int32_t c = 0; c < k; ++c) {
            idx[i * k + c] = c < n ? bi[c] : -1;
            if (d2_out) d2_out[i * k + c] = c < n ? bd[c] : INFINITY;
        }
    }
}

/* Covariance (divisor k) of each point's neighbourhood idx (M x k): M x 9. */
OR_EXPORT void or_neighbourhood_cov(const float* ref, int64_t M, int32_t k, const int64_t* idx, double* cov) {
    for (int64_t i = 0; i < M; ++i) {
        double mu[3] = {0, 0, 0};
        for (int32_t c = 0; c < k; ++c)
            for (int a = 0; a < 3; ++a) mu[a] += (double)ref[3 * idx[i * k + c] + a];
        for (int a = 0; a < 3; ++a) mu[a] /= (double)k;
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) {
                double s = 0.0;
                for (int32_t c = 0; c < k; ++c) {
                    const float* p = ref + 3 * idx[i * k + c];
                    s += ((double)p[a] - mu[a]) * ((double)p[b] - mu[b]);
                }
                cov[9 * i + 3 * a + b] = s / (double)k;
            }
    }
}

/* ------------------------------------------------------------------------ */
/* Priors, Eqs. (trans_prior) and (rot_prior), and G (Eq. posterior, R4)     */
/* ------------------------------------------------------------------------ */

/* G_j = -N gbar_j + grad log prior(theta_j).  prior: 0 uniform, 1 Gaussian
 * (translation, divided by sigma as printed, R6) + von Mises (rotation). */
OR_EXPORT void or_log_post_grad(const double* th, const double* gbar, int32_t K, double N,
                                int32_t prior, const double mu[6], const double sigma[3],
                                const double kappa[3], double* G) {
    for (int32_t j = 0; j < K; ++j)
        for (int a = 0; a < 6; ++a) {
            double p = 0.0;
            if (prior == 1) {
                if (a < 3) p = -(th[6 * j + a] - mu[a]) / sigma[a];
                else p = -kappa[a - 3] * sin(th[6 * j + a] - mu[a]);
            }
            G[6 * j + a] = -N * gbar[6 * j + a] + p;
        }
}

/* ------------------------------------------------------------------------ */
/* Median-heuristic bandwidths (R9) and the Stein direction, Eq. (stein_icp_phi) */
/* ------------------------------------------------------------------------ */

static int or_cmp_f64(const void* a, const void* b) {
    double x = *(const double*)a, y = *(const double*)b;
    return (x > y) - (x < y);
}

OR_EXPORT double or_median(const double* x, int64_t n) {
    double* c = (double*)malloc(sizeof(double) * (size_t)n);
    memcpy(c, x, sizeof(double) * (size_t)n);
    qsort(c, (size_t)n, sizeof(double), or_cmp_f64);
    double med = (n % 2) ? c[n / 2] : 0.5 * (c[n / 2 - 1] + c[n / 2]);
    free(c);
    return med;
}

static double or_wrap(double x) { return atan2(sin(x), cos(x)); }

/* Squared distance between particles j and l in the translation block (block
 * 0) or, with wrapped differences, in the rotation block (block 1). */
static double or_block_d2(const double* th, int32_t j, int32_t l, int block) {
    double s = 0.0;
    for (int a = 0; a < 3; ++a) {
        double d = th[6 * j + 3 * block + a] - th[6 * l + 3 * block + a];
        if (block == 1) d = or_wrap(d);
        s += d * d;
    }
    return s;
}

OR_EXPORT void or_bandwidths(const double* th, int32_t K, double* h_t, double* h_r) {
    int64_t n = (int64_t)K * K;
    double* D = (double*)malloc(sizeof(double) * (size_t)n);
    for (int block = 0; block < 2; ++block) {
        for (int32_t j = 0; j < K; ++j)
            for (int32_t l = 0; l < K; ++l) D[(int64_t)j * K + l] = or_block_d2(th, j, l, block);
        double med = or_median(D, n);
        double h = (med > 0.0) ? med / log((double)K + 1.0) : 1.0;
        if (block == 0) *h_t = h; else *h_r = h;
    }
    free(D);
}

/* phi_i = (1/K) sum_j [ k(theta_j, theta_i) G_j + grad_{theta_j} k(theta_j, theta_i) ]
 * per block, with k = exp(-D/h) and grad_{theta_j} k = (2/h)(theta_i - theta_j) k
 * (differences wrapped in the rotation block). */
OR_EXPORT void or_stein_phi(const double* th, const double* G, int32_t K, double h_t,
                            double h_r, double* phi) {
#pragma omp parallel for schedule(static)
    for (int32_t i = 0; i < K; ++i) {
        double acc[6] = {0, 0, 0, 0, 0, 0};
        for (int32_t j = 0; j < K; ++j) {
            for (int block = 0; block < 2; ++block) {
                double h = block ? h_r : h_t;
                double k = exp(-or_block_d2(th, j, i, block) / h);
                for (int a = 0; a < 3; ++a) {
                    int c = 3 * block + a;
                    double diff = th[6 * i + c] - th[6 * j + c];
                    if (block == 1) diff = or_wrap(diff);
                    acc[c] += k * G[6 * j + c] + (2.0 / h) * diff * k;
                }
            }
        }
        for (int c = 0; c < 6; ++c) phi[6 * i + c] = acc[c] / (double)K;
    }
}

/* ------------------------------------------------------------------------ */
/* Adam (Kingma & Ba), R10: descent on g = -phi                              */
/* ------------------------------------------------------------------------ */

OR_EXPORT void or_adam(double* x, double* mom, double* vel, const double* g, int64_t n,
                       int64_t t, double lr, double b1, double b2, double eps) {
    double c1 = 1.0 - pow(b1, (double)t), c2 = 1.0 - pow(b2, (double)t);
    for (int64_t i = 0; i < n; ++i) {
        mom[i] = b1 * mom[i] + (1.0 - b1) * g[i];
        vel[i] = b2 * vel[i] + (1.0 - b2) * g[i] * g[i];
        double mh = mom[i] / c1, vh = vel[i] / c2;
        x[i] -= lr * mh / (sqrt(vh) + eps);
    }
}

/* ------------------------------------------------------------------------ */
/* Particle mean and covariance                                              */
/* ------------------------------------------------------------------------ */

OR_EXPORT void or_moments(const double* th, int32_t K, double mean[6], double cov[36]) {
    for (int a = 0; a < 6; ++a) {
        double s = 0.0;
        for (int32_t j = 0; j < K; ++j) s += th[6 * j + a];
        mean[a] = s / (double)K;
    }
    for (int a = 0; a < 6; ++a)
        for (int b = 0; b < 6; ++b) {
            double s = 0.0;
            for (int32_t j = 0; j < K; ++j) s += (th[6 * j + a] - mean[a]) * (th[6 * j + b] - mean[b]);
            cov[6 * a + b] = (K > 1) ? s / (double)(K - 1) : 0.0;
        }
}

/* Circular moments (R15): translation as or_moments, rotation angles by their
 * circular mean, covariance of the wrapped deviations. */
OR_EXPORT void or_moments_circular(const double* th, int32_t K, double mean[6], double cov[36]) {
    for (int a = 0; a < 6; ++a) {
        if (a < 3) {
            double s = 0.0;
            for (int32_t j = 0; j < K; ++j) s += th[6 * j + a];
            mean[a] = s / (double)K;
        } else {
            double ss = 0.0, sc = 0.0;
            for (int32_t j = 0; j < K; ++j) {
                ss += sin(th[6 * j + a]);
                sc += cos(th[6 * j + a]);
            }
            mean[a] = (ss == 0.0 && sc == 0.0) ? 0.0 : atan2(ss, sc);
        }
    }
    for (int a = 0; a < 6; ++a)
        for (int b = 0; b < 6; ++b) {
            double s = 0.0;
            for (int32_t j = 0; j < K; ++j) {
                double da = th[6 * j + a] - mean[a], db = th[6 * j + b] - mean[b];
                if (a >= 3) da = or_wrap(da);
                if (b >= 3) db = or_wrap(db);
                s += da * db;
            }
            cov[6 * a + b] = (K > 1) ? s / (double)(K - 1) : 0.0;
        }
}

/* ------------------------------------------------------------------------ */
/* One Stein ICP iteration and a whole run (Sec. IV, summary paragraph)      */
/* ------------------------------------------------------------------------ */

typedef struct {
    int32_t T, m;
    double lr, beta1, beta2, eps;
    uint64_t seed;
    int32_t prior;
    double mu[6], sigma[3], kappa[3];
    const double* normals;   /* NULL: point-to-point; else M x 3: point-to-plane (R16) */
    int32_t independent;     /* 1: independent SGD-ICP runs, phi_j = G_j (R17) */
    const or_kdtree* tree;   /* NULL: exhaustive search; else a k-d tree of ref (same answers, faster) */
} or_params;

/* Iteration t (0-based) in place on th, mom, vel (each K x 6).  Optional
 * outputs of this iteration (NULL to skip): gbar, G, phi (K x 6), h[2]. */
OR_EXPORT void or_step(const float* ref, int64_t M, const float* src, int64_t N,
                       double* th, double* mom, double* vel, int32_t K, const or_params* p,
                       int64_t t, double* gbar_out, double* G_out, double* phi_out,
                       double* h_out) {
    int32_t* mb = (int32_t*)malloc(sizeof(int32_t) * (size_t)p->m);
    double* gbar = (double*)malloc(sizeof(double) * 6 * (size_t)K);
    double* G = (double*)malloc(sizeof(double) * 6 * (size_t)K);
    double* phi = (double*)malloc(sizeof(double) * 6 * (size_t)K);
    double* g = (double*)malloc(sizeof(double) * 6 * (size_t)K);
    if (p->independent) {
        for (int32_t j = 0; j < K; ++j) {
            or_minibatch(p->seed + (uint64_t)j, t, N, p->m, mb);
            or_icp_grad_tree(ref, M, p->tree, src, mb, p->m, th + 6 * j, 1, p->normals, gbar + 6 * j, NULL, NULL);
        }
    } else {
        or_minibatch(p->seed, t, N, p->m, mb);
        or_icp_grad_tree(ref, M, p->tree, src, mb, p->m, th, K, p->normals, gbar, NULL, NULL);
    }
    or_log_post_grad(th, gbar, K, (double)N, p->prior, p->mu, p->sigma, p->kappa, G);
    double h_t = 1.0, h_r = 1.0;
    if (p->independent) {
        memcpy(phi, G, sizeof(double) * 6 * (size_t)K);
    } else {
        or_bandwidths(th, K, &h_t, &h_r);
        or_stein_phi(th, G, K, h_t, h_r, phi);
    }
    for (int64_t i = 0; i < 6 * (int64_t)K; ++i) g[i] = -phi[i];
    or_adam(th, mom, vel, g, 6 * (int64_t)K, t + 1, p->lr, p->beta1, p->beta2, p->eps);
    if (gbar_out) memcpy(gbar_out, gbar, sizeof(double) * 6 * (size_t)K);
    if (G_out) memcpy(G_out, G, sizeof(double) * 6 * (size_t)K);
    if (phi_out) memcpy(phi_out, phi, sizeof(double) * 6 * (size_t)K);
    if (h_out) { h_out[0] = h_t; h_out[1] = h_r; }
    free(mb); free(gbar); free(G); free(phi); free(g);
}

/* Whole run: T iterations from th0 (K x 6, float32 like the library's input).
 * Outputs final particles (K x 6 doubles), mean[6], cov[36]. */
OR_EXPORT int or_register(const float* ref, int64_t M, const float* src, int64_t N,
                          const float* th0, int32_t K, const or_params* p,
                          double* th_out, double* mean, double* cov) {
    if (M < 1 || N < 1 || K < 1 || p->m < 1 || p->m > N || p->T < 0) return -1;
    double* mom = (double*)calloc(6 * (size_t)K, sizeof(double));
    double* vel = (double*)calloc(6 * (size_t)K, sizeof(double));
    for (int64_t i = 0; i < 6 * (int64_t)K; ++i) th_out[i] = (double)th0[i];
    for (int64_t t = 0; t < p->T; ++t)
        or_step(ref, M, src, N, th_out, mom, vel, K, p, t, NULL, NULL, NULL, NULL);
    or_moments(th_out, K, mean, cov);
    free(mom); free(vel);
    return 0;
}

OR_EXPORT int or_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Threads for the parallel loops that follow (n >= 1); timing only, the
 * results do not depend on it. */
OR_EXPORT void or_set_threads(int n) {
#ifdef _OPENMP
    if (n >= 1) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

/* ------------------------------------------------------------------------ */
/* Learned closest-point field (the surrogate of the correspondence search)  */
/* ------------------------------------------------------------------------ */
/*
 * An MLP maps a normalised query q~ = (q - c) / s to the displacement d~ to
 * its nearest reference point (in the same normalised units) and a
 * confidence logit z.  Features: q~ (3 values), then sin and cos of
 * w_f q~_a for frequencies w_f = pi 2^(8 f / 15), f = 0..15, a = 0..2
 * (96 values, index 3 + 6 f + 2 a), then zeros up to 112.
 * Layers: 112 -> 128 (ReLU) -> 128 (ReLU) -> 16, of which outputs 0..2 are
 * d~ and output 3 is z.  Parameters, flat: W1[128][112], b1[128],
 * W2[128][128], b2[128], W3[16][128], b3[16] (33,040 values).
 * Loss over n samples with targets d~*:
 *   (1/n) sum_b [ |d~ - d~*|^2 + lam * (softplus(z) - c* z) ],
 *   c* = exp(-|d~ - d~*|^2 / delta^2), held constant (not differentiated).
 * bf16ops = 1 rounds the operands of every product to bfloat16 (round to
 * nearest even) the way the tensor-core kernels store them: the features,
 * the weights, the hidden activations, and the back-propagated deltas fed to
 * the next product; accumulation stays in double.
 */
#define OR_D_IN 112
#define OR_H 128
#define OR_D_OUT 16
#define OR_NPARAM (OR_H * OR_D_IN + OR_H + OR_H * OR_H + OR_H + OR_D_OUT * OR_H + OR_D_OUT)

OR_EXPORT int or_mlp_nparam(void) { return OR_NPARAM; }

/* Round a double to the nearest bfloat16 value (ties to even), via float. */
OR_EXPORT double or_bf16(double x) {
    float f = (float)x;
    uint32_t u;
    memcpy(&u, &f, 4);
    if ((u & 0x7f800000u) == 0x7f800000u) return x;       /* inf / nan */
    u = (u + 0x7fffu + ((u >> 16) & 1u)) & 0xffff0000u;
    memcpy(&f, &u, 4);
    return (double)f;
}

static double or_q(double x, int bf) { return bf ? or_bf16(x) : x; }

OR_EXPORT void or_mlp_features(const double qn[3], double x[OR_D_IN]) {
    const double pi = 3.14159265358979323846;
    for (int i = 0; i < OR_D_IN; ++i) x[i] = 0.0;
    for (int a = 0; a < 3; ++a) x[a] = qn[a];
    for (int f = 0; f < 16; ++f) {
        double w = pi * pow(2.0, 8.0 * f / 15.0);
        for (int a = 0; a < 3; ++a) {
            x[3 + 6 * f + 2 * a] = sin(w * qn[a]);
            x[3 + 6 * f + 2 * a + 1] = cos(w * qn[a]);
        }
    }
}

typedef struct {
    const double *W1, *b1, *W2, *b2, *W3, *b3;
} or_mlp;

static or_mlp or_mlp_view(const double* p) {
    or_mlp m;
    m.W1 = p;
    m.b1 = m.W1 + OR_H * OR_D_IN;
    m.W2 = m.b1 + OR_H;
    m.b2 = m.W2 + OR_H * OR_H;
    m.W3 = m.b2 + OR_H;
    m.b3 = m.W3 + OR_D_OUT * OR_H;
    return m;
}

/* Forward pass of one sample: the (possibly rounded) features x, hidden
 * activations h1, h2 as fed to the next product, and the 16 outputs. */
static void or_mlp_fwd1(const or_mlp* m, const double xin[OR_D_IN], int bf, double x[OR_D_IN], double h1[OR_H],
                        double h2[OR_H], double out[OR_D_OUT]) {
    for (int i = 0; i < OR_D_IN; ++i) x[i] = or_q(xin[i], bf);
    for (int j = 0; j < OR_H; ++j) {
        double s = 0.0;
        for (int i = 0; i < OR_D_IN; ++i) s += or_q(m->W1[j * OR_D_IN + i], bf) * x[i];
        s += m->b1[j];
        h1[j] = or_q(s > 0.0 ? s : 0.0, bf);
    }
    for (int j = 0; j < OR_H; ++j) {
        double s = 0.0;
        for (int i = 0; i < OR_H; ++i) s += or_q(m->W2[j * OR_H + i], bf) * h1[i];
        s += m->b2[j];
        h2[j] = or_q(s > 0.0 ? s : 0.0, bf);
    }
    for (int o = 0; o < OR_D_OUT; ++o) {
        double s = 0.0;
        for (int i = 0; i < OR_H; ++i) s += or_q(m->W3[o * OR_H + i], bf) * h2[i];
        out[o] = s + m->b3[o];
    }
}

/* Outputs (n x 16) for normalised queries qn (n x 3). */
OR_EXPORT void or_mlp_forward(const double* params, const double* qn, int64_t n, int bf16ops, double* out) {
    or_mlp m = or_mlp_view(params);
#pragma omp parallel for schedule(static)
    for (int64_t b = 0; b < n; ++b) {
        double xin[OR_D_IN], x[OR_D_IN], h1[OR_H], h2[OR_H];
        or_mlp_features(qn + 3 * b, xin);
        or_mlp_fwd1(&m, xin, bf16ops, x, h1, h2, out + OR_D_OUT * b);
    }
}

/* Loss and its gradient with respect to all parameters (grad: OR_NPARAM).
 * cstar_fixed (n, may be NULL) overrides the confidence targets. */
OR_EXPORT double or_mlp_loss_grad(const double* params, const double* qn, const double* dstar, int64_t n,
                                  double lam, double delta, int bf16ops, const double* cstar_fixed, double* grad) {
    or_mlp m = or_mlp_view(params);
    for (int i = 0; i < OR_NPARAM; ++i) grad[i] = 0.0;
    double* gW1 = grad;
    double* gb1 = gW1 + OR_H * OR_D_IN;
    double* gW2 = gb1 + OR_H;
    double* gb2 = gW2 + OR_H * OR_H;
    double* gW3 = gb2 + OR_H;
    double* gb3 = gW3 + OR_D_OUT * OR_H;
    const int bf = bf16ops;
    double loss = 0.0;
    for (int64_t b = 0; b < n; ++b) {
        double xin[OR_D_IN], x[OR_D_IN], h1[OR_H], h2[OR_H], out[OR_D_OUT];
        or_mlp_features(qn + 3 * b, xin);
        or_mlp_fwd1(&m, xin, bf, x, h1, h2, out);
        const double* t = dstar + 3 * b;
        double e2 = 0.0;
        for (int a = 0; a < 3; ++a) e2 += (out[a] - t[a]) * (out[a] - t[a]);
        const double cs = cstar_fixed ? cstar_fixed[b] : exp(-e2 / (delta * delta));
        const double z = out[3];
        const double sp = z > 0 ? z + log1p(exp(-z)) : log1p(exp(z));
        loss += e2 + lam * (sp - cs * z);
        /* delta of the outputs (per sample; the 1/n is applied at the end) */
        double d3[OR_D_OUT];
        for (int o = 0; o < OR_D_OUT; ++o) d3[o] = 0.0;
        for (int a = 0; a < 3; ++a) d3[a] = 2.0 * (out[a] - t[a]);
        d3[3] = lam * (1.0 / (1.0 + exp(-z)) - cs);
        for (int o = 0; o < OR_D_OUT; ++o) {
            gb3[o] += d3[o];
            for (int i = 0; i < OR_H; ++i) gW3[o * OR_H + i] += d3[o] * h2[i];
        }
        double d3q[OR_D_OUT], d2[OR_H], d1[OR_H];
        for (int o = 0; o < OR_D_OUT; ++o) d3q[o] = or_q(d3[o], bf);
        for (int i = 0; i < OR_H; ++i) {
            double s = 0.0;
            for (int o = 0; o < OR_D_OUT; ++o) s += or_q(m.W3[o * OR_H + i], bf) * d3q[o];
            d2[i] = or_q(h2[i] > 0.0 ? s : 0.0, bf);
        }
        for (int j = 0; j < OR_H; ++j) {
            gb2[j] += d2[j];
            for (int i = 0; i < OR_H; ++i) gW2[j * OR_H + i] += d2[j] * h1[i];
        }
        for (int i = 0; i < OR_H; ++i) {
            double s = 0.0;
            for (int j = 0; j < OR_H; ++j) s += or_q(m.W2[j * OR_H + i], bf) * d2[j];
            d1[i] = or_q(h1[i] > 0.0 ? s : 0.0, bf);
        }
        for (int j = 0; j < OR_H; ++j) {
            gb1[j] += d1[j];
            for (int i = 0; i < OR_D_IN; ++i) gW1[j * OR_D_IN + i] += d1[j] * x[i];
        }
    }
    for (int i = 0; i < OR_NPARAM; ++i) grad[i] /= (double)n;
    return loss / (double)n;
}
