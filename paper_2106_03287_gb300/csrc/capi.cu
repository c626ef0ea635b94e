// C ABI of libsteinicp: context, argument checks, staging of host or device
// buffers, and the registration loop (captured once per shape into a CUDA
// graph and replayed).
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <vector>

#include "common.cuh"
#include "nvtx.cuh"

namespace sicp {

int set_err(sicp_ctx* c, int code, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (c) c->err = buf;
    return code;
}

std::vector<CheckReader>& check_registry() {
    static std::vector<CheckReader> r;
    return r;
}

void check_register(CheckReader r) { check_registry().push_back(r); }

#ifdef SICP_CHECKED
constexpr int32_t kCheckedBuild = 1;
#else
constexpr int32_t kCheckedBuild = 0;
#endif

int cuda_err(sicp_ctx* c, cudaError_t e, const char* what) {
    set_err(c, SICP_ECUDA, "%s: %s", what, cudaGetErrorString(e));
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        return SICP_ENOMEM;
    }
    return SICP_ECUDA;
}

int budget_malloc(sicp_ctx* c, void** p, size_t bytes, size_t held) {
    *p = nullptr;
    c->mem_used -= held < c->mem_used ? held : c->mem_used;
    if (c->mem_limit && c->mem_used + bytes > c->mem_limit)
        return set_err(c, SICP_ENOMEM, "device allocation of %zu bytes would pass the context's budget of %zu bytes "
                       "(%zu held)", bytes, c->mem_limit, c->mem_used);
    if (cudaMalloc(p, bytes) != cudaSuccess) {
        *p = nullptr;
        cudaGetLastError();
        return set_err(c, SICP_ENOMEM, "device allocation of %zu bytes failed", bytes);
    }
    c->mem_used += bytes;
    return SICP_OK;
}

int ensure(sicp_ctx* c, Buf& b, size_t bytes) {
    if (bytes == 0) bytes = 16;
    if (b.cap >= bytes) return SICP_OK;
    const size_t held = b.cap;
    if (b.p) cudaFree(b.p);
    b.p = nullptr;
    b.cap = 0;
    const size_t want = bytes + bytes / 4;   // headroom so nearby sizes reuse the buffer
    int rc = budget_malloc(c, &b.p, want, held);
    if (rc) return rc;
    b.cap = want;
    return SICP_OK;
}

// Key of a captured registration loop: everything its kernels read as arguments.
struct LoopKey {
    int64_t N;
    int32_t K, T, m, mode, chunks, stride, tel;   // tel: telemetry rows recorded
    int32_t pi[4];          // T, m, nn_mode, prior
    float pf[16];           // lr, betas, eps, prior mu/sigma/kappa
    int32_t surr_iters;
    float min_conf;
    uint64_t surr_gen;      // surrogate weights / normalisation version
    uint64_t seed;
    int64_t t0;             // first iteration of the run
    int64_t ref_M;          // reference size (the exhaustive kernel takes it by value)
    int64_t wait_polls;     // failure-detection check settings (the kernels take them by value)
    int32_t wait_never, pad2;
    const void* ptrs[16];
    bool operator==(const LoopKey& o) const { return memcmp(this, &o, sizeof *this) == 0; }
};

// One instantiated registration graph.  With profiling on, the graph also
// records three events per profiled iteration (before the gradient kernel,
// between it and the Stein kernel, after the Stein kernel).
struct GraphSlot {
    bool valid = false;
    LoopKey key;
    cudaGraphExec_t exec = nullptr;
    std::vector<cudaEvent_t> ev;
    int n_prof = 0;
    bool pending = false;   // events recorded by a finished launch, not yet read
};

// Two slots alternate while profiling, so the events of one run are read on
// the host while the next run executes on the GPU.
struct GraphCache {
    GraphSlot slot[2];
    int next = 0;
    ~GraphCache() {
        for (GraphSlot& s : slot) {
            if (s.exec) cudaGraphExecDestroy(s.exec);
            for (cudaEvent_t e : s.ev) cudaEventDestroy(e);
        }
    }
};

}  // namespace sicp

using namespace sicp;

namespace {

struct DeviceScope {
    int prev = -1;
    explicit DeviceScope(int d) {
        cudaGetDevice(&prev);
        if (prev != d) cudaSetDevice(d);
    }
    ~DeviceScope() {
        int cur = -1;
        cudaGetDevice(&cur);
        if (prev >= 0 && cur != prev) cudaSetDevice(prev);
    }
};

bool host_finite(const float* x, int64_t n) {
    for (int64_t i = 0; i < n; ++i)
        if (!isfinite(x[i])) return false;
    return true;
}

// Make an input visible to the device: device pointers pass through, host
// buffers are copied into the context buffer `tmp`.
int stage_in(sicp_ctx* ctx, const void* p, size_t bytes, int on_device, Buf& tmp, const void** out) {
    if (on_device) {
        *out = p;
        return SICP_OK;
    }
    int rc = ensure(ctx, tmp, bytes);
    if (rc) return rc;
    SICP_CUDA(cudaMemcpyAsync(tmp.p, p, bytes, cudaMemcpyHostToDevice, ctx->stream));
    *out = tmp.p;
    return SICP_OK;
}

int copy_out(sicp_ctx* ctx, void* dst, const void* src_dev, size_t bytes, int on_device) {
    if (!dst || bytes == 0) return SICP_OK;
    SICP_CUDA(cudaMemcpyAsync(dst, src_dev, bytes, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                              ctx->stream));
    return SICP_OK;
}

int sync(sicp_ctx* ctx) {
    SICP_CUDA(cudaStreamSynchronize(ctx->stream));
    return SICP_OK;
}

int read_flags(sicp_ctx* ctx, int* flags_host) {
    SICP_CUDA(cudaMemcpyAsync(flags_host, ctx->flags.p, 4 * sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    return sync(ctx);
}

// Search mode plus flags: `allowed` is the set of flag bits the caller accepts.
int check_mode(sicp_ctx* ctx, int32_t mode, int32_t allowed, bool allow_surrogate) {
    const int32_t flags = mode & (SICP_POINT_TO_PLANE | SICP_INDEPENDENT);
    if (flags & ~allowed) return set_err(ctx, SICP_EINVAL, "mode flags 0x%x are not accepted here", flags & ~allowed);
    mode &= ~flags;
    if (flags & SICP_POINT_TO_PLANE) {
        if (mode != SICP_NN_GRID && mode != SICP_NN_BRUTE_FP32 && mode != SICP_NN_BRUTE_BF16)
            return set_err(ctx, SICP_EINVAL, "the point-to-plane metric works with the exact searches (grid, FP32, BF16)");
        if (ctx->normals_k == 0)
            return set_err(ctx, SICP_ENOREF, "the point-to-plane metric needs sicp_reference_normals on this reference");
        return SICP_OK;
    }
    if (mode == SICP_NN_BRUTE_FP32 || mode == SICP_NN_GRID || mode == SICP_NN_BRUTE_BF16) return SICP_OK;
    if (mode == SICP_NN_SURROGATE && allow_surrogate) {
        if (surrogate_ready(ctx)) return SICP_OK;
        return set_err(ctx, SICP_ENOSURROGATE, "no trained surrogate on this context");
    }
    return set_err(ctx, SICP_EINVAL, "unknown nn_mode %d", mode);
}

void fill_defaults(sicp_params* p) {
    memset(p, 0, sizeof *p);
    p->T = 100;
    p->m = 100;
    p->lr = 0.01f;
    p->beta1 = 0.9f;
    p->beta2 = 0.999f;
    p->eps = 1e-8f;
    p->nn_mode = SICP_NN_GRID;
    p->surrogate_min_conf = 0.5f;
    for (int a = 0; a < 3; ++a) {
        p->prior_sigma[a] = 1.f;
        p->prior_kappa[a] = 1.f;
    }
}

// Adam constants default when left zero.
sicp_params normalise(const sicp_params* in) {
    sicp_params p = *in;
    if (p.beta1 == 0.f) p.beta1 = 0.9f;
    if (p.beta2 == 0.f) p.beta2 = 0.999f;
    if (p.eps == 0.f) p.eps = 1e-8f;
    return p;
}

int check_params(sicp_ctx* ctx, const sicp_params& p) {
    if (!(p.beta1 >= 0.5f && p.beta1 < 1.f) || !(p.beta2 >= 0.5f && p.beta2 < 1.f))
        return set_err(ctx, SICP_EINVAL, "Adam betas must lie in [0.5, 1)");
    if (!(p.eps > 0.f) || !isfinite(p.lr) || !(p.lr >= 0.f))
        return set_err(ctx, SICP_EINVAL, "lr must be finite and >= 0, eps > 0");
    if (p.prior != 0 && p.prior != 1) return set_err(ctx, SICP_EINVAL, "prior must be 0 or 1");
    if (p.surrogate_iters < 0) return set_err(ctx, SICP_EINVAL, "surrogate_iters must be >= 0");
    if (!(p.surrogate_min_conf >= 0.f && p.surrogate_min_conf <= 1.f))
        return set_err(ctx, SICP_EINVAL, "surrogate_min_conf must lie in [0, 1]");
    if (p.prior == 1) {
        for (int a = 0; a < 3; ++a)
            if (!(p.prior_sigma[a] > 0.f) || !(p.prior_kappa[a] >= 0.f))
                return set_err(ctx, SICP_EINVAL, "prior sigma must be > 0 and kappa >= 0");
    }
    return SICP_OK;
}

SteinArgs stein_args(const sicp_params& p, float* theta, float* am, float* av, const float* partial,
                     int32_t chunks, float inv_m, int32_t K, float N, int64_t t) {
    SteinArgs a;
    a.theta = theta;
    a.adam_m = am;
    a.adam_v = av;
    a.partial = partial;
    a.chunks = chunks;
    a.inv_m = inv_m;
    a.K = K;
    a.N = N;
    a.t = t;
    a.lr = p.lr;
    a.beta1 = p.beta1;
    a.beta2 = p.beta2;
    a.eps = p.eps;
    a.prior = p.prior;
    for (int c = 0; c < 6; ++c) a.mu[c] = p.prior_mu[c];
    for (int c = 0; c < 3; ++c) {
        a.sigma[c] = p.prior_sigma[c];
        a.kappa[c] = p.prior_kappa[c];
    }
    a.out_phi = nullptr;
    a.out_gbar = nullptr;
    a.out_h = nullptr;
    a.med_state = nullptr;
    a.arrive = nullptr;
    a.err = nullptr;
    a.gen = 0;
    a.max_spins = 0;
    a.extra = 0;
    a.cache = 1;
    return a;
}

unsigned long long* stats_ptr(sicp_ctx* ctx) {
    return ctx->stats_on ? (unsigned long long*)ctx->stats.p : nullptr;
}

// Add the kernel durations recorded by a finished launch of `s` to the totals.
void collect_profile(sicp_ctx* ctx, GraphSlot& s) {
    if (!s.pending) return;
    for (int i = 0; i < s.n_prof; ++i) {
        float a = 0.f, b = 0.f;
        if (cudaEventElapsedTime(&a, s.ev[3 * i], s.ev[3 * i + 1]) == cudaSuccess &&
            cudaEventElapsedTime(&b, s.ev[3 * i + 1], s.ev[3 * i + 2]) == cudaSuccess) {
            ctx->prof[0] += a;
            ctx->prof[1] += 1;
            ctx->prof[2] += b;
            ctx->prof[3] += 1;
        } else {
            cudaGetLastError();
        }
    }
    s.pending = false;
}

cudaError_t launch_grad(sicp_ctx* ctx, int32_t mode, const GradArgs& g) {
    if (mode == SICP_NN_GRID)
        return launch_grad_grid(g, (const GridSearch*)ctx->search_dev.p, ctx->search_slot, ctx->stream);
    return launch_grad_brute(g, ctx->ref4, ctx->M, ctx->stream);
}

constexpr int32_t kMaxK = 2048;
constexpr float kSurrogateIcpGradConf = 0.5f;   // confidence threshold of sicp_icp_grad's surrogate mode
constexpr int64_t kMaxN = 0x7fffffff;
constexpr int64_t kMaxM = (int64_t)1 << 30;

}  // namespace

extern "C" {

void sicp_default_params(sicp_params* p) {
    if (p) fill_defaults(p);
}

int sicp_create(sicp_ctx** out, int device, void* cuda_stream) {
    if (!out) return SICP_EINVAL;
    *out = nullptr;
    int n = 0;
    if (cudaGetDeviceCount(&n) != cudaSuccess || device < 0 || device >= n) {
        cudaGetLastError();
        return SICP_ECUDA;
    }
    sicp_ctx* c = new sicp_ctx();
    c->device = device;
    DeviceScope ds(device);
    cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device);
    if (cuda_stream) {
        c->stream = (cudaStream_t)cuda_stream;
    } else {
        if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess) {
            delete c;
            return SICP_ECUDA;
        }
        c->own_stream = true;
    }
    c->graphs = new GraphCache();
    if (kernel_attrs_init() != cudaSuccess || surrogate_kernel_attrs() != cudaSuccess ||
        bf16_kernel_attrs() != cudaSuccess || minibatch_kernel_attrs() != cudaSuccess) {
        cudaGetLastError();
        sicp_destroy(c);
        return SICP_ECUDA;
    }
    if (search_table_init(c) != SICP_OK) {
        sicp_destroy(c);
        return SICP_ENOMEM;
    }
    if (ensure(c, c->flags, 4 * sizeof(int)) != SICP_OK) {
        sicp_destroy(c);
        return SICP_ENOMEM;
    }
    *out = c;
    return SICP_OK;
}

void sicp_destroy(sicp_ctx* c) {
    if (!c) return;
    DeviceScope ds(c->device);
    if (c->stream) cudaStreamSynchronize(c->stream);
    delete c->graphs;
    search_slot_release(c->search_slot);
    if (c->batch) batch_destroy(c->batch);
    if (c->surr) surrogate_destroy(c->surr);
    Buf* bufs[] = {&c->src4, &c->mb, &c->theta, &c->adam_m, &c->adam_v, &c->partial, &c->moments,
                   &c->flags, &c->tmp_in, &c->tmp_out, &c->tmp_aux, &c->bbox, &c->stats, &c->gbar,
                   &c->bf16_tiles, &c->normals, &c->search_dev, &c->bf16_ref, &c->bf16_order, &c->bf16_q, &c->resume, &c->tel,
                   &c->tel_nn, &c->tel_part};
    for (Buf* b : bufs)
        if (b->p) cudaFree(b->p);
    if (c->ref4) cudaFree(c->ref4);
    for (Grid* g : {&c->grid, &c->grid2}) {
        void* gp[] = {g->sorted, g->cell_start, g->cell_of, g->counts, g->scan_sums, g->seed,
                      g->seed_tmp, g->seed4};
        for (void* p : gp)
            if (p) cudaFree(p);
    }
    if (c->tab_off) cudaFree(c->tab_off);
    if (c->tab_lb) cudaFree(c->tab_lb);
    if (c->own_stream) cudaStreamDestroy(c->stream);
    delete c;
}

const char* sicp_last_error(const sicp_ctx* c) { return c ? c->err.c_str() : "null context"; }

int sicp_set_reference(sicp_ctx* ctx, const float* xyz, int64_t M, float cell_size, int on_device) {
    NvtxRange nvtx_("reference_build");
    if (!ctx) return SICP_EINVAL;
    ctx->err.clear();
    if (!xyz || M < 1 || M > kMaxM) return set_err(ctx, SICP_EINVAL, "reference needs 1 <= M <= 2^30 points");
    if (!(cell_size >= 0.f) || !isfinite(cell_size)) return set_err(ctx, SICP_EINVAL, "cell_size must be >= 0");
    if (!on_device && !host_finite(xyz, 3 * M)) return set_err(ctx, SICP_EINVAL, "non-finite reference coordinate");
    DeviceScope ds(ctx->device);
    const void* d_xyz;
    int rc = stage_in(ctx, xyz, sizeof(float) * 3 * M, on_device, ctx->tmp_in, &d_xyz);
    if (rc) return rc;
    if ((size_t)M > ctx->ref_cap) {
        const size_t held = sizeof(float4) * ctx->ref_cap;
        if (ctx->ref4) cudaFree(ctx->ref4);
        ctx->ref4 = nullptr;
        ctx->ref_cap = 0;
        ctx->M = 0;   // the old reference is gone
        if ((rc = budget_malloc(ctx, (void**)&ctx->ref4, sizeof(float4) * M, held))) return rc;
        ctx->ref_cap = M;
    }
    ctx->M = 0;
    surrogate_invalidate(ctx);   // a surrogate belongs to the reference it was trained on
    ctx->bf16_ready = false;
    ctx->normals_k = 0;          // and so do normals
    SICP_CUDA(cudaMemsetAsync(ctx->flags.p, 0, 4 * sizeof(int), ctx->stream));
    SICP_CUDA(launch_pack_points((const float*)d_xyz, M, ctx->ref4, (int*)ctx->flags.p, ctx->stream));
    int flags[4];
    rc = read_flags(ctx, flags);
    if (rc) return rc;
    if (flags[0]) return set_err(ctx, SICP_EINVAL, "non-finite reference coordinate");
    ctx->M = M;
    rc = grid_build(ctx, cell_size);
    if (rc) {
        ctx->M = 0;
        return rc;
    }
    // captured loops stay valid: their kernels read the reference's description from device memory
    return sync(ctx);
}

int sicp_minibatch(sicp_ctx* ctx, uint64_t seed, int64_t t0, int32_t T, int64_t N, int32_t m,
                   int32_t* out_idx, int on_device) {
    NvtxRange nvtx_("sample");
    if (!ctx) return SICP_EINVAL;
    ctx->err.clear();
    if (!out_idx || T < 1 || t0 < 0 || N < 1 || N > kMaxN || m < 1 || m > N)
        return set_err(ctx, SICP_EINVAL, "minibatch needs T >= 1, t0 >= 0, 1 <= m <= N < 2^31");
    DeviceScope ds(ctx->device);
    const size_t bytes = sizeof(int32_t) * (size_t)T * m;
    int32_t* dst = out_idx;
    if (!on_device) {
        int rc = ensure(ctx, ctx->tmp_out, bytes);
        if (rc) return rc;
        dst = (int32_t*)ctx->tmp_out.p;
    }
    SICP_CUDA(launch_minibatch(seed, t0, T, N, m, dst, ctx->stream));
    if (!on_device) {
        int rc = copy_out(ctx, out_idx, dst, bytes, 0);
        if (rc) return rc;
    }
    return sync(ctx);
}

int sicp_nn(sicp_ctx* ctx, const float* q, int64_t n, int32_t mode, int32_t* out_idx, float* out_d2,
            int on_device) {
    NvtxRange nvtx_("nn");
    if (!ctx) return SICP_EINVAL;
    ctx->err.clear();
    if (n < 0 || n > kMaxN) return set_err(ctx, SICP_EINVAL, "query count out of range");
    if (n == 0) return SICP_OK;
    if (!q || !out_idx) return set_err(ctx, SICP_EINVAL, "null query or output pointer");
    int rc = check_mode(ctx, mode, 0, false);
    if (rc) return rc;
    if (ctx->M < 1) return set_err(ctx, SICP_ENOREF, "no reference cloud set");
    if (!on_device && !host_finite(q, 3 * n)) return set_err(ctx, SICP_EINVAL, "non-finite query");
    DeviceScope ds(ctx->device);
    const void* d_q;
    rc = stage_in(ctx, q, sizeof(float) * 3 * n, on_device, ctx->tmp_in, &d_q);
    if (rc) return rc;
    int32_t* d_idx = out_idx;
    float* d_d2 = out_d2;
    if (!on_device) {
        rc = ensure(ctx, ctx->tmp_out, (sizeof(int32_t) + sizeof(float)) * n);
        if (rc) return rc;
        d_idx = (int32_t*)ctx->tmp_out.p;
        d_d2 = (float*)((char*)ctx->tmp_out.p + sizeof(int32_t) * n);
    }
    SICP_CUDA(cudaMemsetAsync(ctx->flags.p, 0, 4 * sizeof(int), ctx->stream));
    if (on_device) SICP_CUDA(launch_check_finite((const float*)d_q, 3 * n, (int*)ctx->flags.p, ctx->stream));
    if (mode == SICP_NN_GRID) {
        SICP_CUDA(launch_nn_grid(ctx->search, (const float*)d_q, n, d_idx, d_d2, stats_ptr(ctx), ctx->stream));
    } else if (mode == SICP_NN_BRUTE_BF16) {
        if ((rc = bf16_prepare(ctx))) return rc;
        if ((rc = bf16_queries(ctx, n))) return rc;
        SICP_CUDA(launch_nn_bf16(ctx, (const float*)d_q, n, d_idx, d_d2, (int*)ctx->flags.p + 3));
    } else {
        SICP_CUDA(launch_nn_brute(ctx->ref4, ctx->M, (const float*)d_q, n, d_idx, d_d2, ctx->stream));
    }
    int flags[4];
    rc = read_flags(ctx, flags);
    if (rc) return rc;
    if (flags[0]) return set_err(ctx, SICP_EINVAL, "non-finite query");
    if (flags[3]) return set_err(ctx, SICP_ETIMEOUT, "a bounded wait of the tensor-core search gave up");
    if (!on_device) {
        if ((rc = copy_out(ctx, out_idx, d_idx, sizeof(int32_t) * n, 0))) return rc;
        if (out_d2 && (rc = copy_out(ctx, out_d2, d_d2, sizeof(float) * n, 0))) return rc;
    }
    return sync(ctx);
}

int sicp_icp_grad(sicp_ctx* ctx, const float* src_xyz, int64_t N, const int32_t* mb, int32_t m,
                  const float* particles, int32_t K, int32_t mode, float* out_gbar, int32_t* out_nn,
                  int on_device) {
    NvtxRange nvtx_("transform_nn_gradient");
    if (!ctx) return SICP_EINVAL;
    ctx->err.clear();
    if (!src_xyz || !mb || !particles || !out_gbar) return set_err(ctx, SICP_EINVAL, "null pointer");
    if (N < 1 || N > kMaxN || m < 1 || K < 1 || K > 65535)
        return set_err(ctx, SICP_EINVAL, "icp_grad needs N >= 1, m >= 1, 1 <= K <= 65535");
    const bool surr = mode == SICP_NN_SURROGATE;
    if (surr && (out_nn || (int64_t)K * m > ((int64_t)1 << 24)))
        return set_err(ctx, SICP_EINVAL, "surrogate mode needs out_nn = NULL and K * m <= 2^24");
    int rc = check_mode(ctx, mode, SICP_POINT_TO_PLANE, true);
    if (rc) return rc;
    if (ctx->M < 1) return set_err(ctx, SICP_ENOREF, "no reference cloud set");
    const bool plane = (mode & SICP_POINT_TO_PLANE) != 0;
    mode &= ~SICP_POINT_TO_PLANE;
    if (!on_device) {
        if (!host_finite(src_xyz, 3 * N) || !host_finite(particles, 6 * (int64_t)K))
            return set_err(ctx, SICP_EINVAL, "non-finite input");
        for (int32_t k = 0; k < m; ++k)
            if (mb[k] < 0 || mb[k] >= N) return set_err(ctx, SICP_EINVAL, "minibatch index out of range");
    }
    DeviceScope ds(ctx->device);
    const size_t b_src = sizeof(float) * 3 * N, b_mb = sizeof(int32_t) * m, b_th = sizeof(float) * 6 * K;
    if ((rc = ensure(ctx, ctx->tmp_aux, b_src + b_mb + b_th + 64))) return rc;
    const void *d_src, *d_mb, *d_th;
    char* aux = (char*)ctx->tmp_aux.p;
    if (on_device) {
        d_src = src_xyz;
        d_mb = mb;
        d_th = particles;
    } else {
        SICP_CUDA(cudaMemcpyAsync(aux, src_xyz, b_src, cudaMemcpyHostToDevice, ctx->stream));
        SICP_CUDA(cudaMemcpyAsync(aux + b_src, mb, b_mb, cudaMemcpyHostToDevice, ctx->stream));
        SICP_CUDA(cudaMemcpyAsync(aux + b_src + b_mb, particles, b_th, cudaMemcpyHostToDevice, ctx->stream));
        d_src = aux;
        d_mb = aux + b_src;
        d_th = aux + b_src + b_mb;
    }
    const bool bf = mode == SICP_NN_BRUTE_BF16;
    if (bf && (int64_t)K * m > ((int64_t)1 << 26))
        return set_err(ctx, SICP_EINVAL, "the tensor-core search needs K * m <= 2^26");
    const int chunks = (mode == SICP_NN_BRUTE_FP32 ? grad_layout(m) : grad_layout_grid(m)).chunks;
    if ((rc = ensure(ctx, ctx->src4, sizeof(float4) * N))) return rc;
    if ((rc = ensure(ctx, ctx->partial, sizeof(float) * 6 * (size_t)((surr || bf) && m > chunks ? m : chunks) * K)))
        return rc;
    if (surr && (rc = surrogate_prepare(ctx, (int64_t)K * m))) return rc;
    if (bf && (rc = bf16_prepare(ctx))) return rc;
    if (bf && (rc = bf16_queries(ctx, (int64_t)K * m))) return rc;
    if ((rc = ensure(ctx, ctx->tmp_out, (sizeof(float) * 6 + sizeof(int32_t) * (size_t)m) * K))) return rc;
    float* d_g = (float*)ctx->tmp_out.p;
    int32_t* d_nn = (int32_t*)((char*)ctx->tmp_out.p + sizeof(float) * 6 * K);
    SICP_CUDA(cudaMemsetAsync(ctx->flags.p, 0, 4 * sizeof(int), ctx->stream));
    SICP_CUDA(launch_pack_points((const float*)d_src, N, (float4*)ctx->src4.p, (int*)ctx->flags.p, ctx->stream));
    ctx->src_n = N;
    SICP_CUDA(launch_check_finite((const float*)d_th, 6 * (int64_t)K, (int*)ctx->flags.p, ctx->stream));
    SICP_CUDA(launch_check_index((const int32_t*)d_mb, m, N, (int*)ctx->flags.p, ctx->stream));
    int flags[4];
    if ((rc = read_flags(ctx, flags))) return rc;
    if (flags[0]) return set_err(ctx, SICP_EINVAL, "non-finite input");
    if (flags[1]) return set_err(ctx, SICP_EINVAL, "minibatch index out of range");
    GradArgs g;
    g.src = (const float4*)ctx->src4.p;
    g.mb = (const int32_t*)d_mb;
    g.m = m;
    g.theta = (const float*)d_th;
    g.K = K;
    g.partial = (float*)ctx->partial.p;
    g.out_nn = d_nn;
    g.stats = stats_ptr(ctx);
    g.gbar = d_g;
    g.inv_m = 1.f / (float)m;
    g.normals = plane ? (const float4*)ctx->normals.p : nullptr;
    g.mb_stride = 0;
    g.n_src = N;
    g.n_ref = ctx->M;
    if (surr) {
        SICP_CUDA(surrogate_launch_grad(ctx, g.src, g.mb, m, g.theta, K, kSurrogateIcpGradConf, (float*)ctx->partial.p,
                                        d_g, g.stats, (int*)ctx->flags.p + 3));
    } else if (bf) {
        SICP_CUDA(launch_grad_bf16(ctx, g.src, g.mb, m, g.theta, K, (float*)ctx->partial.p, d_g, out_nn ? d_nn : nullptr,
                                   (int*)ctx->flags.p + 3, g.normals, 0));
    } else {
        SICP_CUDA(launch_grad(ctx, mode, g));
        if (mode != SICP_NN_GRID)
            SICP_CUDA(launch_partial_to_gbar((const float*)ctx->partial.p, chunks, K, 1.f / (float)m, d_g, ctx->stream));
    }
    if ((rc = copy_out(ctx, out_gbar, d_g, sizeof(float) * 6 * K, on_device))) return rc;
    if (out_nn && (rc = copy_out(ctx, out_nn, d_nn, sizeof(int32_t) * (size_t)m * K, on_device))) return rc;
    if (surr || bf) {
        if ((rc = read_flags(ctx, flags))) return rc;
        if (flags[3]) return set_err(ctx, SICP_ETIMEOUT, "a bounded wait on the GPU gave up");
    }
    return sync(ctx);
}

int sicp_stein_adam(sicp_ctx* ctx, float* particles, float* adam_m, float* adam_v, const float* gbar,
                    int32_t K, int64_t N, int64_t t, const sicp_params* p_in, float* out_phi, float* out_h,
                    int on_device) {
    NvtxRange nvtx_("stein_adam");
    if (!ctx) return SICP_EINVAL;
    ctx->err.clear();
    if (!particles || !adam_m || !adam_v || !gbar || !p_in) return set_err(ctx, SICP_EINVAL, "null pointer");
    if (K < 1 || K > kMaxK || N < 1 || t < 1)
        return set_err(ctx, SICP_EINVAL, "stein_adam needs 1 <= K <= %d, N >= 1, t >= 1", kMaxK);
    const sicp_params p = normalise(p_in);
    int rc = check_params(ctx, p);
    if (rc) return rc;
    DeviceScope ds(ctx->device);
    const size_t b = sizeof(float) * 6 * K;
    if ((rc = ensure(ctx, ctx->tmp_aux, 5 * b + 64))) return rc;
    float* th = (float*)ctx->tmp_aux.p;
    float* am = th + 6 * K;
    float* av = am + 6 * K;
    float* gb = av + 6 * K;
    float* phi = gb + 6 * K;
    float* hh = phi + 6 * K;   // 2 floats in the padding, then the 2 Stein arrival counters
    const cudaMemcpyKind kin = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    SICP_CUDA(cudaMemcpyAsync(th, particles, b, kin, ctx->stream));
    SICP_CUDA(cudaMemcpyAsync(am, adam_m, b, kin, ctx->stream));
    SICP_CUDA(cudaMemcpyAsync(av, adam_v, b, kin, ctx->stream));
    SICP_CUDA(cudaMemcpyAsync(gb, gbar, b, kin, ctx->stream));
    SICP_CUDA(cudaMemsetAsync(ctx->flags.p, 0, 4 * sizeof(int), ctx->stream));
    SICP_CUDA(launch_check_finite(th, 24 * (int64_t)K, (int*)ctx->flags.p, ctx->stream));
    int flags[4];
    if ((rc = read_flags(ctx, flags))) return rc;
    if (flags[0]) return set_err(ctx, SICP_EINVAL, "non-finite input");
    SteinArgs a = stein_args(p, th, am, av, gb, 1, 1.f, K, (float)N, t);
    a.out_phi = phi;
    a.out_h = hh;
    a.arrive = (unsigned*)(hh + 2);
    a.err = (int*)ctx->flags.p + 3;
    a.gen = 1;
    a.max_spins = ctx->wait_polls;
    a.extra = ctx->wait_never ? 1u : 0u;
    SICP_CUDA(cudaMemsetAsync(a.arrive, 0, 2 * sizeof(unsigned), ctx->stream));
    SICP_CUDA(launch_stein_adam(a, ctx->stream));
    if ((rc = read_flags(ctx, flags))) return rc;
    if (flags[3]) return set_err(ctx, SICP_ETIMEOUT, "a bounded wait of the Stein update gave up");
    const cudaMemcpyKind kout = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    SICP_CUDA(cudaMemcpyAsync(particles, th, b, kout, ctx->stream));
    SICP_CUDA(cudaMemcpyAsync(adam_m, am, b, kout, ctx->stream));
    SICP_CUDA(cudaMemcpyAsync(adam_v, av, b, kout, ctx->stream));
    if (out_phi) SICP_CUDA(cudaMemcpyAsync(out_phi, phi, b, kout, ctx->stream));
    if (out_h) SICP_CUDA(cudaMemcpyAsync(out_h, hh, 2 * sizeof(float), kout, ctx->stream));
    return sync(ctx);
}

}  // extern "C"

namespace {

int moments_entry(sicp_ctx* ctx, const float* particles, int32_t K, double* mean6, double* cov36, int on_device,
                  bool circular) {
    if (!ctx) return SICP_EINVAL;
    ctx->err.clear();
    if (!particles || K < 1 || K > kMaxK) return set_err(ctx, SICP_EINVAL, "moments needs 1 <= K <= %d", kMaxK);
    DeviceScope ds(ctx->device);
    const void* d_th;
    int rc = stage_in(ctx, particles, sizeof(float) * 6 * K, on_device, ctx->tmp_in, &d_th);
    if (rc) return rc;
    if ((rc = ensure(ctx, ctx->moments, 42 * sizeof(double)))) return rc;
    if (circular)
        SICP_CUDA(launch_moments_circular((const float*)d_th, K, (double*)ctx->moments.p, ctx->stream));
    else
        SICP_CUDA(launch_moments((const float*)d_th, K, (double*)ctx->moments.p, ctx->stream));
    if ((rc = copy_out(ctx, mean6, ctx->moments.p, 6 * sizeof(double), on_device))) return rc;
    if ((rc = copy_out(ctx, cov36, (double*)ctx->moments.p + 6, 36 * sizeof(double), on_device))) return rc;
    return sync(ctx);
}

}  // namespace

extern "C" {

int sicp_moments(sicp_ctx* ctx, const float* particles, int32_t K, double* mean6, double* cov36, int on_device) {
    NvtxRange nvtx_("moments");
    return moments_entry(ctx, particles, K, mean6, cov36, on_device, false);
}

int sicp_moments_circular(sicp_ctx* ctx, const float* particles, int32_t K, double* mean6, double* cov36,
                          int on_device) {
    return moments_entry(ctx, particles, K, mean6, cov36, on_device, true);
}

}  // extern "C"

namespace {

// One registration run of p->T iterations starting at iteration t0 (minibatch
// stream position and Adam step t0 + 1).  adam_in (2 [K][6] arrays: m then v,
// may be null: zeros) seeds the Adam moments; adam_out (may be null) receives
// them after the run.
int register_run(sicp_ctx* ctx, const float* src_xyz, int64_t N, const float* particles_in, int32_t K,
                 const sicp_params* p_in, float* particles_out, double* mean6, double* cov36, int on_device,
                 int64_t t0, const float* adam_in, float* adam_out) {
    NvtxRange nvtx_("register");
    if (!ctx) return SICP_EINVAL;
    ctx->err.clear();
    if (!src_xyz || !particles_in || !particles_out || !p_in) return set_err(ctx, SICP_EINVAL, "null pointer");
    if (t0 < 0 || t0 > ((int64_t)1 << 40)) return set_err(ctx, SICP_EINVAL, "t0 must lie in [0, 2^40]");
    const sicp_params p = normalise(p_in);
    if (N < 1 || N > kMaxN) return set_err(ctx, SICP_EINVAL, "source needs 1 <= N <= 2^31-1 points");
    if (K < 1 || K > kMaxK) return set_err(ctx, SICP_EINVAL, "particle count must be in [1, %d]", kMaxK);
    if (p.T < 0) return set_err(ctx, SICP_EINVAL, "T must be >= 0");
    if (p.m < 1 || p.m > N) return set_err(ctx, SICP_EINVAL, "minibatch m=%d outside [1, N=%lld]", p.m, (long long)N);
    int rc = check_params(ctx, p);
    if (rc) return rc;
    if ((rc = check_mode(ctx, p.nn_mode, SICP_POINT_TO_PLANE | SICP_INDEPENDENT, true))) return rc;
    if (ctx->M < 1) return set_err(ctx, SICP_ENOREF, "no reference cloud set");
    if (!on_device && (!host_finite(src_xyz, 3 * N) || !host_finite(particles_in, 6 * (int64_t)K)))
        return set_err(ctx, SICP_EINVAL, "non-finite input");
    if (adam_in && !on_device) {
        if (!host_finite(adam_in, 12 * (int64_t)K)) return set_err(ctx, SICP_EINVAL, "non-finite input");
        for (int64_t i = 6 * (int64_t)K; i < 12 * (int64_t)K; ++i)
            if (adam_in[i] < 0.f) return set_err(ctx, SICP_EINVAL, "negative Adam second moment");
    }
    DeviceScope ds(ctx->device);
    const bool plane = (p.nn_mode & SICP_POINT_TO_PLANE) != 0;
    const bool indep = (p.nn_mode & SICP_INDEPENDENT) != 0;
    const int32_t nn_mode = p.nn_mode & ~(SICP_POINT_TO_PLANE | SICP_INDEPENDENT);
    const bool surr = nn_mode == SICP_NN_SURROGATE;
    if (surr && indep) return set_err(ctx, SICP_EINVAL, "independent runs use an exact search (grid, FP32, BF16)");
    if (surr && (int64_t)K * p.m > ((int64_t)1 << 24))
        return set_err(ctx, SICP_EINVAL, "surrogate mode needs K * m <= 2^24 queries per iteration");
    const bool bf = nn_mode == SICP_NN_BRUTE_BF16;
    if (bf && (int64_t)K * p.m > ((int64_t)1 << 26))
        return set_err(ctx, SICP_EINVAL, "the tensor-core search needs K * m <= 2^26");
    // every argument is valid: from here the run replaces the context's run state (the buffers
    // below may be reallocated), which is valid again once the run has finished
    ctx->run_valid = false;
    const bool grid = nn_mode == SICP_NN_GRID || surr;   // the surrogate's exact iterations use the grid
    const int32_t exact_mode = surr ? SICP_NN_GRID : nn_mode;
    const int chunks = (grid ? grad_layout_grid(p.m) : grad_layout(p.m)).chunks;
    const int32_t surr_T = surr ? (p.surrogate_iters < p.T ? p.surrogate_iters : p.T) : 0;
    const size_t b_th = sizeof(float) * 6 * K;
    // partial sums of the exhaustive kernel, or the surrogate's per-query terms
    const size_t partial_floats = 6 * (size_t)K * (size_t)((surr_T > 0 || bf) && p.m > chunks ? p.m : chunks);
    if ((rc = ensure(ctx, ctx->src4, sizeof(float4) * N))) return rc;
    // one minibatch row per iteration, or one per iteration and independent run
    if ((rc = ensure(ctx, ctx->mb, sizeof(int32_t) * (size_t)(p.T > 0 ? p.T : 1) * p.m * (indep ? (size_t)K : 1))))
        return rc;
    if ((rc = ensure(ctx, ctx->theta, b_th))) return rc;
    if ((rc = ensure(ctx, ctx->adam_m, b_th))) return rc;
    if ((rc = ensure(ctx, ctx->adam_v, b_th))) return rc;
    if ((rc = ensure(ctx, ctx->partial, sizeof(float) * partial_floats))) return rc;
    if ((rc = ensure(ctx, ctx->moments, 42 * sizeof(double)))) return rc;
    if ((rc = ensure(ctx, ctx->gbar, b_th + 4 * sizeof(float)))) return rc;   // + the two blocks' medians
    if (surr_T > 0 && (rc = surrogate_prepare(ctx, (int64_t)K * p.m))) return rc;
    if (bf && (rc = bf16_prepare(ctx))) return rc;
    if (bf && (rc = bf16_queries(ctx, (int64_t)K * p.m))) return rc;
    const bool tel = ctx->telemetry;
    ctx->tel_rows = 0;
    if (tel) {
        if ((rc = ensure(ctx, ctx->tel, sizeof(float) * 16 * (size_t)(p.T > 0 ? p.T : 1)))) return rc;
        if ((rc = ensure(ctx, ctx->tel_nn, sizeof(int32_t) * (size_t)K * p.m))) return rc;
        if ((rc = ensure(ctx, ctx->tel_part, sizeof(float) * 2 * (size_t)K + 16))) return rc;
    }

    const void *d_src, *d_th0;
    if ((rc = stage_in(ctx, src_xyz, sizeof(float) * 3 * N, on_device, ctx->tmp_in, &d_src))) return rc;
    if ((rc = stage_in(ctx, particles_in, b_th, on_device, ctx->tmp_aux, &d_th0))) return rc;
    float* theta = (float*)ctx->theta.p;
    SICP_CUDA(cudaMemsetAsync(ctx->flags.p, 0, 4 * sizeof(int), ctx->stream));
    SICP_CUDA(launch_pack_points((const float*)d_src, N, (float4*)ctx->src4.p, (int*)ctx->flags.p, ctx->stream));
    ctx->src_n = N;
    SICP_CUDA(launch_check_finite((const float*)d_th0, 6 * (int64_t)K, (int*)ctx->flags.p, ctx->stream));
    SICP_CUDA(cudaMemcpyAsync(theta, d_th0, b_th, cudaMemcpyDeviceToDevice, ctx->stream));
    if (adam_in) {
        const cudaMemcpyKind kin = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
        SICP_CUDA(cudaMemcpyAsync(ctx->adam_m.p, adam_in, b_th, kin, ctx->stream));
        SICP_CUDA(cudaMemcpyAsync(ctx->adam_v.p, adam_in + 6 * (size_t)K, b_th, kin, ctx->stream));
        if (on_device) {
            SICP_CUDA(launch_check_finite((const float*)ctx->adam_m.p, 6 * (int64_t)K, (int*)ctx->flags.p, ctx->stream));
            SICP_CUDA(launch_check_nonneg((const float*)ctx->adam_v.p, 6 * (int64_t)K, (int*)ctx->flags.p, ctx->stream));
        }
    } else {
        SICP_CUDA(cudaMemsetAsync(ctx->adam_m.p, 0, b_th, ctx->stream));
        SICP_CUDA(cudaMemsetAsync(ctx->adam_v.p, 0, b_th, ctx->stream));
    }
    // after gbar: the two blocks' previous medians, then their Stein arrival counters
    float* med_state = (float*)ctx->gbar.p + 6 * (size_t)K;
    SICP_CUDA(cudaMemsetAsync(med_state, 0, 4 * sizeof(float), ctx->stream));

    const int stride = ctx->prof_stride;
    LoopKey key;
    memset(&key, 0, sizeof key);
    key.N = N;
    key.K = K;
    key.T = p.T;
    key.m = p.m;
    key.mode = p.nn_mode;
    key.chunks = chunks;
    key.stride = stride;
    key.pi[0] = p.T;
    key.pi[1] = p.m;
    key.pi[2] = p.nn_mode;
    key.pi[3] = p.prior;
    key.pf[0] = p.lr;
    key.pf[1] = p.beta1;
    key.pf[2] = p.beta2;
    key.pf[3] = p.eps;
    for (int a = 0; a < 6; ++a) key.pf[4 + a] = p.prior_mu[a];
    for (int a = 0; a < 3; ++a) {
        key.pf[10 + a] = p.prior_sigma[a];
        key.pf[13 + a] = p.prior_kappa[a];
    }
    key.surr_iters = surr_T;
    key.min_conf = surr ? p.surrogate_min_conf : 0.f;
    key.surr_gen = surr ? ctx->surr_gen : 0;
    key.seed = p.seed;
    key.t0 = t0;
    key.ref_M = ctx->M;   // (the grid and BF16 kernels read the reference's description from device memory)
    key.wait_polls = ctx->wait_polls;
    key.wait_never = ctx->wait_never;
    key.ptrs[0] = ctx->src4.p;
    key.ptrs[1] = ctx->mb.p;
    key.ptrs[2] = ctx->theta.p;
    key.ptrs[3] = ctx->adam_m.p;
    key.ptrs[4] = ctx->adam_v.p;
    key.ptrs[5] = ctx->partial.p;
    key.ptrs[6] = ctx->moments.p;
    key.ptrs[7] = ctx->grid.sorted;
    key.ptrs[8] = ctx->ref4;
    key.ptrs[9] = stats_ptr(ctx);
    key.ptrs[10] = ctx->gbar.p;
    key.ptrs[11] = plane ? ctx->normals.p : nullptr;
    key.tel = tel ? 1 : 0;
    key.ptrs[12] = tel ? ctx->tel.p : nullptr;
    key.ptrs[13] = tel ? ctx->tel_nn.p : nullptr;
    key.ptrs[14] = tel ? ctx->tel_part.p : nullptr;
    key.ptrs[15] = bf ? ctx->bf16_q.p : nullptr;   // the tensor-core search's query buffers

    GraphCache& gc = *ctx->graphs;
    GraphSlot& slot = gc.slot[stride > 0 ? gc.next : 0];
    const bool use_graph = getenv("SICP_NO_GRAPH") == nullptr;
    auto record = [&](GraphSlot* prof) -> int {
        {
            NvtxRange r_sample("sample");
            if (indep)
                SICP_CUDA(launch_minibatch_runs(p.seed, t0, p.T, N, p.m, K, (int32_t*)ctx->mb.p, ctx->stream));
            else
                SICP_CUDA(launch_minibatch(p.seed, t0, p.T, N, p.m, (int32_t*)ctx->mb.p, ctx->stream));
        }
        GradArgs g;
        g.src = (const float4*)ctx->src4.p;
        g.m = p.m;
        g.theta = theta;
        g.K = K;
        g.partial = (float*)ctx->partial.p;
        int32_t* tel_nn = tel ? (int32_t*)ctx->tel_nn.p : nullptr;   // the exact searches' correspondences
        int* tel_fb = tel ? (int*)((float*)ctx->tel_part.p + 2 * (size_t)K) : nullptr;
        g.out_nn = tel_nn;
        g.stats = stats_ptr(ctx);
        g.gbar = (float*)ctx->gbar.p;
        g.inv_m = 1.f / (float)p.m;
        g.normals = plane ? (const float4*)ctx->normals.p : nullptr;
        g.mb_stride = indep ? (int64_t)p.T * p.m : 0;   // run j's row of iteration t: mb[(j T + t) m]
        g.n_src = N;
        g.n_ref = ctx->M;
        int np = 0;
        for (int32_t t = 0; t < p.T; ++t) {
            const bool timed = prof && stride > 0 && (t % stride) == 0;
            if (timed) SICP_CUDA(cudaEventRecordWithFlags(prof->ev[3 * np], ctx->stream, cudaEventRecordExternal));
            g.mb = (const int32_t*)ctx->mb.p + (size_t)t * p.m;
            {
                NvtxRange r_grad("transform_nn_gradient");
                if (t < surr_T)
                    SICP_CUDA(surrogate_launch_grad(ctx, g.src, g.mb, p.m, theta, K, p.surrogate_min_conf,
                                                    (float*)ctx->partial.p, (float*)ctx->gbar.p, g.stats,
                                                    (int*)ctx->flags.p + 3, tel_fb));
                else if (bf)
                    SICP_CUDA(launch_grad_bf16(ctx, g.src, g.mb, p.m, theta, K, (float*)ctx->partial.p,
                                               (float*)ctx->gbar.p, tel_nn, (int*)ctx->flags.p + 3, g.normals,
                                               g.mb_stride));
                else
                    SICP_CUDA(launch_grad(ctx, exact_mode, g));
            }
            if (tel) {   // the row of iteration t, from the particles it started from
                NvtxRange r_tel("telemetry");
                TelArgs ta;
                ta.theta = theta;
                ta.K = K;
                ta.m = p.m;
                ta.src = g.src;
                ta.n_src = N;
                ta.mb = g.mb;
                ta.mb_stride = g.mb_stride;
                ta.nn = t < surr_T ? nullptr : tel_nn;
                ta.ref4 = ctx->ref4;
                ta.n_ref = ctx->M;
                ta.qterms = t < surr_T ? (const float*)ctx->partial.p : nullptr;
                ta.fb = t < surr_T ? tel_fb : nullptr;
                ta.part = (float*)ctx->tel_part.p;
                ta.row = (float*)ctx->tel.p + 16 * (size_t)t;
                ta.t_abs = (double)(t0 + t);
                SICP_CUDA(launch_telemetry(ta, ctx->stream));
            }
            if (timed) SICP_CUDA(cudaEventRecordWithFlags(prof->ev[3 * np + 1], ctx->stream, cudaEventRecordExternal));
            // the grid kernel and the surrogate path leave gbar; the exhaustive kernel leaves `chunks` partials
            SteinArgs a = (grid || bf) ? stein_args(p, theta, (float*)ctx->adam_m.p, (float*)ctx->adam_v.p,
                                            (const float*)ctx->gbar.p, 1, 1.f, K, (float)N, t0 + t + 1)
                               : stein_args(p, theta, (float*)ctx->adam_m.p, (float*)ctx->adam_v.p,
                                            (const float*)ctx->partial.p, chunks, 1.f / (float)p.m, K, (float)N,
                                            t0 + t + 1);
            a.med_state = med_state;
            a.arrive = (unsigned*)(med_state + 2);
            a.err = (int*)ctx->flags.p + 3;
            a.gen = (uint32_t)(t + 1);
            a.max_spins = ctx->wait_polls;
            a.extra = ctx->wait_never ? 1u : 0u;
            {
                NvtxRange r_stein("stein_adam");
                if (indep)
                    SICP_CUDA(launch_adam_independent(a, ctx->stream));
                else
                    SICP_CUDA(launch_stein_adam(a, ctx->stream));
            }
            if (timed) SICP_CUDA(cudaEventRecordWithFlags(prof->ev[3 * np + 2], ctx->stream, cudaEventRecordExternal));
            if (timed) ++np;
        }
        if (prof) prof->n_prof = np;
        {
            NvtxRange r_mom("moments");
            SICP_CUDA(launch_moments(theta, K, (double*)ctx->moments.p, ctx->stream));
        }
        return SICP_OK;
    };
    if (use_graph) {
        if (!(slot.valid && slot.key == key)) {
            if (slot.exec) cudaGraphExecDestroy(slot.exec);
            slot.exec = nullptr;
            slot.valid = false;
            slot.pending = false;
            const int need = stride > 0 ? 3 * ((p.T + stride - 1) / stride) : 0;
            while ((int)slot.ev.size() < need) {
                cudaEvent_t e;
                SICP_CUDA(cudaEventCreate(&e));
                slot.ev.push_back(e);
            }
            cudaGraph_t graph;
            SICP_CUDA(cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal));
            rc = record(stride > 0 ? &slot : nullptr);
            cudaError_t e = cudaStreamEndCapture(ctx->stream, &graph);
            if (rc) {
                if (e == cudaSuccess) cudaGraphDestroy(graph);
                return rc;
            }
            if (e != cudaSuccess) return cuda_err(ctx, e, "cudaStreamEndCapture");
            e = cudaGraphInstantiate(&slot.exec, graph, 0);
            cudaGraphDestroy(graph);
            if (e != cudaSuccess) return cuda_err(ctx, e, "cudaGraphInstantiate");
            slot.key = key;
            slot.valid = true;
        }
        {
            NvtxRange r_launch("graph_launch");
            SICP_CUDA(cudaGraphLaunch(slot.exec, ctx->stream));
        }
        if (stride > 0) {
            // the other slot's last launch finished before this call began
            collect_profile(ctx, gc.slot[1 - gc.next]);
            slot.pending = true;
            gc.next = 1 - gc.next;
        }
    } else {
        if ((rc = record(nullptr))) return rc;
    }
    int flags[4];
    if ((rc = read_flags(ctx, flags))) return rc;
    if (flags[0]) return set_err(ctx, SICP_EINVAL, "non-finite input (or a negative Adam second moment)");
    if (flags[3])
        return set_err(ctx, SICP_ETIMEOUT, "a bounded wait on the GPU gave up (tensor-core search or Stein update)");
    if ((rc = copy_out(ctx, particles_out, theta, b_th, on_device))) return rc;
    if ((rc = copy_out(ctx, mean6, ctx->moments.p, 6 * sizeof(double), on_device))) return rc;
    if ((rc = copy_out(ctx, cov36, (double*)ctx->moments.p + 6, 36 * sizeof(double), on_device))) return rc;
    if (adam_out) {
        if ((rc = copy_out(ctx, adam_out, ctx->adam_m.p, b_th, on_device))) return rc;
        if ((rc = copy_out(ctx, adam_out + 6 * (size_t)K, ctx->adam_v.p, b_th, on_device))) return rc;
    }
    if ((rc = sync(ctx))) return rc;
    ctx->tel_rows = tel ? p.T : 0;
    ctx->run_valid = true;
    ctx->run_K = K;
    ctx->run_t = t0 + p.T;
    ctx->run_seed = p.seed;
    return SICP_OK;
}

}  // namespace

// ---- the context's run state as a byte string
//   "SICPRUN1" | u32 version (1) | i32 K | i64 t | u64 seed | f32 state[3][K][6] | u32 CRC-32
// in host byte order; the CRC (IEEE 802.3 polynomial, reflected, as in zlib)
// covers every byte before it.

namespace {

constexpr char kStateMagic[8] = {'S', 'I', 'C', 'P', 'R', 'U', 'N', '1'};
constexpr size_t kStateHead = 8 + 4 + 4 + 8 + 8;

uint32_t crc32_ieee(const unsigned char* p, size_t n) {
    uint32_t c = 0xffffffffu;
    for (size_t i = 0; i < n; ++i) {
        c ^= p[i];
        for (int k = 0; k < 8; ++k) c = (c >> 1) ^ (0xedb88320u & (0u - (c & 1u)));
    }
    return ~c;
}

size_t state_bytes(int32_t K) { return kStateHead + sizeof(float) * 18 * (size_t)K + 4; }

}  // namespace

extern "C" {

int sicp_register(sicp_ctx* ctx, const float* src_xyz, int64_t N, const float* particles_in, int32_t K,
                  const sicp_params* p, float* particles_out, double* mean6, double* cov36, int on_device) {
    return register_run(ctx, src_xyz, N, particles_in, K, p, particles_out, mean6, cov36, on_device, 0, nullptr,
                        nullptr);
}

int sicp_register_continue(sicp_ctx* ctx, const float* src_xyz, int64_t N, float* state, int32_t K, int64_t t0,
                           const sicp_params* p, double* mean6, double* cov36, int on_device) {
    if (!ctx) return SICP_EINVAL;
    if (!state) return set_err(ctx, SICP_EINVAL, "null pointer");
    if (K < 1 || K > kMaxK) return set_err(ctx, SICP_EINVAL, "particle count must be in [1, %d]", kMaxK);
    // the particles are read before they are overwritten (staged into the context first)
    return register_run(ctx, src_xyz, N, state, K, p, state, mean6, cov36, on_device, t0, state + 6 * (size_t)K,
                        state + 6 * (size_t)K);
}

int sicp_export_state(sicp_ctx* ctx, void* buf, size_t* len) {
    if (!ctx) return SICP_EINVAL;
    ctx->err.clear();
    if (!len) return set_err(ctx, SICP_EINVAL, "null pointer");
    if (!ctx->run_valid) return set_err(ctx, SICP_EINVAL, "no finished run in this context");
    const int32_t K = ctx->run_K;
    const size_t need = state_bytes(K);
    if (!buf) {
        *len = need;
        return SICP_OK;
    }
    if (*len < need) {
        *len = need;
        return set_err(ctx, SICP_EINVAL, "buffer too small: %zu bytes needed", need);
    }
    DeviceScope ds(ctx->device);
    unsigned char* o = (unsigned char*)buf;
    const uint32_t version = 1;
    const int64_t t = ctx->run_t;
    const uint64_t seed = ctx->run_seed;
    memcpy(o, kStateMagic, 8);
    memcpy(o + 8, &version, 4);
    memcpy(o + 12, &K, 4);
    memcpy(o + 16, &t, 8);
    memcpy(o + 24, &seed, 8);
    const size_t b = sizeof(float) * 6 * (size_t)K;
    std::vector<float> h(18 * (size_t)K);
    SICP_CUDA(cudaMemcpyAsync(h.data(), ctx->theta.p, b, cudaMemcpyDeviceToHost, ctx->stream));
    SICP_CUDA(cudaMemcpyAsync(h.data() + 6 * (size_t)K, ctx->adam_m.p, b, cudaMemcpyDeviceToHost, ctx->stream));
    SICP_CUDA(cudaMemcpyAsync(h.data() + 12 * (size_t)K, ctx->adam_v.p, b, cudaMemcpyDeviceToHost, ctx->stream));
    int rc = sync(ctx);
    if (rc) return rc;
    memcpy(o + kStateHead, h.data(), 3 * b);
    const uint32_t crc = crc32_ieee(o, need - 4);
    memcpy(o + need - 4, &crc, 4);
    *len = need;
    return SICP_OK;
}

int sicp_import_state(sicp_ctx* ctx, const void* buf, size_t len) {
    if (!ctx) return SICP_EINVAL;
    ctx->err.clear();
    if (!buf) return set_err(ctx, SICP_EINVAL, "null pointer");
    const unsigned char* in = (const unsigned char*)buf;
    if (len < kStateHead + 4 || memcmp(in, kStateMagic, 8) != 0) return set_err(ctx, SICP_EINVAL, "not a run state");
    uint32_t version, crc;
    int32_t K;
    int64_t t;
    uint64_t seed;
    memcpy(&version, in + 8, 4);
    memcpy(&K, in + 12, 4);
    memcpy(&t, in + 16, 8);
    memcpy(&seed, in + 24, 8);
    if (version != 1) return set_err(ctx, SICP_EINVAL, "run state version %u not supported", version);
    if (K < 1 || K > kMaxK) return set_err(ctx, SICP_EINVAL, "particle count must be in [1, %d]", kMaxK);
    if (len != state_bytes(K)) return set_err(ctx, SICP_EINVAL, "run state of %zu bytes, %zu expected", len, state_bytes(K));
    memcpy(&crc, in + len - 4, 4);
    if (crc != crc32_ieee(in, len - 4)) return set_err(ctx, SICP_EINVAL, "run state checksum mismatch");
    if (t < 0 || t > ((int64_t)1 << 40)) return set_err(ctx, SICP_EINVAL, "t must lie in [0, 2^40]");
    std::vector<float> h(18 * (size_t)K);
    memcpy(h.data(), in + kStateHead, sizeof(float) * h.size());
    if (!host_finite(h.data(), (int64_t)h.size())) return set_err(ctx, SICP_EINVAL, "non-finite state");
    for (size_t i = 12 * (size_t)K; i < h.size(); ++i)
        if (h[i] < 0.f) return set_err(ctx, SICP_EINVAL, "negative Adam second moment in the state");
    DeviceScope ds(ctx->device);
    const size_t b = sizeof(float) * 6 * (size_t)K;
    int rc;
    ctx->run_valid = false;
    if ((rc = ensure(ctx, ctx->theta, b)) || (rc = ensure(ctx, ctx->adam_m, b)) || (rc = ensure(ctx, ctx->adam_v, b)))
        return rc;
    SICP_CUDA(cudaMemcpyAsync(ctx->theta.p, h.data(), b, cudaMemcpyHostToDevice, ctx->stream));
    SICP_CUDA(cudaMemcpyAsync(ctx->adam_m.p, h.data() + 6 * (size_t)K, b, cudaMemcpyHostToDevice, ctx->stream));
    SICP_CUDA(cudaMemcpyAsync(ctx->adam_v.p, h.data() + 12 * (size_t)K, b, cudaMemcpyHostToDevice, ctx->stream));
    if ((rc = sync(ctx))) return rc;
    ctx->run_valid = true;
    ctx->run_K = K;
    ctx->run_t = t;
    ctx->run_seed = seed;
    return SICP_OK;
}

int sicp_resume(sicp_ctx* ctx, const float* src_xyz, int64_t N, const sicp_params* p, float* particles_out,
                double* mean6, double* cov36, int on_device) {
    if (!ctx) return SICP_EINVAL;
    ctx->err.clear();
    if (!p) return set_err(ctx, SICP_EINVAL, "null pointer");
    if (!ctx->run_valid) return set_err(ctx, SICP_EINVAL, "no run to resume in this context");
    if (p->seed != ctx->run_seed)
        return set_err(ctx, SICP_EINVAL, "the run draws its minibatches with seed %llu",
                       (unsigned long long)ctx->run_seed);
    DeviceScope ds(ctx->device);
    const int32_t K = ctx->run_K;
    const int64_t t0 = ctx->run_t;
    const size_t b = sizeof(float) * 6 * (size_t)K;
    std::vector<float> h;
    float* st;
    int rc;
    if (on_device) {   // the state as register_run reads it: [3][K][6] in one device buffer
        if ((rc = ensure(ctx, ctx->resume, 3 * b))) return rc;
        st = (float*)ctx->resume.p;
        SICP_CUDA(cudaMemcpyAsync(st, ctx->theta.p, b, cudaMemcpyDeviceToDevice, ctx->stream));
        SICP_CUDA(cudaMemcpyAsync(st + 6 * (size_t)K, ctx->adam_m.p, b, cudaMemcpyDeviceToDevice, ctx->stream));
        SICP_CUDA(cudaMemcpyAsync(st + 12 * (size_t)K, ctx->adam_v.p, b, cudaMemcpyDeviceToDevice, ctx->stream));
    } else {
        h.resize(18 * (size_t)K);
        st = h.data();
        SICP_CUDA(cudaMemcpyAsync(st, ctx->theta.p, b, cudaMemcpyDeviceToHost, ctx->stream));
        SICP_CUDA(cudaMemcpyAsync(st + 6 * (size_t)K, ctx->adam_m.p, b, cudaMemcpyDeviceToHost, ctx->stream));
        SICP_CUDA(cudaMemcpyAsync(st + 12 * (size_t)K, ctx->adam_v.p, b, cudaMemcpyDeviceToHost, ctx->stream));
        if ((rc = sync(ctx))) return rc;
    }
    rc = register_run(ctx, src_xyz, N, st, K, p, st, mean6, cov36, on_device, t0, st + 6 * (size_t)K,
                      st + 6 * (size_t)K);
    if (rc) return rc;
    if (particles_out) {
        if (on_device) {
            SICP_CUDA(cudaMemcpyAsync(particles_out, st, b, cudaMemcpyDeviceToDevice, ctx->stream));
            return sync(ctx);
        }
        memcpy(particles_out, st, b);
    }
    return SICP_OK;
}

int sicp_stats(sicp_ctx* ctx, int enable, uint64_t* out10) {
    if (!ctx) return SICP_EINVAL;
    ctx->err.clear();
    DeviceScope ds(ctx->device);
    int rc = ensure(ctx, ctx->stats, 10 * sizeof(unsigned long long));
    if (rc) return rc;
    if (out10) {
        unsigned long long h[10] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
        if (ctx->stats_on) {
            SICP_CUDA(cudaMemcpyAsync(h, ctx->stats.p, sizeof h, cudaMemcpyDeviceToHost, ctx->stream));
            if ((rc = sync(ctx))) return rc;
        }
        for (int a = 0; a < 10; ++a) out10[a] = (uint64_t)h[a];
    }
    SICP_CUDA(cudaMemsetAsync(ctx->stats.p, 0, 10 * sizeof(unsigned long long), ctx->stream));
    ctx->stats_on = enable != 0;
    return sync(ctx);
}

int sicp_set_wait_check(sicp_ctx* ctx, int on, int64_t polls) {
    if (!ctx) return SICP_EINVAL;
    ctx->err.clear();
    if (polls < 0 || polls > ((int64_t)1 << 30)) return set_err(ctx, SICP_EINVAL, "polls must lie in [0, 2^30]");
    ctx->wait_never = on ? 1 : 0;
    ctx->wait_polls = (long long)polls;
    return SICP_OK;
}

int sicp_check_status(int32_t* checked, uint64_t* first, uint64_t* count) {
    unsigned long long f = 0, c = 0;
    if (cudaDeviceSynchronize() != cudaSuccess) return SICP_ECUDA;
    for (CheckReader r : check_registry()) r(&f, &c);
    if (checked) *checked = kCheckedBuild;
    if (first) *first = f;
    if (count) *count = c;
    return SICP_OK;
}

int sicp_set_telemetry(sicp_ctx* ctx, int on) {
    if (!ctx) return SICP_EINVAL;
    ctx->err.clear();
    ctx->telemetry = on != 0;
    return SICP_OK;
}

int sicp_read_telemetry(sicp_ctx* ctx, float* out, int32_t max_rows, int32_t* rows) {
    if (!ctx) return SICP_EINVAL;
    ctx->err.clear();
    if (max_rows < 0 || (max_rows > 0 && !out)) return set_err(ctx, SICP_EINVAL, "out needs max_rows >= 0 rows");
    if (rows) *rows = ctx->tel_rows;
    const int32_t n = ctx->tel_rows < max_rows ? ctx->tel_rows : max_rows;
    if (n <= 0) return SICP_OK;
    DeviceScope ds(ctx->device);
    SICP_CUDA(cudaMemcpyAsync(out, ctx->tel.p, sizeof(float) * 16 * (size_t)n, cudaMemcpyDeviceToHost, ctx->stream));
    return sync(ctx);
}

int sicp_set_memory_limit(sicp_ctx* ctx, size_t bytes, size_t* held) {
    if (!ctx) return SICP_EINVAL;
    ctx->err.clear();
    ctx->mem_limit = bytes;
    if (held) *held = ctx->mem_used;
    return SICP_OK;
}

int sicp_profile(sicp_ctx* ctx, int stride, double* out4) {
    if (!ctx) return SICP_EINVAL;
    ctx->err.clear();
    if (stride < 0) return set_err(ctx, SICP_EINVAL, "stride must be >= 0");
    DeviceScope ds(ctx->device);
    int rc = sync(ctx);
    if (rc) return rc;
    for (GraphSlot& s : ctx->graphs->slot) collect_profile(ctx, s);
    if (out4)
        for (int a = 0; a < 4; ++a) out4[a] = ctx->prof[a];
    for (int a = 0; a < 4; ++a) ctx->prof[a] = 0.0;
    ctx->prof_stride = stride;
    return SICP_OK;
}

}  // extern "C"
