// Host runtime and C ABI of the solver: argument validation, operator
// assembly (Supplementary Note 1), the RK4 driver with CUDA-graph capture and
// device-side stop decision, and the host/device pointer handling.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <cstdlib>
#include <numeric>
#include <string>
#include <vector>

#include "qpr_internal.cuh"

using qpr::Ctl;
using qpr::HostOps;

struct qpr_ctx {
    int device = 0;
    int64_t n = 0;
    int np = 0;
    double alpha = 0.0, omega = 0.0;
    qpr_options opt{};
    double spread = 0.0;   // estimated lambda_max - lambda_min of H
    double cmax = 1.0;     // max column sum of G
    // device operators
    double *d_H = nullptr;
    int *d_hptr = nullptr, *d_hcol = nullptr;
    double *d_hval = nullptr;
    int *d_rowseg = nullptr;
    int2 *d_seg = nullptr;
    int backend = QPR_BACKEND_SPARSE;
    int *d_sptr = nullptr, *d_scol = nullptr;
    double *d_sval = nullptr;
    unsigned char *d_dang = nullptr;
    double *d_c = nullptr;
    // device work
    double *d_state = nullptr;  // y, z, ya, yb: 2 planes each
    double *d_mix64 = nullptr;  // mixed form: R, F (2 planes each)
    float *d_mix32 = nullptr;   // mixed form: F32, D, Dlo, da, db, Ghi, Glo (2 planes each)
    float *d_g32 = nullptr, *d_hval32 = nullptr, *d_c32 = nullptr, *d_sval32 = nullptr, *d_partials32 = nullptr;
    __nv_bfloat16 *d_hsplit = nullptr;  // dense mixed form: H split into 3 BF16 planes
    __nv_bfloat16 *d_dsplit = nullptr;  // dense mixed form: 3 delta-split buffers of 6 planes
    int2 *d_pairs_tc = nullptr;
    qpr::TcMaps tcmaps{};
    int2 *d_colkh = nullptr;    // column-block form: packed CSR, plan arrays, X = H delta
    int *d_colint = nullptr;    // q | sb | wb
    int4 *d_colpieces = nullptr;
    float *d_X = nullptr;
    qpr::ColMaps colmaps{};
    int persist_grid = 0;       // > 0: the persistent column-block form, CTAs per launch
    int persist_smem = 0, epi_off = 0;
    qpr::MixedWork mw{};
    double *d_g = nullptr;
    double *d_partials = nullptr;
    int2 *d_pairs = nullptr;
    int4 *d_epi_pairs = nullptr;
    Ctl *d_ctl = nullptr;
    double *d_io = nullptr;     // staging for host density matrices (interleaved)
    double *d_p = nullptr;      // populations staging
    float *d_rkf = nullptr;     // RKF45: D1, Dlo1, acc, Flo (2 planes each), the two compact diagonals
    cudaGraphExec_t graph_rkf = nullptr;  // RKF45: refresh + ref_refresh attempts
    double rkf_key[3] = {0, 0, 0};        // h0, Tol, h_max of the captured graph's first block (unused by kernels)
    Ctl *h_ctl = nullptr;       // pinned
    cudaStream_t stream = nullptr;
    cudaEvent_t ev = nullptr;
    cudaGraphExec_t graph = nullptr;
    cudaGraphExec_t graph_c = nullptr;  // mixed form: a block of steps without the refresh
    int graph_steps = 0;
    qpr::DevOps ops{};
    qpr::Work work{};
    std::string err;
    bool poisoned = false;
    int64_t launches = 0;  // kernels launched by the current call
};

namespace {

thread_local std::string g_create_error;

const char *kStatusNames[] = {"QPR_OK",         "QPR_E_ARG",           "QPR_E_GRAPH",
                              "QPR_E_CUDA",     "QPR_E_OOM",           "QPR_E_UNSTABLE",
                              "QPR_E_NOT_CONVERGED", "QPR_E_TIMEOUT",  "QPR_E_NONFINITE"};

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

qpr_status fail(qpr_ctx *ctx, qpr_status st, const std::string &msg) {
    if (ctx) ctx->err = msg;
    return st;
}

qpr_status cuda_fail(qpr_ctx *ctx, cudaError_t e, const char *what) {
    std::string msg = std::string(what) + ": " + cudaGetErrorString(e);
    if (e == cudaErrorMemoryAllocation) return fail(ctx, QPR_E_OOM, msg);
    if (ctx) ctx->poisoned = true;
    return fail(ctx, QPR_E_CUDA, msg);
}

#define QPR_CUDA(ctx, call)                                   \
    do {                                                      \
        cudaError_t e_ = (call);                              \
        if (e_ != cudaSuccess) return cuda_fail(ctx, e_, #call); \
    } while (0)

// A pointer the kernels can read directly: device or managed memory.
bool is_device_ptr(const void *p) {
    cudaPointerAttributes attr;
    if (cudaPointerGetAttributes(&attr, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return attr.type == cudaMemoryTypeDevice || attr.type == cudaMemoryTypeManaged;
}

qpr_status sync_ctx(qpr_ctx *ctx) {
    cudaError_t e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaStreamSynchronize");
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(ctx, e, "kernel launch");
    return QPR_OK;
}

void launch_stage(qpr_ctx *ctx, int s) {
    if (ctx->backend == QPR_BACKEND_DENSE) qpr::launch_stage_fp64(s, ctx->ops, ctx->work, ctx->stream);
    else qpr::launch_stage_sparse(s, ctx->ops, ctx->work, ctx->stream);
}

void enqueue_step(qpr_ctx *ctx) {
    const qpr::Work &w = ctx->work;
    const double *yin[5] = {w.y, w.y, w.ya, w.yb, w.ya};
    for (int s = 1; s <= 4; ++s) {
        qpr::launch_gain(s, ctx->ops, yin[s], w, ctx->stream);
        launch_stage(ctx, s);
    }
}

qpr_status ensure_graph(qpr_ctx *ctx) {
    if (ctx->graph || ctx->opt.graph_steps <= 0) return QPR_OK;
    cudaGraph_t g = nullptr;
    QPR_CUDA(ctx, cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal));
    for (int s = 0; s < ctx->opt.graph_steps; ++s) enqueue_step(ctx);
    cudaError_t e = cudaStreamEndCapture(ctx->stream, &g);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaStreamEndCapture");
    e = cudaGraphInstantiate(&ctx->graph, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        ctx->graph = nullptr;
        return cuda_fail(ctx, e, "cudaGraphInstantiate");
    }
    ctx->graph_steps = ctx->opt.graph_steps;
    return QPR_OK;
}

// Bring a caller density matrix (host or device) into the y planes.
qpr_status import_rho(qpr_ctx *ctx, const void *rho, double *planes) {
    const size_t bytes = (size_t)ctx->n * ctx->n * 2 * sizeof(double);
    const double *src = (const double *)rho;
    if (!is_device_ptr(rho)) {
        QPR_CUDA(ctx, cudaMemcpyAsync(ctx->d_io, rho, bytes, cudaMemcpyHostToDevice, ctx->stream));
        src = ctx->d_io;
    }
    qpr::launch_import(src, (int)ctx->n, ctx->np, planes, ctx->stream);
    ctx->launches += 1;
    return QPR_OK;
}

// The solver's starting state: y (FP64 form) or R with a zero delta (mixed
// form, whose first refresh normalises R + delta).
qpr_status import_state(qpr_ctx *ctx, const void *rho) {
    if (ctx->opt.precision != QPR_MIXED) return import_rho(ctx, rho, ctx->work.y);
    qpr_status st = import_rho(ctx, rho, ctx->mw.R);
    if (st != QPR_OK) return st;
    const size_t plane = (size_t)ctx->np * ctx->np;
    QPR_CUDA(ctx, cudaMemsetAsync(ctx->mw.D, 0, 4 * plane * sizeof(float), ctx->stream));
    return QPR_OK;
}

qpr_status export_rho(qpr_ctx *ctx, const double *planes, int use_scale, void *rho) {
    const size_t bytes = (size_t)ctx->n * ctx->n * 2 * sizeof(double);
    ctx->launches += 1;
    if (is_device_ptr(rho)) {
        qpr::launch_export(planes, (int)ctx->n, ctx->np, ctx->d_ctl, use_scale, (double *)rho, ctx->stream);
    } else {
        qpr::launch_export(planes, (int)ctx->n, ctx->np, ctx->d_ctl, use_scale, ctx->d_io, ctx->stream);
        QPR_CUDA(ctx, cudaMemcpyAsync(rho, ctx->d_io, bytes, cudaMemcpyDeviceToHost, ctx->stream));
    }
    return QPR_OK;
}

qpr_status check_usable(qpr_ctx *ctx) {
    if (!ctx) return QPR_E_ARG;
    if (ctx->poisoned) return fail(ctx, QPR_E_CUDA, "context poisoned by an earlier CUDA error: " + ctx->err);
    return QPR_OK;
}

// Run RK4 steps until the device sets `done`. Leaves the unnormalised state
// in y and 1 / tr(y) in ctl->scale.
qpr_status run_rk4(qpr_ctx *ctx, double dt, double tol, int64_t max_steps) {
    Ctl *h = ctx->h_ctl;
    memset(h, 0, sizeof(Ctl));
    h->max_steps = max_steps;
    h->tol = tol;
    h->dt = dt;
    h->scale = 1.0;
    QPR_CUDA(ctx, cudaMemcpyAsync(ctx->d_ctl, h, sizeof(Ctl), cudaMemcpyHostToDevice, ctx->stream));
    qpr_status st = ensure_graph(ctx);
    if (st != QPR_OK) return st;
    const int chunk = ctx->graph ? ctx->graph_steps : 1;
    // Each stage-2 gain kernel stops the run once max_steps is reached, so
    // the loop ends after at most ceil((max_steps + 1) / chunk) launches.
    for (;;) {
        if (ctx->graph) {
            QPR_CUDA(ctx, cudaGraphLaunch(ctx->graph, ctx->stream));
        } else {
            enqueue_step(ctx);
        }
        ctx->launches += 8 * (int64_t)chunk;
        QPR_CUDA(ctx, cudaMemcpyAsync(h, ctx->d_ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, ctx->stream));
        st = sync_ctx(ctx);
        if (st != QPR_OK) return st;
        if (h->done) break;
    }
    return QPR_OK;
}

// One block of the persistent mixed form: the exact refresh (unless
// `refresh` is false), then `steps` delta steps in one launch.
qpr_status launch_mixed_block(qpr_ctx *ctx, int steps, bool refresh) {
    if (refresh) {
        qpr::launch_mixed_refresh(ctx->ops, ctx->mw, ctx->stream);
        ctx->launches += qpr::kMixedLaunchesPerRefresh;
    }
    QPR_CUDA(ctx, qpr::launch_cols_block(ctx->ops, ctx->mw, steps, ctx->persist_grid, ctx->stream));
    ctx->launches += 1;
    return QPR_OK;
}

int mixed_launches_per_step(const qpr_ctx *ctx) {
    if (ctx->mw.cmaps) return qpr::kMixedLaunchesPerStepCols;
    return (ctx->mw.splitD ? 2 : 1) * qpr::kMixedLaunchesPerStep;
}

void enqueue_mixed_block(qpr_ctx *ctx, int steps, bool refresh = true) {
    if (refresh) qpr::launch_mixed_refresh(ctx->ops, ctx->mw, ctx->stream);
    for (int k = 0; k < steps; ++k)
        for (int s = 1; s <= 4; ++s) qpr::launch_mixed_stage(s, ctx->ops, ctx->mw, ctx->stream);
}

// Two graphs: refresh + ref_refresh steps, and ref_refresh steps alone.
qpr_status ensure_mixed_graph(qpr_ctx *ctx) {
    if (ctx->graph || ctx->opt.graph_steps <= 0 || ctx->persist_grid > 0) return QPR_OK;
    for (int k = 0; k < 2; ++k) {
        cudaGraph_t g = nullptr;
        cudaGraphExec_t *dst = k == 0 ? &ctx->graph : &ctx->graph_c;
        QPR_CUDA(ctx, cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal));
        enqueue_mixed_block(ctx, ctx->opt.ref_refresh, k == 0);
        cudaError_t e = cudaStreamEndCapture(ctx->stream, &g);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaStreamEndCapture");
        e = cudaGraphInstantiate(dst, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) {
            *dst = nullptr;
            if (ctx->graph) cudaGraphExecDestroy(ctx->graph);
    if (ctx->graph_c) cudaGraphExecDestroy(ctx->graph_c);
            ctx->graph = nullptr;
            return cuda_fail(ctx, e, "cudaGraphInstantiate");
        }
    }
    ctx->graph_steps = ctx->opt.ref_refresh;
    return QPR_OK;
}

qpr_status read_ctl(qpr_ctx *ctx) {
    QPR_CUDA(ctx, cudaMemcpyAsync(ctx->h_ctl, ctx->d_ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, ctx->stream));
    return sync_ctx(ctx);
}

// Mixed form: blocks of (exact refresh + ref_refresh delta steps) until the
// device stops. A stop on the FP32-accurate estimate is confirmed by an exact
// refresh at the same step; the run always ends with a refresh, so R holds
// the normalised returned state and resid_exact its exact FP64 residual.
//
// Steady-state solves (tol > 0) with adaptive_refresh lengthen the window
// between refreshes as the residual falls: the FP32 error a window adds to
// the state grows about as (window steps)^2 x ||f||, so a block continues
// without a refresh while (steps since the refresh)^2 x r stays within
// ref_refresh^2 x r0 (r: the residual estimate of the last step, r0: the
// one after the first block), at most kMaxRefreshGrowth x ref_refresh steps.
// The batched solver applies the same rule per problem.
using qpr::kMaxRefreshGrowth;
qpr_status run_mixed(qpr_ctx *ctx, double dt, double tol, int64_t max_steps) {
    Ctl *h = ctx->h_ctl;
    memset(h, 0, sizeof(Ctl));
    h->max_steps = max_steps;
    h->tol = tol;
    h->dt = dt;
    h->scale = 1.0;
    h->resid_exact_step = -1;
    h->gb_extra = (ctx->persist_grid > 0 && ctx->opt.test_fault) ? 1u : 0u;
    QPR_CUDA(ctx, cudaMemcpyAsync(ctx->d_ctl, h, sizeof(Ctl), cudaMemcpyHostToDevice, ctx->stream));
    qpr_status st = ensure_mixed_graph(ctx);
    if (st != QPR_OK) return st;
    const int block = ctx->opt.ref_refresh;
    const bool adaptive = tol > 0.0 && ctx->opt.adaptive_refresh != 0;
    bool refresh = true;
    int64_t since = 0;  // steps since the last refresh
    double r0 = -1.0;
    for (;;) {
        qpr::NvtxRange nvtx_block(refresh ? "block (refresh + steps)" : "block (steps)");
        if (ctx->persist_grid > 0) {
            st = launch_mixed_block(ctx, block, refresh);
            if (st != QPR_OK) return st;
        } else {
            cudaGraphExec_t g = refresh ? ctx->graph : ctx->graph_c;
            if (g) {
                QPR_CUDA(ctx, cudaGraphLaunch(g, ctx->stream));
            } else {
                enqueue_mixed_block(ctx, block, refresh);
            }
            ctx->launches += (refresh ? qpr::kMixedLaunchesPerRefresh : 0) +
                             mixed_launches_per_step(ctx) * (int64_t)block;
        }
        since = (refresh ? 0 : since) + block;
        st = read_ctl(ctx);
        if (st != QPR_OK) return st;
        if (h->err_timeout) return fail(ctx, QPR_E_TIMEOUT, "a device-side wait gave up (err_timeout set by a stage kernel)");
        if (!h->done) {
            refresh = true;
            if (adaptive) {
                const double r = h->resid;
                if (r0 < 0.0) r0 = r;
                const double next = (double)(since + block);
                refresh = !(r > 0.0 && next <= (double)kMaxRefreshGrowth * block &&
                            next * next * r <= (double)block * block * r0);
            }
            continue;
        }
        if (h->status == qpr::kCtlNonFinite) return QPR_OK;
        if (h->resid_exact_step == h->step) return QPR_OK;  // stopped by an exact refresh at this step
        // confirm (or finish) with an exact refresh at the current step
        h->done = 0;
        const int prev = h->status;
        h->status = qpr::kCtlRunning;
        QPR_CUDA(ctx, cudaMemcpyAsync(ctx->d_ctl, h, sizeof(Ctl), cudaMemcpyHostToDevice, ctx->stream));
        qpr::launch_mixed_refresh(ctx->ops, ctx->mw, ctx->stream);
        ctx->launches += qpr::kMixedLaunchesPerRefresh;
        st = read_ctl(ctx);
        if (st != QPR_OK) return st;
        if (h->err_timeout) return fail(ctx, QPR_E_TIMEOUT, "a device-side wait gave up (err_timeout set by a stage kernel)");
        if (h->done) return QPR_OK;  // converged, max steps or non-finite, decided exactly
        if (prev == qpr::kCtlMaxSteps) return QPR_OK;
        // the estimate passed but the exact residual did not: keep stepping
        // from this refresh
        refresh = !adaptive;
        since = 0;
    }
}

// RKF45 needs the column-block form of the mixed sparse stage: allocate
// its buffers (the second delta pair, the running sum, the low part of F,
// the two compact diagonals), its tensor map and kernel attributes on the
// first call.
qpr_status ensure_rkf(qpr_ctx *ctx) {
    if (ctx->opt.precision != QPR_MIXED || !ctx->mw.cmaps)
        return fail(ctx, QPR_E_ARG, "qpr_rkf45 needs QPR_MIXED with a column-block sparse form "
                                    "(COLUMNS, COLUMNS_PERSISTENT or COLUMNS_GATHER)");
    if (ctx->d_rkf) return QPR_OK;
    const size_t plane = (size_t)ctx->np * ctx->np;
    QPR_CUDA(ctx, cudaMalloc(&ctx->d_rkf, (8 * plane + 2 * (size_t)ctx->np) * sizeof(float)));
    QPR_CUDA(ctx, cudaMemsetAsync(ctx->d_rkf, 0, (8 * plane + 2 * (size_t)ctx->np) * sizeof(float), ctx->stream));
    qpr::MixedWork &mw = ctx->mw;
    mw.D1 = ctx->d_rkf;
    mw.Dlo1 = ctx->d_rkf + 2 * plane;
    mw.acc = ctx->d_rkf + 4 * plane;
    mw.Flo = ctx->d_rkf + 6 * plane;
    mw.pvd = ctx->d_rkf + 8 * plane;
    if (!qpr::make_rkf_map(ctx->ops, mw.D1, &ctx->colmaps)) return fail(ctx, QPR_E_CUDA, "cuTensorMapEncodeTiled failed");
    QPR_CUDA(ctx, qpr::init_rkf(ctx->ops.col_launch_smem, ctx->ops.col_gather != 0));
    return QPR_OK;
}

void enqueue_rkf_block(qpr_ctx *ctx, int attempts) {
    qpr::launch_rkf_refresh(ctx->ops, ctx->mw, ctx->stream);
    for (int k = 0; k < attempts; ++k)
        for (int s = 1; s <= qpr::kRkfStages; ++s) qpr::launch_rkf_stage(s, ctx->ops, ctx->mw, ctx->stream);
}

qpr_status ensure_rkf_graph(qpr_ctx *ctx) {
    if (ctx->graph_rkf || ctx->opt.graph_steps <= 0) return QPR_OK;
    cudaGraph_t g = nullptr;
    QPR_CUDA(ctx, cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal));
    enqueue_rkf_block(ctx, ctx->opt.ref_refresh);
    cudaError_t e = cudaStreamEndCapture(ctx->stream, &g);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaStreamEndCapture");
    e = cudaGraphInstantiate(&ctx->graph_rkf, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        ctx->graph_rkf = nullptr;
        return cuda_fail(ctx, e, "cudaGraphInstantiate");
    }
    return QPR_OK;
}

// Blocks of (exact refresh + ref_refresh RKF45 attempts) until the device
// stops: the time end of a trajectory, max_steps accepted steps, a
// non-finite value, or a residual estimate below tol, which an exact
// refresh confirms (as in run_mixed). The run ends with a refresh, so R
// holds the returned state. Bounded: at most max_attempts attempts.
qpr_status run_rkf45(qpr_ctx *ctx, double h0, double step_tol, double hmax, double tend, double tol,
                     int64_t max_steps, int64_t max_attempts, int order) {
    Ctl *h = ctx->h_ctl;
    memset(h, 0, sizeof(Ctl));
    h->max_steps = max_steps;
    h->tol = tol;
    h->dt = h0;
    h->scale = 1.0;
    h->resid_exact_step = -1;
    h->rk_h = h0;
    h->rk_hmax = hmax;
    h->rk_tol = step_tol;
    h->rk_tend = tend;
    h->rk_order = order;
    h->rk_hf = (float)h0;
    h->rk_hl = (float)(h0 - (double)(float)h0);
    QPR_CUDA(ctx, cudaMemcpyAsync(ctx->d_ctl, h, sizeof(Ctl), cudaMemcpyHostToDevice, ctx->stream));
    qpr_status st = ensure_rkf_graph(ctx);
    if (st != QPR_OK) return st;
    const int block = ctx->opt.ref_refresh;
    int64_t attempts = 0;
    for (;;) {
        if (ctx->graph_rkf) {
            QPR_CUDA(ctx, cudaGraphLaunch(ctx->graph_rkf, ctx->stream));
        } else {
            enqueue_rkf_block(ctx, block);
        }
        ctx->launches += qpr::kRkfLaunchesPerRefresh + (int64_t)qpr::kRkfLaunchesPerAttempt * block;
        attempts += block;
        st = read_ctl(ctx);
        if (st != QPR_OK) return st;
        if (h->err_timeout) return fail(ctx, QPR_E_TIMEOUT, "a device-side wait gave up (err_timeout set by a stage kernel)");
        if (!h->done) {
            if (attempts >= max_attempts) break;
            continue;
        }
        if (h->status == qpr::kCtlNonFinite) return QPR_OK;
        if (h->status != qpr::kCtlTimeReached && h->resid_exact_step == h->step) return QPR_OK;
        // confirm a candidate (or fold the final delta into R) with an exact refresh
        h->done = 0;
        const int prev = h->status;
        h->status = qpr::kCtlRunning;
        QPR_CUDA(ctx, cudaMemcpyAsync(ctx->d_ctl, h, sizeof(Ctl), cudaMemcpyHostToDevice, ctx->stream));
        qpr::launch_rkf_refresh(ctx->ops, ctx->mw, ctx->stream);
        ctx->launches += qpr::kRkfLaunchesPerRefresh;
        st = read_ctl(ctx);
        if (st != QPR_OK) return st;
        if (h->err_timeout) return fail(ctx, QPR_E_TIMEOUT, "a device-side wait gave up (err_timeout set by a stage kernel)");
        if (prev == qpr::kCtlTimeReached || prev == qpr::kCtlMaxSteps) {
            if (h->status != qpr::kCtlNonFinite) h->status = prev;
            return QPR_OK;
        }
        if (h->done) return QPR_OK;  // converged, max steps or non-finite, decided exactly
        if (attempts >= max_attempts) break;
    }
    // attempt budget spent: fold the delta into R and report the state reached
    h->done = 0;
    h->status = qpr::kCtlRunning;
    QPR_CUDA(ctx, cudaMemcpyAsync(ctx->d_ctl, h, sizeof(Ctl), cudaMemcpyHostToDevice, ctx->stream));
    qpr::launch_rkf_refresh(ctx->ops, ctx->mw, ctx->stream);
    ctx->launches += qpr::kRkfLaunchesPerRefresh;
    st = read_ctl(ctx);
    if (st != QPR_OK) return st;
    if (!h->done) h->status = qpr::kCtlMaxSteps;
    return QPR_OK;
}

}  // namespace

namespace qpr {

// Power iteration for the extreme eigenvalues of the symmetric CSR matrix
// H; returns an estimate of lambda_max - lambda_min (with a 2% margin, and
// never above the Gershgorin bound).
double estimate_spread(int64_t n, const std::vector<int64_t> &ptr, const std::vector<int> &col,
                       const std::vector<double> &val) {
    if (val.empty()) return 0.0;
    auto matvec = [&](const std::vector<double> &x, std::vector<double> &y, double shift) {
        for (int64_t i = 0; i < n; ++i) {
            double s = -shift * x[i];
            for (int64_t q = ptr[i]; q < ptr[i + 1]; ++q) s += val[q] * x[col[q]];
            y[i] = s;
        }
    };
    auto dominant = [&](double shift) {
        std::vector<double> x(n), y(n);
        for (int64_t i = 0; i < n; ++i) x[i] = 1.0 + 0.37 * sin(0.7 * (double)i + 0.1);
        double lam = 0.0;
        for (int it = 0; it < 400; ++it) {
            double nx = 0.0;
            for (double v : x) nx += v * v;
            nx = sqrt(nx);
            if (nx == 0.0) return 0.0;
            for (double &v : x) v /= nx;
            matvec(x, y, shift);
            double rq = 0.0;
            for (int64_t i = 0; i < n; ++i) rq += x[i] * y[i];
            lam = rq;
            x.swap(y);
        }
        return lam;
    };
    double gersh = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        double r = 0.0;
        for (int64_t q = ptr[i]; q < ptr[i + 1]; ++q) r += fabs(val[q]);
        gersh = std::max(gersh, r);
    }
    const double l1 = dominant(0.0);
    const double l2 = dominant(l1);  // eigenvalue of H - l1 I farthest from 0
    double spread = fabs(l2) * 1.02 + 1e-12;
    return std::min(spread, 2.0 * gersh);
}

void set_create_error(const std::string &msg) { g_create_error = msg; }

void row_segments(const HostOps &h, int np, int len, std::vector<int> &rowseg, std::vector<int2> &seg) {
    rowseg.assign((size_t)np + 1, 0);
    seg.clear();
    for (int i = 0; i < np; ++i) {
        rowseg[i] = (int)seg.size();
        if (i < h.n)
            for (int64_t q = h.hptr[i]; q < h.hptr[i + 1]; q += len)
                seg.push_back(make_int2((int)q, (int)std::min<int64_t>(q + len, h.hptr[i + 1])));
    }
    rowseg[np] = (int)seg.size();
}

// Operators of Supplementary Note 1 on the host: adjacency (A_ij = w for the
// link j -> i, duplicates summed, self-loops and zero weights dropped),
// out-degrees, CSR of H (Eq. S6) and of S (column-normalised adjacency
// restricted to columns with out-links), dangling flags.
qpr_status assemble_host(int64_t n, int64_t m, const int64_t *src, const int64_t *dst, const double *w, int h_diag,
                         HostOps &out, std::string &err) {
    out.n = n;
    for (int64_t e = 0; e < m; ++e) {
        const double we = w ? w[e] : 1.0;
        if (src[e] < 0 || src[e] >= n || dst[e] < 0 || dst[e] >= n)
            { err = "edge " + std::to_string(e) + " has a node index outside [0, n)"; return QPR_E_GRAPH; }
        if (!std::isfinite(we) || we < 0.0)
            { err = "edge " + std::to_string(e) + " has a negative or non-finite weight"; return QPR_E_GRAPH; }
    }

    // ---- adjacency: A_ij = w for the link j -> i; duplicates sum ----
    struct Ent { int64_t i, j; double a; };
    std::vector<Ent> ents;
    ents.reserve((size_t)m);
    for (int64_t e = 0; e < m; ++e) {
        const double we = w ? w[e] : 1.0;
        if (src[e] == dst[e] || we == 0.0) continue;
        ents.push_back({dst[e], src[e], we});
    }
    std::stable_sort(ents.begin(), ents.end(), [](const Ent &x, const Ent &y) {
        return x.i != y.i ? x.i < y.i : x.j < y.j;
    });
    std::vector<Ent> A;
    for (const Ent &x : ents) {
        if (!A.empty() && A.back().i == x.i && A.back().j == x.j) A.back().a += x.a;
        else A.push_back(x);
    }
    std::vector<double> &outdeg = out.outdeg;
    outdeg.assign(n, 0.0);
    for (const Ent &x : A) outdeg[x.j] += x.a;

    // ---- H (Eq. S6): H_ij = -max(A_ij, A_ji) off the diagonal ----
    std::vector<Ent> Hs;
    Hs.reserve(A.size() * 2);
    for (const Ent &x : A) {
        Hs.push_back({x.i, x.j, x.a});
        Hs.push_back({x.j, x.i, x.a});
    }
    std::sort(Hs.begin(), Hs.end(), [](const Ent &x, const Ent &y) {
        return x.i != y.i ? x.i < y.i : x.j < y.j;
    });
    std::vector<Ent> Hu;  // unique (i, j) with -max
    for (const Ent &x : Hs) {
        if (!Hu.empty() && Hu.back().i == x.i && Hu.back().j == x.j) Hu.back().a = std::max(Hu.back().a, x.a);
        else Hu.push_back(x);
    }
    std::vector<int64_t> &hptr = out.hptr;
    std::vector<int> &hcol = out.hcol;
    std::vector<double> &hval = out.hval;
    hptr.assign(n + 1, 0);
    {
        size_t q = 0;
        for (int64_t i = 0; i < n; ++i) {
            hptr[i] = (int64_t)hcol.size();
            bool diag_done = false;
            const double hd = (h_diag == QPR_HDIAG_NEG_OUTDEG) ? -outdeg[i] : 0.0;
            while (q < Hu.size() && Hu[q].i == i) {
                if (!diag_done && Hu[q].j > i) {
                    if (hd != 0.0) { hcol.push_back((int)i); hval.push_back(hd); }
                    diag_done = true;
                }
                hcol.push_back((int)Hu[q].j);
                hval.push_back(-Hu[q].a);
                ++q;
            }
            if (!diag_done && hd != 0.0) { hcol.push_back((int)i); hval.push_back(hd); }
        }
        hptr[n] = (int64_t)hcol.size();
    }

    // ---- S restricted to columns with out-links, CSR by rows ----
    std::vector<int> &sptr = out.sptr, &scol = out.scol;
    std::vector<double> &sval = out.sval;
    sptr.assign(n + 1, 0);
    scol.reserve(A.size());
    sval.reserve(A.size());
    {
        size_t q = 0;
        for (int64_t i = 0; i < n; ++i) {
            sptr[i] = (int)scol.size();
            while (q < A.size() && A[q].i == i) {
                scol.push_back((int)A[q].j);
                sval.push_back(A[q].a / outdeg[A[q].j]);
                ++q;
            }
        }
        sptr[n] = (int)scol.size();
    }
    std::vector<unsigned char> &dang = out.dang;
    dang.assign(n, 0);
    for (int64_t j = 0; j < n; ++j) dang[j] = (outdeg[j] > 0.0) ? 0 : 1;
    return QPR_OK;
}

// c_j = sum_i G_ij = alpha (column sum of S) + (1 - alpha) (column sum of F),
// padded with zeros to np; *cmax receives the largest.
std::vector<double> column_sums_G(const HostOps &h, double alpha, int np, double *cmax) {
    std::vector<double> c(np, 0.0), scs(h.n, 0.0);
    for (size_t q = 0; q < h.sval.size(); ++q) scs[h.scol[q]] += h.sval[q];
    const double fcol = (double)(h.n - 1) / (double)(h.n - 1);
    double mx = 0.0;
    for (int64_t j = 0; j < h.n; ++j) {
        const double sj = h.dang[j] ? 1.0 : scs[j];
        c[j] = alpha * sj + (1.0 - alpha) * fcol;
        mx = std::max(mx, c[j]);
    }
    if (cmax) *cmax = mx;
    return c;
}

}  // namespace qpr

namespace {

}  // namespace

extern "C" {

qpr_status qpr_default_options(qpr_options *opt) {
    if (!opt) return QPR_E_ARG;
    memset(opt, 0, sizeof(*opt));
    opt->precision = QPR_FP64;
    opt->h_diag = QPR_HDIAG_ZERO;
    opt->dangling = QPR_DANGLING_F;
    opt->graph_steps = 32;
    opt->cuda_stream = nullptr;
    opt->device = -1;
    opt->backend = QPR_BACKEND_AUTO;
    opt->ref_refresh = 32;
    opt->adaptive_refresh = 1;
    return QPR_OK;
}

const char *qpr_status_string(qpr_status s) {
    if ((int)s < 0 || (int)s > 8) return "QPR_E_UNKNOWN";
    return kStatusNames[(int)s];
}

const char *qpr_last_error(const qpr_ctx *ctx) {
    if (!ctx) return g_create_error.c_str();
    return ctx->err.c_str();
}

int64_t qpr_n(const qpr_ctx *ctx) { return ctx ? ctx->n : 0; }
int32_t qpr_backend(const qpr_ctx *ctx) { return ctx ? ctx->backend : 0; }

int32_t qpr_sparse_form(const qpr_ctx *ctx) {
    if (!ctx || ctx->opt.precision != QPR_MIXED || ctx->mw.splitD) return 0;
    if (!ctx->mw.cmaps) return QPR_SPARSE_FORM_TILES;
    if (ctx->ops.col_gather) return QPR_SPARSE_FORM_COLUMNS_GATHER;
    return ctx->persist_grid > 0 ? QPR_SPARSE_FORM_COLUMNS_PERSISTENT : QPR_SPARSE_FORM_COLUMNS;
}
qpr_status qpr_sparse_plan(const qpr_ctx *ctx, int32_t *out) {
    if (!ctx || !out) return QPR_E_ARG;
    out[0] = out[1] = out[2] = out[3] = 0;
    if (!ctx->mw.cmaps) return QPR_OK;
    const qpr::DevOps &o = ctx->ops;
    out[0] = o.col_splits;
    out[1] = o.col_gather ? qpr::kColGatherWidth : qpr::kColWidth;
    out[2] = (o.np / out[1]) * o.col_splits;
    out[3] = o.col_smem;
    return QPR_OK;
}
double qpr_h_spread(const qpr_ctx *ctx) { return ctx ? ctx->spread : 0.0; }

double qpr_max_stable_dt(const qpr_ctx *ctx) {
    if (!ctx) return 0.0;
    const double rate = (1.0 - ctx->omega) * ctx->spread + 2.0 * ctx->omega * ctx->cmax;
    return rate > 0.0 ? 2.5 / rate : INFINITY;
}

void qpr_destroy(qpr_ctx *ctx) {
    if (!ctx) return;
    DeviceGuard dg(ctx->device);
    if (ctx->stream) cudaStreamSynchronize(ctx->stream);
    if (ctx->graph) cudaGraphExecDestroy(ctx->graph);
    if (ctx->graph_c) cudaGraphExecDestroy(ctx->graph_c);
    if (ctx->graph_rkf) cudaGraphExecDestroy(ctx->graph_rkf);
    cudaFree(ctx->d_rkf);
    cudaFree(ctx->d_H);
    cudaFree(ctx->d_hptr);
    cudaFree(ctx->d_rowseg);
    cudaFree(ctx->d_seg);
    cudaFree(ctx->d_hcol);
    cudaFree(ctx->d_hval);
    cudaFree(ctx->d_sptr);
    cudaFree(ctx->d_scol);
    cudaFree(ctx->d_sval);
    cudaFree(ctx->d_dang);
    cudaFree(ctx->d_c);
    cudaFree(ctx->d_state);
    cudaFree(ctx->d_mix64);
    cudaFree(ctx->d_mix32);
    cudaFree(ctx->d_g32);
    cudaFree(ctx->d_colkh);
    cudaFree(ctx->d_colint);
    cudaFree(ctx->d_colpieces);
    cudaFree(ctx->d_X);
    cudaFree(ctx->d_sval32);
    cudaFree(ctx->d_partials32);
    cudaFree(ctx->d_hval32);
    cudaFree(ctx->d_c32);
    cudaFree(ctx->d_hsplit);
    cudaFree(ctx->d_dsplit);
    cudaFree(ctx->d_pairs_tc);
    cudaFree(ctx->d_g);
    cudaFree(ctx->d_partials);
    cudaFree(ctx->d_pairs);
    cudaFree(ctx->d_epi_pairs);
    cudaFree(ctx->d_ctl);
    cudaFree(ctx->d_io);
    cudaFree(ctx->d_p);
    if (ctx->h_ctl) cudaFreeHost(ctx->h_ctl);
    if (ctx->ev) cudaEventDestroy(ctx->ev);
    if (ctx->stream) cudaStreamDestroy(ctx->stream);
    cudaGetLastError();
    delete ctx;
}

qpr_status qpr_create(qpr_ctx **out, int64_t n, int64_t m, const int64_t *src, const int64_t *dst,
                      const double *w, double alpha, double omega, const qpr_options *opt) {
    qpr::NvtxRange nvtx_range("qpr_create");
    g_create_error.clear();
    if (!out) {
        g_create_error = "out is NULL";
        return QPR_E_ARG;
    }
    *out = nullptr;
    qpr_options o;
    qpr_default_options(&o);
    if (opt) o = *opt;
    auto arg_err = [&](qpr_status st, const std::string &msg) {
        g_create_error = msg;
        return st;
    };
    if (n < 2) return arg_err(QPR_E_ARG, "n must be at least 2");
    if (n > 65536) return arg_err(QPR_E_ARG, "n above 65536 is not supported");
    if (m < 0 || (m > 0 && (!src || !dst))) return arg_err(QPR_E_ARG, "edge arrays missing");
    if (!(alpha >= 0.0 && alpha <= 1.0)) return arg_err(QPR_E_ARG, "alpha must lie in [0, 1]");
    if (!(omega >= 0.0 && omega <= 1.0)) return arg_err(QPR_E_ARG, "omega must lie in [0, 1]");
    if (o.precision != QPR_FP64 && o.precision != QPR_MIXED) return arg_err(QPR_E_ARG, "unsupported precision");
    if (o.precision == QPR_MIXED && (o.ref_refresh < 1 || o.ref_refresh > 4096))
        return arg_err(QPR_E_ARG, "ref_refresh outside [1, 4096]");
    if (o.h_diag != QPR_HDIAG_ZERO && o.h_diag != QPR_HDIAG_NEG_OUTDEG)
        return arg_err(QPR_E_ARG, "unknown h_diag mode");
    if (o.dangling != QPR_DANGLING_F && o.dangling != QPR_DANGLING_UNIFORM)
        return arg_err(QPR_E_ARG, "unknown dangling mode");
    if (o.graph_steps < 0 || o.graph_steps > 4096) return arg_err(QPR_E_ARG, "graph_steps outside [0, 4096]");
    if (o.backend < QPR_BACKEND_AUTO || o.backend > QPR_BACKEND_SPARSE) return arg_err(QPR_E_ARG, "unknown backend");
    if (o.sparse_form < QPR_SPARSE_FORM_AUTO || o.sparse_form > QPR_SPARSE_FORM_COLUMNS_GATHER || o.sparse_form == 4)
        return arg_err(QPR_E_ARG, "unknown sparse_form");
    if (o.test_fault != 0 && o.test_fault != 1) return arg_err(QPR_E_ARG, "test_fault must be 0 or 1");
    if (o.row_splits < 0 || o.row_splits > 64) return arg_err(QPR_E_ARG, "row_splits outside [0, 64]");
    HostOps hops;
    {
        std::string aerr;
        const qpr_status ast = assemble_host(n, m, src, dst, w, o.h_diag, hops, aerr);
        if (ast != QPR_OK) return arg_err(ast, aerr);
    }
    const std::vector<int64_t> &hptr = hops.hptr;
    const std::vector<int> &hcol = hops.hcol;
    const std::vector<double> &hval = hops.hval;
    const std::vector<int> &sptr = hops.sptr, &scol = hops.scol;
    const std::vector<double> &sval = hops.sval;
    const std::vector<unsigned char> &dang = hops.dang;

    qpr_ctx *ctx = new (std::nothrow) qpr_ctx();
    if (!ctx) return arg_err(QPR_E_OOM, "host allocation failed");
    ctx->n = n;
    ctx->alpha = alpha;
    ctx->omega = omega;
    ctx->opt = o;
    ctx->np = (int)(((n + qpr::kPadFp64 - 1) / qpr::kPadFp64) * qpr::kPadFp64);
    const bool tc = (o.precision == QPR_MIXED) &&
                    (o.backend == QPR_BACKEND_DENSE ||
                     (o.backend == QPR_BACKEND_AUTO && (double)hval.size() >= (double)n * (double)n / 8.0));
    if (tc) ctx->np = (int)(((n + qpr::kTileTc - 1) / qpr::kTileTc) * qpr::kTileTc);
    ctx->spread = qpr::estimate_spread(n, hptr, hcol, hval);
    if (o.backend == QPR_BACKEND_AUTO)
        ctx->backend = ((double)hval.size() < (double)n * (double)n / 8.0) ? QPR_BACKEND_SPARSE : QPR_BACKEND_DENSE;
    else
        ctx->backend = o.backend;
    std::vector<double> c = qpr::column_sums_G(hops, alpha, ctx->np, &ctx->cmax);

    if (o.device < 0) {
        if (cudaGetDevice(&ctx->device) != cudaSuccess) {
            cudaGetLastError();
            delete ctx;
            return arg_err(QPR_E_CUDA, "no CUDA device available");
        }
    } else {
        ctx->device = o.device;
    }
    DeviceGuard dg(ctx->device);
    auto bail = [&](qpr_status st) {
        g_create_error = ctx->err;
        qpr_destroy(ctx);
        return st;
    };
#define CREATE_CUDA(call)                                            \
    do {                                                             \
        cudaError_t e_ = (call);                                     \
        if (e_ != cudaSuccess) return bail(cuda_fail(ctx, e_, #call)); \
    } while (0)
    if (getenv("QPR_FAULT") && strcmp(getenv("QPR_FAULT"), "oom") == 0) {
        ctx->err = "injected allocation failure (QPR_FAULT=oom)";
        return bail(QPR_E_OOM);
    }
    CREATE_CUDA(qpr::init_stage_fp64());
    CREATE_CUDA(qpr::init_stage_sparse());
    CREATE_CUDA(qpr::init_stage_mixed());
    const int np = ctx->np;
    const size_t plane = (size_t)np * np;
    // dense H, np x np with zero padding
    {
        std::vector<double> Hd(plane, 0.0);
        for (int64_t i = 0; i < n; ++i)
            for (int64_t q = hptr[i]; q < hptr[i + 1]; ++q) Hd[(size_t)i * np + hcol[q]] = hval[q];
        CREATE_CUDA(cudaMalloc(&ctx->d_H, plane * sizeof(double)));
        CREATE_CUDA(cudaMemcpy(ctx->d_H, Hd.data(), plane * sizeof(double), cudaMemcpyHostToDevice));
    }
    {
        std::vector<int> hptr32(n + 1);
        for (int64_t i = 0; i <= n; ++i) hptr32[i] = (int)hptr[i];
        CREATE_CUDA(cudaMalloc(&ctx->d_hptr, (n + 1) * sizeof(int)));
        CREATE_CUDA(cudaMalloc(&ctx->d_hcol, std::max<size_t>(1, hcol.size()) * sizeof(int)));
        CREATE_CUDA(cudaMalloc(&ctx->d_hval, std::max<size_t>(1, hval.size()) * sizeof(double)));
        CREATE_CUDA(cudaMemcpy(ctx->d_hptr, hptr32.data(), (n + 1) * sizeof(int), cudaMemcpyHostToDevice));
        if (!hcol.empty()) {
            CREATE_CUDA(cudaMemcpy(ctx->d_hcol, hcol.data(), hcol.size() * sizeof(int), cudaMemcpyHostToDevice));
            CREATE_CUDA(cudaMemcpy(ctx->d_hval, hval.data(), hval.size() * sizeof(double), cudaMemcpyHostToDevice));
        }
    }
    CREATE_CUDA(cudaMalloc(&ctx->d_sptr, (n + 1) * sizeof(int)));
    CREATE_CUDA(cudaMalloc(&ctx->d_scol, std::max<size_t>(1, scol.size()) * sizeof(int)));
    CREATE_CUDA(cudaMalloc(&ctx->d_sval, std::max<size_t>(1, sval.size()) * sizeof(double)));
    CREATE_CUDA(cudaMalloc(&ctx->d_dang, n));
    CREATE_CUDA(cudaMalloc(&ctx->d_c, np * sizeof(double)));
    CREATE_CUDA(cudaMemcpy(ctx->d_sptr, sptr.data(), (n + 1) * sizeof(int), cudaMemcpyHostToDevice));
    if (!scol.empty()) {
        CREATE_CUDA(cudaMemcpy(ctx->d_scol, scol.data(), scol.size() * sizeof(int), cudaMemcpyHostToDevice));
        CREATE_CUDA(cudaMemcpy(ctx->d_sval, sval.data(), sval.size() * sizeof(double), cudaMemcpyHostToDevice));
    }
    CREATE_CUDA(cudaMemcpy(ctx->d_dang, dang.data(), n, cudaMemcpyHostToDevice));
    CREATE_CUDA(cudaMemcpy(ctx->d_c, c.data(), np * sizeof(double), cudaMemcpyHostToDevice));

    const int T = np / qpr::kTileFp64;
    std::vector<int2> pairs;
    pairs.reserve((size_t)T * (T + 1) / 2);
    for (int I = 0; I < T; ++I)
        for (int J = I + 1; J < T; ++J) pairs.push_back(make_int2(I, J));
    for (int I = 0; I < T; ++I) pairs.push_back(make_int2(I, I));
    CREATE_CUDA(cudaMalloc(&ctx->d_pairs, pairs.size() * sizeof(int2)));
    CREATE_CUDA(cudaMemcpy(ctx->d_pairs, pairs.data(), pairs.size() * sizeof(int2), cudaMemcpyHostToDevice));
    {
        // The order of the column-block epilogues' CTAs. Each pair keeps its
        // index in `pairs` (its residual partial slot), so only the schedule
        // changes, never a result. When an epilogue's operands (X, the stage
        // input, F32, D and the next input: 40 bytes per element) exceed the
        // L2 cache, the pairs go row by row from the last tile row to the
        // first, each row from the last column down to the diagonal: the
        // SpMM grid before writes X by column blocks in increasing order, so
        // the epilogue starts on the X tiles written last (the ones still in
        // L2), and it writes the first column blocks of the next stage input
        // last, which the next SpMM grid reads first (N = 2048: 0.736 ->
        // 0.715 s to steady state; N = 4096: 2.134 -> 2.099 s). Otherwise
        // (everything L2-resident) they keep the order of `pairs`, which
        // measured 0.6% faster at N = 922.
        int l2 = 0;
        if (cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, ctx->device) != cudaSuccess) {
            cudaGetLastError();
            l2 = 0;
        }
        const bool reverse = 40.0 * (double)np * (double)np > (double)l2;
        std::vector<int4> epi;
        epi.reserve(pairs.size());
        const int off = T * (T - 1) / 2;  // index of the first diagonal pair
        if (reverse) {
            for (int I = T - 1; I >= 0; --I)
                for (int J = T - 1; J >= I; --J) {
                    const int q = (I == J) ? off + I : I * (T - 1) - I * (I - 1) / 2 + (J - I - 1);
                    epi.push_back(make_int4(I, J, q, 0));
                }
        } else {
            for (size_t q = 0; q < pairs.size(); ++q) epi.push_back(make_int4(pairs[q].x, pairs[q].y, (int)q, 0));
        }
        for (const int4 &e : epi)
            if (pairs[e.z].x != e.x || pairs[e.z].y != e.y) {
                ctx->err = "epilogue pair order: inconsistent pair index";
                g_create_error = ctx->err;
                qpr_destroy(ctx);
                return QPR_E_ARG;
            }
        CREATE_CUDA(cudaMalloc(&ctx->d_epi_pairs, epi.size() * sizeof(int4)));
        CREATE_CUDA(cudaMemcpy(ctx->d_epi_pairs, epi.data(), epi.size() * sizeof(int4), cudaMemcpyHostToDevice));
    }
    CREATE_CUDA(cudaMalloc(&ctx->d_state, 8 * plane * sizeof(double)));
    CREATE_CUDA(cudaMemset(ctx->d_state, 0, 8 * plane * sizeof(double)));
    CREATE_CUDA(cudaMalloc(&ctx->d_g, np * sizeof(double)));
    CREATE_CUDA(cudaMalloc(&ctx->d_partials, pairs.size() * sizeof(double)));
    {
        std::vector<float> hv32(std::max<size_t>(1, hval.size()));
        for (size_t q = 0; q < hval.size(); ++q) hv32[q] = (float)hval[q];
        std::vector<float> c32(np);
        for (int j = 0; j < np; ++j) c32[j] = (float)c[j];
        std::vector<int> rowseg;
        std::vector<int2> segs;
        qpr::row_segments(hops, np, 32, rowseg, segs);
        CREATE_CUDA(cudaMalloc(&ctx->d_rowseg, rowseg.size() * sizeof(int)));
        CREATE_CUDA(cudaMemcpy(ctx->d_rowseg, rowseg.data(), rowseg.size() * sizeof(int), cudaMemcpyHostToDevice));
        CREATE_CUDA(cudaMalloc(&ctx->d_seg, std::max<size_t>(1, segs.size()) * sizeof(int2)));
        if (!segs.empty())
            CREATE_CUDA(cudaMemcpy(ctx->d_seg, segs.data(), segs.size() * sizeof(int2), cudaMemcpyHostToDevice));
        CREATE_CUDA(cudaMalloc(&ctx->d_hval32, hv32.size() * sizeof(float)));
        CREATE_CUDA(cudaMemcpy(ctx->d_hval32, hv32.data(), hv32.size() * sizeof(float), cudaMemcpyHostToDevice));
        CREATE_CUDA(cudaMalloc(&ctx->d_c32, np * sizeof(float)));
        CREATE_CUDA(cudaMemcpy(ctx->d_c32, c32.data(), np * sizeof(float), cudaMemcpyHostToDevice));
    }
    int npairs_tc = 0;
    if (tc) {
        CREATE_CUDA(qpr::init_mixed_tc());
        // H = H0 + H1 + H2, each the BF16 rounding of what the previous left
        std::vector<__nv_bfloat16> hs(3 * plane, __float2bfloat16_rn(0.0f));
        for (int64_t i = 0; i < n; ++i)
            for (int64_t q = hptr[i]; q < hptr[i + 1]; ++q) {
                const double h = hval[q];
                const __nv_bfloat16 h0 = __double2bfloat16(h);
                const double r1 = h - (double)__bfloat162float(h0);
                const __nv_bfloat16 h1 = __double2bfloat16(r1);
                const double r2 = r1 - (double)__bfloat162float(h1);
                const __nv_bfloat16 h2 = __double2bfloat16(r2);
                const size_t o2 = (size_t)i * np + hcol[q];
                hs[o2] = h0;
                hs[plane + o2] = h1;
                hs[2 * plane + o2] = h2;
            }
        CREATE_CUDA(cudaMalloc(&ctx->d_hsplit, 3 * plane * sizeof(__nv_bfloat16)));
        CREATE_CUDA(cudaMemcpy(ctx->d_hsplit, hs.data(), 3 * plane * sizeof(__nv_bfloat16), cudaMemcpyHostToDevice));
        CREATE_CUDA(cudaMalloc(&ctx->d_dsplit, 18 * plane * sizeof(__nv_bfloat16)));
        CREATE_CUDA(cudaMemset(ctx->d_dsplit, 0, 18 * plane * sizeof(__nv_bfloat16)));
        const int Ttc = np / qpr::kTileTc;
        std::vector<int2> ptc;
        for (int I = 0; I < Ttc; ++I)
            for (int J = I + 1; J < Ttc; ++J) ptc.push_back(make_int2(I, J));
        for (int I = 0; I < Ttc; ++I) ptc.push_back(make_int2(I, I));
        npairs_tc = (int)ptc.size();
        CREATE_CUDA(cudaMalloc(&ctx->d_pairs_tc, ptc.size() * sizeof(int2)));
        CREATE_CUDA(cudaMemcpy(ctx->d_pairs_tc, ptc.data(), ptc.size() * sizeof(int2), cudaMemcpyHostToDevice));
    }
    if (o.precision == QPR_MIXED) {
        CREATE_CUDA(cudaMalloc(&ctx->d_mix64, 4 * plane * sizeof(double)));
        CREATE_CUDA(cudaMemset(ctx->d_mix64, 0, 4 * plane * sizeof(double)));
        CREATE_CUDA(cudaMalloc(&ctx->d_mix32, 14 * plane * sizeof(float)));
        CREATE_CUDA(cudaMemset(ctx->d_mix32, 0, 14 * plane * sizeof(float)));
        CREATE_CUDA(cudaMalloc(&ctx->d_g32, 2 * np * sizeof(float)));  // g, then the diagonal vector pv
        CREATE_CUDA(cudaMemset(ctx->d_g32, 0, 2 * np * sizeof(float)));
        CREATE_CUDA(cudaMalloc(&ctx->d_partials32, std::max<size_t>(pairs.size(), (size_t)npairs_tc) * sizeof(float)));
        std::vector<float> sv32(std::max<size_t>(1, sval.size()));
        for (size_t q = 0; q < sval.size(); ++q) sv32[q] = (float)sval[q];
        CREATE_CUDA(cudaMalloc(&ctx->d_sval32, sv32.size() * sizeof(float)));
        CREATE_CUDA(cudaMemcpy(ctx->d_sval32, sv32.data(), sv32.size() * sizeof(float), cudaMemcpyHostToDevice));
    }
    // column-block form: the whole column block staged in shared memory, or
    // (larger N) the gather form reading row segments through L1/L2
    qpr::ColPlan cplan;
    const int form = o.sparse_form;
    const bool want_cols = (o.precision == QPR_MIXED) && !tc && form != QPR_SPARSE_FORM_TILES;
    bool cols = want_cols && form != QPR_SPARSE_FORM_COLUMNS_GATHER &&
                qpr::plan_columns(hops, np, ctx->device, cplan, o.row_splits);
    const bool gathered = want_cols && !cols && (form == QPR_SPARSE_FORM_AUTO || form == QPR_SPARSE_FORM_COLUMNS_GATHER) &&
                          qpr::plan_columns(hops, np, ctx->device, cplan, o.row_splits, true);
    cols = cols || gathered;
    if (o.precision == QPR_MIXED && !tc && !cols && form != QPR_SPARSE_FORM_AUTO && form != QPR_SPARSE_FORM_TILES) {
        ctx->err = form == QPR_SPARSE_FORM_COLUMNS_GATHER
                       ? "sparse_form COLUMNS_GATHER: no row split fits one CTA's shared memory"
                       : "sparse_form COLUMNS: the staged operands of N = " + std::to_string(n) +
                             " do not fit one CTA's shared memory";
        return bail(QPR_E_ARG);
    }
    if (cols) {
        const std::vector<int2> &kh = cplan.kh;
        // the bundle descriptors, then the cut rows
        std::vector<int4> pieces(cplan.pieces);
        pieces.insert(pieces.end(), cplan.cuts.begin(), cplan.cuts.end());
        std::vector<int> ints;
        for (const std::vector<int> *v : {&cplan.q, &cplan.sb, &cplan.wb, &cplan.cutb})
            ints.insert(ints.end(), v->begin(), v->end());
        CREATE_CUDA(cudaMalloc(&ctx->d_colkh, kh.size() * sizeof(int2)));
        CREATE_CUDA(cudaMemcpy(ctx->d_colkh, kh.data(), kh.size() * sizeof(int2), cudaMemcpyHostToDevice));
        CREATE_CUDA(cudaMalloc(&ctx->d_colint, ints.size() * sizeof(int)));
        CREATE_CUDA(cudaMemcpy(ctx->d_colint, ints.data(), ints.size() * sizeof(int), cudaMemcpyHostToDevice));
        CREATE_CUDA(cudaMalloc(&ctx->d_colpieces, std::max<size_t>(1, pieces.size()) * sizeof(int4)));
        CREATE_CUDA(cudaMemcpy(ctx->d_colpieces, pieces.data(), pieces.size() * sizeof(int4),
                               cudaMemcpyHostToDevice));
        CREATE_CUDA(cudaMalloc(&ctx->d_X, 2 * plane * sizeof(float)));
        CREATE_CUDA(cudaMemset(ctx->d_X, 0, 2 * plane * sizeof(float)));
        if (o.sparse_form == QPR_SPARSE_FORM_COLUMNS_PERSISTENT) {
            ctx->persist_grid =
                qpr::persist_grid(np, cplan.splits, cplan.smem, ctx->device, &ctx->persist_smem, &ctx->epi_off);
            if (ctx->persist_grid <= 0) {
                ctx->err = "sparse_form COLUMNS_PERSISTENT: no cooperative launch of the block kernel fits";
                return bail(QPR_E_ARG);
            }
        }
    }
    CREATE_CUDA(cudaMalloc(&ctx->d_ctl, sizeof(Ctl)));
    CREATE_CUDA(cudaMemset(ctx->d_ctl, 0, sizeof(Ctl)));
    CREATE_CUDA(cudaMalloc(&ctx->d_io, (size_t)n * n * 2 * sizeof(double)));
    CREATE_CUDA(cudaMalloc(&ctx->d_p, n * sizeof(double)));
    CREATE_CUDA(cudaMallocHost(&ctx->h_ctl, sizeof(Ctl)));
    CREATE_CUDA(cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking));
    CREATE_CUDA(cudaEventCreateWithFlags(&ctx->ev, cudaEventDisableTiming));
#undef CREATE_CUDA

    qpr::DevOps &ops = ctx->ops;
    ops.n = (int)n;
    ops.np = np;
    ops.alpha = alpha;
    ops.omega = omega;
    ops.dangling = o.dangling;
    ops.H = ctx->d_H;
    ops.h_ptr = ctx->d_hptr;
    ops.h_col = ctx->d_hcol;
    ops.h_val = ctx->d_hval;
    ops.s_ptr = ctx->d_sptr;
    ops.s_col = ctx->d_scol;
    ops.s_val = ctx->d_sval;
    ops.dang = ctx->d_dang;
    ops.c = ctx->d_c;
    ops.c32 = ctx->d_c32;
    ops.h_val32 = ctx->d_hval32;
    ops.s_val32 = ctx->d_sval32;
    ops.alpha32 = (float)alpha;
    ops.oma32 = (float)(1.0 - alpha);
    ops.omega32 = (float)omega;
    ops.inv_nm1_32 = (float)(1.0 / (double)(n - 1));
    ops.inv_n32 = (float)(1.0 / (double)n);
    ops.rowseg = ctx->d_rowseg;
    ops.seg = ctx->d_seg;
    qpr::Work &wk = ctx->work;
    wk.y = ctx->d_state;
    wk.z = ctx->d_state + 2 * plane;
    wk.ya = ctx->d_state + 4 * plane;
    wk.yb = ctx->d_state + 6 * plane;
    wk.g = ctx->d_g;
    wk.partials = ctx->d_partials;
    wk.pairs = ctx->d_pairs;
    wk.npairs = (int)pairs.size();
    wk.tiles = T;
    wk.ctl = ctx->d_ctl;
    if (o.precision == QPR_MIXED) {
        qpr::MixedWork &mw = ctx->mw;
        mw.R = ctx->d_mix64;
        mw.F = ctx->d_mix64 + 2 * plane;
        mw.F32 = ctx->d_mix32;
        mw.D = ctx->d_mix32 + 2 * plane;  // D and Dlo adjacent: one memset clears the delta
        mw.Dlo = ctx->d_mix32 + 4 * plane;
        mw.da = ctx->d_mix32 + 6 * plane;
        mw.db = ctx->d_mix32 + 8 * plane;
        mw.Ghi = ctx->d_mix32 + 10 * plane;
        mw.Glo = ctx->d_mix32 + 12 * plane;
        mw.partials32 = ctx->d_partials32;
        if (cols) {
            const size_t nq = cplan.q.size();
            const size_t nsb = cplan.sb.size();
            const size_t nwb = cplan.wb.size();
            ops.col_kh = ctx->d_colkh;
            ops.col_q = ctx->d_colint;
            ops.col_sb = ctx->d_colint + nq;
            ops.col_wb = ctx->d_colint + nq + nsb;
            ops.col_cutb = ctx->d_colint + nq + nsb + nwb;
            ops.col_pieces = ctx->d_colpieces;
            ops.col_cut = ctx->d_colpieces + cplan.pieces.size();
            ops.col_part_off = cplan.part_off;
            ops.col_gather = gathered ? 1 : 0;
            ops.col_splits = cplan.splits;
            ops.col_smem = cplan.smem;
            ops.col_p_off = cplan.p_off;
            ops.col_sp_off = cplan.sp_off;
            ops.col_epi_off = ctx->epi_off;
            ops.col_psmem = ctx->persist_smem;
            mw.X = ctx->d_X;
            const float *din[3] = {mw.D, mw.da, mw.db};
            if (!qpr::make_col_maps(ops, din, &ctx->colmaps)) {
                ctx->err = "cuTensorMapEncodeTiled failed";
                g_create_error = ctx->err;
                qpr_destroy(ctx);
                return QPR_E_CUDA;
            }
            // the SpMM grid's leading CTAs form the gain, on the SMs the product leaves free (at least 8)
            int sms = 0;
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device);
            const int units = gathered ? cplan.splits * (np / qpr::kColGatherWidth) : (np / qpr::kColWidth) * cplan.splits;
            ops.col_gain_ctas = std::min(64, std::max(8, sms - units));
            ops.col_launch_smem = std::max(cplan.smem, (int)(np * sizeof(float)) + 16);
            const cudaError_t ea = gathered ? qpr::set_gather_smem(ops.col_launch_smem)
                                            : qpr::set_cols_smem(ops.col_launch_smem);
            if (ea != cudaSuccess) {
                cudaGetLastError();
                ctx->err = std::string("kernel attribute: ") + cudaGetErrorString(ea);
                g_create_error = ctx->err;
                qpr_destroy(ctx);
                return QPR_E_CUDA;
            }
            mw.cmaps = &ctx->colmaps;
        }
        mw.g = ctx->d_g32;
        mw.pv = ctx->d_g32 + np;
        mw.g64 = ctx->d_g;
        mw.partials = ctx->d_partials;
        mw.pairs = ctx->d_pairs;
        mw.epi_pairs = ctx->d_epi_pairs;
        mw.npairs = (int)pairs.size();
        mw.tiles = T;
        mw.ctl = ctx->d_ctl;
        mw.nstage_partials = (int)pairs.size();
        if (tc) {
            mw.pairs_tc = ctx->d_pairs_tc;
            mw.npairs_tc = npairs_tc;
            mw.nstage_partials = npairs_tc;
            mw.splitD = ctx->d_dsplit;
            mw.splitA = ctx->d_dsplit + 6 * plane;
            mw.splitB = ctx->d_dsplit + 12 * plane;
            const __nv_bfloat16 *ds[3] = {mw.splitD, mw.splitA, mw.splitB};
            if (!qpr::make_tc_maps(ops, ctx->d_hsplit, ds, &ctx->tcmaps)) {
                ctx->err = "cuTensorMapEncodeTiled failed";
                g_create_error = ctx->err;
                qpr_destroy(ctx);
                return QPR_E_CUDA;
            }
            mw.maps = &ctx->tcmaps;
        }
    }
    *out = ctx;
    return QPR_OK;
}

// Make the context stream wait for work the caller queued on its stream.
static qpr_status begin_call(qpr_ctx *ctx) {
    qpr_status st = check_usable(ctx);
    if (st != QPR_OK) return st;
    ctx->launches = 0;
    cudaStream_t user = (cudaStream_t)ctx->opt.cuda_stream;
    QPR_CUDA(ctx, cudaEventRecord(ctx->ev, user));
    QPR_CUDA(ctx, cudaStreamWaitEvent(ctx->stream, ctx->ev, 0));
    return QPR_OK;
}

static qpr_status rhs_impl(qpr_ctx *ctx, const void *rho, void *out, double *resid) {
    qpr_status st = begin_call(ctx);
    if (st != QPR_OK) return st;
    if (!rho) return fail(ctx, QPR_E_ARG, "rho is NULL");
    st = import_rho(ctx, rho, ctx->work.y);
    if (st != QPR_OK) return st;
    Ctl *h = ctx->h_ctl;
    memset(h, 0, sizeof(Ctl));
    h->scale = 1.0;
    QPR_CUDA(ctx, cudaMemcpyAsync(ctx->d_ctl, h, sizeof(Ctl), cudaMemcpyHostToDevice, ctx->stream));
    qpr::launch_gain(0, ctx->ops, ctx->work.y, ctx->work, ctx->stream);
    launch_stage(ctx, 0);
    if (out) {
        st = export_rho(ctx, ctx->work.z, 0, out);
        if (st != QPR_OK) return st;
    }
    std::vector<double> part(ctx->work.npairs);
    if (resid)
        QPR_CUDA(ctx, cudaMemcpyAsync(part.data(), ctx->d_partials, part.size() * sizeof(double),
                                      cudaMemcpyDeviceToHost, ctx->stream));
    st = sync_ctx(ctx);
    if (st != QPR_OK) return st;
    if (resid) {
        double s = 0.0;
        for (double v : part) s += v;
        *resid = sqrt(s);
    }
    return QPR_OK;
}

qpr_status qpr_rhs(qpr_ctx *ctx, const void *rho, void *out) {
    if (!ctx) return QPR_E_ARG;
    if (!out) return fail(ctx, QPR_E_ARG, "out is NULL");
    DeviceGuard dg(ctx->device);
    return rhs_impl(ctx, rho, out, nullptr);
}

qpr_status qpr_residual(qpr_ctx *ctx, const void *rho, double *resid_out) {
    if (!ctx) return QPR_E_ARG;
    if (!resid_out) return fail(ctx, QPR_E_ARG, "resid_out is NULL");
    DeviceGuard dg(ctx->device);
    return rhs_impl(ctx, rho, nullptr, resid_out);
}

qpr_status qpr_evolve(qpr_ctx *ctx, void *rho, double dt, int64_t steps) {
    qpr::NvtxRange nvtx_range("qpr_evolve");
    if (!ctx) return QPR_E_ARG;
    DeviceGuard dg(ctx->device);
    qpr_status st = begin_call(ctx);
    if (st != QPR_OK) return st;
    if (!rho) return fail(ctx, QPR_E_ARG, "rho is NULL");
    if (!(dt > 0.0) || !std::isfinite(dt)) return fail(ctx, QPR_E_ARG, "dt must be positive and finite");
    if (steps < 0) return fail(ctx, QPR_E_ARG, "steps must be non-negative");
    if (dt > qpr_max_stable_dt(ctx))
        return fail(ctx, QPR_E_UNSTABLE, "dt exceeds the RK4 stability estimate " +
                                             std::to_string(qpr_max_stable_dt(ctx)));
    st = import_state(ctx, rho);
    if (st != QPR_OK) return st;
    const bool mixed = ctx->opt.precision == QPR_MIXED;
    st = mixed ? run_mixed(ctx, dt, 0.0, steps) : run_rk4(ctx, dt, 0.0, steps);
    if (st != QPR_OK) return st;
    if (ctx->h_ctl->status == qpr::kCtlNonFinite)
        return fail(ctx, QPR_E_NONFINITE, "non-finite trace or residual during the integration");
    st = mixed ? export_rho(ctx, ctx->mw.R, 0, rho) : export_rho(ctx, ctx->work.y, 1, rho);
    if (st != QPR_OK) return st;
    return sync_ctx(ctx);
}

qpr_status qpr_steady_state(qpr_ctx *ctx, void *rho, double dt, double tol, int64_t max_steps,
                            qpr_stats *out) {
    qpr::NvtxRange nvtx_range("qpr_steady_state");
    if (!ctx) return QPR_E_ARG;
    DeviceGuard dg(ctx->device);
    auto t0 = std::chrono::steady_clock::now();
    qpr_status st = begin_call(ctx);
    if (st != QPR_OK) return st;
    if (!rho) return fail(ctx, QPR_E_ARG, "rho is NULL");
    if (!(dt > 0.0) || !std::isfinite(dt)) return fail(ctx, QPR_E_ARG, "dt must be positive and finite");
    if (!(tol > 0.0)) return fail(ctx, QPR_E_ARG, "tol must be positive");
    if (max_steps < 0) return fail(ctx, QPR_E_ARG, "max_steps must be non-negative");
    const double dmax = qpr_max_stable_dt(ctx);
    int64_t m = 1;
    if (dt > dmax) m = (int64_t)ceil(dt / dmax);
    const double h = dt / (double)m;
    st = import_state(ctx, rho);
    if (st != QPR_OK) return st;
    const bool mixed = ctx->opt.precision == QPR_MIXED;
    st = mixed ? run_mixed(ctx, h, tol, max_steps) : run_rk4(ctx, h, tol, max_steps);
    if (st != QPR_OK) return st;
    Ctl c = *ctx->h_ctl;
    if (mixed) c.resid = c.resid_exact;
    st = mixed ? export_rho(ctx, ctx->mw.R, 0, rho) : export_rho(ctx, ctx->work.y, 1, rho);
    if (st != QPR_OK) return st;
    st = sync_ctx(ctx);
    if (st != QPR_OK) return st;
    if (out) {
        memset(out, 0, sizeof(*out));
        out->steps = c.step;
        out->substeps_m = m;
        out->t = (double)c.step * h;
        out->residual = c.resid;
        out->trace_before = c.trace;
        out->converged = (c.status == qpr::kCtlConverged) ? 1 : 0;
        out->kernel_launches = ctx->launches;
        out->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    }
    if (qpr::log_enabled())
        fprintf(stderr, "qpr_steady_state: N=%lld steps=%lld dt=%g residual=%.3e status=%d launches=%lld %.4f s\n",
                (long long)ctx->n, (long long)c.step, h, c.resid, c.status, (long long)ctx->launches,
                std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count());
    if (c.status == qpr::kCtlNonFinite) return fail(ctx, QPR_E_NONFINITE, "non-finite trace or residual");
    if (c.status != qpr::kCtlConverged)
        return fail(ctx, QPR_E_NOT_CONVERGED, "max_steps reached with residual " + std::to_string(c.resid));
    return QPR_OK;
}

qpr_status qpr_profile_chain(qpr_ctx *ctx, const void *rho, double dt, int32_t reps, double *out_ms) {
    qpr::NvtxRange nvtx_range("qpr_profile_chain");
    if (!ctx) return QPR_E_ARG;
    DeviceGuard dg(ctx->device);
    qpr_status st = begin_call(ctx);
    if (st != QPR_OK) return st;
    if (!rho || !out_ms || reps < 1 || reps > 4096) return fail(ctx, QPR_E_ARG, "rho/out_ms NULL or reps not in [1, 4096]");
    if (!(dt > 0.0) || dt > qpr_max_stable_dt(ctx)) return fail(ctx, QPR_E_ARG, "dt not positive or unstable");
    if (ctx->opt.precision != QPR_MIXED || !ctx->mw.cmaps)
        return fail(ctx, QPR_E_ARG, "qpr_profile_chain needs QPR_MIXED with a column-block sparse form");
    st = import_state(ctx, rho);
    if (st != QPR_OK) return st;
    Ctl *h = ctx->h_ctl;
    memset(h, 0, sizeof(Ctl));
    h->max_steps = 1 << 30;
    h->tol = 0.0;
    h->dt = dt;
    h->scale = 1.0;
    h->resid_exact_step = -1;
    QPR_CUDA(ctx, cudaMemcpyAsync(ctx->d_ctl, h, sizeof(Ctl), cudaMemcpyHostToDevice, ctx->stream));
    // the stage-2 input: a refresh, then stage 1 (SpMM and epilogue)
    qpr::launch_mixed_refresh(ctx->ops, ctx->mw, ctx->stream);
    qpr::launch_mixed_stage(1, ctx->ops, ctx->mw, ctx->stream, 1, true);
    qpr::launch_mixed_stage(1, ctx->ops, ctx->mw, ctx->stream, 2, true);
    cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
    auto destroy = [&]() {
        for (cudaEvent_t &e : ev)
            if (e) cudaEventDestroy(e);
    };
    for (cudaEvent_t &e : ev) {
        if (cudaEventCreate(&e) != cudaSuccess) {
            destroy();
            return fail(ctx, QPR_E_CUDA, "cudaEventCreate failed");
        }
    }
    // each chain repeats one kernel: the SpMM grid reads the stage input and
    // writes X and g, the epilogue reads X and the stage input and writes the
    // next stage input, so every launch does the same work on the same data
    cudaEventRecord(ev[0], ctx->stream);
    for (int r = 0; r < reps; ++r) qpr::launch_mixed_stage(2, ctx->ops, ctx->mw, ctx->stream, 1, false);
    cudaEventRecord(ev[1], ctx->stream);
    cudaEventRecord(ev[2], ctx->stream);
    for (int r = 0; r < reps; ++r) qpr::launch_mixed_stage(2, ctx->ops, ctx->mw, ctx->stream, 2, false);
    cudaEventRecord(ev[3], ctx->stream);
    ctx->launches += 3 + qpr::kMixedLaunchesPerRefresh + 2 * (int64_t)reps;
    st = sync_ctx(ctx);
    if (st == QPR_OK) {
        float a = 0.f, b = 0.f;
        cudaEventElapsedTime(&a, ev[0], ev[1]);
        cudaEventElapsedTime(&b, ev[2], ev[3]);
        out_ms[0] = a / reps;
        out_ms[1] = b / reps;
    }
    destroy();
    return st;
}

qpr_status qpr_profile_step(qpr_ctx *ctx, const void *rho, double dt, int64_t steps, qpr_profile *out) {
    qpr::NvtxRange nvtx_range("qpr_profile_step");
    if (!ctx) return QPR_E_ARG;
    DeviceGuard dg(ctx->device);
    qpr_status st = begin_call(ctx);
    if (st != QPR_OK) return st;
    if (!rho || !out || steps < 1) return fail(ctx, QPR_E_ARG, "rho/out NULL or steps < 1");
    if (!(dt > 0.0) || dt > qpr_max_stable_dt(ctx)) return fail(ctx, QPR_E_ARG, "dt not positive or unstable");
    st = import_state(ctx, rho);
    if (st != QPR_OK) return st;
    Ctl *h = ctx->h_ctl;
    memset(h, 0, sizeof(Ctl));
    h->max_steps = steps + 1;
    h->tol = 0.0;
    h->dt = dt;
    h->scale = 1.0;
    h->resid_exact_step = -1;
    QPR_CUDA(ctx, cudaMemcpyAsync(ctx->d_ctl, h, sizeof(Ctl), cudaMemcpyHostToDevice, ctx->stream));
    const bool mixed = ctx->opt.precision == QPR_MIXED;
    const bool cols = mixed && ctx->mw.cmaps;
    // every kernel alone on the stream, between two events: kind 0 product,
    // 1 epilogue, 2 gain; the refresh's kernels together (kind 3)
    struct Mark { int kind; cudaEvent_t a, b; };
    std::vector<Mark> marks;
    auto timed = [&](int kind, auto &&launch) -> qpr_status {
        Mark mk{kind, nullptr, nullptr};
        QPR_CUDA(ctx, cudaEventCreate(&mk.a));
        marks.push_back(mk);
        QPR_CUDA(ctx, cudaEventCreate(&marks.back().b));
        QPR_CUDA(ctx, cudaEventRecord(marks.back().a, ctx->stream));
        launch();
        QPR_CUDA(ctx, cudaEventRecord(marks.back().b, ctx->stream));
        return QPR_OK;
    };
    auto destroy = [&]() {
        for (Mark &m : marks) {
            if (m.a) cudaEventDestroy(m.a);
            if (m.b) cudaEventDestroy(m.b);
        }
    };
    const qpr::Work &w = ctx->work;
    const double *yin[5] = {w.y, w.y, w.ya, w.yb, w.ya};
    int per_step = 0;
    if (mixed) {
        st = timed(3, [&] { qpr::launch_mixed_refresh(ctx->ops, ctx->mw, ctx->stream); });
        if (st != QPR_OK) { destroy(); return st; }
    }
    for (int64_t k = 0; k < steps && st == QPR_OK; ++k) {
        for (int s = 1; s <= 4 && st == QPR_OK; ++s) {
            if (cols) {
                st = timed(0, [&] { qpr::launch_mixed_stage(s, ctx->ops, ctx->mw, ctx->stream, 1, true); });
                if (st == QPR_OK)
                    st = timed(1, [&] { qpr::launch_mixed_stage(s, ctx->ops, ctx->mw, ctx->stream, 2, true); });
                if (k == 0) per_step += 2;
            } else if (mixed) {
                if (ctx->mw.splitD) {
                    st = timed(2, [&] { qpr::launch_mixed_stage(s, ctx->ops, ctx->mw, ctx->stream, 1, true); });
                    if (k == 0) per_step += 1;
                }
                if (st == QPR_OK)
                    st = timed(0, [&] { qpr::launch_mixed_stage(s, ctx->ops, ctx->mw, ctx->stream, 2, true); });
                if (k == 0) per_step += 1;
            } else {
                st = timed(2, [&] { qpr::launch_gain(s, ctx->ops, yin[s], w, ctx->stream); });
                if (st == QPR_OK) st = timed(0, [&] { launch_stage(ctx, s); });
                if (k == 0) per_step += 2;
            }
        }
    }
    if (st == QPR_OK) st = sync_ctx(ctx);
    if (st != QPR_OK) {
        destroy();
        return st;
    }
    double sum[4] = {0, 0, 0, 0};
    int cnt[4] = {0, 0, 0, 0};
    for (const Mark &m : marks) {
        float ms = 0.f;
        cudaEventElapsedTime(&ms, m.a, m.b);
        sum[m.kind] += ms;
        cnt[m.kind] += 1;
    }
    destroy();
    memset(out, 0, sizeof(*out));
    out->product_ms = cnt[0] ? sum[0] / cnt[0] : 0.0;
    out->epilogue_ms = cnt[1] ? sum[1] / cnt[1] : 0.0;
    out->gain_ms = cnt[2] ? sum[2] / cnt[2] : 0.0;
    out->refresh_ms = cnt[3] ? sum[3] / cnt[3] : 0.0;
    out->step_ms = (sum[0] + sum[1] + sum[2]) / (double)steps;
    out->launches_per_step = per_step;
    return QPR_OK;
}

qpr_status qpr_populations(qpr_ctx *ctx, const void *rho, double *p, int64_t *rank) {
    if (!ctx) return QPR_E_ARG;
    DeviceGuard dg(ctx->device);
    qpr_status st = begin_call(ctx);
    if (st != QPR_OK) return st;
    if (!rho || !p) return fail(ctx, QPR_E_ARG, "rho or p is NULL");
    const int64_t n = ctx->n;
    const double *src = (const double *)rho;
    if (!is_device_ptr(rho)) {
        QPR_CUDA(ctx, cudaMemcpyAsync(ctx->d_io, rho, (size_t)n * n * 2 * sizeof(double),
                                      cudaMemcpyHostToDevice, ctx->stream));
        src = ctx->d_io;
    }
    qpr::launch_diag(src, (int)n, ctx->d_p, ctx->stream);
    std::vector<double> ph(n);
    QPR_CUDA(ctx, cudaMemcpyAsync(ph.data(), ctx->d_p, n * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    const bool p_dev = is_device_ptr(p);
    if (p_dev)
        QPR_CUDA(ctx, cudaMemcpyAsync(p, ctx->d_p, n * sizeof(double), cudaMemcpyDeviceToDevice, ctx->stream));
    st = sync_ctx(ctx);
    if (st != QPR_OK) return st;
    if (!p_dev) memcpy(p, ph.data(), n * sizeof(double));
    if (rank) {
        std::vector<int64_t> r(n);
        std::iota(r.begin(), r.end(), 0);
        std::stable_sort(r.begin(), r.end(), [&](int64_t a, int64_t b) { return ph[a] > ph[b]; });
        if (is_device_ptr(rank)) {
            QPR_CUDA(ctx, cudaMemcpy(rank, r.data(), n * sizeof(int64_t), cudaMemcpyHostToDevice));
        } else {
            memcpy(rank, r.data(), n * sizeof(int64_t));
        }
    }
    return QPR_OK;
}

qpr_status qpr_rkf45(qpr_ctx *ctx, void *rho, const qpr_rkf45_options *opt, double tol, int64_t max_steps,
                     qpr_rkf45_stats *out) {
    qpr::NvtxRange nvtx_range("qpr_rkf45");
    if (!ctx) return QPR_E_ARG;
    DeviceGuard dg(ctx->device);
    auto t0 = std::chrono::steady_clock::now();
    qpr_status st = begin_call(ctx);
    if (st != QPR_OK) return st;
    if (!rho) return fail(ctx, QPR_E_ARG, "rho is NULL");
    qpr_rkf45_options o{};
    if (opt) o = *opt;
    const double hmax = o.h_max > 0.0 ? o.h_max : qpr_max_stable_dt(ctx);
    const double step_tol = o.step_tol > 0.0 ? o.step_tol : 1e-6;
    const bool traj = o.t_end > 0.0;
    double h0 = o.h0 > 0.0 ? o.h0 : 0.01;
    if (!std::isfinite(h0) || !std::isfinite(step_tol) || !(hmax > 0.0) || !std::isfinite(hmax) ||
        (traj && !std::isfinite(o.t_end)))
        return fail(ctx, QPR_E_ARG, "h0, step_tol, h_max and t_end must be finite");
    if (!traj && !(tol > 0.0)) return fail(ctx, QPR_E_ARG, "tol must be positive for a steady-state solve");
    if (max_steps < 0) return fail(ctx, QPR_E_ARG, "max_steps must be non-negative");
    const int order = o.order == 0 ? 4 : o.order;
    if (order != 4 && order != 5) return fail(ctx, QPR_E_ARG, "order must be 0, 4 or 5");
    h0 = std::min(h0, hmax);
    if (traj) h0 = std::min(h0, o.t_end);
    st = ensure_rkf(ctx);
    if (st != QPR_OK) return st;
    st = import_state(ctx, rho);
    if (st != QPR_OK) return st;
    const int64_t max_attempts = 16 * max_steps + 64 * (int64_t)ctx->opt.ref_refresh;
    st = run_rkf45(ctx, h0, step_tol, hmax, traj ? o.t_end : 0.0, traj ? 0.0 : tol, max_steps, max_attempts, order);
    if (st != QPR_OK) return st;
    Ctl c = *ctx->h_ctl;
    st = export_rho(ctx, ctx->mw.R, 0, rho);
    if (st != QPR_OK) return st;
    st = sync_ctx(ctx);
    if (st != QPR_OK) return st;
    if (out) {
        memset(out, 0, sizeof(*out));
        out->accepted = c.step;
        out->rejected = c.rk_rejected;
        out->t = c.rk_t;
        out->h_next = c.rk_h;
        out->residual = c.resid_exact;
        out->last_discrepancy = c.rk_err;
        out->kernel_launches = ctx->launches;
        out->converged = (c.status == qpr::kCtlConverged || c.status == qpr::kCtlTimeReached) ? 1 : 0;
        out->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    }
    if (c.status == qpr::kCtlNonFinite) return fail(ctx, QPR_E_NONFINITE, "non-finite state, residual or discrepancy");
    if (c.status == qpr::kCtlTimeReached || c.status == qpr::kCtlConverged) return QPR_OK;
    return fail(ctx, QPR_E_NOT_CONVERGED, traj ? "max_steps reached before t_end"
                                              : "max_steps reached with residual " + std::to_string(c.resid_exact));
}

qpr_status qpr_pagerank(qpr_ctx *ctx, double tol, int64_t max_iter, double *pi, int64_t *iters) {
    qpr::NvtxRange nvtx_range("qpr_pagerank");
    if (!ctx) return QPR_E_ARG;
    DeviceGuard dg(ctx->device);
    qpr_status st = begin_call(ctx);
    if (st != QPR_OK) return st;
    if (!pi) return fail(ctx, QPR_E_ARG, "pi is NULL");
    if (!(tol > 0.0) || max_iter < 1) return fail(ctx, QPR_E_ARG, "tol must be positive and max_iter >= 1");
    const int64_t n = ctx->n;
    // scratch: the host staging buffer (2 n^2 doubles >= 2 n + grid for n >= 2)
    if ((size_t)2 * n * n < (size_t)(2 * n + qpr::pagerank_grid((int)n)))
        return fail(ctx, QPR_E_ARG, "n too small for the staging buffer");
    int64_t it = 0;
    double delta = 0.0;
    QPR_CUDA(ctx, qpr::pagerank(ctx->ops, tol, max_iter, ctx->d_io, ctx->d_p, &it, &delta, ctx->stream));
    ctx->launches += 2 + it;
    if (is_device_ptr(pi)) {
        QPR_CUDA(ctx, cudaMemcpyAsync(pi, ctx->d_p, n * sizeof(double), cudaMemcpyDeviceToDevice, ctx->stream));
    } else {
        QPR_CUDA(ctx, cudaMemcpyAsync(pi, ctx->d_p, n * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    }
    st = sync_ctx(ctx);
    if (st != QPR_OK) return st;
    if (iters) *iters = it;
    if (!std::isfinite(delta)) return fail(ctx, QPR_E_NONFINITE, "non-finite PageRank iterate");
    if (delta >= tol)
        return fail(ctx, QPR_E_NOT_CONVERGED, "max_iter reached with L1 change " + std::to_string(delta));
    return QPR_OK;
}

qpr_status qpr_hub_classes(qpr_ctx *ctx, const double *p, double c, int32_t *classes, int64_t *counts) {
    if (!ctx) return QPR_E_ARG;
    DeviceGuard dg(ctx->device);
    qpr_status st = begin_call(ctx);
    if (st != QPR_OK) return st;
    if (!p) return fail(ctx, QPR_E_ARG, "p is NULL");
    if (!(c >= 1.0) || !std::isfinite(c)) return fail(ctx, QPR_E_ARG, "c must be finite and at least 1");
    const int64_t n = ctx->n;
    const double *src = p;
    if (!is_device_ptr(p)) {
        QPR_CUDA(ctx, cudaMemcpyAsync(ctx->d_p, p, n * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
        src = ctx->d_p;
    }
    // the classes and the counts in the staging buffer (2 n^2 doubles)
    int *d_cls = reinterpret_cast<int *>(ctx->d_io);
    unsigned long long *d_cnt = reinterpret_cast<unsigned long long *>(ctx->d_io + (n + 1) / 2 + 1);
    QPR_CUDA(ctx, qpr::hub_classes(src, (int)n, c, d_cls, d_cnt, ctx->stream));
    ctx->launches += 1;
    unsigned long long cnt[3] = {0, 0, 0};
    QPR_CUDA(ctx, cudaMemcpyAsync(cnt, d_cnt, sizeof(cnt), cudaMemcpyDeviceToHost, ctx->stream));
    if (classes) {
        const cudaMemcpyKind kind = is_device_ptr(classes) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
        QPR_CUDA(ctx, cudaMemcpyAsync(classes, d_cls, n * sizeof(int32_t), kind, ctx->stream));
    }
    st = sync_ctx(ctx);
    if (st != QPR_OK) return st;
    if (counts)
        for (int k = 0; k < 3; ++k) counts[k] = (int64_t)cnt[k];
    return QPR_OK;
}

}  // extern "C"
