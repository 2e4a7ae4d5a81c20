// Autotuner: picks, for one problem, the kernel family (sparse CSR or dense
// tensor-core stage), for the mixed sparse form the stage form (whole-block
// column SpMM, gather SpMM or tile pairs) and its row splits, and the
// reference-refresh block length, by timing short real runs on the device,
// and caches the choice in a text file keyed by GPU name, precision and
// size/density buckets.
//
// Search (mixed precision): first every (backend, form, row splits)
// candidate with ref_refresh 32, then ref_refresh in {16, 32, 64} for the
// winner. Row splits: the plan's own choice and its neighbours (whole-block
// form 1..4, gather form half and twice the plan's), candidates whose plan
// repeats an earlier one are skipped.
//
// Cache line format (one per key, later lines win):
//   <key> <backend> <ref_refresh> <ms_per_step> <sparse_form> <row_splits>
// with key = "<gpu name without spaces>|p<precision>|n<floor log2 N>|d<floor log2 (nnz(H)/N + 1)>"
// (lines with only the first four fields are read with form AUTO and 0 splits).
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <fstream>
#include <sstream>
#include <string>
#include <vector>

#include "qpr_internal.cuh"

namespace {

std::string tune_key(int device, int precision, int64_t n, size_t nnz) {
    cudaDeviceProp prop;
    std::string name = "gpu";
    if (cudaGetDeviceProperties(&prop, device) == cudaSuccess) name = prop.name;
    else cudaGetLastError();
    for (char &c : name)
        if (c == ' ' || c == '|') c = '_';
    const int nb = (int)floor(log2((double)n));
    const int db = (int)floor(log2((double)nnz / (double)n + 1.0));
    std::ostringstream k;
    k << name << "|p" << precision << "|n" << nb << "|d" << db;
    return k.str();
}

bool cache_lookup(const char *path, const std::string &key, qpr_tune_result *out) {
    if (!path) return false;
    std::ifstream f(path);
    if (!f) return false;
    std::string line;
    bool found = false;
    while (std::getline(f, line)) {
        std::istringstream is(line);
        std::string k;
        int be = 0, rr = 0, form = 0, splits = 0;
        double ms = 0.0;
        if (is >> k >> be >> rr >> ms && k == key) {
            if (!(is >> form >> splits)) form = splits = 0;
            out->backend = be;
            out->ref_refresh = rr;
            out->ms_per_step = ms;
            out->sparse_form = form;
            out->row_splits = splits;
            found = true;
        }
    }
    return found;
}

}  // namespace

extern "C" qpr_status qpr_autotune(int64_t n, int64_t m, const int64_t *src, const int64_t *dst, const double *w,
                                   double alpha, double omega, double dt, const qpr_options *base,
                                   const char *cache_path, qpr_tune_result *out) {
    qpr::NvtxRange nvtx_range("qpr_autotune");
    if (!out) return QPR_E_ARG;
    memset(out, 0, sizeof(*out));
    qpr_options o;
    qpr_default_options(&o);
    if (base) o = *base;
    qpr::HostOps h;
    std::string err;
    qpr_status st = qpr::assemble_host(n, m, src, dst, w, o.h_diag, h, err);
    if (st != QPR_OK) {
        qpr::set_create_error(err);
        return st;
    }
    int dev = o.device;
    if (dev < 0 && cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        qpr::set_create_error("no CUDA device available");
        return QPR_E_CUDA;
    }
    const std::string key = tune_key(dev, o.precision, n, h.hval.size());
    if (cache_lookup(cache_path, key, out)) {
        out->from_cache = 1;
        return QPR_OK;
    }
    // rho0 = I/N on the device
    const size_t bytes = (size_t)n * n * 16;
    void *rho = nullptr;
    if (cudaMalloc(&rho, bytes) != cudaSuccess) {
        cudaGetLastError();
        qpr::set_create_error("device allocation failed");
        return QPR_E_OOM;
    }
    std::vector<double> eye((size_t)n * n * 2, 0.0);
    for (int64_t i = 0; i < n; ++i) eye[2 * ((size_t)i * n + i)] = 1.0 / (double)n;
    struct Cand { int backend, form, splits, rr; };
    double best = INFINITY;
    qpr_status ret = QPR_OK;
    std::vector<std::vector<int32_t>> seen_plans;
    // ms per step of one candidate (INFINITY if it does not run); the plan of
    // a mixed sparse candidate that repeats an earlier one is skipped
    auto measure = [&](const Cand &c, bool dedup) {
        qpr_options oc = o;
        oc.backend = c.backend;
        oc.sparse_form = c.form;
        oc.row_splits = c.splits;
        oc.ref_refresh = c.rr;
        oc.device = dev;
        qpr_ctx *ctx = nullptr;
        if (qpr_create(&ctx, n, m, src, dst, w, alpha, omega, &oc) != QPR_OK) return (double)INFINITY;
        if (dedup && o.precision == QPR_MIXED) {
            std::vector<int32_t> plan(6, 0);
            qpr_sparse_plan(ctx, plan.data());
            plan[4] = qpr_sparse_form(ctx);
            plan[5] = qpr_backend(ctx);
            for (const auto &p : seen_plans)
                if (p == plan) {
                    qpr_destroy(ctx);
                    return (double)INFINITY;
                }
            seen_plans.push_back(plan);
        }
        const int steps = o.precision == QPR_MIXED ? std::max(32, 2 * c.rr) : 16;
        double ms = INFINITY;
        if (cudaMemcpy(rho, eye.data(), bytes, cudaMemcpyHostToDevice) == cudaSuccess &&
            qpr_evolve(ctx, rho, dt, 4) == QPR_OK) {
            auto t0 = std::chrono::steady_clock::now();
            if (qpr_evolve(ctx, rho, dt, steps) == QPR_OK)
                ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count() /
                     (double)steps;
        }
        qpr_destroy(ctx);
        return ms;
    };
    auto consider = [&](const Cand &c, double ms) {
        if (ms < best) {
            best = ms;
            out->backend = c.backend;
            out->ref_refresh = c.rr;
            out->ms_per_step = ms;
            out->sparse_form = c.form;
            out->row_splits = c.splits;
        }
    };
    std::vector<Cand> cands;
    if (o.precision == QPR_MIXED) {
        cands.push_back({QPR_BACKEND_DENSE, QPR_SPARSE_FORM_AUTO, 0, 32});
        for (int sp : {0, 1, 2, 3, 4}) cands.push_back({QPR_BACKEND_SPARSE, QPR_SPARSE_FORM_COLUMNS, sp, 32});
        cands.push_back({QPR_BACKEND_SPARSE, QPR_SPARSE_FORM_COLUMNS_GATHER, 0, 32});
        cands.push_back({QPR_BACKEND_SPARSE, QPR_SPARSE_FORM_TILES, 0, 32});
    } else {
        cands.push_back({QPR_BACKEND_SPARSE, QPR_SPARSE_FORM_AUTO, 0, o.ref_refresh});
        cands.push_back({QPR_BACKEND_DENSE, QPR_SPARSE_FORM_AUTO, 0, o.ref_refresh});
    }
    for (const Cand &c : cands) consider(c, measure(c, true));
    if (o.precision == QPR_MIXED && best < INFINITY && out->backend == QPR_BACKEND_SPARSE &&
        out->sparse_form == QPR_SPARSE_FORM_COLUMNS_GATHER) {
        // the gather form's splits around its plan's choice
        qpr_options oc = o;
        oc.backend = QPR_BACKEND_SPARSE;
        oc.sparse_form = QPR_SPARSE_FORM_COLUMNS_GATHER;
        oc.device = dev;
        qpr_ctx *ctx = nullptr;
        int32_t plan[4] = {0, 0, 0, 0};
        if (qpr_create(&ctx, n, m, src, dst, w, alpha, omega, &oc) == QPR_OK) {
            qpr_sparse_plan(ctx, plan);
            qpr_destroy(ctx);
        }
        for (int sp : {plan[0] / 2, plan[0] * 2})
            if (sp >= 1 && sp <= 64) {
                const Cand c{QPR_BACKEND_SPARSE, QPR_SPARSE_FORM_COLUMNS_GATHER, sp, 32};
                consider(c, measure(c, true));
            }
    }
    if (o.precision == QPR_MIXED && best < INFINITY) {
        const Cand w0{out->backend, out->sparse_form, out->row_splits, 32};
        for (int rr : {16, 64}) {
            const Cand c{w0.backend, w0.form, w0.splits, rr};
            consider(c, measure(c, false));
        }
    }
    cudaFree(rho);
    if (!(best < INFINITY)) {
        qpr::set_create_error("no candidate configuration ran");
        return QPR_E_CUDA;
    }
    if (cache_path) {
        std::ofstream f(cache_path, std::ios::app);
        if (f)
            f << key << " " << out->backend << " " << out->ref_refresh << " " << out->ms_per_step << " "
              << out->sparse_form << " " << out->row_splits << "\n";
    }
    return ret;
}
