// Autotuner: picks the kernel family (sparse CSR or dense tensor-core stage)
// and, for the mixed form, the reference-refresh block length for one problem
// by timing short real runs on the device, and caches the choice in a text
// file keyed by GPU name, precision and size/density buckets.
//
// Cache line format (one per key, later lines win):
//   <key> <backend> <ref_refresh> <ms_per_step>
// with key = "<gpu name without spaces>|p<precision>|n<floor log2 N>|d<floor log2 (nnz(H)/N + 1)>".
#include <math.h>
#include <stdio.h>
#include <string.h>

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
        int be = 0, rr = 0;
        double ms = 0.0;
        if (is >> k >> be >> rr >> ms && k == key) {
            out->backend = be;
            out->ref_refresh = rr;
            out->ms_per_step = ms;
            found = true;
        }
    }
    return found;
}

}  // namespace

extern "C" qpr_status qpr_autotune(int64_t n, int64_t m, const int64_t *src, const int64_t *dst, const double *w,
                                   double alpha, double omega, double dt, const qpr_options *base,
                                   const char *cache_path, qpr_tune_result *out) {
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
    // candidates
    struct Cand { int backend, rr; };
    std::vector<Cand> cands;
    const int backends[2] = {QPR_BACKEND_SPARSE, QPR_BACKEND_DENSE};
    for (int be : backends) {
        if (o.precision == QPR_MIXED) {
            for (int rr : {8, 16, 32, 64}) cands.push_back({be, rr});
        } else {
            cands.push_back({be, o.ref_refresh});
        }
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
    double best = INFINITY;
    qpr_status ret = QPR_OK;
    for (const Cand &c : cands) {
        qpr_options oc = o;
        oc.backend = c.backend;
        oc.ref_refresh = c.rr;
        oc.device = dev;
        qpr_ctx *ctx = nullptr;
        if (qpr_create(&ctx, n, m, src, dst, w, alpha, omega, &oc) != QPR_OK) continue;  // e.g. out of memory
        const int steps = o.precision == QPR_MIXED ? std::max(16, 2 * c.rr) : 16;
        double ms = INFINITY;
        if (cudaMemcpy(rho, eye.data(), bytes, cudaMemcpyHostToDevice) == cudaSuccess &&
            qpr_evolve(ctx, rho, dt, 4) == QPR_OK) {
            auto t0 = std::chrono::steady_clock::now();
            if (qpr_evolve(ctx, rho, dt, steps) == QPR_OK)
                ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count() /
                     (double)steps;
        }
        qpr_destroy(ctx);
        if (ms < best) {
            best = ms;
            out->backend = c.backend;
            out->ref_refresh = c.rr;
            out->ms_per_step = ms;
        }
    }
    cudaFree(rho);
    if (!(best < INFINITY)) {
        qpr::set_create_error("no candidate configuration ran");
        return QPR_E_CUDA;
    }
    if (cache_path) {
        std::ofstream f(cache_path, std::ios::app);
        if (f) f << key << " " << out->backend << " " << out->ref_refresh << " " << out->ms_per_step << "\n";
    }
    return ret;
}
