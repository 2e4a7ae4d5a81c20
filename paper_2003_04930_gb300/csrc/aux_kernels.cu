// O(N^2) and O(E + N) kernels around the stage GEMM: Hermitising import,
// export with trace normalisation, diagonal extraction, and the gain
// g = G p of the dissipator.
#include <math.h>

#include "gain_body.cuh"
#include "qpr_internal.cuh"

namespace qpr {
namespace {

constexpr int kGainThreads = 256;

using gain64::block_sum;
using gain64::warp_sum;

__global__ void import_kernel(const double *__restrict__ rho, int n, int np, double *__restrict__ out) {
    const size_t plane = (size_t)np * np;
    for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < plane;
         idx += (size_t)gridDim.x * blockDim.x) {
        const int a = (int)(idx / np), b = (int)(idx - (size_t)a * np);
        double re = 0.0, im = 0.0;
        if (a < n && b < n) {
            const double *x = rho + 2 * ((size_t)a * n + b);
            const double *xt = rho + 2 * ((size_t)b * n + a);
            re = 0.5 * (x[0] + xt[0]);
            im = 0.5 * (x[1] - xt[1]);
        }
        out[idx] = re;
        out[plane + idx] = im;
    }
}

__global__ void export_kernel(const double *__restrict__ planes, int n, int np, const Ctl *ctl,
                              int use_scale, double *__restrict__ rho) {
    const size_t plane = (size_t)np * np;
    const double s = use_scale ? ctl->scale : 1.0;
    const size_t nn = (size_t)n * n;
    for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < nn;
         idx += (size_t)gridDim.x * blockDim.x) {
        const int a = (int)(idx / n), b = (int)(idx - (size_t)a * n);
        const size_t src = (size_t)a * np + b;
        rho[2 * idx] = s * planes[src];
        rho[2 * idx + 1] = s * planes[plane + src];
    }
}

__global__ void diag_kernel(const double *__restrict__ rho, int n, double *__restrict__ p) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        p[i] = rho[2 * ((size_t)i * n + i)];
}

template <int STAGE>
__global__ void __launch_bounds__(kGainThreads)
gain_kernel(DevOps ops, Work w, const double *__restrict__ yin) {
    __shared__ int s_done;
    // CTA 0 of this very kernel may set `done` while other CTAs start: read
    // it once per CTA so that every thread of a CTA takes the same branch.
    if (threadIdx.x == 0) s_done = *(volatile int *)&w.ctl->done;
    __syncthreads();
    if (s_done) return;
    gain64::gain_fp64_body<STAGE>(ops, w, yin, blockIdx.x, gridDim.x);
}

int grid_for(size_t work, int threads) {
    size_t b = (work + threads - 1) / threads;
    if (b > 152 * 16) b = 152 * 16;
    if (b < 1) b = 1;
    return (int)b;
}

}  // namespace

void launch_import(const double *rho_il, int n, int np, double *planes, cudaStream_t s) {
    import_kernel<<<grid_for((size_t)np * np, 256), 256, 0, s>>>(rho_il, n, np, planes);
}

void launch_export(const double *planes, int n, int np, const Ctl *ctl, int use_scale,
                   double *rho_il, cudaStream_t s) {
    export_kernel<<<grid_for((size_t)n * n, 256), 256, 0, s>>>(planes, n, np, ctl, use_scale, rho_il);
}

void launch_diag(const double *rho_il, int n, double *p, cudaStream_t s) {
    diag_kernel<<<grid_for((size_t)n, 256), 256, 0, s>>>(rho_il, n, p);
}

void launch_gain(int stage, const DevOps &ops, const double *yin, const Work &w, cudaStream_t s) {
    const int wpb = kGainThreads / 32;
    int blocks = (ops.np + wpb - 1) / wpb;
    if (blocks > 152) blocks = 152;
    switch (stage) {
        case 0: gain_kernel<0><<<blocks, kGainThreads, 0, s>>>(ops, w, yin); break;
        case 1: gain_kernel<1><<<blocks, kGainThreads, 0, s>>>(ops, w, yin); break;
        case 2: gain_kernel<2><<<blocks, kGainThreads, 0, s>>>(ops, w, yin); break;
        case 3: gain_kernel<3><<<blocks, kGainThreads, 0, s>>>(ops, w, yin); break;
        default: gain_kernel<4><<<blocks, kGainThreads, 0, s>>>(ops, w, yin); break;
    }
}

}  // namespace qpr
