// Classical PageRank and hub classes (main text, the airline ranking: the
// quantum PageRank populations compared with the classical PageRank vector,
// nodes sorted into main and secondary hubs).
//
// The classical PageRank is the stationary vector pi of the Google matrix
// G = alpha S + (1 - alpha) F (Eq. S4 with the column-normalised adjacency,
// F of Eq. S2): G pi = pi, sum pi = 1. It is also the populations of the
// omega = 1 steady state of the Lindblad equation (Eq. 1 with only the
// dissipator, whose populations follow dp/dt = G p - c o p with c = 1).
// Power iteration pi <- G pi from the uniform vector, in FP64: each
// iteration is one kernel whose CTAs form G pi for their rows (CSR of S,
// the dangling columns, the teleport part) and per-CTA partials of the L1
// change, which the host sums in index order every few iterations.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <utility>
#include <vector>

#include "gain_body.cuh"
#include "qpr_internal.cuh"

namespace qpr {
namespace {

constexpr int kPrThreads = 256;

using gain64::block_sum;

// One power-iteration step: out = G pi / sum(pi) for rows of this CTA
// (rows blk, blk + grid, ... in warps), and this CTA's partial of
// sum |out_i - pi_i| / sum(pi) (delta[blk]). Every CTA sums pi and its
// dangling part itself, in the same order, so the iteration is
// deterministic.
__global__ void __launch_bounds__(kPrThreads) pagerank_step_kernel(DevOps ops, const double *__restrict__ pi,
                                                                  double *__restrict__ out,
                                                                  double *__restrict__ delta) {
    __shared__ double red[32];
    const int n = ops.n;
    double P = 0.0, Dd = 0.0;
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
        const double pj = pi[j];
        P += pj;
        if (ops.dang[j]) Dd += pj;
    }
    P = block_sum(P, red);
    Dd = block_sum(Dd, red);
    const double inv = 1.0 / P;
    const int lane = threadIdx.x & 31, warps = blockDim.x >> 5;
    double dl = 0.0;
    for (int i = blockIdx.x * warps + (threadIdx.x >> 5); i < n; i += gridDim.x * warps) {
        double s = 0.0;
        for (int q = ops.s_ptr[i] + lane; q < ops.s_ptr[i + 1]; q += 32) s += ops.s_val[q] * pi[ops.s_col[q]];
        s = gain64::warp_sum(s);
        if (lane == 0) {
            const double pii = pi[i];
            const double dterm = (ops.dangling == QPR_DANGLING_F) ? (Dd - (ops.dang[i] ? pii : 0.0)) / (n - 1)
                                                                  : Dd / n;
            const double g = (ops.alpha * (s + dterm) + (1.0 - ops.alpha) * (P - pii) / (n - 1)) * inv;
            out[i] = g;
            dl += fabs(g - pii * inv);
        }
    }
    dl = block_sum(dl, red);
    if (threadIdx.x == 0) delta[blockIdx.x] = dl;
}

__global__ void uniform_kernel(double *pi, int n) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) pi[i] = 1.0 / n;
}

// pi / sum(pi) into out (one CTA; fixed-order sum).
__global__ void __launch_bounds__(1024) normalize_kernel(const double *__restrict__ pi, int n,
                                                         double *__restrict__ out) {
    __shared__ double red[32];
    double P = 0.0;
    for (int j = threadIdx.x; j < n; j += blockDim.x) P += pi[j];
    P = block_sum(P, red);
    for (int j = threadIdx.x; j < n; j += blockDim.x) out[j] = pi[j] / P;
}

// classes[i] = 2 (main hub, p_i > c / N), 1 (secondary, 1/N < p_i <= c/N),
// 0 otherwise; counts[k] += the nodes of class k.
__global__ void hub_kernel(const double *__restrict__ p, int n, double c, int *__restrict__ classes,
                           unsigned long long *__restrict__ counts) {
    __shared__ unsigned int cnt[3];
    if (threadIdx.x < 3) cnt[threadIdx.x] = 0;
    __syncthreads();
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const double v = p[i];
        const int k = (v > c / (double)n) ? 2 : (v > 1.0 / (double)n ? 1 : 0);
        classes[i] = k;
        atomicAdd(&cnt[k], 1u);
    }
    __syncthreads();
    if (threadIdx.x < 3) atomicAdd(&counts[threadIdx.x], (unsigned long long)cnt[threadIdx.x]);
}

}  // namespace

int pagerank_grid(int n) {
    int sms = 0, dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) {
        cudaGetLastError();
        sms = 1;
    }
    const int rows_per_cta = kPrThreads / 32;
    int grid = (n + rows_per_cta - 1) / rows_per_cta;
    if (grid > 2 * sms) grid = 2 * sms;
    return grid < 1 ? 1 : grid;
}

cudaError_t pagerank(const DevOps &ops, double tol, int64_t max_iter, double *scratch, double *pi_out_dev,
                     int64_t *iters, double *delta_out, cudaStream_t s) {
    const int n = ops.n;
    const int grid = pagerank_grid(n);
    cudaError_t e = cudaSuccess;
    double *a = scratch, *b = scratch + n, *delta = scratch + 2 * (size_t)n;
    uniform_kernel<<<(n + 255) / 256, 256, 0, s>>>(a, n);
    std::vector<double> part(grid);
    // check convergence every `chunk` iterations (the host reads the last
    // iteration's partials)
    const int chunk = 8;
    int64_t it = 0;
    double d = INFINITY;
    while (it < max_iter) {
        const int64_t k1 = std::min<int64_t>(max_iter, it + chunk);
        for (; it < k1; ++it) {
            pagerank_step_kernel<<<grid, kPrThreads, 0, s>>>(ops, a, b, delta);
            std::swap(a, b);
        }
        e = cudaMemcpyAsync(part.data(), delta, grid * sizeof(double), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) break;
        d = 0.0;
        for (double v : part) d += v;
        if (!(d >= tol)) break;  // converged (or not finite)
    }
    if (e == cudaSuccess) {
        normalize_kernel<<<1, 1024, 0, s>>>(a, n, pi_out_dev);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (iters) *iters = it;
    if (delta_out) *delta_out = d;
    return e;
}

cudaError_t hub_classes(const double *p, int n, double c, int *classes_dev, unsigned long long *counts_dev,
                        cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(counts_dev, 0, 3 * sizeof(unsigned long long), s);
    if (e != cudaSuccess) return e;
    int grid = (n + 255) / 256;
    if (grid > 1024) grid = 1024;
    hub_kernel<<<grid, 256, 0, s>>>(p, n, c, classes_dev, counts_dev);
    return cudaGetLastError();
}

}  // namespace qpr
