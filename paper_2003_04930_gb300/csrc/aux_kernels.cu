// O(N^2) and O(E + N) kernels around the stage GEMM: Hermitising import,
// export with trace normalisation, diagonal extraction, and the gain
// g = G p of the dissipator.
#include <math.h>

#include "qpr_internal.cuh"

namespace qpr {
namespace {

constexpr int kGainThreads = 256;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Fixed-order block sum, broadcast to every thread (blockDim.x <= 1024).
__device__ double block_sum(double v, double *red) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    v = warp_sum(v);
    __syncthreads();  // red may still be read by a previous call
    if (lane == 0) red[warp] = v;
    __syncthreads();
    double s = 0.0;
    const int nw = (blockDim.x + 31) >> 5;
    for (int q = 0; q < nw; ++q) s += red[q];
    return s;
}

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

// g = G p with G = alpha S + (1 - alpha) F (Eq. S2, Eq. S4), p_j = sig Y_jj:
//   (S p)_i = sum_{j with out-links} A_ij / outDeg(j) p_j  +  dangling part,
//   dangling part = (D - [i dangles] p_i) / (N - 1)  (F columns)  or  D / N,
//   (F p)_i = (P - p_i) / (N - 1),
// with P = sum_j p_j and D = sum over dangling j of p_j.
// Stage 1 also fixes sig = 1 / Re tr(y) for the whole step. Stage 2 first
// reduces the residual partials of stage 1 into ||f(y_n)||_F and takes the
// stop decision (one CTA).
template <int STAGE>
__global__ void __launch_bounds__(kGainThreads)
gain_kernel(DevOps ops, Work w, const double *__restrict__ yin) {
    __shared__ double red[kGainThreads / 32];
    __shared__ int s_done;
    Ctl *ctl = w.ctl;
    // CTA 0 of this very kernel may set `done` while other CTAs start: read
    // it once per CTA so that every thread of a CTA takes the same branch.
    if (threadIdx.x == 0) s_done = *(volatile int *)&ctl->done;
    __syncthreads();
    if (s_done) return;
    const int n = ops.n, np = ops.np;

    if (STAGE == 2 && blockIdx.x == 0) {
        double s = 0.0;
        for (int i = threadIdx.x; i < w.npairs; i += blockDim.x) s += w.partials[i];
        s = block_sum(s, red);
        if (threadIdx.x == 0) {
            const double r = sqrt(s);
            ctl->resid = r;
            ctl->resid_step = ctl->step;
            if (!isfinite(r)) {
                ctl->status = kCtlNonFinite;
                ctl->done = 1;
            } else if (r < ctl->tol) {
                ctl->status = kCtlConverged;
                ctl->done = 1;
            } else if (ctl->step >= ctl->max_steps) {
                ctl->status = kCtlMaxSteps;
                ctl->done = 1;
            }
        }
    }

    double P = 0.0, D = 0.0;
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
        const double pj = yin[(size_t)j * np + j];
        P += pj;
        if (ops.dang[j]) D += pj;
    }
    P = block_sum(P, red);
    D = block_sum(D, red);
    double sig = 1.0;
    if (STAGE == 1) {
        sig = 1.0 / P;
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            ctl->scale = sig;
            ctl->trace = P;
            if (!(P > 0.0) || !isfinite(P)) {
                ctl->status = kCtlNonFinite;
                ctl->done = 1;
            }
        }
    }
    const double Ps = sig * P, Ds = sig * D;
    const double inv_nm1 = 1.0 / (double)(n - 1);
    const int lane = threadIdx.x & 31;
    const int wpb = blockDim.x >> 5;
    for (int i = blockIdx.x * wpb + (threadIdx.x >> 5); i < np; i += gridDim.x * wpb) {
        double s = 0.0;
        if (i < n) {
            for (int q = ops.s_ptr[i] + lane; q < ops.s_ptr[i + 1]; q += 32) {
                const int j = ops.s_col[q];
                s += ops.s_val[q] * (sig * yin[(size_t)j * np + j]);
            }
        }
        s = warp_sum(s);
        if (lane == 0) {
            double gi = 0.0;
            if (i < n) {
                const double pi = sig * yin[(size_t)i * np + i];
                const double dterm = (ops.dangling == QPR_DANGLING_F)
                                         ? (Ds - (ops.dang[i] ? pi : 0.0)) * inv_nm1
                                         : Ds / (double)n;
                gi = ops.alpha * (s + dterm) + (1.0 - ops.alpha) * (Ps - pi) * inv_nm1;
            }
            w.g[i] = gi;
        }
    }
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
