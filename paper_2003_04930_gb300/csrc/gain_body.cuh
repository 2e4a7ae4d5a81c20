// FP64 gain g = G p as a device function (single-problem and batched kernels).
#pragma once

#include <math.h>

#include "qpr_internal.cuh"

namespace qpr {
namespace gain64 {

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Fixed-order block sum, broadcast to every thread (blockDim.x <= 1024).
__device__ __forceinline__ double block_sum(double v, double *red) {
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

// g = G p with G = alpha S + (1 - alpha) F (Eq. S2, Eq. S4), p_j = sig Y_jj:
//   (S p)_i = sum_{j with out-links} A_ij / outDeg(j) p_j  +  dangling part,
//   dangling part = (D - [i dangles] p_i) / (N - 1)  (F columns)  or  D / N,
//   (F p)_i = (P - p_i) / (N - 1),
// with P = sum_j p_j and D = sum over dangling j of p_j.
// Stage 1 also fixes sig = 1 / Re tr(y) for the whole step. Stage 2 first
// reduces the residual partials of stage 1 into ||f(y_n)||_F and takes the
// stop decision (one CTA).
// blk / nblk: this CTA's index and the number of CTAs sharing the rows; the
// residual decision (stage 2) is taken by blk 0.
template <int STAGE>
__device__ __forceinline__ void gain_fp64_body(const DevOps &ops, const Work &w, const double *__restrict__ yin,
                                               int blk, int nblk) {
    __shared__ double red[32];
    Ctl *ctl = w.ctl;
    const int n = ops.n, np = ops.np;

    if (STAGE == 2 && blk == 0) {
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
        if (blk == 0 && threadIdx.x == 0) {
            ctl->scale = sig;
            ctl->trace = P;
            if (!(P > 0.0) || !isfinite(P)) {
                ctl->status = kCtlNonFinite;
                ctl->done = 1;
            }
        }
    }
    const double Ps = __dmul_rn(sig, P), Ds = __dmul_rn(sig, D);
    const double inv_nm1 = __drcp_rn((double)(n - 1));
    const int lane = threadIdx.x & 31;
    const int wpb = blockDim.x >> 5;
    for (int i = blk * wpb + (threadIdx.x >> 5); i < np; i += nblk * wpb) {
        double s = 0.0;
        if (i < n) {
            for (int q = ops.s_ptr[i] + lane; q < ops.s_ptr[i + 1]; q += 32) {
                const int j = ops.s_col[q];
                s = __fma_rn(ops.s_val[q], __dmul_rn(sig, yin[(size_t)j * np + j]), s);
            }
        }
        s = warp_sum(s);
        if (lane == 0) {
            double gi = 0.0;
            if (i < n) {
                const double pi = __dmul_rn(sig, yin[(size_t)i * np + i]);
                const double dterm = (ops.dangling == QPR_DANGLING_F)
                                         ? __dmul_rn(__dsub_rn(Ds, ops.dang[i] ? pi : 0.0), inv_nm1)
                                         : __ddiv_rn(Ds, (double)n);
                gi = __fma_rn(ops.alpha, __dadd_rn(s, dterm),
                              __dmul_rn(__dmul_rn(__dsub_rn(1.0, ops.alpha), __dsub_rn(Ps, pi)), inv_nm1));
            }
            w.g[i] = gi;
        }
    }
}

}  // namespace gain64
}  // namespace qpr
