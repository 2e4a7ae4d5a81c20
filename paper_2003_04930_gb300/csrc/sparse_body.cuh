// FP64 sparse stage: one tile pair as a device function (shared by the
// single-problem kernel and the batched kernels).
#pragma once

#include "qpr_internal.cuh"
#include "stage_epilogue.cuh"

namespace qpr {
namespace sparse64 {

constexpr int TS = kEpiTS;
constexpr int NTHREADS = kEpiThreads;
constexpr int LDX = 2 * TS + 1;
constexpr int LDO = kEpiLDO;
constexpr int SMEM_BYTES = (2 * TS * LDX + 4 * TS * LDO) * (int)sizeof(double);

// rows `rowtile` of H times columns `coltile` of Y into sX ([TS][LDX]).
__device__ __forceinline__ void spmm_tile(const DevOps &ops, const double *__restrict__ yin, size_t plane,
                                          int rowtile, int coltile, double *sX) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int np = ops.np, n = ops.n;
    const int col = coltile * TS + lane;
    const double *__restrict__ yre = yin + col;
    const double *__restrict__ yim = yin + plane + col;
    for (int a = warp; a < TS; a += NTHREADS / 32) {
        const int ga = rowtile * TS + a;
        double xr = 0.0, xi = 0.0;
        if (ga < n) {
            const int q1 = ops.h_ptr[ga + 1];
            int q = ops.h_ptr[ga];
            for (; q + 4 <= q1; q += 4) {
                const int k0 = ops.h_col[q], k1 = ops.h_col[q + 1], k2 = ops.h_col[q + 2], k3 = ops.h_col[q + 3];
                const double h0 = ops.h_val[q], h1 = ops.h_val[q + 1], h2 = ops.h_val[q + 2], h3 = ops.h_val[q + 3];
                const double r0 = yre[(size_t)k0 * np], r1 = yre[(size_t)k1 * np];
                const double r2 = yre[(size_t)k2 * np], r3 = yre[(size_t)k3 * np];
                const double i0 = yim[(size_t)k0 * np], i1 = yim[(size_t)k1 * np];
                const double i2 = yim[(size_t)k2 * np], i3 = yim[(size_t)k3 * np];
                // explicit fused multiply-adds: the same rounding in every kernel
                // that inlines this function
                xr = __fma_rn(h0, r0, xr); xi = __fma_rn(h0, i0, xi);
                xr = __fma_rn(h1, r1, xr); xi = __fma_rn(h1, i1, xi);
                xr = __fma_rn(h2, r2, xr); xi = __fma_rn(h2, i2, xi);
                xr = __fma_rn(h3, r3, xr); xi = __fma_rn(h3, i3, xi);
            }
            for (; q < q1; ++q) {
                const int k = ops.h_col[q];
                const double h = ops.h_val[q];
                xr = __fma_rn(h, yre[(size_t)k * np], xr);
                xi = __fma_rn(h, yim[(size_t)k * np], xi);
            }
        }
        sX[a * LDX + lane] = xr;
        sX[a * LDX + TS + lane] = -xi;
    }
}

// One tile pair (I, J) of stage STAGE; smem: SMEM_BYTES of dynamic shared
// memory. Ends with a barrier so that the caller may reuse shared memory.
template <int STAGE>
__device__ __forceinline__ void tile(const DevOps &ops, const Work &w, int I, int J, int pidx, bool first,
                                     double *smem) {
    __shared__ double red[NTHREADS / 32];
    const bool diag = (I == J);
    const size_t plane = (size_t)ops.np * ops.np;
    const double *__restrict__ yin = (STAGE <= 1) ? w.y : (STAGE == 3 ? w.yb : w.ya);
    double *sX1 = smem;
    double *sX2 = smem + TS * LDX;
    double *sO = smem + 2 * TS * LDX;
    spmm_tile(ops, yin, plane, I, J, sX1);
    if (!diag) spmm_tile(ops, yin, plane, J, I, sX2);
    __syncthreads();
    stage_epilogue<STAGE>(ops, w, I, J, diag, sX1, sX2, LDX, sO, red, pidx, first);
    __syncthreads();
}

}  // namespace sparse64
}  // namespace qpr
