// Fused epilogue shared by the RK4 stage kernels (dense DMMA, sparse CSR).
//
// Input, in shared memory, for the tile pair (I, J), I <= J, of 32 x 32
// complex tiles: sX1 holds X = H Y restricted to rows I and columns J,
// sX2 the same for rows J and columns I (sX2 == sX1 when I == J), each as
// [32][ldx] doubles with
//     sX[a * ldx + b]      = (H Re Y)_ab,
//     sX[a * ldx + 32 + b] = -(H Im Y)_ab.
// With X = A + iB the Lindblad right-hand side (Eq. 1 / Eq. S7, with the
// jump operators L_ij = sqrt(G_ij)|i><j|) of entry (a, b) is
//     k_ab = (1-omega) [ (B_ab + B_ba) - i (A_ab - A_ba) ]
//            + omega [ delta_ab g_a - 1/2 (c_a + c_b) Y_ab ],
// and the classical RK4 stage update (Supplementary Note 2) is applied to
// it. Tile (I, J) is written directly and tile (J, I) as its conjugate
// transpose through shared memory, so every state stays exactly Hermitian.
#pragma once

#include "qpr_internal.cuh"

namespace qpr {

constexpr int kEpiTS = 32;
constexpr int kEpiLDO = kEpiTS + 1;
constexpr int kEpiThreads = 128;

__device__ __forceinline__ double epi_warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// sO: 4 * 32 * kEpiLDO doubles of shared memory, disjoint from sX1/sX2.
// Must be called by all kEpiThreads threads of the CTA after the X tiles
// are complete and visible (__syncthreads()).
// pidx: slot of this tile pair's residual partial; first: the tile pair
// that advances the step counter at stage 4.
template <int STAGE>
__device__ __forceinline__ void stage_epilogue(const DevOps &ops, const Work &w, int I, int J, bool diag,
                                               const double *sX1, const double *sX2, int ldx,
                                               double *sO, double *red, int pidx, bool first) {
    constexpr int TS = kEpiTS, LDO = kEpiLDO;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int np = ops.np;
    const size_t plane = (size_t)np * np;
    const double *__restrict__ yin = (STAGE <= 1) ? w.y : (STAGE == 3 ? w.yb : w.ya);
    const double *X2 = diag ? sX1 : sX2;
    const Ctl *ctl = w.ctl;

    const double om = ops.omega, cm = 1.0 - om;
    const double scale = ctl->scale;
    const double gsig = (STAGE == 1) ? scale : 1.0;                 // stage-1 input is unnormalised y
    const double ysig = (STAGE >= 1 && STAGE <= 3) ? scale : 1.0;  // Y1 = y / tr(y)
    const double dt = ctl->dt;
    const double dt6 = __ddiv_rn(dt, 6.0), dt3 = __ddiv_rn(dt, 3.0);
    const double cg = __dmul_rn(cm, gsig);
    double nrm = 0.0;

    // Every operation below is an explicit round-to-nearest intrinsic, so the
    // result does not depend on how a compiler contracts it in the kernel that
    // inlines this function (single-problem and batched kernels agree bitwise).
    for (int e = tid; e < TS * TS; e += kEpiThreads) {
        const int a = e / TS, b = e - (e / TS) * TS;
        const int ga = I * TS + a, gb = J * TS + b;
        const size_t off = (size_t)ga * np + gb;
        const double Aab = sX1[a * ldx + b], Bab = -sX1[a * ldx + TS + b];
        const double Aba = X2[b * ldx + a], Bba = -X2[b * ldx + TS + a];
        const double ysr = __dmul_rn(gsig, yin[off]), ysi = __dmul_rn(gsig, yin[plane + off]);
        const double omhc = __dmul_rn(om, __dmul_rn(0.5, __dadd_rn(ops.c[ga], ops.c[gb])));
        double kr = __fma_rn(-omhc, ysr, __dmul_rn(cg, __dadd_rn(Bab, Bba)));
        const double ki = __fma_rn(-omhc, ysi, __dmul_rn(-cg, __dsub_rn(Aab, Aba)));
        if (ga == gb) kr = __fma_rn(om, w.g[ga], kr);
        if (STAGE <= 1) nrm = __fma_rn(kr, kr, __fma_rn(ki, ki, nrm));

        double o0, o1, o2 = 0.0, o3 = 0.0;
        if (STAGE == 0) {
            o0 = kr;
            o1 = ki;
            w.z[off] = o0;
            w.z[plane + off] = o1;
        } else if (STAGE <= 3) {
            const double y1r = __dmul_rn(ysig, w.y[off]), y1i = __dmul_rn(ysig, w.y[plane + off]);
            if (STAGE == 1) {
                o0 = __fma_rn(dt6, kr, y1r);
                o1 = __fma_rn(dt6, ki, y1i);
            } else {
                o0 = __fma_rn(dt3, kr, w.z[off]);
                o1 = __fma_rn(dt3, ki, w.z[plane + off]);
            }
            const double cst = (STAGE == 3) ? dt : __dmul_rn(0.5, dt);
            o2 = __fma_rn(cst, kr, y1r);
            o3 = __fma_rn(cst, ki, y1i);
            double *yn = (STAGE == 2) ? w.yb : w.ya;
            w.z[off] = o0;
            w.z[plane + off] = o1;
            yn[off] = o2;
            yn[plane + off] = o3;
        } else {
            o0 = __fma_rn(dt6, kr, w.z[off]);
            o1 = __fma_rn(dt6, ki, w.z[plane + off]);
            w.y[off] = o0;
            w.y[plane + off] = o1;
        }
        sO[0 * TS * LDO + a * LDO + b] = o0;
        sO[1 * TS * LDO + a * LDO + b] = o1;
        if (STAGE >= 1 && STAGE <= 3) {
            sO[2 * TS * LDO + a * LDO + b] = o2;
            sO[3 * TS * LDO + a * LDO + b] = o3;
        }
    }

    if (STAGE <= 1) {
        nrm = epi_warp_sum(nrm);
        if (lane == 0) red[warp] = nrm;
        __syncthreads();
        if (tid == 0) {
            double s = 0.0;
            for (int q = 0; q < kEpiThreads / 32; ++q) s += red[q];
            w.partials[pidx] = diag ? s : 2.0 * s;
        }
    }

    if (!diag) {
        __syncthreads();
        // tile (J, I) = conjugate transpose of tile (I, J)
        double *d0, *d1, *d2 = nullptr, *d3 = nullptr;
        if (STAGE == 0) {
            d0 = w.z;
            d1 = w.z + plane;
        } else if (STAGE <= 3) {
            double *yn = (STAGE == 2) ? w.yb : w.ya;
            d0 = w.z;
            d1 = w.z + plane;
            d2 = yn;
            d3 = yn + plane;
        } else {
            d0 = w.y;
            d1 = w.y + plane;
        }
        for (int e = tid; e < TS * TS; e += kEpiThreads) {
            const int b = e / TS, a = e - (e / TS) * TS;
            const size_t off = (size_t)(J * TS + b) * np + I * TS + a;
            d0[off] = sO[0 * TS * LDO + a * LDO + b];
            d1[off] = -sO[1 * TS * LDO + a * LDO + b];
            if (STAGE >= 1 && STAGE <= 3) {
                d2[off] = sO[2 * TS * LDO + a * LDO + b];
                d3[off] = -sO[3 * TS * LDO + a * LDO + b];
            }
        }
    }

    if (STAGE == 4 && first && tid == 0) w.ctl->step += 1;
}

}  // namespace qpr
