// Mixed-precision RK4 with an exact FP64 reference ("delta form").
//
// f is linear, so for any reference state R and stage input Y_s
//     f(Y_s) = f(R) + f(Y_s - R).
// Every refresh (start of every block of `ref_refresh` steps) sets
// R = y / tr(y), computes F = f(R) exactly in FP64 (the sparse FP64 stage
// kernel, stage 0), and takes ||F||_F as the exact FP64 residual of that step.
// Between refreshes the stage inputs are carried as FP32 deltas
// delta_s = Y_s - R and only f(delta_s) is evaluated, in FP32:
//   stage 1: k1 = F + f(D),   S  = f(D),     da = D + dt/2 k1   (D = y - R)
//   stage 2: k2 = F + f(da),  S += 2 f(da),  db = D + dt/2 k2
//   stage 3: k3 = F + f(db),  S += 2 f(db),  da = D + dt k3
//   stage 4: k4 = F + f(da),  y += dt F + dt/6 (S + f(da)) in FP64,  D = y - R
// (the weights sum to 6, so the F part of the RK4 sum is added once, in FP64)
// FP64 is used for the RK accumulation into y, the trace renormalisation and
// the exact residual; everything else runs on the FP32 pipe (GB300 has
// roughly 1/64 of its FP32 rate in FP64). The error of an FP32 f(delta) is
// relative to |H| |delta|, and |delta| shrinks with the residual, so the
// steady state reached is the FP64 one (the final answer is always
// re-checked with an exact FP64 residual).
//
// The stage kernel forms X = H delta from the CSR of H in FP32 (one warp per
// row, four nonzeros per warp instruction, float4 per lane, fixed-order
// reduction) and fuses the Lindblad right-hand side and the stage update
// into the epilogue, writing tile (I, J) and its conjugate transpose.
#include <math.h>

#include "qpr_internal.cuh"
#include "stage_epilogue.cuh"

namespace qpr {
namespace {

constexpr int TS = 32;
constexpr int NT = 256;           // threads per CTA
constexpr int LDX = 2 * TS + 1;   // X tile row: real part, then imaginary part
constexpr int LDO = TS + 1;

__device__ __forceinline__ float4 f4fma(float h, float4 v, float4 acc) {
    acc.x = fmaf(h, v.x, acc.x);
    acc.y = fmaf(h, v.y, acc.y);
    acc.z = fmaf(h, v.z, acc.z);
    acc.w = fmaf(h, v.w, acc.w);
    return acc;
}
__device__ __forceinline__ float4 f4xor(float4 v, int m) {
    v.x += __shfl_xor_sync(0xffffffffu, v.x, m);
    v.y += __shfl_xor_sync(0xffffffffu, v.y, m);
    v.z += __shfl_xor_sync(0xffffffffu, v.z, m);
    v.w += __shfl_xor_sync(0xffffffffu, v.w, m);
    return v;
}

// sX[a][b] = (H Re d)_ab, sX[a][TS + b] = (H Im d)_ab for rows of tile rt and
// columns of tile ct, in FP32.
__device__ __forceinline__ void spmm32_tile(const DevOps &ops, const float *__restrict__ d, size_t plane,
                                            int rt, int ct, float *sX) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int grp = lane >> 3, sub = lane & 7;
    const int np = ops.np, n = ops.n;
    const float *__restrict__ re = d + ct * TS + 4 * sub;
    const float *__restrict__ im = d + plane + ct * TS + 4 * sub;
    for (int a = warp; a < TS; a += NT / 32) {
        const int ga = rt * TS + a;
        float4 xr = make_float4(0.f, 0.f, 0.f, 0.f), xi = xr;
        if (ga < n) {
            const int q1 = ops.h_ptr[ga + 1];
            int q = ops.h_ptr[ga] + grp;
            for (; q + 4 < q1; q += 8) {
                const int k0 = ops.h_col[q], k1 = ops.h_col[q + 4];
                const float h0 = ops.h_val32[q], h1 = ops.h_val32[q + 4];
                const float4 r0 = *reinterpret_cast<const float4 *>(re + (size_t)k0 * np);
                const float4 i0 = *reinterpret_cast<const float4 *>(im + (size_t)k0 * np);
                const float4 r1 = *reinterpret_cast<const float4 *>(re + (size_t)k1 * np);
                const float4 i1 = *reinterpret_cast<const float4 *>(im + (size_t)k1 * np);
                xr = f4fma(h0, r0, xr);
                xi = f4fma(h0, i0, xi);
                xr = f4fma(h1, r1, xr);
                xi = f4fma(h1, i1, xi);
            }
            if (q < q1) {
                const int k0 = ops.h_col[q];
                const float h0 = ops.h_val32[q];
                xr = f4fma(h0, *reinterpret_cast<const float4 *>(re + (size_t)k0 * np), xr);
                xi = f4fma(h0, *reinterpret_cast<const float4 *>(im + (size_t)k0 * np), xi);
            }
        }
        xr = f4xor(xr, 8);
        xr = f4xor(xr, 16);
        xi = f4xor(xi, 8);
        xi = f4xor(xi, 16);
        if (grp == 0) {
            float *row = sX + a * LDX;
            row[4 * sub + 0] = xr.x; row[4 * sub + 1] = xr.y; row[4 * sub + 2] = xr.z; row[4 * sub + 3] = xr.w;
            row[TS + 4 * sub + 0] = xi.x; row[TS + 4 * sub + 1] = xi.y;
            row[TS + 4 * sub + 2] = xi.z; row[TS + 4 * sub + 3] = xi.w;
        }
    }
}

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

template <int STAGE>
__global__ void __launch_bounds__(NT)
stage_mixed_sparse_kernel(DevOps ops, MixedWork w) {
    __shared__ __align__(16) float sX1[TS * LDX];
    __shared__ __align__(16) float sX2[TS * LDX];
    // outputs of tile (I, J) kept for the mirrored write: stages 1-3 keep S and
    // the next delta (4 FP32 planes), stage 4 the new y (2 FP64 planes) and D
    // (2 FP32 planes); 25.3 KB either way
    __shared__ __align__(16) double sOraw[(2 * TS * LDO * 8 + 2 * TS * LDO * 4) / 8];
    double *sO64 = sOraw;
    float *sO32 = (STAGE == 4) ? reinterpret_cast<float *>(sOraw + 2 * TS * LDO) : reinterpret_cast<float *>(sOraw);
    __shared__ double red[NT / 32];
    __shared__ int s_done;
    if (threadIdx.x == 0) s_done = *(volatile int *)&w.ctl->done;
    __syncthreads();
    if (s_done) return;

    const int I = w.pairs[blockIdx.x].x, J = w.pairs[blockIdx.x].y;
    const bool diag = (I == J);
    const int np = ops.np;
    const size_t plane = (size_t)np * np;
    const float *__restrict__ din = (STAGE == 1) ? w.D : (STAGE == 3 ? w.db : w.da);
    float *dnext = (STAGE == 2) ? w.db : w.da;

    spmm32_tile(ops, din, plane, I, J, sX1);
    if (!diag) spmm32_tile(ops, din, plane, J, I, sX2);
    __syncthreads();
    const float *X2 = diag ? sX1 : sX2;

    const float om = (float)ops.omega, cm = 1.0f - om;
    const double dt = w.ctl->dt;
    const float dtf = (float)dt;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    double nrm = 0.0;
    for (int e = tid; e < TS * TS; e += NT) {
        const int a = e / TS, b = e - (e / TS) * TS;
        const int ga = I * TS + a, gb = J * TS + b;
        const size_t off = (size_t)ga * np + gb;
        const float Aab = sX1[a * LDX + b], Bab = sX1[a * LDX + TS + b];
        const float Aba = X2[b * LDX + a], Bba = X2[b * LDX + TS + a];
        const float dr = din[off], di = din[plane + off];
        const float hc = 0.5f * (ops.c32[ga] + ops.c32[gb]);
        // kd = f(delta) in FP32; k = F + kd
        float kdr = cm * (Bab + Bba) - om * hc * dr;
        const float kdi = -cm * (Aab - Aba) - om * hc * di;
        if (ga == gb) kdr += om * w.g[ga];
        if (STAGE <= 3) {
            const float kr = kdr + w.F32[off], ki = kdi + w.F32[plane + off];
            if (STAGE == 1) nrm += (double)kr * kr + (double)ki * ki;
            const float Dr = w.D[off], Di = w.D[plane + off];
            float sr, si;
            if (STAGE == 1) { sr = kdr; si = kdi; }
            else { sr = w.S[off] + 2.0f * kdr; si = w.S[plane + off] + 2.0f * kdi; }
            const float cst = (STAGE == 3) ? dtf : 0.5f * dtf;
            const float nr = Dr + cst * kr, ni = Di + cst * ki;
            w.S[off] = sr; w.S[plane + off] = si;
            dnext[off] = nr; dnext[plane + off] = ni;
            sO32[0 * TS * LDO + a * LDO + b] = sr;
            sO32[1 * TS * LDO + a * LDO + b] = si;
            sO32[2 * TS * LDO + a * LDO + b] = nr;
            sO32[3 * TS * LDO + a * LDO + b] = ni;
        } else {
            const double sr = (double)(w.S[off] + kdr), si = (double)(w.S[plane + off] + kdi);
            const double yr = w.y[off] + dt * w.F[off] + (dt / 6.0) * sr;
            const double yi = w.y[plane + off] + dt * w.F[plane + off] + (dt / 6.0) * si;
            const float Dr = (float)(yr - w.R[off]), Di = (float)(yi - w.R[plane + off]);
            w.y[off] = yr; w.y[plane + off] = yi;
            w.D[off] = Dr; w.D[plane + off] = Di;
            sO64[0 * TS * LDO + a * LDO + b] = yr;
            sO64[1 * TS * LDO + a * LDO + b] = yi;
            sO32[0 * TS * LDO + a * LDO + b] = Dr;
            sO32[1 * TS * LDO + a * LDO + b] = Di;
        }
    }
    if (STAGE == 1) {
        nrm = warp_sum_d(nrm);
        if (lane == 0) red[warp] = nrm;
        __syncthreads();
        if (tid == 0) {
            double s = 0.0;
            for (int q = 0; q < NT / 32; ++q) s += red[q];
            w.partials[blockIdx.x] = diag ? s : 2.0 * s;
        }
    }
    if (!diag) {
        __syncthreads();
        for (int e = tid; e < TS * TS; e += NT) {
            const int b = e / TS, a = e - (e / TS) * TS;
            const size_t off = (size_t)(J * TS + b) * np + I * TS + a;
            if (STAGE <= 3) {
                w.S[off] = sO32[0 * TS * LDO + a * LDO + b];
                w.S[plane + off] = -sO32[1 * TS * LDO + a * LDO + b];
                dnext[off] = sO32[2 * TS * LDO + a * LDO + b];
                dnext[plane + off] = -sO32[3 * TS * LDO + a * LDO + b];
            } else {
                w.y[off] = sO64[0 * TS * LDO + a * LDO + b];
                w.y[plane + off] = -sO64[1 * TS * LDO + a * LDO + b];
                w.D[off] = sO32[0 * TS * LDO + a * LDO + b];
                w.D[plane + off] = -sO32[1 * TS * LDO + a * LDO + b];
            }
        }
    }
    if (STAGE == 4 && blockIdx.x == 0 && tid == 0) w.ctl->step += 1;
}

__device__ double block_sum_d(double v, double *red) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    v = warp_sum_d(v);
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    double s = 0.0;
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) s += red[q];
    return s;
}

// g = G p(delta) for an FP32 delta (the gain is linear in p; no trace
// normalisation inside a block of delta steps). Stage 2 first takes the stop
// decision from the stage-1 residual partials (an FP32-accurate estimate of
// ||f(y_n)||_F; a pass is confirmed by an exact FP64 refresh on the host
// side of the loop).
template <int STAGE>
__global__ void __launch_bounds__(256)
gain_mixed_kernel(DevOps ops, MixedWork w, const float *__restrict__ din) {
    __shared__ double red[8];
    __shared__ int s_done;
    Ctl *ctl = w.ctl;
    if (threadIdx.x == 0) s_done = *(volatile int *)&ctl->done;
    __syncthreads();
    if (s_done) return;
    const int n = ops.n, np = ops.np;
    // (a step index whose exact residual the refresh already judged is not
    // judged again on the estimate)
    if (STAGE == 2 && blockIdx.x == 0 && ctl->resid_exact_step != ctl->step) {
        double s = 0.0;
        for (int i = threadIdx.x; i < w.nstage_partials; i += blockDim.x) s += w.partials[i];
        s = block_sum_d(s, red);
        if (threadIdx.x == 0) {
            const double r = sqrt(s);
            ctl->resid = r;
            ctl->resid_step = ctl->step;
            if (!isfinite(r)) {
                ctl->status = kCtlNonFinite;
                ctl->done = 1;
            } else if (r < ctl->tol) {
                ctl->status = kCtlCandidate;
                ctl->done = 1;
            } else if (ctl->step >= ctl->max_steps) {
                ctl->status = kCtlMaxSteps;
                ctl->done = 1;
            }
        }
    }
    double P = 0.0, Dd = 0.0;
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
        const double pj = (double)din[(size_t)j * np + j];
        P += pj;
        if (ops.dang[j]) Dd += pj;
    }
    P = block_sum_d(P, red);
    Dd = block_sum_d(Dd, red);
    const double inv_nm1 = 1.0 / (double)(n - 1);
    const int lane = threadIdx.x & 31, wpb = blockDim.x >> 5;
    for (int i = blockIdx.x * wpb + (threadIdx.x >> 5); i < np; i += gridDim.x * wpb) {
        double s = 0.0;
        if (i < n)
            for (int q = ops.s_ptr[i] + lane; q < ops.s_ptr[i + 1]; q += 32) {
                const int j = ops.s_col[q];
                s += ops.s_val[q] * (double)din[(size_t)j * np + j];
            }
        s = warp_sum_d(s);
        if (lane == 0) {
            double gi = 0.0;
            if (i < n) {
                const double pi = (double)din[(size_t)i * np + i];
                const double dterm = (ops.dangling == QPR_DANGLING_F) ? (Dd - (ops.dang[i] ? pi : 0.0)) * inv_nm1
                                                                       : Dd / (double)n;
                gi = ops.alpha * (s + dterm) + (1.0 - ops.alpha) * (P - pi) * inv_nm1;
            }
            w.g[i] = (float)gi;
        }
    }
}

// Refresh, part 1: sigma = 1 / Re tr(y) (one CTA).
__global__ void __launch_bounds__(256) refresh_trace_kernel(DevOps ops, MixedWork w) {
    __shared__ double red[8];
    __shared__ int s_done;
    if (threadIdx.x == 0) s_done = *(volatile int *)&w.ctl->done;
    __syncthreads();
    if (s_done) return;
    double P = 0.0;
    for (int j = threadIdx.x; j < ops.n; j += blockDim.x) P += w.y[(size_t)j * ops.np + j];
    P = block_sum_d(P, red);
    if (threadIdx.x == 0) {
        w.ctl->trace = P;
        w.ctl->scale = 1.0 / P;
        if (!(P > 0.0) || !isfinite(P)) {
            w.ctl->status = kCtlNonFinite;
            w.ctl->done = 1;
        }
    }
}

// Refresh, part 2: R = y = sigma y, D = 0 (and its BF16 split, dense backend).
__global__ void refresh_normalize_kernel(DevOps ops, MixedWork w) {
    if (*(volatile int *)&w.ctl->done) return;  // set before this kernel started, uniform
    const double sig = w.ctl->scale;
    const size_t tot = 2 * (size_t)ops.np * ops.np;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < tot; i += (size_t)gridDim.x * blockDim.x) {
        const double v = sig * w.y[i];
        w.y[i] = v;
        w.R[i] = v;
        w.D[i] = 0.0f;
    }
    if (w.splitD) {
        const __nv_bfloat16 z = __float2bfloat16_rn(0.0f);
        for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < 3 * tot;
             i += (size_t)gridDim.x * blockDim.x)
            w.splitD[i] = z;
    }
}

// Refresh, part 4 (after F = f(R) in FP64): F32 = F; CTA 0 reduces the exact
// residual ||F||_F and takes the stop decision for this step index.
__global__ void __launch_bounds__(256) refresh_post_kernel(DevOps ops, MixedWork w) {
    __shared__ double red[8];
    __shared__ int s_done;
    Ctl *ctl = w.ctl;
    if (threadIdx.x == 0) s_done = *(volatile int *)&ctl->done;
    __syncthreads();
    if (s_done) return;
    const size_t tot = 2 * (size_t)ops.np * ops.np;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < tot; i += (size_t)gridDim.x * blockDim.x)
        w.F32[i] = (float)w.F[i];
    if (blockIdx.x == 0) {
        double s = 0.0;
        for (int i = threadIdx.x; i < w.npairs; i += blockDim.x) s += w.partials[i];
        s = block_sum_d(s, red);
        if (threadIdx.x == 0) {
            const double r = sqrt(s);
            ctl->resid_exact = r;
            ctl->resid_exact_step = ctl->step;
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
}

int grid_elems(size_t work) {
    size_t b = (work + 255) / 256;
    if (b > 152 * 8) b = 152 * 8;
    return (int)(b < 1 ? 1 : b);
}

}  // namespace

void launch_mixed_refresh(const DevOps &ops, const MixedWork &w, cudaStream_t s) {
    const size_t tot = 2 * (size_t)ops.np * ops.np;
    refresh_trace_kernel<<<1, 256, 0, s>>>(ops, w);
    refresh_normalize_kernel<<<grid_elems(tot), 256, 0, s>>>(ops, w);
    // F = f(R) with the exact FP64 sparse stage kernel (stage 0: reads w.y, writes w.z)
    Work w64{};
    w64.y = w.R;
    w64.z = w.F;
    w64.ya = w.R;
    w64.yb = w.R;
    w64.g = w.g64;
    w64.partials = w.partials;
    w64.pairs = w.pairs;
    w64.npairs = w.npairs;
    w64.tiles = w.tiles;
    w64.ctl = w.ctl;
    launch_gain(0, ops, w.R, w64, s);
    launch_stage_sparse(0, ops, w64, s);
    refresh_post_kernel<<<grid_elems(tot), 256, 0, s>>>(ops, w);
}

void launch_mixed_stage(int stage, const DevOps &ops, const MixedWork &w, cudaStream_t s, int parts) {
    const float *din = (stage == 1) ? w.D : (stage == 3 ? w.db : w.da);
    int gb = (ops.np + 7) / 8;
    if (gb > 152) gb = 152;
    if (parts & 1) {
        switch (stage) {
            case 1: gain_mixed_kernel<1><<<gb, 256, 0, s>>>(ops, w, din); break;
            case 2: gain_mixed_kernel<2><<<gb, 256, 0, s>>>(ops, w, din); break;
            case 3: gain_mixed_kernel<3><<<gb, 256, 0, s>>>(ops, w, din); break;
            default: gain_mixed_kernel<4><<<gb, 256, 0, s>>>(ops, w, din); break;
        }
    }
    if ((parts & 2) && w.splitD) {
        launch_mixed_tc(stage, ops, w, *w.maps, s);
        return;
    }
    if (parts & 2) {
        switch (stage) {
            case 1: stage_mixed_sparse_kernel<1><<<w.npairs, NT, 0, s>>>(ops, w); break;
            case 2: stage_mixed_sparse_kernel<2><<<w.npairs, NT, 0, s>>>(ops, w); break;
            case 3: stage_mixed_sparse_kernel<3><<<w.npairs, NT, 0, s>>>(ops, w); break;
            default: stage_mixed_sparse_kernel<4><<<w.npairs, NT, 0, s>>>(ops, w); break;
        }
    }
}

}  // namespace qpr
