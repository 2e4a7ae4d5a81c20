// Adaptive RKF45 (Supplementary Note 2, Eq. S10 - S13) in the mixed
// column-block form.
//
// f is linear and does not depend on t, so one RKF45 attempt of step h is a
// polynomial in z = h L applied to the state y: the fourth-order solution of
// Eq. S11 is P4(z) y and the fifth-order solution of Eq. S12 is P5(z) y, with
//     P4(z) = 1 + z + z^2/2 + z^3/6 + z^4/24 + z^5/104,
//     P5(z) = 1 + z + z^2/2 + z^3/6 + z^4/24 + z^5/120 + z^6/2080
// (the stage coefficients of Eq. S10 with the two 4101 denominators read as
// 4104 multiply out to these; the CPU oracle takes the six stages literally
// and the tests hold both to the same results). So an attempt evaluates the
// powers u_k = z^k y, k = 1..6, one stage each:
//     y_{k+1} = y + sum_{k<=5} pi_k u_k,   pi = 1, 1/2, 1/6, 1/24, 1/104,
//     z_{k+1} - y_{k+1} = -u_5/780 + u_6/2080,
// and the discrepancy |z - y| (the largest modulus over the entries) never
// needs z itself: no cancellation between two nearly equal solutions.
//
// Delta form, as in the RK4 mixed form: y = R + D with R and F = f(R) exact
// in FP64 from the last refresh and D a float-float pair. Stage 1 evaluates
// f(y) = F + f(D): its norm is the residual estimate, u_1 = h f(y) its next
// input, and the running sum starts as acc = h f(D) (the h F part of u_1 is
// added at the end in float-float from F = F32 + Flo). Stages 2-5 evaluate
// u_k = h f(u_{k-1}) in FP32 and add pi_k u_k to acc; stage 6 evaluates u_6,
// the discrepancy, and the candidate D' = D + h F + acc in float-float, into
// the other delta pair (or D + h F + acc + (z - y), the fifth-order z of
// Eq. S12, when the caller chose the note's alternative). The last CTA of
// stage 6 takes the controller's decision (one thread, FP64): accept when
// |z - y| <= Tol h (then the other pair becomes the state), s = (Tol h / (2 |z - y|))^(1/4) clipped to
// [1/10, 4], next h = min(s h, h_max) (shortened to end a trajectory at its
// end time). Every stage is an SpMM launch (whose leading CTAs form the gain)
// and an epilogue launch, exactly as an RK4 stage of the column-block form.
#include <math.h>

#include "cols_body.cuh"
#include "cols_spmm.cuh"
#include "mixed_body.cuh"
#include "qpr_internal.cuh"
#include "tma_util.cuh"

namespace qpr {
namespace {

using namespace cols;
using mixed::ff;
using mixed::ff_add;
using mixed::ff_mul_f;

// Weight of u_k in y_{k+1} (the coefficients of P4), k = 1..5, and of u_5,
// u_6 in z_{k+1} - y_{k+1}.
__device__ __forceinline__ float rkf_pi(int k) {
    return k == 1 ? 1.0f : k == 2 ? 0.5f : k == 3 ? (1.0f / 6.0f) : k == 4 ? (1.0f / 24.0f) : (1.0f / 104.0f);
}
constexpr float kE5 = -1.0f / 780.0f;
constexpr float kE6 = 1.0f / 2080.0f;

// Stage inputs: stage 1 the current delta (D or D1), then the powers
// alternate between da (u_1, u_3, u_5) and db (u_2, u_4).
template <int S>
__device__ __forceinline__ const float *rkf_input(const MixedWork &w, int cur) {
    return S == 1 ? (cur ? w.D1 : w.D) : ((S & 1) ? w.db : w.da);
}
template <int S>
__device__ __forceinline__ float *rkf_output(const MixedWork &w) {
    return (S & 1) ? w.da : w.db;
}

__device__ __forceinline__ int read_cur(const MixedWork &w) { return *(volatile int *)&w.ctl->rk_cur; }

// The SpMM kernels of stage S: the leading ops.col_gain_ctas CTAs form the
// gain of the stage input (stage 1 from the compact diagonal of the current
// delta, later stages from the one the previous epilogue wrote), the others
// one product unit each, as in the RK4 kernels.
template <int S>
__device__ __forceinline__ const float *rkf_pv(const DevOps &ops, const MixedWork &w) {
    return (S == 1) ? w.pvd + (size_t)read_cur(w) * ops.np : w.pv;
}

template <int S>
__global__ void __launch_bounds__(kANT) rkf_spmm_kernel(const __grid_constant__ CUtensorMap tm_d0,
                                                        const __grid_constant__ CUtensorMap tm_d1,
                                                        const __grid_constant__ CUtensorMap tm_a,
                                                        const __grid_constant__ CUtensorMap tm_b, DevOps ops,
                                                        MixedWork w) {
    const int b = blockIdx.x, ng = ops.col_gain_ctas;
    if (b < ng) {
        gain_role<S == 2>(ops, w, b, ng, [&] { return rkf_pv<S>(ops, w); });
        return;
    }
    const int u = b - ng, ncb = ops.np / kCW;
    spmm_block_body(
        [&]() -> const CUtensorMap * {
            if (S == 1) return read_cur(w) ? &tm_d1 : &tm_d0;
            return (S & 1) ? &tm_b : &tm_a;
        },
        ops, w, u % ncb, u / ncb);
}

template <int S>
__global__ void __launch_bounds__(kANT, kGatherCtasPerSm) rkf_gather_kernel(DevOps ops, MixedWork w) {
    const int b = blockIdx.x, ng = ops.col_gain_ctas;
    if (b < ng) {
        gain_role<S == 2>(ops, w, b, ng, [&] { return rkf_pv<S>(ops, w); });
        return;
    }
    const int u = b - ng;
    spmm_gather_body([&] { return rkf_input<S>(w, S == 1 ? read_cur(w) : 0); }, ops, w, u % ops.col_splits,
                     u / ops.col_splits);
}

// Operands of one thread's elements e = tid + k kENT of tile (I, J).
template <int S>
struct RkfIn {
    static constexpr int K = TS * TS / kENT;
    float dr[K], di[K];  // the stage input
    float ur[K], ui[K];  // stage 1, 6: F32
    float ar[K], ai[K];  // stages 2-6: acc
    float vr[K], vi[K], sr[K], si[K];  // stage 6: D, Dlo of the current pair
    float lr[K], li[K];  // stage 6: Flo
    float ca[K];
    float cb;
};

template <int S>
__device__ __forceinline__ void rkf_load(const DevOps &ops, const MixedWork &w, int I, int J, int cur,
                                         RkfIn<S> &in) {
    const int np = ops.np;
    const size_t plane = (size_t)np * np;
    const float *__restrict__ din = rkf_input<S>(w, cur);
    const float *__restrict__ Dc = cur ? w.D1 : w.D;
    const float *__restrict__ Lc = cur ? w.Dlo1 : w.Dlo;
    const int tid = threadIdx.x;
#pragma unroll
    for (int k = 0; k < RkfIn<S>::K; ++k) {
        const int e = tid + k * kENT;
        const int a = e / TS, b = e - (e / TS) * TS;
        const size_t off = (size_t)(I * TS + a) * np + J * TS + b;
        in.dr[k] = __ldcg(din + off);
        in.di[k] = __ldcg(din + plane + off);
        if (S == 1 || S == 6) {
            in.ur[k] = __ldcg(w.F32 + off);
            in.ui[k] = __ldcg(w.F32 + plane + off);
        }
        if (S >= 2) {
            in.ar[k] = __ldcg(w.acc + off);
            in.ai[k] = __ldcg(w.acc + plane + off);
        }
        if (S == 6) {
            in.vr[k] = __ldcg(Dc + off);
            in.vi[k] = __ldcg(Dc + plane + off);
            in.sr[k] = __ldcg(Lc + off);
            in.si[k] = __ldcg(Lc + plane + off);
            in.lr[k] = __ldcg(w.Flo + off);
            in.li[k] = __ldcg(w.Flo + plane + off);
        }
        in.ca[k] = ops.c32[I * TS + a];
    }
    in.cb = ops.c32[J * TS + (tid % TS)];
}

// h F in float-float from F = fh + fl and h = hh + hl (the product of the
// high parts exactly by FMA, the cross terms in FP32), then added to the
// float-float delta (dh, dl) and to the FP32 sum a.
__device__ __forceinline__ ff candidate(float dh, float dl, float fh, float fl, float hh, float hl, float a) {
    const float p = __fmul_rn(fh, hh);
    const float e = __fmaf_rn(fh, hh, -p);
    const float c = __fmaf_rn(fh, hl, __fmul_rn(fl, hh));
    const float q = __fadd_rn(e, c);
    const ff hf = {__fadd_rn(p, q), __fsub_rn(q, __fsub_rn(__fadd_rn(p, q), p))};
    const ff t = ff_add(dh, dl, hf.hi, hf.lo);
    return ff_add(t.hi, t.lo, a, 0.0f);
}

// Largest value over the CTA (every thread receives it); NaN propagates.
__device__ __forceinline__ float block_max(float v, float *red) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float u = __shfl_xor_sync(0xffffffffu, v, o);
        v = (u > v || isnan(u)) ? u : v;
    }
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    float m = red[0];
    for (int q = 1; q < (int)(blockDim.x >> 5); ++q) m = (red[q] > m || isnan(red[q])) ? red[q] : m;
    return m;
}

// The controller (Eq. S13), taken by the last CTA of the stage-6 epilogue
// (a ticket in the control block) from the tiles' discrepancy partials.
__device__ __forceinline__ void rkf_decide(const MixedWork &w, int nparts) {
    __shared__ int s_last;
    __shared__ float red[32];
    Ctl *ctl = w.ctl;
    if (threadIdx.x == 0) {
        __threadfence();
        s_last = (atomicAdd(&ctl->ticket, 1) == nparts - 1);
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    float m = 0.0f;
    for (int i = threadIdx.x; i < nparts; i += blockDim.x) {
        const float v = __ldcg(w.partials32 + i);
        m = (v > m || isnan(v)) ? v : m;
    }
    m = block_max(m, red);
    if (threadIdx.x != 0) return;
    ctl->ticket = 0;
    const double err = (double)m;
    const double h = ctl->rk_h;
    ctl->rk_err = err;
    if (!isfinite(err)) {
        ctl->status = kCtlNonFinite;
        ctl->done = 1;
        return;
    }
    const double tol = ctl->rk_tol;
    const bool ok = err <= tol * h;
    double s = err > 0.0 ? pow(tol * h / (2.0 * err), 0.25) : 4.0;
    s = fmin(fmax(s, 0.1), 4.0);
    if (ok) {
        ctl->rk_cur ^= 1;
        ctl->step += 1;
        ctl->rk_t += h;
    } else {
        ctl->rk_rejected += 1;
    }
    double hn = fmin(s * h, ctl->rk_hmax);
    if (ctl->rk_tend > 0.0) {
        const double rem = ctl->rk_tend - ctl->rk_t;
        if (rem <= 1e-15 * ctl->rk_tend) {
            ctl->rk_t = ctl->rk_tend;
            ctl->status = kCtlTimeReached;
            ctl->done = 1;
        } else {
            hn = fmin(hn, rem);
        }
    }
    ctl->rk_h = hn;
    ctl->rk_hf = (float)hn;
    ctl->rk_hl = (float)(hn - (double)(float)hn);
}

// Epilogue of stage S for tile pair (I, J), I <= J: X tiles and the gain
// from L2 (the SpMM and the gain kernels wrote them), the operands loaded
// before the grid dependency wait (written two or more kernels back).
// Writes tile (I, J) and its conjugate mirror (J, I) of the outputs:
// stages 1-5 u_S and acc, stage 6 the candidate delta pair.
template <int S>
__global__ void __launch_bounds__(kENT, 3) rkf_epi_kernel(DevOps ops, MixedWork w) {
    __shared__ __align__(16) float sX1[TS * LDX];
    __shared__ __align__(16) float sX2[TS * LDX];
    __shared__ __align__(16) float sO[4 * TS * LDO];
    __shared__ float sg[TS];
    __shared__ float red[kENT / 32];
    __shared__ int s_done;
    const int4 pr = w.epi_pairs[blockIdx.x];  // {I, J, partial slot}: the column forms' epilogue order
    const int I = pr.x, J = pr.y;
    const int cur = read_cur(w);
    RkfIn<S> in;
    rkf_load<S>(ops, w, I, J, cur, in);
    tma::grid_dependency_wait();
    tma::launch_dependents();
    const int np = ops.np;
    const size_t plane = (size_t)np * np;
    const bool diag = (I == J);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    // the stop flag and the X tiles in one round trip (X is read whatever the
    // flag says; nothing is written unless the run goes on)
    const int done = (tid == 0) ? *(volatile int *)&w.ctl->done : 0;
    // X tiles as [a][LDX] rows (real part, then imaginary part)
    for (int t = tid; t < (diag ? 1 : 2) * TS * (2 * TS / 4); t += kENT) {
        const int which = t / (TS * (2 * TS / 4));
        const int u = t - which * (TS * (2 * TS / 4));
        const int a = u / (2 * TS / 4), q = u - a * (2 * TS / 4);
        const int R = which ? J : I, C = which ? I : J;
        const size_t o = (size_t)(R * TS + a) * np + C * TS + 4 * (q & 7);
        const float4 v = __ldcg(reinterpret_cast<const float4 *>(w.X + (q < 8 ? 0 : plane) + o));
        float *dst = (which ? sX2 : sX1) + a * LDX + 4 * q;
        dst[0] = v.x;
        dst[1] = v.y;
        dst[2] = v.z;
        dst[3] = v.w;
    }
    if (diag && tid < TS) sg[tid] = __ldcg(w.g + I * TS + tid);
    if (tid == 0) s_done = done;
    __syncthreads();
    if (s_done) return;
    const float *X2 = diag ? sX1 : sX2;
    const float om = ops.omega32, cm = __fsub_rn(1.0f, om);
    const float hh = w.ctl->rk_hf, hl = w.ctl->rk_hl;
    const bool fifth = (S == 6) && w.ctl->rk_order == 5;
    float *out = (S <= 5) ? rkf_output<S>(w) : nullptr;
    float *Dn = cur ? w.D : w.D1;  // stage 6: the other pair
    float *Ln = cur ? w.Dlo : w.Dlo1;
    float nrm = 0.f, emax = 0.f;
#pragma unroll
    for (int k = 0; k < RkfIn<S>::K; ++k) {
        const int e = tid + k * kENT;
        const int a = e / TS, b = e - (e / TS) * TS;
        const int ga = I * TS + a, gb = J * TS + b;
        const size_t off = (size_t)ga * np + gb;
        float kdr, kdi;
        mixed::lindblad_elem(om, cm, in.ca[k], in.cb, sX1[a * LDX + b], sX1[a * LDX + TS + b], X2[b * LDX + a],
                             X2[b * LDX + TS + a], in.dr[k], in.di[k], ga == gb, ga == gb ? sg[a] : 0.f, kdr, kdi);
        float o0, o1, o2, o3;  // outputs of this element (mirrored below)
        if (S == 1) {
            // f(y) = F + f(D): the residual estimate; u_1 = h f(y); acc = h f(D)
            const float kr = __fadd_rn(in.ur[k], kdr), ki = __fadd_rn(in.ui[k], kdi);
            nrm = __fmaf_rn(kr, kr, __fmaf_rn(ki, ki, nrm));
            o0 = __fmul_rn(hh, kr);
            o1 = __fmul_rn(hh, ki);
            o2 = __fmul_rn(hh, kdr);
            o3 = __fmul_rn(hh, kdi);
        } else if (S <= 5) {
            // u_S = h f(u_{S-1}); acc += pi_S u_S
            o0 = __fmul_rn(hh, kdr);
            o1 = __fmul_rn(hh, kdi);
            o2 = __fmaf_rn(rkf_pi(S), o0, in.ar[k]);
            o3 = __fmaf_rn(rkf_pi(S), o1, in.ai[k]);
        } else {
            // u_6 = h f(u_5); z - y = e5 u_5 + e6 u_6; D' = D + h F + acc
            const float u6r = __fmul_rn(hh, kdr), u6i = __fmul_rn(hh, kdi);
            const float er = __fmaf_rn(kE6, u6r, __fmul_rn(kE5, in.dr[k]));
            const float ei = __fmaf_rn(kE6, u6i, __fmul_rn(kE5, in.di[k]));
            const float em = sqrtf(__fmaf_rn(er, er, __fmul_rn(ei, ei)));
            emax = (em > emax || isnan(em)) ? em : emax;
            // fourth order: D + h F + acc; fifth order: z = y + (z - y)
            const float ar = fifth ? __fadd_rn(in.ar[k], er) : in.ar[k];
            const float ai = fifth ? __fadd_rn(in.ai[k], ei) : in.ai[k];
            const ff nr = candidate(in.vr[k], in.sr[k], in.ur[k], in.lr[k], hh, hl, ar);
            const ff ni = candidate(in.vi[k], in.si[k], in.ui[k], in.li[k], hh, hl, ai);
            o0 = nr.hi;
            o1 = ni.hi;
            o2 = nr.lo;
            o3 = ni.lo;
        }
        if (S <= 5) {
            out[off] = o0;
            out[plane + off] = o1;
            w.acc[off] = o2;
            w.acc[plane + off] = o3;
            if (ga == gb) w.pv[ga] = o0;
        } else {
            Dn[off] = o0;
            Dn[plane + off] = o1;
            Ln[off] = o2;
            Ln[plane + off] = o3;
            if (ga == gb) w.pvd[(size_t)(cur ^ 1) * np + ga] = o0;
        }
        sO[0 * TS * LDO + a * LDO + b] = o0;
        sO[1 * TS * LDO + a * LDO + b] = o1;
        sO[2 * TS * LDO + a * LDO + b] = o2;
        sO[3 * TS * LDO + a * LDO + b] = o3;
    }
    if (S == 1 || S == 6) {
        // this tile pair's partial: the sum of |f(y)|^2 (stage 1, both tiles of
        // an off-diagonal pair) or the largest |z - y| (stage 6)
        float v = (S == 1) ? mixed::warp_sum_f(nrm) : emax;
        if (S == 6) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const float u = __shfl_xor_sync(0xffffffffu, v, o);
                v = (u > v || isnan(u)) ? u : v;
            }
        }
        if (lane == 0) red[warp] = v;
        __syncthreads();
        if (tid == 0) {
            float acc = red[0];
            for (int q = 1; q < kENT / 32; ++q)
                acc = (S == 1) ? __fadd_rn(acc, red[q]) : ((red[q] > acc || isnan(red[q])) ? red[q] : acc);
            w.partials32[pr.z] = (S == 1 && !diag) ? __fmul_rn(2.0f, acc) : acc;
        }
    }
    if (!diag) {
        __syncthreads();
        float *m0 = (S <= 5) ? out : Dn;
        float *m1 = (S <= 5) ? w.acc : Ln;
        for (int e = tid; e < TS * TS; e += kENT) {
            const int b = e / TS, a = e - (e / TS) * TS;
            const size_t off = (size_t)(J * TS + b) * np + I * TS + a;
            m0[off] = sO[0 * TS * LDO + a * LDO + b];
            m0[plane + off] = -sO[1 * TS * LDO + a * LDO + b];
            m1[off] = sO[2 * TS * LDO + a * LDO + b];
            m1[plane + off] = -sO[3 * TS * LDO + a * LDO + b];
        }
    }
    __syncthreads();
    // (the stop decision of stage 1 is taken by the stage-2 SpMM grid, gain_role)
    if (S == 6) rkf_decide(w, w.npairs);
}

// ---- refresh: y = R + D (current pair) folded into R, F = f(R) exactly ----
__device__ __forceinline__ double rkf_state(const MixedWork &w, int cur, size_t i) {
    const float *D = cur ? w.D1 : w.D;
    const float *L = cur ? w.Dlo1 : w.Dlo;
    return w.R[i] + ((double)D[i] + (double)L[i]);
}

__global__ void __launch_bounds__(256) rkf_refresh_trace_kernel(DevOps ops, MixedWork w) {
    __shared__ double red[32];
    if (*(volatile int *)&w.ctl->done) return;  // uniform: set before this kernel started
    const int cur = read_cur(w);
    double P = 0.0;
    for (int j = threadIdx.x; j < ops.n; j += blockDim.x) P += rkf_state(w, cur, (size_t)j * ops.np + j);
    P = mixed::block_sum_d(P, red);
    if (threadIdx.x == 0) {
        Ctl *ctl = w.ctl;
        ctl->trace = P;
        ctl->scale = 1.0 / P;
        if (!(P > 0.0) || !isfinite(P)) {
            ctl->status = kCtlNonFinite;
            ctl->done = 1;
        }
    }
}

// R = sigma (R + delta), both delta pairs and their diagonals zeroed.
__global__ void rkf_refresh_normalize_kernel(DevOps ops, MixedWork w) {
    if (*(volatile int *)&w.ctl->done) return;
    const int cur = read_cur(w);
    const double sig = w.ctl->scale;
    const size_t tot = 2 * (size_t)ops.np * ops.np;
    const size_t i0 = blockIdx.x * (size_t)blockDim.x + threadIdx.x, stride = (size_t)gridDim.x * blockDim.x;
    for (size_t i = i0; i < tot; i += stride) {
        w.R[i] = sig * rkf_state(w, cur, i);
        w.D[i] = 0.0f;
        w.Dlo[i] = 0.0f;
        w.D1[i] = 0.0f;
        w.Dlo1[i] = 0.0f;
    }
    for (size_t i = i0; i < 2 * (size_t)ops.np; i += stride) w.pvd[i] = 0.0f;
}

// F32 = fl(F), Flo = fl(F - F32); the exact residual ||F||_F and the stop
// decision (CTA 0).
__global__ void __launch_bounds__(256) rkf_refresh_post_kernel(DevOps ops, MixedWork w) {
    __shared__ double red[32];
    __shared__ int s_done;
    if (threadIdx.x == 0) s_done = *(volatile int *)&w.ctl->done;
    __syncthreads();
    if (s_done) return;
    const size_t tot = 2 * (size_t)ops.np * ops.np;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < tot; i += (size_t)gridDim.x * blockDim.x) {
        const double f = w.F[i];
        const float fh = (float)f;
        w.F32[i] = fh;
        w.Flo[i] = (float)(f - (double)fh);
    }
    if (blockIdx.x == 0) {
        Ctl *ctl = w.ctl;
        double s = 0.0;
        for (int i = threadIdx.x; i < w.npairs; i += blockDim.x) s += w.partials[i];
        s = mixed::block_sum_d(s, red);
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

int elems_grid(size_t work) {
    size_t b = (work + 255) / 256;
    if (b > 152 * 8) b = 152 * 8;
    return (int)(b < 1 ? 1 : b);
}

template <typename K, typename... A>
void launch_ex(K kernel, dim3 grid, dim3 block, size_t smem, cudaStream_t s, A... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    cudaLaunchKernelEx(&cfg, kernel, args...);
}

template <int S>
void stage_s(const DevOps &ops, const MixedWork &w, cudaStream_t s) {
    const ColMaps &m = *w.cmaps;
    const size_t sm = (size_t)ops.col_launch_smem;
    if (ops.col_gather) {
        const dim3 ga(ops.col_gain_ctas + ops.col_splits * (ops.np / kCWWide));
        launch_ex(rkf_gather_kernel<S>, ga, dim3(kANT), sm, s, ops, w);
    } else {
        const dim3 ga(ops.col_gain_ctas + (ops.np / kCW) * ops.col_splits);
        launch_ex(rkf_spmm_kernel<S>, ga, dim3(kANT), sm, s, m.d[0], m.d1, m.d[1], m.d[2], ops, w);
    }
    launch_ex(rkf_epi_kernel<S>, dim3(w.npairs), dim3(kENT), 0, s, ops, w);
}

template <int S>
cudaError_t set_rkf_smem(int bytes, bool gather) {
    if (gather) return raise_smem_limit_t(rkf_gather_kernel<S>, bytes);
    return raise_smem_limit_t(rkf_spmm_kernel<S>, bytes);
}

}  // namespace

cudaError_t init_rkf(int spmm_smem, bool gather) {
    cudaError_t e = set_rkf_smem<1>(spmm_smem, gather);
    if (e == cudaSuccess) e = set_rkf_smem<2>(spmm_smem, gather);
    if (e == cudaSuccess) e = set_rkf_smem<3>(spmm_smem, gather);
    if (e == cudaSuccess) e = set_rkf_smem<4>(spmm_smem, gather);
    if (e == cudaSuccess) e = set_rkf_smem<5>(spmm_smem, gather);
    if (e == cudaSuccess) e = set_rkf_smem<6>(spmm_smem, gather);
    return e;
}

bool make_rkf_map(const DevOps &ops, const float *d1, ColMaps *maps) {
    PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
    if (!enc) return false;
    const cuuint64_t np = (cuuint64_t)ops.np;
    cuuint64_t dims[3] = {np, 2, np};
    cuuint64_t strides[2] = {np * np * sizeof(float), np * sizeof(float)};
    cuuint32_t box[3] = {kCW, 2, kBoxRows};
    cuuint32_t es[3] = {1, 1, 1};
    return enc(&maps->d1, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, (void *)d1, dims, strides, box, es,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

void launch_rkf_stage(int stage, const DevOps &ops, const MixedWork &w, cudaStream_t s) {
    switch (stage) {
        case 1: stage_s<1>(ops, w, s); break;
        case 2: stage_s<2>(ops, w, s); break;
        case 3: stage_s<3>(ops, w, s); break;
        case 4: stage_s<4>(ops, w, s); break;
        case 5: stage_s<5>(ops, w, s); break;
        default: stage_s<6>(ops, w, s); break;
    }
}

void launch_rkf_refresh(const DevOps &ops, const MixedWork &w, cudaStream_t s) {
    const size_t tot = 2 * (size_t)ops.np * ops.np;
    rkf_refresh_trace_kernel<<<1, 256, 0, s>>>(ops, w);
    rkf_refresh_normalize_kernel<<<elems_grid(tot), 256, 0, s>>>(ops, w);
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
    rkf_refresh_post_kernel<<<elems_grid(tot), 256, 0, s>>>(ops, w);
}

}  // namespace qpr
