// Device functions of the mixed-precision form (sparse backend and the
// refresh), shared by the single-problem kernels and the batched kernels.
#pragma once

#include <math.h>

#include "qpr_internal.cuh"

namespace qpr {
namespace mixed {

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

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ float warp_sum_f(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = __fadd_rn(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// Sum over the CTA in a fixed order (the same bits in every CTA and run).
__device__ __forceinline__ float block_sum_f(float v, float *red) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    v = warp_sum_f(v);
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    float s = 0.f;
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) s = __fadd_rn(s, red[q]);
    return s;
}

// Float-float arithmetic: a value is hi + lo with |lo| <= ulp(hi) / 2, about
// 48 significant bits, carried by FP32 instructions only (the FP64 pipe of
// this part runs at 1/64 of the FP32 rate). ff_add is Knuth's TwoSum of the
// high parts with the low parts added to its error, then Dekker's
// FastTwoSum to renormalise; ff_mul_f multiplies by an FP32 factor with the
// FMA form of TwoProduct. Explicit round-to-nearest intrinsics: no
// contraction may change these error-free transformations.
struct ff {
    float hi, lo;
};
__device__ __forceinline__ ff ff_add(float ah, float al, float bh, float bl) {
    const float s = __fadd_rn(ah, bh);
    const float v = __fsub_rn(s, ah);
    float e = __fadd_rn(__fsub_rn(ah, __fsub_rn(s, v)), __fsub_rn(bh, v));
    e = __fadd_rn(e, __fadd_rn(al, bl));
    const float h = __fadd_rn(s, e);
    return {h, __fsub_rn(e, __fsub_rn(h, s))};
}
__device__ __forceinline__ ff ff_mul_f(float ah, float al, float b) {
    const float p = __fmul_rn(ah, b);
    const float e = __fmaf_rn(al, b, __fmaf_rn(ah, b, -p));
    const float h = __fadd_rn(p, e);
    return {h, __fsub_rn(e, __fsub_rn(h, p))};
}

// Delta update of stage 4 for one real component: delta + dt F + c s4 in
// float-float, with dt F = (gh, gl) and the step weight c = (ch, cl) (dt in
// the nested RK4 form).
__device__ __forceinline__ ff delta_update(float dh, float dl, float gh, float gl, float ch, float cl, float s4) {
    const ff u = ff_mul_f(ch, cl, s4);
    const ff t = ff_add(u.hi, u.lo, gh, gl);
    return ff_add(dh, dl, t.hi, t.lo);
}

__device__ __forceinline__ double block_sum_d(double v, double *red) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    v = warp_sum_d(v);
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    double s = 0.0;
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) s += red[q];
    return s;
}

constexpr int kSegSlots = 96;      // segment partials held at once (24 KB)
constexpr int kSegLen = 32;        // nonzeros per segment (one warp-wide load)

// The gathers of one segment (len <= kSegLen nonzeros; lane e < len holds
// column myk and value myh of nonzero e): 8-lane group grp takes nonzeros
// grp, grp + 4, ..., each lane a float4 of the real and of the imaginary row
// slice, and returns its partial sums (before the sum over the groups).
// Batches of 16 nonzeros, branch-free inside a batch: slots past len load
// the segment's first row with weight 0, so that the 8 loads of a batch are
// all issued before its first FMA (one L2 round trip per batch, 32
// registers of loads in flight).
__device__ __forceinline__ void gather_segment(const float *__restrict__ re, const float *__restrict__ im, int np,
                                               int myk, float myh, int len, int grp, float4 &xr, float4 &xi) {
    constexpr int R = 4;  // rounds of 4 nonzeros per batch
    const int k0 = __shfl_sync(0xffffffffu, myk, 0);
    for (int e0 = 0; e0 < len; e0 += 4 * R) {  // warp-uniform
        float4 vr[R], vi[R];
#pragma unroll
        for (int it = 0; it < R; ++it) {
            const int e = e0 + it * 4 + grp;
            int k = __shfl_sync(0xffffffffu, myk, e & 31);
            k = (e < len) ? k : k0;
            vr[it] = *reinterpret_cast<const float4 *>(re + (size_t)k * np);
            vi[it] = *reinterpret_cast<const float4 *>(im + (size_t)k * np);
        }
#pragma unroll
        for (int it = 0; it < R; ++it) {
            const int e = e0 + it * 4 + grp;
            float h = __shfl_sync(0xffffffffu, myh, e & 31);
            h = (e < len) ? h : 0.f;
            xr = f4fma(h, vr[it], xr);
            xi = f4fma(h, vi[it], xi);
        }
    }
}

// sX[a][b] = (H Re d)_ab, sX[a][TS + b] = (H Im d)_ab for rows of tile rt and
// columns of tile ct, in FP32. The nonzeros of every row are cut into
// segments of at most kSegLen (ops.seg, rows' ranges in ops.rowseg); warps
// take segments round-robin, so a hub row no longer holds one warp while
// the others wait. A warp loads a segment's columns and values with one
// coalesced load, broadcasts them by shuffle and keeps all of the
// segment's 2 x 8 float4 gathers in flight; segment partials go to shared
// memory and are summed per row in segment order (deterministic).
// slots: kSegSlots * 2 * TS floats of shared memory, free during the call.
__device__ __forceinline__ void spmm32_tile(const DevOps &ops, const float *__restrict__ d, size_t plane,
                                            int rt, int ct, float *sX, float *slots) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int grp = lane >> 3, sub = lane & 7;
    const int np = ops.np;
    const float *__restrict__ re = d + ct * TS + 4 * sub;
    const float *__restrict__ im = d + plane + ct * TS + 4 * sub;
    const int s0 = ops.rowseg[rt * TS], s1 = ops.rowseg[rt * TS + TS];
    int base = s0;
    do {
        const int cnt = min(kSegSlots, s1 - base);
        for (int si = warp; si < cnt; si += NT / 32) {
            const int2 sg = ops.seg[base + si];
            const int len = sg.y - sg.x;
            int myk = 0;
            float myh = 0.f;
            if (lane < len) {
                myk = ops.h_col[sg.x + lane];
                myh = ops.h_val32[sg.x + lane];
            }
            float4 xr = make_float4(0.f, 0.f, 0.f, 0.f), xi = xr;
            gather_segment(re, im, np, myk, myh, len, grp, xr, xi);
            xr = f4xor(xr, 8);
            xr = f4xor(xr, 16);
            xi = f4xor(xi, 8);
            xi = f4xor(xi, 16);
            if (grp == 0) {
                float4 *slot = reinterpret_cast<float4 *>(slots + si * 2 * TS);
                slot[sub] = xr;
                slot[TS / 4 + sub] = xi;
            }
        }
        __syncthreads();
        // per row: sum its segments of this round in order (rows without
        // nonzeros, and padding rows, get zeros)
        for (int t = threadIdx.x; t < TS * 2 * TS; t += NT) {
            const int a = t / (2 * TS), c = t - a * (2 * TS);
            const int ga = rt * TS + a;
            const int r0 = max(ops.rowseg[ga], base), r1 = min(ops.rowseg[ga + 1], base + cnt);
            float acc = (base == s0) ? 0.f : sX[a * LDX + c];
            for (int q = r0; q < r1; ++q) acc = __fadd_rn(acc, slots[(q - base) * 2 * TS + c]);
            sX[a * LDX + c] = acc;
        }
        __syncthreads();
        base += cnt;
    } while (base < s1);
}

constexpr int kStageEntries = 3072;  // staged CSR entries of the two row tiles (24 KB)
// Dynamic shared memory of the sparse mixed stage: segment slots, staged
// segment headers, staged columns and values; the epilogue's output stash
// (16.9 KB) reuses the same bytes afterwards.
constexpr int kMixedDynSmem = kSegSlots * 2 * TS * 4 + kSegSlots * 8 + kStageEntries * 8;
static_assert(kMixedDynSmem >= 4 * TS * LDO * 4, "output stash fits the dynamic buffer");

// Both products of a tile pair, X_IJ (rows of I, columns of J, into sX1)
// and, unless I == J, X_JI (into sX2). When the segments of both row tiles
// fit the slots and their CSR entries fit the staging buffer, the segment
// headers, columns and values are first copied to shared memory with
// coalesced loads, so that each segment costs one round of gathers from
// L2; otherwise one tile after the other without staging. The sums per row
// are formed exactly as in spmm32_tile (segment order), so the result does
// not depend on the path taken.
__device__ __forceinline__ void spmm32_pair(const DevOps &ops, const float *__restrict__ d, size_t plane, int I,
                                            int J, bool diag, float *sX1, float *sX2, uint8_t *dyn) {
    float *slots = reinterpret_cast<float *>(dyn);
    int2 *hdr = reinterpret_cast<int2 *>(dyn + kSegSlots * 2 * TS * 4);
    int *scol = reinterpret_cast<int *>(hdr + kSegSlots);
    float *sval = reinterpret_cast<float *>(scol + kStageEntries);
    const int sI0 = ops.rowseg[I * TS], sI1 = ops.rowseg[I * TS + TS];
    const int sJ0 = diag ? 0 : ops.rowseg[J * TS], sJ1 = diag ? 0 : ops.rowseg[J * TS + TS];
    const int cI = sI1 - sI0, cJ = sJ1 - sJ0;
    const int qI0 = cI ? ops.seg[sI0].x : 0, qI1 = cI ? ops.seg[sI1 - 1].y : 0;
    const int qJ0 = cJ ? ops.seg[sJ0].x : 0, qJ1 = cJ ? ops.seg[sJ1 - 1].y : 0;
    const int lenI = qI1 - qI0, lenJ = qJ1 - qJ0;
    if (cI + cJ > kSegSlots || lenI + lenJ > kStageEntries) {
        spmm32_tile(ops, d, plane, I, J, sX1, slots);
        if (!diag) spmm32_tile(ops, d, plane, J, I, sX2, slots);
        return;
    }
    for (int t = threadIdx.x; t < cI + cJ; t += NT) {
        const bool ti = t < cI;
        const int2 sg = ops.seg[ti ? sI0 + t : sJ0 + (t - cI)];
        const int base = ti ? -qI0 : lenI - qJ0;
        hdr[t] = make_int2(sg.x + base, sg.y + base);
    }
    for (int t = threadIdx.x; t < lenI + lenJ; t += NT) {
        const int q = t < lenI ? qI0 + t : qJ0 + (t - lenI);
        scol[t] = ops.h_col[q];
        sval[t] = ops.h_val32[q];
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int grp = lane >> 3, sub = lane & 7;
    const int np = ops.np;
    for (int si = warp; si < cI + cJ; si += NT / 32) {
        const int ct = si < cI ? J : I;
        const float *__restrict__ re = d + ct * TS + 4 * sub;
        const float *__restrict__ im = d + plane + ct * TS + 4 * sub;
        const int2 sg = hdr[si];
        const int len = sg.y - sg.x;
        int myk = 0;
        float myh = 0.f;
        if (lane < len) {
            myk = scol[sg.x + lane];
            myh = sval[sg.x + lane];
        }
        float4 xr = make_float4(0.f, 0.f, 0.f, 0.f), xi = xr;
        gather_segment(re, im, np, myk, myh, len, grp, xr, xi);
        xr = f4xor(xr, 8);
        xr = f4xor(xr, 16);
        xi = f4xor(xi, 8);
        xi = f4xor(xi, 16);
        if (grp == 0) {
            float4 *slot = reinterpret_cast<float4 *>(slots + si * 2 * TS);
            slot[sub] = xr;
            slot[TS / 4 + sub] = xi;
        }
    }
    __syncthreads();
    const int ntiles = diag ? 1 : 2;
    for (int t = threadIdx.x; t < ntiles * TS * 2 * TS; t += NT) {
        const int which = t / (TS * 2 * TS);  // 0: rows of I into sX1, 1: rows of J into sX2
        const int u = t - which * (TS * 2 * TS);
        const int a = u / (2 * TS), c = u - a * (2 * TS);
        const int ga = (which ? J : I) * TS + a;
        const int off = which ? cI - sJ0 : -sI0;  // slot index = segment index + off
        float acc = 0.f;
        for (int q = ops.rowseg[ga]; q < ops.rowseg[ga + 1]; ++q) acc = __fadd_rn(acc, slots[(q + off) * 2 * TS + c]);
        (which ? sX2 : sX1)[a * LDX + c] = acc;
    }
    __syncthreads();
}

// g = G p(delta) for an FP32 delta (the gain is linear in p; there is no
// trace normalisation inside a block of delta steps) for rows
// r_begin, r_begin + r_step, ... < r_end (one warp per row), written to
// out[i - out_base]. Every CTA computes the trace and dangling mass itself.
// FP32 throughout, in a fixed order.
__device__ __forceinline__ void gain_rows(const DevOps &ops, const float *__restrict__ din, int r_begin, int r_step,
                                          int r_end, int out_base, float *out) {
    __shared__ float red[32];
    const int n = ops.n, np = ops.np;
    float P = 0.f, Dd = 0.f;
    // __ldcg: the diagonal may have been written by another CTA of the same
    // (persistent) launch, so it is read from L2
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
        const float pj = __ldcg(din + (size_t)j * np + j);
        P = __fadd_rn(P, pj);
        if (ops.dang[j]) Dd = __fadd_rn(Dd, pj);
    }
    P = block_sum_f(P, red);
    Dd = block_sum_f(Dd, red);
    const int lane = threadIdx.x & 31;
    for (int i = r_begin + (threadIdx.x >> 5); i < r_end; i += r_step) {
        float s = 0.f;
        if (i < n) {
            const int q1 = ops.s_ptr[i + 1];
#pragma unroll 4
            for (int q = ops.s_ptr[i] + lane; q < q1; q += 32) {
                const int j = ops.s_col[q];
                s = __fmaf_rn(ops.s_val32[q], __ldcg(din + (size_t)j * np + j), s);
            }
        }
        s = warp_sum_f(s);
        if (lane == 0) {
            float gi = 0.f;
            if (i < n) {
                const float pi = __ldcg(din + (size_t)i * np + i);
                const float dterm = (ops.dangling == QPR_DANGLING_F)
                                        ? __fmul_rn(__fsub_rn(Dd, ops.dang[i] ? pi : 0.f), ops.inv_nm1_32)
                                        : __fmul_rn(Dd, ops.inv_n32);
                gi = __fmaf_rn(ops.alpha32, __fadd_rn(s, dterm),
                               __fmul_rn(__fmul_rn(ops.oma32, __fsub_rn(P, pi)), ops.inv_nm1_32));
            }
            out[i - out_base] = gi;
        }
    }
}

// Stop decision of stage 2 from the stage-1 residual partials (an
// FP32-accurate estimate of ||f(y_n)||_F; a pass is confirmed by an exact
// FP64 refresh on the host side of the loop). Every CTA sums the partials in
// the same order and reaches the same decision; the one with `first`
// records it. A step index whose exact residual a refresh already decided is
// not decided again. Returns true when the run stops (uniform over the CTA).
__device__ __forceinline__ bool stage2_decide(const MixedWork &w, bool first) {
    __shared__ float red[32];
    __shared__ int s_status;
    Ctl *ctl = w.ctl;
    if (ctl->resid_exact_step == ctl->step) return false;
    float s = 0.f;
    for (int i = threadIdx.x; i < w.nstage_partials; i += blockDim.x) s = __fadd_rn(s, w.partials32[i]);
    s = block_sum_f(s, red);
    if (threadIdx.x == 0) {
        const double r = sqrt((double)s);  // one thread: the FP64 here is negligible
        int status = kCtlRunning;
        if (!isfinite(r)) status = kCtlNonFinite;
        else if (r < ctl->tol) status = kCtlCandidate;
        else if (ctl->step >= ctl->max_steps) status = kCtlMaxSteps;
        s_status = status;
        if (first) {
            ctl->resid = r;
            ctl->resid_step = ctl->step;
            if (status != kCtlRunning) {
                ctl->status = status;
                ctl->done = 1;
            }
        }
    }
    __syncthreads();
    return s_status != kCtlRunning;
}

// f(delta)_ab of the Lindblad right-hand side (Eq. 1) in FP32 from the
// products X = H delta at (a, b) (Aab + i Bab) and at (b, a) (Aba + i Bba),
// the element delta_ab = dr + i di, the column sums c_a and c_b of G and, on
// the diagonal, the gain g_a = (G p(delta))_a:
//   (1 - omega)[(Bab + Bba) - i (Aab - Aba)] + omega[delta_ab g_a - (c_a + c_b)/2 delta_ab].
// Explicit round-to-nearest intrinsics: the same rounding in every kernel
// inlining this code.
__device__ __forceinline__ void lindblad_elem(float om, float cm, float ca, float cb, float Aab, float Bab, float Aba,
                                              float Bba, float dr, float di, bool on_diag, float ga, float &kdr,
                                              float &kdi) {
    const float omhc = __fmul_rn(om, __fmul_rn(0.5f, __fadd_rn(ca, cb)));
    kdr = __fmaf_rn(-omhc, dr, __fmul_rn(cm, __fadd_rn(Bab, Bba)));
    kdi = __fmaf_rn(-omhc, di, __fmul_rn(-cm, __fsub_rn(Aab, Aba)));
    if (on_diag) kdr = __fmaf_rn(om, ga, kdr);
}

// The RK4 step in nested form. f is linear, so the classical step
// y + dt/6 (k1 + 2 k2 + 2 k3 + k4) equals
//     y + dt L (y + dt/2 L (y + dt/3 L (y + dt/4 L y)))
// (the same polynomial I + dt L + ... + (dt L)^4 / 24 of dt L). Stage s
// evaluates k = L w_s = F + f(delta_s) of its input w_s = R + delta_s
// (delta_1 = D) and writes the next input delta_{s+1} = D + c_s dt k with
// c = 1/4, 1/3, 1/2; stage 4 adds dt k to the state: D + Dlo += dt F +
// dt f(delta_4) in float-float (dt F = Ghi + Glo). No running sum of the
// stages is kept, so a stage reads the product, its input, F32 and D and
// writes one plane pair (stage 4: D and Dlo).
//
// Operands of one thread's elements e = tid + k NTH (k < K) of tile (I, J)
// of stage STAGE, loaded into registers ahead of the products (one round
// trip to memory for the whole epilogue): the stage input d; stages 1-3:
// F32 (u) and, at stages 2-3, D (v; at stage 1 the input is D); stage 4: D
// (v), Dlo (s), Ghi (g), Glo (l); and c32 of the element's row (ca) and
// column (cb).
template <int STAGE, int NTH>
struct EpiIn {
    static constexpr int K = TS * TS / NTH;
    float dr[K], di[K], ur[K], ui[K], vr[K], vi[K], sr[K], si[K], gr[K], gi[K], lr[K], li[K], ca[K];
    float cb;
};

template <int STAGE, int NTH>
__device__ __forceinline__ void epi_load(const DevOps &ops, const MixedWork &w, int I, int J, EpiIn<STAGE, NTH> &in) {
    const int np = ops.np;
    const size_t plane = (size_t)np * np;
    const float *__restrict__ din = (STAGE == 1) ? w.D : (STAGE == 3 ? w.db : w.da);
    const int tid = threadIdx.x;
    // from L2: another CTA (or SM) of an earlier kernel wrote these, and the
    // caller may read them before its grid dependency wait
#pragma unroll
    for (int k = 0; k < EpiIn<STAGE, NTH>::K; ++k) {
        const int e = tid + k * NTH;
        const int a = e / TS, b = e - (e / TS) * TS;
        const size_t off = (size_t)(I * TS + a) * np + J * TS + b;
        in.dr[k] = __ldcg(din + off);
        in.di[k] = __ldcg(din + plane + off);
        if (STAGE <= 3) {
            in.ur[k] = __ldcg(w.F32 + off);
            in.ui[k] = __ldcg(w.F32 + plane + off);
            if (STAGE >= 2) {
                in.vr[k] = __ldcg(w.D + off);
                in.vi[k] = __ldcg(w.D + plane + off);
            }
        } else {
            in.vr[k] = __ldcg(w.D + off);
            in.vi[k] = __ldcg(w.D + plane + off);
            in.sr[k] = __ldcg(w.Dlo + off);
            in.si[k] = __ldcg(w.Dlo + plane + off);
            in.gr[k] = __ldcg(w.Ghi + off);
            in.gi[k] = __ldcg(w.Ghi + plane + off);
            in.lr[k] = __ldcg(w.Glo + off);
            in.li[k] = __ldcg(w.Glo + plane + off);
        }
        in.ca[k] = ops.c32[I * TS + a];
    }
    in.cb = ops.c32[J * TS + (tid % TS)];  // the column of every element of this thread
}

// Epilogue of one tile pair (I, J) of stage STAGE from the products
// sX1 = X_IJ and (unless I == J) sX2 = X_JI of X = H delta, [a][LDX] rows
// (real part, then imaginary part), and, on a diagonal pair, the gain of
// its rows in sg, with the operands `in` loaded by epi_load. Writes tile
// (I, J) and its conjugate mirror (J, I); stage 1 leaves this pair's
// residual-estimate partial in partials32[pidx]. sO32: 4 * TS * LDO floats
// of shared memory; NTH threads. Ends with a barrier.
template <int STAGE, int NTH>
__device__ __forceinline__ void tile_epilogue_in(const DevOps &ops, const MixedWork &w, int I, int J, int pidx,
                                                 const float *sX1, const float *sX2, const float *sg, float *sO32,
                                                 const EpiIn<STAGE, NTH> &in) {
    __shared__ float red[NTH / 32];
    const bool diag = (I == J);
    const int np = ops.np;
    const size_t plane = (size_t)np * np;
    float *dnext = (STAGE == 2) ? w.db : w.da;
    const float *X2 = diag ? sX1 : sX2;

    const float om = ops.omega32, cm = __fsub_rn(1.0f, om);
    const float dtf = w.ctl->dtf;
    // c_s dt of the next stage input (dt / 4 and dt / 2 exact from fl(dt); fl(dt / 3))
    const float cst = (STAGE == 1) ? __fmul_rn(0.25f, dtf) : (STAGE == 2 ? w.ctl->dt3 : __fmul_rn(0.5f, dtf));
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    float nrm = 0.f;  // this thread's share of ||k1||^2 (an FP32-accurate estimate)
#pragma unroll
    for (int k = 0; k < EpiIn<STAGE, NTH>::K; ++k) {
        const int e = tid + k * NTH;
        const int a = e / TS, b = e - (e / TS) * TS;
        const int ga = I * TS + a, gb = J * TS + b;
        const size_t off = (size_t)ga * np + gb;
        const float Aab = sX1[a * LDX + b], Bab = sX1[a * LDX + TS + b];
        const float Aba = X2[b * LDX + a], Bba = X2[b * LDX + TS + a];
        const float dr = in.dr[k], di = in.di[k];
        // kd = f(delta) in FP32; k = F + kd
        float kdr, kdi;
        lindblad_elem(om, cm, in.ca[k], in.cb, Aab, Bab, Aba, Bba, dr, di, ga == gb, ga == gb ? sg[a] : 0.f, kdr,
                      kdi);
        if (STAGE <= 3) {
            const float kr = __fadd_rn(kdr, in.ur[k]), ki = __fadd_rn(kdi, in.ui[k]);
            if (STAGE == 1) nrm = __fmaf_rn(kr, kr, __fmaf_rn(ki, ki, nrm));
            const float Dr = (STAGE == 1) ? dr : in.vr[k], Di = (STAGE == 1) ? di : in.vi[k];
            const float nr = __fmaf_rn(cst, kr, Dr), ni = __fmaf_rn(cst, ki, Di);
            dnext[off] = nr; dnext[plane + off] = ni;
            if (ga == gb && w.pv) w.pv[ga] = nr;
            sO32[0 * TS * LDO + a * LDO + b] = nr;
            sO32[1 * TS * LDO + a * LDO + b] = ni;
        } else {
            // delta += dt F + dt f(delta_4) in float-float
            const ff vr = delta_update(in.vr[k], in.sr[k], in.gr[k], in.lr[k], dtf, w.ctl->dtl, kdr);
            const ff vi = delta_update(in.vi[k], in.si[k], in.gi[k], in.li[k], dtf, w.ctl->dtl, kdi);
            w.D[off] = vr.hi; w.D[plane + off] = vi.hi;
            w.Dlo[off] = vr.lo; w.Dlo[plane + off] = vi.lo;
            if (ga == gb && w.pv) w.pv[ga] = vr.hi;
            sO32[0 * TS * LDO + a * LDO + b] = vr.hi;
            sO32[1 * TS * LDO + a * LDO + b] = vi.hi;
            sO32[2 * TS * LDO + a * LDO + b] = vr.lo;
            sO32[3 * TS * LDO + a * LDO + b] = vi.lo;
        }
    }
    if (STAGE == 1) {
        const float nrm_w = warp_sum_f(nrm);
        if (lane == 0) red[warp] = nrm_w;
        __syncthreads();
        if (tid == 0) {
            float s = 0.f;
            for (int q = 0; q < NTH / 32; ++q) s = __fadd_rn(s, red[q]);
            w.partials32[pidx] = diag ? s : __fmul_rn(2.0f, s);
        }
    }
    if (!diag) {
        __syncthreads();
        for (int e = tid; e < TS * TS; e += NTH) {
            const int b = e / TS, a = e - (e / TS) * TS;
            const size_t off = (size_t)(J * TS + b) * np + I * TS + a;
            if (STAGE <= 3) {
                dnext[off] = sO32[0 * TS * LDO + a * LDO + b];
                dnext[plane + off] = -sO32[1 * TS * LDO + a * LDO + b];
            } else {
                w.D[off] = sO32[0 * TS * LDO + a * LDO + b];
                w.D[plane + off] = -sO32[1 * TS * LDO + a * LDO + b];
                w.Dlo[off] = sO32[2 * TS * LDO + a * LDO + b];
                w.Dlo[plane + off] = -sO32[3 * TS * LDO + a * LDO + b];
            }
        }
    }
    __syncthreads();
}

// The same with the operands loaded here.
template <int STAGE, int NTH = NT>
__device__ __forceinline__ void tile_epilogue(const DevOps &ops, const MixedWork &w, int I, int J, int pidx,
                                              const float *sX1, const float *sX2, const float *sg, float *sO32) {
    EpiIn<STAGE, NTH> in;
    epi_load<STAGE, NTH>(ops, w, I, J, in);
    tile_epilogue_in<STAGE, NTH>(ops, w, I, J, pidx, sX1, sX2, sg, sO32, in);
}

// One tile pair (I, J) of stage STAGE of the sparse mixed form: products
// from the segments of H gathered from L2, the gain on a diagonal pair, the
// epilogue. pidx is the slot of its residual partial, first marks the pair
// that advances the step counter. dyn: kMixedDynSmem bytes of dynamic shared
// memory (16-byte aligned). Ends with a barrier so that the caller may
// reuse shared memory.
template <int STAGE>
__device__ __forceinline__ void mixed_sparse_tile(const DevOps &ops, const MixedWork &w, int I, int J, int pidx,
                                                  bool first, uint8_t *dyn) {
    __shared__ __align__(16) float sX1[TS * LDX];
    __shared__ __align__(16) float sX2[TS * LDX];
    __shared__ float sg[TS];
    const bool diag = (I == J);
    if (STAGE == 2 && stage2_decide(w, first)) return;
    const int np = ops.np;
    const size_t plane = (size_t)np * np;
    const float *__restrict__ din = (STAGE == 1) ? w.D : (STAGE == 3 ? w.db : w.da);
    spmm32_pair(ops, din, plane, I, J, diag, sX1, sX2, dyn);
    // only diagonal tiles add the gain g = G p(delta); they compute it for
    // their own rows
    if (diag) {
        gain_rows(ops, din, I * TS, NT / 32, I * TS + TS, I * TS, sg);
        __syncthreads();
    }
    // the output stash reuses the dynamic buffer (free after the products)
    tile_epilogue<STAGE>(ops, w, I, J, pidx, sX1, sX2, sg, reinterpret_cast<float *>(dyn));
    if (STAGE == 4 && first && threadIdx.x == 0) w.ctl->step += 1;
    __syncthreads();
}


// The gain kernel of the dense (tensor-core) stage: stage 2 also takes the
// stop decision (CTA blk 0).
template <int STAGE>
__device__ __forceinline__ void gain_mixed_body(const DevOps &ops, const MixedWork &w, const float *__restrict__ din,
                                                int blk, int nblk) {
    if (STAGE == 2) stage2_decide(w, blk == 0);
    const int wpb = blockDim.x >> 5;
    gain_rows(ops, din, blk * wpb, nblk * wpb, ops.np, 0, w.g);
}

// Refresh, part 1 (one CTA): sigma = 1 / Re tr(y) for y = R + delta, in
// FP64, and the FP32 forms of dt that the delta stages use.
__device__ __forceinline__ double state_value(const MixedWork &w, size_t i) {
    // (double)hi + (double)lo is exact: the pair spans at most 48 bits
    return w.R[i] + ((double)w.D[i] + (double)w.Dlo[i]);
}

__device__ __forceinline__ void refresh_trace_body(const DevOps &ops, const MixedWork &w) {
    __shared__ double red[32];
    double P = 0.0;
    for (int j = threadIdx.x; j < ops.n; j += blockDim.x) P += state_value(w, (size_t)j * ops.np + j);
    P = block_sum_d(P, red);
    if (threadIdx.x == 0) {
        Ctl *ctl = w.ctl;
        ctl->trace = P;
        ctl->scale = 1.0 / P;
        if (!(P > 0.0) || !isfinite(P)) {
            ctl->status = kCtlNonFinite;
            ctl->done = 1;
        }
        ctl->dtf = (float)ctl->dt;
        ctl->dtl = (float)(ctl->dt - (double)ctl->dtf);
        ctl->dt3 = (float)(ctl->dt / 3.0);
    }
}

// Refresh, part 2: R = sigma (R + delta), delta = 0 (and the BF16 split of
// D, dense backend); elements i0, i0 + stride, ...
__device__ __forceinline__ void refresh_normalize_body(const DevOps &ops, const MixedWork &w, size_t i0,
                                                       size_t stride) {
    const double sig = w.ctl->scale;
    const size_t tot = 2 * (size_t)ops.np * ops.np;
    for (size_t i = i0; i < tot; i += stride) {
        w.R[i] = sig * state_value(w, i);
        w.D[i] = 0.0f;
        w.Dlo[i] = 0.0f;
    }
    if (w.pv)
        for (size_t i = i0; i < (size_t)ops.np; i += stride) w.pv[i] = 0.0f;
    if (w.splitD) {
        const __nv_bfloat16 z = __float2bfloat16_rn(0.0f);
        for (size_t i = i0; i < 3 * tot; i += stride) w.splitD[i] = z;
    }
}

// Refresh, part 4 (after F = f(R) in FP64): F32 = fl(F) and dt F as the
// float-float pair (Ghi, Glo); the CTA with first set reduces the exact
// residual ||F||_F and takes the stop decision.
__device__ __forceinline__ void refresh_post_body(const DevOps &ops, const MixedWork &w, size_t i0, size_t stride,
                                                  bool first) {
    __shared__ double red[32];
    Ctl *ctl = w.ctl;
    const size_t tot = 2 * (size_t)ops.np * ops.np;
    const double dt = ctl->dt;
    for (size_t i = i0; i < tot; i += stride) {
        const double f = w.F[i];
        const double g = dt * f;
        const float gh = (float)g;
        w.F32[i] = (float)f;
        w.Ghi[i] = gh;
        w.Glo[i] = (float)(g - (double)gh);
    }
    if (first) {
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

}  // namespace mixed
}  // namespace qpr
