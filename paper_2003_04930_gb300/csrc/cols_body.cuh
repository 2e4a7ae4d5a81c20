// Column-block form of the sparse mixed stage: device functions shared by
// the single-problem kernels (stage_cols.cu) and the batched kernels
// (batch.cu).
//
// A stage is two kernels. The SpMM kernel computes X = H delta one block J
// of kCW complex columns at a time: the CTA stages delta[:, J] for all rows
// (one 128-byte row: 16 real, then 16 imaginary values), its row split's CSR
// entries and its work list in shared memory, then forms X[i, J] =
// sum_q H_iq delta[q, J] with shared-memory reads only. The epilogue kernel
// applies the RK4 stage to every tile pair (I, J), I <= J, from X_IJ and
// X_JI, as the tile-pair form does.
//
// Work list: the rows of a split are cut into bundles of 4 row pieces, one
// per 8-lane group of a warp (lane p of a group holds 4 of the 32 values of
// the row: one 16-byte read per nonzero, a whole row per group and no bank
// conflict); a row longer than kLongRow nonzeros is a bundle of its own,
// its nonzeros dealt to the 4 groups in turn. Bundles go to warps longest
// first, each to the least loaded warp.
#pragma once

#include "mixed_body.cuh"

namespace qpr {
namespace cols {

using mixed::LDO;
using mixed::LDX;
using mixed::NT;
using mixed::TS;

constexpr int kCW = 16;            // complex columns per block
constexpr int kRowFloats = 2 * kCW; // staged row: kCW real, then kCW imaginary values (128 bytes)
constexpr int kBoxRows = 32;       // rows of one TMA box
constexpr int kANT = 512;          // threads of the SpMM kernel
constexpr int kAWarps = kANT / 32;
constexpr int kLongRow = 48;       // longer rows: one bundle, nonzeros dealt to all 4 groups
constexpr int kPieceLong = 1;      // flags bit 0 of piece 0: long-row bundle; flags >> 1: rounds

// Shared memory of the SpMM kernel for np rows, `kh` CSR entries and
// `bundles` bundles (+ 128 bytes of alignment slack).
__host__ __device__ __forceinline__ size_t spmm_smem_bytes(int np, int kh, int bundles) {
    return (size_t)np * kRowFloats * 4 + ((size_t)kh * 8 + 15) / 16 * 16 + (size_t)bundles * 64 + 128;
}

__device__ __forceinline__ float4 f4fma(float h, float4 v, float4 acc) { return mixed::f4fma(h, v, acc); }

// Bundles [b0, b1) of one warp: X[row, J] for each row piece, from the
// staged block sD ([row][kRowFloats]), the staged CSR entries sKH (entry q
// at sKH[q - q_base]) and the staged bundles sP (bundle b at sP[4 (b -
// p_base)]). Sums are formed in a fixed order (per group in entry order,
// then over the groups of a long row by xor-shuffle), so the result does
// not depend on timing.
__device__ __forceinline__ void warp_bundles(const float *__restrict__ sD, const int2 *__restrict__ sKH,
                                             const int4 *__restrict__ sP, int q_base, int p_base, int b0, int b1,
                                             int J, int np, float *__restrict__ X) {
    const int lane = threadIdx.x & 31, g = lane >> 3, p = lane & 7;
    const float *__restrict__ sDp = sD + 4 * p;
    const size_t plane = (size_t)np * np;
    const int col = J * kCW + 4 * (p & 3);
    float *__restrict__ Xp = X + (p < 4 ? 0 : plane) + col;
    for (int b = b0; b < b1; ++b) {
        const int4 pc = sP[4 * (b - p_base) + g];
        const int f0 = sP[4 * (b - p_base)].w;
        float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
        if (f0 & kPieceLong) {
            const int4 p0 = sP[4 * (b - p_base)];
            const int T = f0 >> 1;
#pragma unroll 4
            for (int t = 0; t < T; ++t) {
                const int e = 4 * t + g;
                const bool v = e < p0.z;
                const int2 kh = v ? sKH[p0.y + e - q_base] : make_int2(0, 0);
                const float h = __int_as_float(kh.y);
                acc = f4fma(h, *reinterpret_cast<const float4 *>(sDp + kh.x * kRowFloats), acc);
            }
            acc = mixed::f4xor(acc, 8);
            acc = mixed::f4xor(acc, 16);
            if (g == 0) *reinterpret_cast<float4 *>(Xp + (size_t)p0.x * np) = acc;
        } else {
            const int T = f0 >> 1;  // longest piece of the bundle
#pragma unroll 4
            for (int t = 0; t < T; ++t) {
                const bool v = t < pc.z;
                const int2 kh = v ? sKH[pc.y + t - q_base] : make_int2(0, 0);
                const float h = __int_as_float(kh.y);
                acc = f4fma(h, *reinterpret_cast<const float4 *>(sDp + kh.x * kRowFloats), acc);
            }
            if (pc.x >= 0) *reinterpret_cast<float4 *>(Xp + (size_t)pc.x * np) = acc;
        }
    }
}

// Stage input of stage STAGE: D (stage 1), da (stages 2 and 4), db (stage 3).
template <int STAGE>
__device__ __forceinline__ const float *stage_input(const MixedWork &w) {
    return (STAGE == 1) ? w.D : (STAGE == 3 ? w.db : w.da);
}

// The gain g = G p(delta): CTA b of the nb SpMM CTAs computes rows
// [b np / nb, (b + 1) np / nb), at most a few per warp, while its operands
// are in flight.
__device__ __forceinline__ void cta_gain(const DevOps &ops, const MixedWork &w, const float *din, int b, int nb) {
    const int np = ops.np;
    const int r0 = (int)((long long)b * np / nb), r1 = (int)((long long)(b + 1) * np / nb);
    mixed::gain_rows(ops, din, r0, (int)(blockDim.x >> 5), r1, 0, w.g);
}

// Stop decision after stage 1, taken by the last epilogue CTA to finish
// (a ticket in the control block; release/acquire through fences): it sums
// the nparts residual-estimate partials in index order, records the
// estimate and, when the run stops here, sets done so that the kernels of
// stages 2..4 return at once. A step whose exact residual a refresh already
// judged is not judged again. Called by every thread after tile_epilogue.
__device__ __forceinline__ void stage1_last_decides(const MixedWork &w, int nparts) {
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
    float s = 0.f;
    for (int i = threadIdx.x; i < nparts; i += blockDim.x) s = __fadd_rn(s, __ldcg(w.partials32 + i));
    s = mixed::block_sum_f(s, red);
    if (threadIdx.x == 0) {
        ctl->ticket = 0;
        if (ctl->resid_exact_step != ctl->step) {
            const double r = sqrt((double)s);
            int status = kCtlRunning;
            if (!isfinite(r)) status = kCtlNonFinite;
            else if (r < ctl->tol) status = kCtlCandidate;
            else if (ctl->step >= ctl->max_steps) status = kCtlMaxSteps;
            ctl->resid = r;
            ctl->resid_step = ctl->step;
            if (status != kCtlRunning) {
                ctl->status = status;
                ctl->done = 1;
            }
        }
    }
}

// Epilogue of tile pair (I, J) from X (global, written by the SpMM kernel)
// and the gain w.g; stage 1 ends with the ticket of the stop decision,
// stage 4 advances the step counter (first pair). Shared memory: sX1, sX2
// (TS * LDX floats each), sg (TS), sO (4 * TS * LDO).
template <int STAGE>
__device__ __forceinline__ void epilogue_pair(const DevOps &ops, const MixedWork &w, int I, int J, int pidx,
                                              bool first, int nparts, float *sX1, float *sX2, float *sg, float *sO) {
    const int np = ops.np;
    const size_t plane = (size_t)np * np;
    const bool diag = (I == J);
    const int ntiles = diag ? 1 : 2;
    // X tiles as [a][LDX] rows (real part, then imaginary part), float4 loads
    for (int t = threadIdx.x; t < ntiles * TS * (2 * TS / 4); t += NT) {
        const int which = t / (TS * (2 * TS / 4));
        const int u = t - which * (TS * (2 * TS / 4));
        const int a = u / (2 * TS / 4), q = u - a * (2 * TS / 4);  // q: 0..7 real quads, 8..15 imaginary
        const int R = which ? J : I, C = which ? I : J;
        const size_t o = (size_t)(R * TS + a) * np + C * TS + 4 * (q & 7);
        const float4 v = *reinterpret_cast<const float4 *>(w.X + (q < 8 ? 0 : plane) + o);
        float *dst = (which ? sX2 : sX1) + a * LDX + 4 * q;
        dst[0] = v.x;
        dst[1] = v.y;
        dst[2] = v.z;
        dst[3] = v.w;
    }
    if (diag && threadIdx.x < TS) sg[threadIdx.x] = w.g[I * TS + threadIdx.x];
    __syncthreads();
    mixed::tile_epilogue<STAGE>(ops, w, I, J, pidx, sX1, sX2, sg, sO);
    if (STAGE == 1) stage1_last_decides(w, nparts);
    if (STAGE == 4 && first && threadIdx.x == 0) w.ctl->step += 1;
}

}  // namespace cols
}  // namespace qpr
