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
// Work list: the rows of a split are cut into bundles handled by one warp.
// Whole-block (narrow) layout: a bundle is 8 rows of similar length, one
// per lane quad, or one row longer than kLongRow nonzeros whose nonzeros
// are dealt to the 8 quads. Lane l of a quad holds 8 of the 32 values of a
// staged row (two 16-byte chunks), the two quads of a quarter-warp reading
// complementary halves of their rows so that their 8 lanes hit 8 distinct
// bank quads whatever rows they read. A bundle's CSR entries are stored
// interleaved and zero-padded to its T rounds (round t, quad q at 8 t + q),
// so each round's 8 entries are 64 contiguous bytes (one 8-byte read per
// lane: 2 wavefronts for 8 nonzeros, against 4 when 8 lanes share a row and
// read its entry together). Gather (wide) layout: a pair of 8-lane groups
// per row (one per plane of a 32-column block), kRPG rows per pair and
// round (entries at 4 t + kRPG h + s). Bundles go to warps longest first,
// each to the least loaded warp.
#pragma once

#include "mixed_body.cuh"

namespace qpr {
namespace cols {

using mixed::LDO;
using mixed::LDX;
using mixed::NT;
using mixed::TS;

constexpr int kCW = 16;            // complex columns per block
constexpr int kCWWide = 32;        // complex columns per block of the gather form (one 128-byte line per plane)
constexpr int kRowFloats = 2 * kCW; // staged row: kCW real, then kCW imaginary values (128 bytes)
static_assert(kCW == kColWidth && kCWWide == kColGatherWidth, "host and device block widths agree");
constexpr int kBoxRows = 32;       // rows of one TMA box
constexpr int kANT = 512;          // threads of the SpMM kernel
constexpr int kAWarps = kANT / 32;   // (32 warps measured slower)
// Gather form (measured sweeps: 2 CTAs per SM with 8 rounds of loads in
// flight beat 3 CTAs per SM with 4 or fewer by 10-30%)
constexpr int kGatherCtasPerSm = 2;   // resident CTAs per SM the gather form's plan sizes for
constexpr int kGatherUnroll = 8;      // rounds whose row loads the gather form issues together
constexpr int kGatherWaves = 3;       // waves of CTAs the gather form's plan asks for at least
constexpr int kGatherSplitBytes = 56 << 10;  // largest staged entries + bundles of one gather split
constexpr int kLongRow = 48;       // longer rows: one bundle, nonzeros dealt to all 4 groups
constexpr int kENT = 512;          // threads of the epilogue (2 elements of a tile pair each; 256 measured slower)
constexpr int kPieceLong = 1;      // bundle flags: long-row bundle
constexpr int kPiecePart = 2;      // bundle flags: one part of a cut row (its sum goes to a partial slot)
// For np above kColMaxNp (the gather form, many row splits, when its grid
// has fewer than kCutMaxWaves waves), rows
// longer than kPartMax nonzeros are cut into parts of at most kPartMax,
// each a long-row bundle of its own (possibly on another warp) whose sum goes
// to a partial slot in shared memory; after all warps, the parts of a row are
// added in part order (combine_cuts). A long row's bundle is otherwise one
// warp's work, which made the warp holding a hub row of a heavy-tailed graph
// the critical path of its CTA (N = 2048: 79 -> 67 us per gather launch).
// With the few splits of smaller problems a hub row is about one warp's
// share and cutting measured slower, so those plans cut nothing and every
// form there sums each row the same way.
constexpr int kPartMax = 256;
constexpr int kCutMaxWaves = 12;
constexpr int kRPG = 2;            // gather layout: rows (slots) per group pair and round
constexpr int kNarrowRows = 8;     // whole-block layout: rows per round (one per lane quad)
constexpr int kNarrowUnroll = 4;   // whole-block layout: rounds whose shared-memory reads are issued together

// A bundle descriptor is 3 int4: {first entry (relative to its split's
// entries, even), rounds T, flags, 0} and its row slots rows[0..7] (int4
// 1 + j / 4, component j % 4; -1: none; a long-row bundle has only
// rows[0]). Slot s of group g is rows[g + groups s]: rows[quad] in the
// whole-block layout, rows[h + 2 s] (pair h) in the gather layout.
constexpr int kBundleInt4 = 3;

__device__ __forceinline__ float4 f4fma(float h, float4 v, float4 acc) { return mixed::f4fma(h, v, acc); }
__device__ __forceinline__ float4 f4add(float4 a, float4 b) {
    return make_float4(__fadd_rn(a.x, b.x), __fadd_rn(a.y, b.y), __fadd_rn(a.z, b.z), __fadd_rn(a.w, b.w));
}
__device__ __forceinline__ int pick(int4 v, int g) { return (g == 0) ? v.x : (g == 1) ? v.y : (g == 2) ? v.z : v.w; }

// Bundles [b0, b1) of one warp in the gather layout: X[row, J] for each
// row, from the split's staged entries sKH and bundles sP (bundle b at
// sP[kBundleInt4 (b - p_base)]). Sums are formed in a fixed order (per row
// in entry order; for a long row per group kRPG interleaved sums added in
// slot order, then over the group pairs by xor-shuffle), so the result does
// not depend on timing.
//
// sD is the stage input in global memory (two np x np planes); row q's 32
// values per plane of block J are read there with L1-cached loads (hub
// rows, referenced by many rows of a split, hit L1). The input was written
// by the previous kernel; every load is issued after griddepcontrol.wait,
// which makes that kernel's writes visible, and no kernel reads the stage
// inputs through L1 before it.
template <bool GMEM = true, bool WIDE = true>
__device__ __forceinline__ void wide_bundles(const float *__restrict__ sD, const int2 *__restrict__ sKH,
                                             const int4 *__restrict__ sP, int p_base, int b0, int b1, int J, int np,
                                             float *__restrict__ X, float *parts) {
    static_assert(WIDE && GMEM, "the wide layout is the gather form's");
    const int lane = threadIdx.x & 31, g = lane >> 3, p = lane & 7;
    const size_t plane = (size_t)np * np;
    // narrow: group g = one row, lanes 0-3 real and 4-7 imaginary values of
    // 16 columns; wide: group pair h = one row, group 2h + pl its plane pl,
    // 32 columns (one 128-byte line per plane)
    const int h = WIDE ? (g >> 1) : g;
    const int pl = WIDE ? (g & 1) : (p < 4 ? 0 : 1);
    const int col = WIDE ? J * kCWWide + 4 * p : J * kCW + 4 * (p & 3);
    const float *__restrict__ sDp = GMEM ? sD + pl * plane + col : sD + 4 * p;
    auto row_of = [&](int q) {
        if (GMEM) return __ldca(reinterpret_cast<const float4 *>(sDp + (size_t)q * np));
        return *reinterpret_cast<const float4 *>(sDp + q * kRowFloats);
    };
    float *__restrict__ Xp = X + pl * plane + col;
    auto put = [&](int row, float4 v) { *reinterpret_cast<float4 *>(Xp + (size_t)row * np) = v; };
    // int4 entries per round: kRPG / 2 per group (narrow) or group pair (wide)
    constexpr int RS = (WIDE ? 2 : 4) * (kRPG / 2);
    constexpr int RowF = WIDE ? 2 * kRowFloats : kRowFloats;  // floats of a partial row
    const int part_off = WIDE ? pl * kRowFloats + 4 * p : 4 * p;
    for (int b = b0; b < b1; ++b) {
        const int4 *bd = sP + kBundleInt4 * (b - p_base);
        const int4 d0 = bd[0];
        const int4 *__restrict__ kh = reinterpret_cast<const int4 *>(sKH + d0.x) + h * (kRPG / 2);
        const int T = d0.y;
        float4 acc[kRPG];
#pragma unroll
        for (int s = 0; s < kRPG; ++s) acc[s] = make_float4(0.f, 0.f, 0.f, 0.f);
        // (the same pipelining of the shared-memory loads measured no faster)
        constexpr int U = GMEM ? kGatherUnroll : 0;
        // a row load; from global memory, padding entries (value 0) load nothing
        auto fetch = [&](int q, int hbits) {
            if (GMEM && hbits == 0) return make_float4(0.f, 0.f, 0.f, 0.f);
            return row_of(q);
        };
        if (U > 0) {
            // U rounds at a time: their entries, then all their row loads,
            // then the FMAs in round order (the same sums as one round at a
            // time)
            int t = 0;
            for (; t + U <= T; t += U) {
                int4 e[U > 0 ? U : 1][kRPG / 2];
                float4 v[U > 0 ? U : 1][kRPG];
#pragma unroll
                for (int u = 0; u < U; ++u)
#pragma unroll
                    for (int s2 = 0; s2 < kRPG / 2; ++s2) e[u][s2] = kh[RS * (t + u) + s2];
#pragma unroll
                for (int u = 0; u < U; ++u)
#pragma unroll
                    for (int s2 = 0; s2 < kRPG / 2; ++s2) {
                        v[u][2 * s2] = fetch(e[u][s2].x, e[u][s2].y);
                        v[u][2 * s2 + 1] = fetch(e[u][s2].z, e[u][s2].w);
                    }
#pragma unroll
                for (int u = 0; u < U; ++u)
#pragma unroll
                    for (int s2 = 0; s2 < kRPG / 2; ++s2) {
                        acc[2 * s2] = f4fma(__int_as_float(e[u][s2].y), v[u][2 * s2], acc[2 * s2]);
                        acc[2 * s2 + 1] = f4fma(__int_as_float(e[u][s2].w), v[u][2 * s2 + 1], acc[2 * s2 + 1]);
                    }
            }
            for (; t < T; ++t) {
#pragma unroll
                for (int s2 = 0; s2 < kRPG / 2; ++s2) {
                    const int4 e = kh[RS * t + s2];
                    const float4 v0 = fetch(e.x, e.y), v1 = fetch(e.z, e.w);
                    acc[2 * s2] = f4fma(__int_as_float(e.y), v0, acc[2 * s2]);
                    acc[2 * s2 + 1] = f4fma(__int_as_float(e.w), v1, acc[2 * s2 + 1]);
                }
            }
        } else {
#pragma unroll 2
            for (int t = 0; t < T; ++t) {
#pragma unroll
                for (int s2 = 0; s2 < kRPG / 2; ++s2) {
                    const int4 e = kh[RS * t + s2];
                    acc[2 * s2] = f4fma(__int_as_float(e.y), row_of(e.x), acc[2 * s2]);
                    acc[2 * s2 + 1] = f4fma(__int_as_float(e.w), row_of(e.z), acc[2 * s2 + 1]);
                }
            }
        }
        if (d0.z & kPieceLong) {
            float4 a = acc[0];
#pragma unroll
            for (int s = 1; s < kRPG; ++s) a = f4add(a, acc[s]);
            if (!WIDE) a = mixed::f4xor(a, 8);
            a = mixed::f4xor(a, 16);
            if (h == 0) {
                if (d0.z & kPiecePart)
                    *reinterpret_cast<float4 *>(parts + bd[1].x * RowF + part_off) = a;
                else
                    put(bd[1].x, a);
            }
        } else {
#pragma unroll
            for (int s = 0; s < kRPG; ++s) {
                const int row = pick(bd[1], h + 2 * s);
                if (row >= 0) put(row, acc[s]);
            }
        }
    }
}

// Bundles [b0, b1) of one warp in the whole-block layout: X[row, J] for
// each row from the staged block sD ([row][kRowFloats]), the split's staged
// entries sKH and bundles sP. Each row's sum runs over its entries in CSR
// order (one FMA chain per column); a long row's 8 partial sums are added
// by an xor butterfly over the quads. The result does not depend on timing.
template <int UNROLL>
__device__ __forceinline__ void narrow_bundles(const float *__restrict__ sD, const int2 *__restrict__ sKH,
                                               const int4 *__restrict__ sP, int p_base, int b0, int b1, int J,
                                               int np, float *__restrict__ X, float *parts) {
    const int lane = threadIdx.x & 31, quad = lane >> 2, l = lane & 3, par = quad & 1;
    const size_t plane = (size_t)np * np;
    // lane l of a quad holds chunks 2l and 2l + 1 (16 bytes each) of a staged
    // row; read i takes chunk 2l + (i ^ par), so the two quads of a
    // quarter-warp read complementary halves of their rows (no bank conflict)
    const int c0 = 2 * l + par, c1 = 2 * l + (1 - par);
    const int o0 = 4 * c0, o1 = 4 * c1;
    float *__restrict__ X0 = X + (c0 < 4 ? 0 : plane) + J * kCW + 4 * (c0 & 3);
    float *__restrict__ X1 = X + (c1 < 4 ? 0 : plane) + J * kCW + 4 * (c1 & 3);
    for (int b = b0; b < b1; ++b) {
        const int4 *bd = sP + kBundleInt4 * (b - p_base);
        const int4 d0 = bd[0];
        const int2 *__restrict__ kh = sKH + d0.x + quad;
        const int T = d0.y;
        float4 a0 = make_float4(0.f, 0.f, 0.f, 0.f), a1 = a0;
        int t = 0;
        // UNROLL rounds at a time: their entries, then their row reads, then
        // the FMAs in round order (the same sums as one round at a time)
        for (; UNROLL > 1 && t + UNROLL <= T; t += UNROLL) {
            int2 e[UNROLL];
            float4 v0[UNROLL], v1[UNROLL];
#pragma unroll
            for (int u = 0; u < UNROLL; ++u) e[u] = kh[kNarrowRows * (t + u)];
#pragma unroll
            for (int u = 0; u < UNROLL; ++u) {
                const float *__restrict__ row = sD + e[u].x * kRowFloats;
                v0[u] = *reinterpret_cast<const float4 *>(row + o0);
                v1[u] = *reinterpret_cast<const float4 *>(row + o1);
            }
#pragma unroll
            for (int u = 0; u < UNROLL; ++u) {
                a0 = f4fma(__int_as_float(e[u].y), v0[u], a0);
                a1 = f4fma(__int_as_float(e[u].y), v1[u], a1);
            }
        }
#pragma unroll 1
        for (; t < T; ++t) {
            const int2 e = kh[kNarrowRows * t];
            const float hv = __int_as_float(e.y);
            const float *__restrict__ row = sD + e.x * kRowFloats;
            a0 = f4fma(hv, *reinterpret_cast<const float4 *>(row + o0), a0);
            a1 = f4fma(hv, *reinterpret_cast<const float4 *>(row + o1), a1);
        }
        if (d0.z & kPieceLong) {
            // chunks 2l and 2l + 1, then the sum over the 8 quads
            float4 u0 = par ? a1 : a0, u1 = par ? a0 : a1;
            u0 = mixed::f4xor(mixed::f4xor(mixed::f4xor(u0, 4), 8), 16);
            u1 = mixed::f4xor(mixed::f4xor(mixed::f4xor(u1, 4), 8), 16);
            if (quad == 0) {
                const int row = bd[1].x;
                if (d0.z & kPiecePart) {
                    *reinterpret_cast<float4 *>(parts + row * kRowFloats + 8 * l) = u0;
                    *reinterpret_cast<float4 *>(parts + row * kRowFloats + 8 * l + 4) = u1;
                } else {
                    // quad 0 has par = 0: c0 = 2l, c1 = 2l + 1
                    *reinterpret_cast<float4 *>(X0 + (size_t)row * np) = u0;
                    *reinterpret_cast<float4 *>(X1 + (size_t)row * np) = u1;
                }
            }
        } else {
            const int row = pick(bd[1 + (quad >> 2)], quad & 3);
            if (row >= 0) {
                *reinterpret_cast<float4 *>(X0 + (size_t)row * np) = a0;
                *reinterpret_cast<float4 *>(X1 + (size_t)row * np) = a1;
            }
        }
    }
}

// Bundles [b0, b1) of one warp: the whole-block layout from shared memory
// (default), or the gather layout from global memory (GMEM, WIDE).
template <bool GMEM = false, bool WIDE = false, int UNROLL = kNarrowUnroll>
__device__ __forceinline__ void warp_bundles(const float *__restrict__ sD, const int2 *__restrict__ sKH,
                                             const int4 *__restrict__ sP, int p_base, int b0, int b1, int J, int np,
                                             float *__restrict__ X, float *parts) {
    static_assert(GMEM == WIDE, "whole-block layout from shared memory, gather layout from global memory");
    if constexpr (WIDE) wide_bundles<true, true>(sD, sKH, sP, p_base, b0, b1, J, np, X, parts);
    else narrow_bundles<UNROLL>(sD, sKH, sP, p_base, b0, b1, J, np, X, parts);
}

// The rows cut into parts, cuts[0 .. ncut) = {row, first slot, parts, 0}:
// X[row, J] = the sum of the parts' partial rows in slot order. Called by all
// threads after every warp's bundles (and a barrier).
template <bool WIDE = false>
__device__ __forceinline__ void combine_cuts(const int4 *__restrict__ cuts, int ncut, const float *parts, int J,
                                             int np, float *__restrict__ X) {
    const size_t plane = (size_t)np * np;
    constexpr int Q = WIDE ? 2 * kRowFloats / 4 : kRowFloats / 4;  // float4 per partial row
    for (int e = threadIdx.x; e < ncut * Q; e += blockDim.x) {
        const int4 c = __ldg(cuts + e / Q);
        const int p = e % Q;  // wide: plane p / 8, columns 4 (p % 8) ..
        float4 s = *reinterpret_cast<const float4 *>(parts + c.y * 4 * Q + 4 * p);
        for (int k = 1; k < c.z; ++k)
            s = f4add(s, *reinterpret_cast<const float4 *>(parts + (c.y + k) * 4 * Q + 4 * p));
        if (WIDE) {
            *reinterpret_cast<float4 *>(X + (p / 8) * plane + (size_t)c.x * np + J * kCWWide + 4 * (p % 8)) = s;
        } else {
            *reinterpret_cast<float4 *>(X + (p < 4 ? 0 : plane) + (size_t)c.x * np + J * kCW + 4 * (p & 3)) = s;
        }
    }
}

// Stage input of stage STAGE: D (stage 1), da (stages 2 and 4), db (stage 3).
template <int STAGE>
__device__ __forceinline__ const float *stage_input(const MixedWork &w) {
    return (STAGE == 1) ? w.D : (STAGE == 3 ? w.db : w.da);
}

// The gain g = G p(delta) of rows [b np / nb, (b + 1) np / nb) (CTA b of
// nb), from the compact diagonal p = w.pv (or pv_in) of the stage input
// (written by the previous epilogue): p is staged in shared memory (sp: np floats) with one
// coalesced round trip, together with the rows' S entries. The sums are
// those of gain_rows on the strided diagonal, in the same order.
__device__ __forceinline__ void cta_gain(const DevOps &ops, const MixedWork &w, int b, int nb, float *sp,
                                         const float *pv_in = nullptr) {
    const float *pv = pv_in ? pv_in : w.pv;
    __shared__ float red[32];
    const int n = ops.n, np = ops.np;
    const int r0 = (int)((long long)b * np / nb), r1 = (int)((long long)(b + 1) * np / nb);
    float P = 0.f, Dd = 0.f;
    for (int j = threadIdx.x; j < np; j += blockDim.x) {
        const float pj = __ldcg(pv + j);
        sp[j] = pj;
        if (j < n) {
            P = __fadd_rn(P, pj);
            if (ops.dang[j]) Dd = __fadd_rn(Dd, pj);
        }
    }
    P = mixed::block_sum_f(P, red);  // its barriers also publish sp
    Dd = mixed::block_sum_f(Dd, red);
    const int lane = threadIdx.x & 31;
    for (int i = r0 + (int)(threadIdx.x >> 5); i < r1; i += (int)(blockDim.x >> 5)) {
        float s = 0.f;
        if (i < n) {
            const int q1 = ops.s_ptr[i + 1];
            for (int q = ops.s_ptr[i] + lane; q < q1; q += 32) s = __fmaf_rn(ops.s_val32[q], sp[ops.s_col[q]], s);
        }
        s = mixed::warp_sum_f(s);
        if (lane == 0) {
            float gi = 0.f;
            if (i < n) {
                const float pi = sp[i];
                const float dterm = (ops.dangling == QPR_DANGLING_F)
                                        ? __fmul_rn(__fsub_rn(Dd, ops.dang[i] ? pi : 0.f), ops.inv_nm1_32)
                                        : __fmul_rn(Dd, ops.inv_n32);
                gi = __fmaf_rn(ops.alpha32, __fadd_rn(s, dterm),
                               __fmul_rn(__fmul_rn(ops.oma32, __fsub_rn(P, pi)), ops.inv_nm1_32));
            }
            w.g[i] = gi;
        }
    }
}

// Stop decision from the nparts stage-1 residual-estimate partials of step
// `step` (every thread of the CTA calls it; every caller forms the same sum
// in index order with a 512-thread block): the CTA with `record` writes the
// estimate to ctl and, when the run stops here, sets done so that the later
// kernels of the step return at once. A step whose exact residual a refresh
// already decided is not decided again. Returns the status. Callers: the
// first gain CTA of the stage-2 SpMM grid (single-problem column forms, RK4
// and RKF45), every CTA of the persistent form's stage 2, and the last CTA
// of a problem's stage-1 epilogue in the batched solver.
__device__ __forceinline__ int stage1_decision(const MixedWork &w, int nparts, long long step, bool record) {
    __shared__ float red[32];
    __shared__ int s_status;
    Ctl *ctl = w.ctl;
    float s = 0.f;
    for (int i = threadIdx.x; i < nparts; i += blockDim.x) s = __fadd_rn(s, __ldcg(w.partials32 + i));
    s = mixed::block_sum_f(s, red);
    if (threadIdx.x == 0) {
        int status = kCtlRunning;
        if (*(volatile long long *)&ctl->resid_exact_step != step) {
            const double r = sqrt((double)s);
            if (!isfinite(r)) status = kCtlNonFinite;
            else if (r < ctl->tol) status = kCtlCandidate;
            else if (step >= ctl->max_steps) status = kCtlMaxSteps;
            if (record) {
                ctl->resid = r;
                ctl->resid_step = step;
                if (status != kCtlRunning) {
                    ctl->status = status;
                    ctl->done = 1;
                }
            }
        }
        s_status = status;
    }
    __syncthreads();
    return s_status;
}

// The last CTA to finish a stage-1 epilogue (a ticket in the control block;
// release/acquire through fences) takes the stop decision.
__device__ __forceinline__ void stage1_last_decides(const MixedWork &w, int nparts) {
    __shared__ int s_last;
    if (threadIdx.x == 0) {
        __threadfence();
        s_last = (atomicAdd(&w.ctl->ticket, 1) == nparts - 1);
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    if (threadIdx.x == 0) w.ctl->ticket = 0;
    stage1_decision(w, nparts, *(volatile long long *)&w.ctl->step, true);
}

// Epilogue of tile pair (I, J) from X (global, written by the SpMM kernel)
// and the gain w.g (both read from L2: other CTAs wrote them); stage 1 ends
// with the ticket of the stop decision (TICKET),
// stage 4 advances the step counter (first pair). kENT threads. Shared
// memory: sX1, sX2 (TS * LDX floats each), sg (TS), sO (4 * TS * LDO).
// The X tiles of pair (I, J) into sX1 (X_IJ) and sX2 (X_JI, off-diagonal
// pairs), and the gain of a diagonal pair into sg; no barrier at the end.
__device__ __forceinline__ void epilogue_load_x(const DevOps &ops, const MixedWork &w, int I, int J, float *sX1,
                                                float *sX2, float *sg) {
    const int np = ops.np;
    const size_t plane = (size_t)np * np;
    const bool diag = (I == J);
    const int ntiles = diag ? 1 : 2;
    // X tiles as [a][LDX] rows (real part, then imaginary part), float4 loads
    for (int t = threadIdx.x; t < ntiles * TS * (2 * TS / 4); t += kENT) {
        const int which = t / (TS * (2 * TS / 4));
        const int u = t - which * (TS * (2 * TS / 4));
        const int a = u / (2 * TS / 4), q = u - a * (2 * TS / 4);  // q: 0..7 real quads, 8..15 imaginary
        const int R = which ? J : I, C = which ? I : J;
        const size_t o = (size_t)(R * TS + a) * np + C * TS + 4 * (q & 7);
        const float4 v = __ldcg(reinterpret_cast<const float4 *>(w.X + (q < 8 ? 0 : plane) + o));
        float *dst = (which ? sX2 : sX1) + a * LDX + 4 * q;
        dst[0] = v.x;
        dst[1] = v.y;
        dst[2] = v.z;
        dst[3] = v.w;
    }
    if (diag && threadIdx.x < TS) sg[threadIdx.x] = __ldcg(w.g + I * TS + threadIdx.x);
}

// The epilogue of pair (I, J) once its X tiles and gain are in shared memory
// (after a barrier).
template <int STAGE, bool TICKET = true>
__device__ __forceinline__ void epilogue_pair_staged(const DevOps &ops, const MixedWork &w, int I, int J, int pidx,
                                                     bool first, int nparts, const float *sX1, const float *sX2,
                                                     const float *sg, float *sO, const mixed::EpiIn<STAGE, kENT> &in) {
    mixed::tile_epilogue_in<STAGE, kENT>(ops, w, I, J, pidx, sX1, sX2, sg, sO, in);
    if (STAGE == 1 && TICKET) stage1_last_decides(w, nparts);
    if (STAGE == 4 && first && threadIdx.x == 0) w.ctl->step += 1;
}

template <int STAGE, bool TICKET = true>
__device__ __forceinline__ void epilogue_pair_in(const DevOps &ops, const MixedWork &w, int I, int J, int pidx,
                                                 bool first, int nparts, float *sX1, float *sX2, float *sg, float *sO,
                                                 const mixed::EpiIn<STAGE, kENT> &in) {
    epilogue_load_x(ops, w, I, J, sX1, sX2, sg);
    __syncthreads();
    epilogue_pair_staged<STAGE, TICKET>(ops, w, I, J, pidx, first, nparts, sX1, sX2, sg, sO, in);
}

// The same with the elementwise operands loaded first, so that their loads
// and the X tiles' are in flight together.
template <int STAGE, bool TICKET = true>
__device__ __forceinline__ void epilogue_pair(const DevOps &ops, const MixedWork &w, int I, int J, int pidx,
                                              bool first, int nparts, float *sX1, float *sX2, float *sg, float *sO) {
    mixed::EpiIn<STAGE, kENT> in;
    mixed::epi_load<STAGE, kENT>(ops, w, I, J, in);
    epilogue_pair_in<STAGE, TICKET>(ops, w, I, J, pidx, first, nparts, sX1, sX2, sg, sO, in);
}

}  // namespace cols
}  // namespace qpr
