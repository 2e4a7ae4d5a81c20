// Kernel bodies of the column-block SpMM (the whole-block form staging a
// column block of the stage input with TMA, and the gather form reading row
// lines through L1/L2), shared by the RK4 stage kernels (stage_cols.cu) and
// the RKF45 stage kernels (stage_rkf.cu). The caller supplies the stage
// input: a function returning the tensor map (whole-block form) or the
// pointer (gather form), called after the grid dependency wait.
#pragma once

#include "cols_body.cuh"
#include "qpr_internal.cuh"
#include "timeline.cuh"
#include "tma_util.cuh"

namespace qpr {
namespace cols {

// Body of the whole-block SpMM kernel for column block J and row split r,
// with the stage input staged through the tensor map that `pick_map`
// returns (called after the grid dependency wait, so it may read what the
// previous kernel wrote). Launched with programmatic dependent launch: the
// prologue (barriers, this CTA's CSR entries and bundles, which no kernel
// writes) overlaps the end of the previous kernel; the stage input is read
// after grid_dependency_wait. TL: record the timeline marks of the
// diagnostic build (timeline.cuh).
template <bool TL = false, typename PickMap>
__device__ __forceinline__ void spmm_block_body(PickMap pick_map, const DevOps &ops, const MixedWork &w, int J,
                                                int r) {
    extern __shared__ uint8_t dyn_raw[];
    __shared__ __align__(8) uint64_t bar_csr, bar_d;
    __shared__ int s_done;
    const int tid = threadIdx.x, warp = tid >> 5;
    const int np = ops.np;
    const uint32_t s0 = tma::smem_u32(dyn_raw);
    uint8_t *base = dyn_raw + (((s0 + 127) & ~127u) - s0);  // 128-byte aligned, shared provenance kept
    float *sD = reinterpret_cast<float *>(base);
    int2 *sKH = reinterpret_cast<int2 *>(base + (size_t)np * kRowFloats * 4);
    int4 *sP = reinterpret_cast<int4 *>(base + ops.col_p_off);
    const int q_base = ops.col_q[2 * r], q_end = ops.col_q[2 * r + 1];
    const int p_base = ops.col_sb[r], p_end = ops.col_sb[r + 1];
    const uint32_t kh_bytes = (uint32_t)((q_end - q_base) * 8);  // an even count of entries
    const uint32_t p_bytes = (uint32_t)((p_end - p_base) * 16 * kBundleInt4);
    if (tid == 0) {
        tma::mbar_init(&bar_csr, 1);
        tma::mbar_init(&bar_d, 1);
        tma::mbar_init_fence();
        tma::mbar_expect_tx(&bar_csr, kh_bytes + p_bytes);
        if (kh_bytes) tma::load_bulk(sKH, ops.col_kh + q_base, kh_bytes, &bar_csr);
        if (p_bytes) tma::load_bulk(sP, ops.col_pieces + kBundleInt4 * (size_t)p_base, p_bytes, &bar_csr);
    }
    const int wb0 = ops.col_wb[r * kAWarps + warp], wb1 = ops.col_wb[r * kAWarps + warp + 1];
    tma::grid_dependency_wait();
    tma::launch_dependents();
    // the stop flag and the column block in one round trip (the block is
    // staged whatever the flag says; nothing is written unless the run goes on)
    if (tid == 0) {
        const int done = *(volatile int *)&w.ctl->done;
        const CUtensorMap *tm = pick_map();
        tma::mbar_expect_tx(&bar_d, (uint32_t)np * kRowFloats * 4);
        for (int b = 0; b < np; b += kBoxRows) tma::load_3d(sD + (size_t)b * kRowFloats, tm, &bar_d, J * kCW, 0, b);
        s_done = done;
    }
    __syncthreads();
    if (s_done) {
        // the copies in flight land before the CTA leaves (bounded)
        tma::mbar_wait(&bar_csr, 0);
        tma::mbar_wait(&bar_d, 0);
        return;
    }
    const bool ok = tma::mbar_wait(&bar_csr, 0) && tma::mbar_wait(&bar_d, 0);
    timeline::mark<TL>(2);
    if (__syncthreads_or(!ok)) {
        // bounded wait gave up: report, give the copies one more bounded wait, return
        if (tid == 0) atomicExch(&w.ctl->err_timeout, 1);
        tma::mbar_wait(&bar_csr, 0);
        tma::mbar_wait(&bar_d, 0);
        return;
    }
    float *parts = reinterpret_cast<float *>(base + ops.col_part_off);
    warp_bundles(sD, sKH, sP, p_base, wb0, wb1, J, np, w.X, parts);
    const int cb0 = ops.col_cutb[r], cb1 = ops.col_cutb[r + 1];
    if (cb1 > cb0) {
        __syncthreads();
        combine_cuts(ops.col_cut + cb0, cb1 - cb0, parts, J, np, w.X);
    }
    timeline::mark_all<TL>(3);
}

// Body of the gather form of the SpMM, for N too large to stage a column
// block: CTA (r, J) stages only its split's entries and bundles and reads
// each nonzero's 32 values of the 32-column block J straight from the stage
// input that `pick_input` returns (called after the grid dependency wait;
// one 128-byte line per plane and row, L1-cached loads; the wide layout of
// warp_bundles: a group pair per row). The grid runs the row splits of one
// column block next to each other, so the block's rows (np x 128 bytes) are
// read from DRAM about once and then served by L2 to the splits.
template <typename PickInput>
__device__ __forceinline__ void spmm_gather_body(PickInput pick_input, const DevOps &ops, const MixedWork &w, int r,
                                                 int J) {
    extern __shared__ uint8_t dyn_raw[];
    __shared__ __align__(8) uint64_t bar_csr;
    __shared__ int s_done;
    const int tid = threadIdx.x, warp = tid >> 5;
    const uint32_t s0 = tma::smem_u32(dyn_raw);
    uint8_t *base = dyn_raw + (((s0 + 127) & ~127u) - s0);
    int2 *sKH = reinterpret_cast<int2 *>(base);
    int4 *sP = reinterpret_cast<int4 *>(base + ops.col_p_off);
    const int q_base = ops.col_q[2 * r], q_end = ops.col_q[2 * r + 1];
    const int p_base = ops.col_sb[r], p_end = ops.col_sb[r + 1];
    const uint32_t kh_bytes = (uint32_t)((q_end - q_base) * 8);
    const uint32_t p_bytes = (uint32_t)((p_end - p_base) * 16 * kBundleInt4);
    if (tid == 0) {
        tma::mbar_init(&bar_csr, 1);
        tma::mbar_init_fence();
        tma::mbar_expect_tx(&bar_csr, kh_bytes + p_bytes);
        if (kh_bytes) tma::load_bulk(sKH, ops.col_kh + q_base, kh_bytes, &bar_csr);
        if (p_bytes) tma::load_bulk(sP, ops.col_pieces + kBundleInt4 * (size_t)p_base, p_bytes, &bar_csr);
    }
    const int wb0 = ops.col_wb[r * kAWarps + warp], wb1 = ops.col_wb[r * kAWarps + warp + 1];
    tma::grid_dependency_wait();
    if (tid == 0) s_done = *(volatile int *)&w.ctl->done;
    __syncthreads();
    const bool ok = tma::mbar_wait(&bar_csr, 0);  // also before leaving: the copies land first (bounded)
    if (s_done) return;
    tma::launch_dependents();
    if (__syncthreads_or(!ok)) {
        if (tid == 0) atomicExch(&w.ctl->err_timeout, 1);
        return;
    }
    float *parts = reinterpret_cast<float *>(base + ops.col_part_off);
    warp_bundles<true, true>(pick_input(), sKH, sP, p_base, wb0, wb1, J, ops.np, w.X, parts);
    const int cb0 = ops.col_cutb[r], cb1 = ops.col_cutb[r + 1];
    if (cb1 > cb0) {
        __syncthreads();
        combine_cuts<true>(ops.col_cut + cb0, cb1 - cb0, parts, J, ops.np, w.X);
    }
}

// The gain of the stage input by CTA b of the nb leading CTAs of an SpMM
// grid (rows shared over them), from the compact diagonal that `pick_pv`
// returns (written by the previous epilogue; called after the grid
// dependency wait). The dynamic shared memory holds the staged diagonal (np
// floats).
//
// DECIDE (the stage-2 grid): CTA 0 first takes the stop decision of the
// step from the stage-1 epilogue's residual partials (stage1_decision, the
// same sum as the epilogue's last CTA would form: both kernels have 512
// threads). The gain CTAs finish well before the product CTAs, so the
// decision is off the critical path; the product CTAs of this grid do not
// wait for it (a stage-2 product of a step that stops is scratch), and the
// stage-2 epilogue, which reads `done` after its grid dependency wait,
// leaves the state as it was.
template <bool DECIDE = false, typename PickPv>
__device__ __forceinline__ void gain_role(const DevOps &ops, const MixedWork &w, int b, int nb, PickPv pick_pv) {
    extern __shared__ uint8_t dyn_raw[];
    __shared__ int s_done;
    tma::grid_dependency_wait();
    if (threadIdx.x == 0) s_done = *(volatile int *)&w.ctl->done;
    __syncthreads();
    if (s_done) return;
    tma::launch_dependents();
    if (DECIDE && b == 0) stage1_decision(w, w.npairs, *(volatile long long *)&w.ctl->step, true);
    cta_gain(ops, w, b, nb, reinterpret_cast<float *>(dyn_raw), pick_pv());
}

}  // namespace cols
}  // namespace qpr
