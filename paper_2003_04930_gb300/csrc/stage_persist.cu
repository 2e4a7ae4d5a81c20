// Persistent form of the column-block sparse mixed stage: one cooperative
// launch (one CTA per SM, all resident) runs a block of RK4 steps. Each
// stage is the SpMM phase (CTA c < ncb x splits: column block c / splits,
// row split c % splits) and the epilogue phase (tile pairs c, c + grid, ...),
// separated by grid barriers. The CTA stages its split's CSR entries and
// bundles once per launch; per stage only the column block of the stage
// input is loaded (3-D TMA box). The stop decision of stage 2 is taken by
// every CTA from the stage-1 partials in index order, so all CTAs leave the
// step loop together.
//
// The arithmetic is the two-launch column form's (warp_bundles, cta_gain,
// the 512-thread epilogue and the same decision sum), so both forms and the
// batched solver give bitwise the same results.
#include <math.h>

#include "cols_body.cuh"
#include "qpr_internal.cuh"
#include "tma_util.cuh"

namespace qpr {
namespace {

using namespace cols;

// Epilogue buffers: sX1, sX2 (TS x LDX), sO (4 TS x LDO), sg (TS), in floats.
constexpr int kEpiFloats = 2 * TS * LDX + 4 * TS * LDO + TS;
// Time a grid-barrier wait may take before the kernel reports a timeout
// (one second on the global nanosecond timer; a legitimate wait at these
// sizes is microseconds).
constexpr unsigned long long kBarrierTimeoutNs = 1000000000ull;

// Grid-wide barrier by generation count. Release: every CTA's writes are
// fenced before it arrives; acquire: the waiter fences after it sees the new
// generation. The barrier completes when ncta + ctl->gb_extra CTAs have
// arrived (gb_extra is 0 except under qpr_options.test_fault). Bounded:
// returns false (and sets err_timeout) when it gave up.
__device__ __forceinline__ bool grid_sync(Ctl *ctl, unsigned ncta, unsigned &gen, int *s_ok) {
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        const unsigned g = gen;
        const unsigned expect = ncta + *(volatile unsigned *)&ctl->gb_extra;
        __threadfence();
        if (atomicAdd(&ctl->gb_count, 1u) == expect - 1) {
            atomicExch(&ctl->gb_count, 0u);
            __threadfence();
            atomicExch(&ctl->gb_gen, g + 1);
        } else {
            const unsigned long long t0 = tma::global_ns();
            while (*(volatile unsigned *)&ctl->gb_gen == g) {
                if (tma::global_ns() - t0 > kBarrierTimeoutNs) {
                    ok = 0;
                    atomicExch(&ctl->err_timeout, 1);
                    break;
                }
                __nanosleep(100);
            }
        }
        __threadfence();
        gen = g + 1;
        *s_ok = ok;
    }
    __syncthreads();
    return *s_ok != 0;
}

struct Smem {
    float *sD;   // staged column block; the epilogue buffers overlay it
    int2 *sKH;
    int4 *sP;
    float *sp;   // staged diagonal of the stage input (the gain)
    float *epi;  // epilogue buffers (over the column block when it is large enough)
    float *parts;  // partial slots of the rows cut into parts
    uint64_t *bar;
    int *flag;
};

// One stage. Returns 0 to go on, 1 when the stop decision ends the block,
// -1 on a timeout.
template <int STAGE>
__device__ __forceinline__ int persist_stage(const CUtensorMap *tm, const DevOps &ops, const MixedWork &w,
                                             const Smem &sm, bool has_unit, int J, int r, long long step,
                                             uint32_t &phase, unsigned &gen) {
    const int tid = threadIdx.x, warp = tid >> 5;
    const int np = ops.np;
    const unsigned C = gridDim.x;
    const int c = blockIdx.x;
    if (STAGE == 2 && stage1_decision(w, w.npairs, step, c == 0) != kCtlRunning) return 1;
    // ---- SpMM phase ----
    if (has_unit && tid == 0) {
        // the previous phases read and wrote this buffer, and other CTAs wrote
        // the stage input, through the generic proxy; the copy is async-proxy
        asm volatile("fence.proxy.async;\n" ::: "memory");
        tma::mbar_expect_tx(sm.bar, (uint32_t)np * kRowFloats * 4);
        for (int b = 0; b < np; b += kBoxRows) tma::load_3d(sm.sD + (size_t)b * kRowFloats, tm, sm.bar, J * kCW, 0, b);
    }
    // the gain: by the CTAs without an SpMM unit when there are any
    const int units = (np / kCW) * ops.col_splits;
    if (units < (int)C) {
        if (!has_unit) cta_gain(ops, w, c - units, (int)C - units, sm.sp);
    } else {
        cta_gain(ops, w, c, (int)C, sm.sp);
    }
    if (has_unit) {
        const bool ok = tma::mbar_wait(sm.bar, phase & 1);
        ++phase;
        if (__syncthreads_or(!ok)) {
            if (tid == 0) atomicExch(&w.ctl->err_timeout, 1);
            tma::mbar_wait(sm.bar, (phase - 1) & 1);
            return -1;
        }
        warp_bundles(sm.sD, sm.sKH, sm.sP, ops.col_sb[r], ops.col_wb[r * kAWarps + warp],
                     ops.col_wb[r * kAWarps + warp + 1], J, np, w.X, sm.parts);
        const int cb0 = ops.col_cutb[r], cb1 = ops.col_cutb[r + 1];
        if (cb1 > cb0) {
            __syncthreads();
            combine_cuts(ops.col_cut + cb0, cb1 - cb0, sm.parts, J, np, w.X);
        }
    }
    if (!grid_sync(w.ctl, C, gen, sm.flag)) return -1;
    // ---- epilogue phase (buffers overlay the column block) ----
    float *sX1 = sm.epi, *sX2 = sX1 + TS * LDX, *sO = sX2 + TS * LDX, *sg = sO + 4 * TS * LDO;
    for (int p = c; p < w.npairs; p += (int)C) {
        const int2 pr = w.pairs[p];
        epilogue_pair<STAGE, false>(ops, w, pr.x, pr.y, p, p == 0, w.npairs, sX1, sX2, sg, sO);
        __syncthreads();
    }
    if (!grid_sync(w.ctl, C, gen, sm.flag)) return -1;
    return 0;
}

__global__ void __launch_bounds__(kANT, 1) cols_block_kernel(const __grid_constant__ ColMaps maps, DevOps ops,
                                                             MixedWork w, int nsteps) {
    extern __shared__ uint8_t dyn_raw[];
    __shared__ __align__(8) uint64_t bar;
    __shared__ int s_flag;
    __shared__ long long s_step;
    Ctl *ctl = w.ctl;
    const int tid = threadIdx.x;
    unsigned gen = 0;  // meaningful in thread 0
    if (tid == 0) {
        s_flag = *(volatile int *)&ctl->done;
        s_step = *(volatile long long *)&ctl->step;
        gen = *(volatile unsigned *)&ctl->gb_gen;
        tma::mbar_init(&bar, 1);
        tma::mbar_init_fence();
    }
    __syncthreads();
    if (s_flag) return;  // every CTA reads the same value: done changes only after a grid barrier
    long long step = s_step;
    const int np = ops.np;
    const uint32_t s0 = tma::smem_u32(dyn_raw);
    uint8_t *base = dyn_raw + (((s0 + 127) & ~127u) - s0);
    Smem sm;
    sm.sD = reinterpret_cast<float *>(base);
    sm.sKH = reinterpret_cast<int2 *>(base + (size_t)np * kRowFloats * 4);
    sm.sP = reinterpret_cast<int4 *>(base + ops.col_p_off);
    sm.sp = reinterpret_cast<float *>(base + ops.col_sp_off);
    sm.epi = reinterpret_cast<float *>(base + ops.col_epi_off);
    sm.parts = reinterpret_cast<float *>(base + ops.col_part_off);
    sm.bar = &bar;
    sm.flag = &s_flag;
    const int c = blockIdx.x;
    const bool has_unit = c < (np / kCW) * ops.col_splits;
    const int J = has_unit ? c / ops.col_splits : 0, r = has_unit ? c % ops.col_splits : 0;
    uint32_t phase = 0;
    // this CTA's CSR entries and bundles, once per launch
    if (has_unit) {
        const int q_base = ops.col_q[2 * r], q_end = ops.col_q[2 * r + 1];
        const int p_base = ops.col_sb[r], p_end = ops.col_sb[r + 1];
        if (tid == 0) {
            const uint32_t kh_bytes = (uint32_t)((q_end - q_base) * 8);  // an even count of entries
            const uint32_t p_bytes = (uint32_t)((p_end - p_base) * 16 * kBundleInt4);
            tma::mbar_expect_tx(&bar, kh_bytes + p_bytes);
            if (kh_bytes) tma::load_bulk(sm.sKH, ops.col_kh + q_base, kh_bytes, &bar);
            if (p_bytes) tma::load_bulk(sm.sP, ops.col_pieces + kBundleInt4 * (size_t)p_base, p_bytes, &bar);
        }
        const bool ok = tma::mbar_wait(&bar, 0);
        ++phase;
        if (__syncthreads_or(!ok)) {
            if (tid == 0) atomicExch(&ctl->err_timeout, 1);
            tma::mbar_wait(&bar, 0);
            return;  // the other CTAs give up at their next grid barrier
        }
    }
    for (int k = 0; k < nsteps; ++k) {
        int st = persist_stage<1>(&maps.d[0], ops, w, sm, has_unit, J, r, step, phase, gen);
        if (st == 0) st = persist_stage<2>(&maps.d[1], ops, w, sm, has_unit, J, r, step, phase, gen);
        if (st == 0) st = persist_stage<3>(&maps.d[2], ops, w, sm, has_unit, J, r, step, phase, gen);
        if (st == 0) st = persist_stage<4>(&maps.d[1], ops, w, sm, has_unit, J, r, step, phase, gen);
        if (st != 0) break;
        ++step;
    }
}

}  // namespace

int persist_grid(int np, int splits, int smem, int device, int *persist_smem, int *epi_off) {
    int coop = 0, sms = 0, per_sm = 0, optin = 0;
    if (cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, device) != cudaSuccess || !coop ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess ||
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    // the epilogue buffers go over the column block when it is large enough
    // (it is reloaded after the epilogue phase), else after the plan's buffers
    const int epi_bytes = kEpiFloats * 4;
    const bool over = (size_t)np * kRowFloats * 4 >= (size_t)epi_bytes;
    const int off = over ? 0 : (smem - 128 + 15) / 16 * 16;
    const int total = over ? smem : off + epi_bytes + 128;
    if (total > optin - 1024) return 0;
    if (set_persist_smem(total) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, cols_block_kernel, kANT, total) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    const int units = (np / kCW) * splits;
    if (per_sm < 1 || units > sms) return 0;
    *persist_smem = total;
    *epi_off = off;
    return sms;
}

cudaError_t set_persist_smem(int bytes) { return raise_smem_limit_t(cols_block_kernel, bytes); }

cudaError_t launch_cols_block(const DevOps &ops, const MixedWork &w, int steps, int grid, cudaStream_t s) {
    ColMaps maps = *w.cmaps;
    DevOps o = ops;
    MixedWork mw = w;
    int n = steps;
    void *args[4] = {&maps, &o, &mw, &n};
    return cudaLaunchCooperativeKernel((const void *)cols_block_kernel, dim3(grid), dim3(kANT), args,
                                       (size_t)ops.col_psmem, s);
}

}  // namespace qpr
