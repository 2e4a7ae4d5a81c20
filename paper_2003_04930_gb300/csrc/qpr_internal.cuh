// Internal declarations shared by the solver's translation units.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>
#include <stdint.h>

#include <stdio.h>
#include <stdlib.h>

#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "qpr.h"

namespace qpr {

// A named NVTX range for the length of a scope: every C-ABI call and every
// block of steps shows up on an Nsight timeline (a no-op when no tool is
// attached).
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

// QPR_LOG=1 in the environment: one line per solve on stderr.
inline bool log_enabled() {
    static const bool on = [] {
        const char *v = getenv("QPR_LOG");
        return v && v[0] && v[0] != '0';
    }();
    return on;
}


struct HostOps;

// Device control block. The host writes tol, dt and max_steps before a
// solve; the kernels read them (so a captured CUDA graph serves every dt)
// and write the stop decision and the residual. Kernels of a step read
// `done` on entry and return at once when it is set.
struct Ctl {
    int done;           // 1: every later kernel returns immediately
    int status;         // kCtlRunning / kCtlConverged / kCtlMaxSteps / kCtlNonFinite
    long long step;     // completed RK4 steps in this solve
    long long max_steps;
    double tol;         // stop when ||f(y_n)||_F < tol (0: never)
    double dt;
    double scale;       // 1 / Re tr(y) of the current step (set by the stage-1 gain kernel)
    double trace;       // Re tr(y) of the current step
    double resid;       // residual of step index `resid_step`
    long long resid_step;
    double resid_exact; // exact FP64 residual of the last reference refresh (mixed form)
    long long resid_exact_step;
    int err_timeout;    // a bounded device-side wait gave up
    int ticket;         // CTAs that finished the current ticketed epilogue (a problem's stage 1 in the batch, RKF45 stage 6)
    // FP32 forms of dt for the mixed form's delta stages, written by its
    // refresh: dtf = fl(dt), dt = dtf + dtl as a float-float pair, dt3 =
    // fl(dt / 3)
    float dtf, dtl, dt3, pad2_;
    // grid barrier of the persistent column-block kernel: arrivals, generation
    unsigned gb_count, gb_gen;
    // testing only: arrivals a grid barrier waits for beyond its grid (0, or 1
    // to make every barrier wait run out; qpr_options.test_fault)
    unsigned gb_extra, pad3_;
    // RKF45 (qpr_rkf45): the step of the next attempt and its largest value,
    // the tolerance Tol of Eq. S13, the integrated time and its end (0: none),
    // the discrepancy |z - y| of the last attempt, the rejected attempts, the
    // delta pair holding the current state (0: D, Dlo; 1: D1, Dlo1), the
    // order of the solution an accepted attempt keeps (4: y of Eq. S11, 5: z
    // of Eq. S12) and the step as a float-float pair (hf + hl) for the delta
    // stages
    double rk_h, rk_hmax, rk_tol, rk_t, rk_tend, rk_err;
    long long rk_rejected;
    int rk_cur, rk_order;
    float rk_hf, rk_hl;
};

// kCtlCandidate: the mixed form's FP32-accurate residual estimate passed;
// the host confirms it with an exact FP64 refresh.
// kCtlTimeReached: an RKF45 trajectory reached its end time.
enum { kCtlRunning = 0, kCtlConverged = 1, kCtlMaxSteps = 2, kCtlNonFinite = 3, kCtlCandidate = 4,
       kCtlTimeReached = 5 };

// Operators on the device (built once by qpr_create).
struct DevOps {
    int n;                // nodes
    int np;               // padded edge of every N x N plane (multiple of kPadFp64)
    double alpha, omega;
    int dangling;         // QPR_DANGLING_F / QPR_DANGLING_UNIFORM
    const double *H;      // np x np row-major, zero padding
    const int *h_ptr;     // CSR of H (same values; zeros skipped): n + 1 row pointers
    const int *h_col;
    const double *h_val;
    const float *h_val32; // the same values rounded to FP32 (mixed form)
    // rows of H cut into segments of at most 32 nonzeros (mixed form):
    // segments of row i are seg[rowseg[i] .. rowseg[i+1]), each {q0, q1}
    // into h_col / h_val; rowseg has np + 1 entries (empty for padding)
    const int *rowseg;
    const int2 *seg;
    const int *s_ptr;     // CSR of S restricted to columns with out-links: n + 1 row pointers
    const int *s_col;
    const double *s_val;  // A_ij / outDeg(j)
    const unsigned char *dang;  // n flags: column j has no out-links
    const double *c;      // np column sums of G (0 on padding)
    const float *c32;     // the same in FP32 (mixed form)
    // FP32 copies for the mixed form's delta stages (no FP64 instruction in
    // a delta stage): S values, alpha, 1 - alpha, omega, 1 / (n - 1), 1 / n
    const float *s_val32;
    float alpha32, oma32, omega32, inv_nm1_32, inv_n32;
    // column-block form of the sparse mixed stage (plan of ColPlan; 0 splits:
    // not used): the entries of H as (column, FP32 value bits), per bundle
    // interleaved and zero-padded; per row split its entry range {first
    // (even), end} and bundle range; bundle descriptors (2 int4 each); per
    // (split, warp) the first bundle
    const int2 *col_kh;
    const int *col_q;      // 2 per split
    const int *col_sb;     // splits + 1: bundles of split r are [col_sb[r], col_sb[r + 1])
    const int4 *col_pieces;
    const int *col_wb;     // splits * 16 + 1, absolute bundle indices
    int col_splits;
    int col_smem;          // dynamic shared memory of the SpMM kernel
    int col_p_off;         // byte offset of the staged bundles in it
    int col_sp_off;        // byte offset of the staged diagonal (np floats) in it
    int col_gather;        // 1: the gather form (the SpMM reads delta from L2; plan of ColPlan, gather)
    // rows cut into parts (kPartMax): per split the cut range [col_cutb[k], col_cutb[k + 1]) of col_cut; the partial
    // slots at byte col_part_off of the SpMM's shared memory
    const int4 *col_cut;
    const int *col_cutb;
    int col_part_off;
    int col_epi_off;       // persistent form: byte offset of the epilogue buffers (0: over the column block)
    int col_psmem;         // persistent form: dynamic shared memory of its launch
    int col_gain_ctas;     // two-launch forms: leading CTAs of the SpMM grid that form the gain instead
    int col_launch_smem;   // two-launch forms: dynamic shared memory of the SpMM launch (>= np floats)
};

// RK4 work buffers. Every state buffer holds two np x np FP64 planes,
// real part first, then imaginary part.
struct Work {
    double *y;            // state at the start of a step (unnormalised)
    double *z;            // RK4 accumulator
    double *ya, *yb;      // stage inputs (ping-pong)
    double *g;            // gain G p of the current stage, np entries
    double *partials;     // one residual partial per stage-kernel CTA
    int2 *pairs;          // tile pairs (I, J), I <= J, off-diagonal first
    int npairs;
    int tiles;            // np / kTileFp64
    Ctl *ctl;
};

// Buffers of the mixed-precision form (stage_mixed.cu). The state is
// y = R + delta: FP64 R = y / tr(y) at the last refresh and F = f(R); the
// delta since that refresh as a float-float pair of FP32 planes, D (high
// part, the FP32 delta the stages read) and Dlo (low part). FP32 (two np x np
// planes each): F32 = fl(F), dt F = Ghi + Glo (float-float) and the stage
// inputs da/db (the nested RK4 form keeps no running stage sum).
struct TcMaps;
struct MixedWork {
    double *R, *F;
    float *F32, *D, *Dlo, *da, *db, *Ghi, *Glo;
    float *g;             // gain of the stage delta, np
    float *pv;            // np: diagonal of the next stage input (written by every epilogue, zeroed by a refresh)
    double *g64;          // FP64 gain used by the refresh, np
    double *partials;     // exact residual partials of the refresh
    float *partials32;    // residual-estimate partials of the stage-1 kernel
    int2 *pairs;          // 32 x 32 tile pairs (refresh and sparse stage kernel)
    int4 *epi_pairs;      // the same pairs in the column-block epilogues' CTA order: {I, J, index in pairs, 0}
    int npairs;
    int tiles;
    Ctl *ctl;
    int nstage_partials;  // residual partials the stage-1 kernel writes
    // dense backend (tcgen05): 128 x 128 tile pairs and the BF16 split planes
    // [3 levels][2 planes: Re, -Im][np][np] of the stage-1, stage-2 and
    // stage-3 inputs (D, da, db); null for the sparse backend
    int2 *pairs_tc;
    int npairs_tc;
    __nv_bfloat16 *splitD, *splitA, *splitB;
    const TcMaps *maps;   // host pointer, used only by the launch code
    // column-block form of the sparse backend: X = H delta (2 planes) and the
    // TMA maps of the stage inputs D, da, db (host pointer; null: tile-pair
    // kernel)
    float *X;
    const struct ColMaps *cmaps;
    // RKF45 in the column-block form (null until the first qpr_rkf45 call):
    // the second delta pair (D1, Dlo1; the controller's rk_cur selects the
    // current one), the running sum of the step's power terms (acc, 2
    // planes), the low part of F as a float-float pair with F32 (Flo, 2
    // planes), and the compact diagonals of D and D1 (pvd, 2 np)
    float *D1, *Dlo1, *acc, *Flo, *pvd;
};

// TMA descriptors of the stage inputs D, da, db for the column-block SpMM:
// each pair of planes seen as 2 np rows of np FP32, boxes of 8 x 256.
struct ColMaps {
    CUtensorMap d[3];
    CUtensorMap d1;  // D1 of the RKF45 form (encoded by its first call)
};

constexpr int kTileTc = 128;

// TMA descriptors of the dense mixed stage: H split planes [3][np][np] and
// the three delta-split buffers.
struct TcMaps {
    CUtensorMap h;
    CUtensorMap d[3];
};

constexpr int kTileFp64 = 32;
constexpr int kPadFp64 = 32;

// ---- kernels (aux_kernels.cu) ----
// Hermitise an interleaved complex128 n x n matrix into two np x np planes.
void launch_import(const double *rho_il, int n, int np, double *planes, cudaStream_t s);
// planes * ctl->scale (use_scale) -> interleaved complex128 n x n.
void launch_export(const double *planes, int n, int np, const Ctl *ctl, int use_scale,
                   double *rho_il, cudaStream_t s);
// p[i] = Re rho_ii of an interleaved complex128 matrix.
void launch_diag(const double *rho_il, int n, double *p, cudaStream_t s);
// g = G p_s for stage `stage` (0: plain right-hand side, 1..4: RK4 stages).
void launch_gain(int stage, const DevOps &ops, const double *yin, const Work &w, cudaStream_t s);

// ---- FP64 tile-pair stage kernel (stage_fp64.cu) ----
// stage 0: out = f(yin) into w.z, residual partials.
// stage 1..4: one classical RK4 stage with the fused update.
void launch_stage_fp64(int stage, const DevOps &ops, const Work &w, cudaStream_t s);
// Opt in to the kernel's dynamic shared memory on the current device.
cudaError_t init_stage_fp64();

// ---- sparse (CSR H) FP64 stage kernel (stage_sparse.cu), same contract ----
void launch_stage_sparse(int stage, const DevOps &ops, const Work &w, cudaStream_t s);
cudaError_t init_stage_sparse();

// ---- mixed-precision form (stage_mixed.cu) ----
// Reference refresh: R = y = y / tr(y), F = f(R) exactly (FP64), D = 0, exact
// residual and stop decision.
void launch_mixed_refresh(const DevOps &ops, const MixedWork &w, cudaStream_t s);
// One RK4 stage: parts & 1 launches the gain of the stage delta (the
// tensor-core form; the tile-pair stage kernel forms the gain itself), parts
// & 2 the stage kernel (3 = both, in that order). Column-block form: parts &
// 1 the SpMM (its leading CTAs form the gain), parts & 2 the epilogue;
// serial (profiling): no programmatic dependent launch.
void launch_mixed_stage(int stage, const DevOps &ops, const MixedWork &w, cudaStream_t s, int parts = 3,
                        bool serial = false);
// Opt in to the dynamic shared memory of the sparse mixed stage kernels.
cudaError_t init_stage_mixed();
// Dense backend of the mixed form (stage_mixed_tc.cu).
cudaError_t init_mixed_tc();
bool make_tc_maps(const DevOps &ops, const __nv_bfloat16 *hsplit, const __nv_bfloat16 *const dsplit[3],
                  TcMaps *maps);
void launch_mixed_tc(int stage, const DevOps &ops, const MixedWork &w, const TcMaps &m, cudaStream_t s);
// Column-block form of the sparse mixed stage (stage_cols.cu): per stage a
// column-block SpMM X = H delta from TMA-staged columns, then the tile-pair
// epilogue. Used where its staged operands fit (np <= kColMaxNp and a plan).
constexpr int kColMaxNp = 1536;
// Complex columns per block of the whole-block and of the gather SpMM.
constexpr int kColWidth = 16;
constexpr int kColGatherWidth = 32;
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder();
bool make_col_maps(const DevOps &ops, const float *const din[3], ColMaps *maps);
// Host plan of the column-block SpMM (device copies go to DevOps col_*).
struct ColPlan {
    int splits = 0;
    int smem = 0;                 // dynamic shared memory per CTA
    int p_off = 0;                // byte offset of the staged bundles
    int sp_off = 0;               // byte offset of the staged diagonal
    std::vector<int2> kh;         // entries of the bundles, interleaved and padded
    std::vector<int> q;           // 2 per split
    std::vector<int> sb;          // splits + 1
    std::vector<int4> pieces;     // 2 per bundle
    std::vector<int> wb;          // splits * 16 + 1
    std::vector<int4> cuts;       // rows cut into parts: {row, first partial slot, parts, 0}
    std::vector<int> cutb;        // splits + 1: the cuts of split r are [cutb[r], cutb[r + 1])
    int part_off = 0;             // byte offset of the partial slots in the SpMM's shared memory
};
// Plans the column-block form of an np x np problem on `device`; false if
// its staged operands do not fit one CTA's shared memory. Row splits: the
// fewest from min_splits up that fit (0: enough CTAs for every SM when the
// problem runs alone). A row's product does not depend on the plan (its
// group sums its entries in order; zero padding never changes a sum that
// starts at +0), so every plan gives bitwise the same X.
// gather: the plan of the gather form (no staged column block, any np; row
// splits from enough CTAs for every SM several times over).
bool plan_columns(const HostOps &h, int np, int device, ColPlan &plan, int min_splits = 0, bool gather = false);
cudaError_t set_gather_smem(int bytes);
// Opt in to `bytes` of dynamic shared memory for the SpMM kernels.
cudaError_t set_cols_smem(int bytes);
void launch_cols_stage(int stage, const DevOps &ops, const MixedWork &w, cudaStream_t s, int parts = 3,
                       bool serial = false);
// RKF45 in the column-block form (stage_rkf.cu). One attempt is six
// stages, each the SpMM (its leading CTAs form the gain) and the epilogue;
// stage 6 ends with the step-size controller. The refresh folds the current delta into R and
// recomputes F = f(R) exactly, as the RK4 refresh does.
constexpr int kRkfStages = 6;
constexpr int kRkfLaunchesPerAttempt = 2 * kRkfStages;
bool make_rkf_map(const DevOps &ops, const float *d1, ColMaps *maps);
void launch_rkf_stage(int stage, const DevOps &ops, const MixedWork &w, cudaStream_t s);
void launch_rkf_refresh(const DevOps &ops, const MixedWork &w, cudaStream_t s);
constexpr int kRkfLaunchesPerRefresh = 5;
cudaError_t init_rkf(int spmm_smem, bool gather);

// Persistent form (stage_persist.cu): one cooperative launch runs up to
// `steps` RK4 steps of the column-block form, grid barriers between the
// phases. persist_grid: CTAs of that launch for an np x np problem with the
// given plan on `device` (0: the form does not apply).
// On success also the launch's dynamic shared memory and the offset of the
// epilogue buffers in it.
int persist_grid(int np, int splits, int smem, int device, int *persist_smem, int *epi_off);
cudaError_t set_persist_smem(int bytes);
cudaError_t launch_cols_block(const DevOps &ops, const MixedWork &w, int steps, int grid, cudaStream_t s);
// Kernel launches per RK4 step and per refresh of the mixed form.
constexpr int kMixedLaunchesPerStep = 4;   // tile-pair sparse kernel (the dense one adds 4 gain kernels)
constexpr int kMixedLaunchesPerStepCols = 8;  // column-block form: SpMM (with the gain) and epilogue per stage
constexpr int kMixedLaunchesPerRefresh = 5;
// Steady-state solves with adaptive_refresh: the longest window between
// refreshes, in multiples of ref_refresh.
constexpr int kMaxRefreshGrowth = 8;

// ---- classical PageRank and hub classes (pagerank.cu) ----
// CTAs of one power-iteration kernel for n nodes.
int pagerank_grid(int n);
// Power iteration pi <- G pi / sum(pi) from the uniform vector until the L1
// change of an iteration (checked every 8) is below tol or after max_iter
// iterations; pi (normalised) into pi_out_dev (n doubles). scratch: device,
// 2 n + pagerank_grid(n) doubles. Synchronises the stream.
cudaError_t pagerank(const DevOps &ops, double tol, int64_t max_iter, double *scratch, double *pi_out_dev,
                     int64_t *iters, double *delta_out, cudaStream_t s);
// classes_dev[i] in {0, 1, 2} (rest, secondary hub, main hub) of the
// probabilities p (device, n doubles) with threshold factor c; counts_dev
// (3 values) receives the class sizes.
cudaError_t hub_classes(const double *p, int n, double c, int *classes_dev, unsigned long long *counts_dev,
                        cudaStream_t s);

// Raise the dynamic shared-memory limit of `kernel` on the current device to
// at least `bytes`; never lower it (contexts with different plans share the
// kernel, and a limit above a launch's request is harmless). Serialised
// over host threads.
cudaError_t raise_smem_limit(const void *kernel, int bytes);
template <typename K>
cudaError_t raise_smem_limit_t(K *kernel, int bytes) {
    return raise_smem_limit(reinterpret_cast<const void *>(kernel), bytes);
}

// ---- host assembly (qpr_api.cu) ----
struct HostOps {
    int64_t n = 0;
    std::vector<double> outdeg;
    std::vector<int64_t> hptr;
    std::vector<int> hcol;
    std::vector<double> hval;
    std::vector<int> sptr, scol;
    std::vector<double> sval;
    std::vector<unsigned char> dang;
};
qpr_status assemble_host(int64_t n, int64_t m, const int64_t *src, const int64_t *dst, const double *w, int h_diag,
                         HostOps &out, std::string &err);
// Segments of at most `len` nonzeros of every row of the CSR of H, for np
// rows (rowseg: np + 1 entries, seg: {q0, q1}).
void row_segments(const HostOps &h, int np, int len, std::vector<int> &rowseg, std::vector<int2> &seg);
std::vector<double> column_sums_G(const HostOps &h, double alpha, int np, double *cmax);
// Message returned by qpr_last_error(NULL) on this thread.
void set_create_error(const std::string &msg);
// Opt in to the dynamic shared memory of the batched kernels (batch.cu).
cudaError_t init_batch();
cudaError_t set_bcols_smem(int bytes);
// Resident CTAs per SM of the batched SpMM with `bytes` of dynamic shared memory.
cudaError_t bcols_ctas_per_sm(int bytes, int *ctas);
double estimate_spread(int64_t n, const std::vector<int64_t> &ptr, const std::vector<int> &col,
                       const std::vector<double> &val);

}  // namespace qpr
