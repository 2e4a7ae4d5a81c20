// Batched steady-state solver: many independent problems (graphs of uneven
// N, each with its own omega) integrated together by the mixed-precision RK4
// form.
//
// Every problem keeps its own operators, buffers and control block; a
// device array of per-problem descriptors lets one kernel launch serve all of
// them. Work is described by lists: the active problems (one CTA per problem
// for the trace and gain kernels of the refresh), the (problem, column
// block, split) units of the SpMM in size classes of the padded edge (each
// class one launch with its own shared memory), and the (problem, I, J) tile
// pairs (grid-stride persistent kernels for the epilogue and the refresh
// products). A block of steps (the refreshes that are due, then ref_refresh
// steps) is one captured CUDA graph over the lists; a problem that stops is
// retired on the device (its kernels return at once) and leaves the lists
// when they are rebuilt, once the active set has shrunk by a quarter. The
// per-tile and per-problem arithmetic is the single-problem code (the same
// device functions in the same order), so every problem's result is bitwise
// the one qpr_steady_state returns for it alone with the same options.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <string>
#include <vector>

#include "cols_body.cuh"
#include "gain_body.cuh"
#include "mixed_body.cuh"
#include "qpr_internal.cuh"
#include "sparse_body.cuh"
#include "tma_util.cuh"

namespace qpr {

struct BatchGraph {
    DevOps ops;
    MixedWork mw;
    Work w64;              // the FP64 refresh: y = R, z = F
    const ColMaps *dmaps;  // column form: tensor maps of D, da, db (device memory); else null
};
static_assert(sizeof(BatchGraph) % 4 == 0, "descriptor copied as 32-bit words");

namespace {

constexpr int kStageNT = 256;  // threads of the mixed stage kernel (mixed_body.cuh)

// Copy problem g's descriptor into shared memory (all threads; ends synced).
__device__ __forceinline__ void load_graph(const BatchGraph *gs, int g, BatchGraph &sg) {
    const int *src = reinterpret_cast<const int *>(gs + g);
    int *dst = reinterpret_cast<int *>(&sg);
    for (int i = threadIdx.x; i < (int)(sizeof(BatchGraph) / 4); i += blockDim.x) dst[i] = src[i];
    __syncthreads();
}

// load_graph and the stop flag of problem g (ctls: the problems' control
// blocks) in the same round trip; returns the flag, the same value for
// every thread of the CTA (ends synced).
__device__ __forceinline__ int load_graph_done(const BatchGraph *gs, const Ctl *ctls, int g, BatchGraph &sg,
                                               int *s_flag) {
    if (threadIdx.x == 0) *s_flag = *(volatile const int *)&ctls[g].done;
    load_graph(gs, g, sg);
    return *s_flag;
}

// 1 if problem `sg` has stopped; the same value for every thread of the CTA.
__device__ __forceinline__ int graph_done(const BatchGraph &sg, int *s_flag) {
    if (threadIdx.x == 0) *s_flag = *(volatile int *)&sg.mw.ctl->done;
    __syncthreads();
    return *s_flag;
}

// The refresh kernels skip problem g when it has stopped or, with a due
// array (one byte per problem, written by the host before each block), when
// its refresh is not due this block.
__device__ __forceinline__ int skip_refresh(const BatchGraph &sg, int g, const uint8_t *due, int *s_flag) {
    if (graph_done(sg, s_flag)) return 1;
    return due && !due[g];
}

__global__ void __launch_bounds__(256) b_trace_kernel(const BatchGraph *gs, const int *act, const uint8_t *due) {
    __shared__ BatchGraph sg;
    __shared__ int s_flag;
    load_graph(gs, act[blockIdx.x], sg);
    if (skip_refresh(sg, act[blockIdx.x], due, &s_flag)) return;
    mixed::refresh_trace_body(sg.ops, sg.mw);
}

__global__ void __launch_bounds__(256) b_normalize_kernel(const BatchGraph *gs, const int *act,
                                                          const uint8_t *due) {
    __shared__ BatchGraph sg;
    __shared__ int s_flag;
    load_graph(gs, act[blockIdx.y], sg);
    if (skip_refresh(sg, act[blockIdx.y], due, &s_flag)) return;
    mixed::refresh_normalize_body(sg.ops, sg.mw, blockIdx.x * (size_t)blockDim.x + threadIdx.x,
                                  (size_t)gridDim.x * blockDim.x);
}

__global__ void __launch_bounds__(256) b_gain64_kernel(const BatchGraph *gs, const int *act, const uint8_t *due) {
    __shared__ BatchGraph sg;
    __shared__ int s_flag;
    load_graph(gs, act[blockIdx.x], sg);
    if (skip_refresh(sg, act[blockIdx.x], due, &s_flag)) return;
    gain64::gain_fp64_body<0>(sg.ops, sg.w64, sg.w64.y, 0, 1);
}

__global__ void __launch_bounds__(sparse64::NTHREADS)
b_sparse64_kernel(const BatchGraph *gs, const int4 *items, int nitems, const uint8_t *due) {
    extern __shared__ __align__(16) double smem[];
    __shared__ BatchGraph sg;
    __shared__ int s_flag;
    for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
        const int4 t = items[it];
        load_graph(gs, t.x, sg);
        if (!skip_refresh(sg, t.x, due, &s_flag)) sparse64::tile<0>(sg.ops, sg.w64, t.y, t.z, t.w, t.w == 0, smem);
        __syncthreads();
    }
}

__global__ void __launch_bounds__(256) b_post_kernel(const BatchGraph *gs, const int *act, const uint8_t *due) {
    __shared__ BatchGraph sg;
    __shared__ int s_flag;
    load_graph(gs, act[blockIdx.y], sg);
    if (skip_refresh(sg, act[blockIdx.y], due, &s_flag)) return;
    mixed::refresh_post_body(sg.ops, sg.mw, blockIdx.x * (size_t)blockDim.x + threadIdx.x,
                             (size_t)gridDim.x * blockDim.x, blockIdx.x == 0);
}

template <int STAGE>
__global__ void __launch_bounds__(kStageNT) b_stage_mixed_kernel(const BatchGraph *gs, const int4 *items, int nitems) {
    extern __shared__ __align__(16) uint8_t tile_smem[];
    __shared__ BatchGraph sg;
    __shared__ int s_flag;
    for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
        const int4 t = items[it];
        load_graph(gs, t.x, sg);
        if (!graph_done(sg, &s_flag))
            mixed::mixed_sparse_tile<STAGE>(sg.ops, sg.mw, t.y, t.z, t.w, t.w == 0, tile_smem);
        __syncthreads();
    }
}

// Column-block form: the SpMM over (problem, J, split) items. The split's
// entries and bundles (two bulk copies) and the column block (3-D tensor
// loads through the problem's own tensor map, kept in device memory) land
// on one mbarrier while the CTA forms its share of the problem's gain; the
// arithmetic is the single-problem form's (warp_bundles, cta_gain), so the
// results are bitwise the same. Registers are capped for two resident CTAs
// per SM, so that the small size classes (less shared memory) overlap one
// CTA's staging with another's products.
template <int STAGE>
__global__ void __launch_bounds__(cols::kANT, 2) b_cols_spmm_kernel(const BatchGraph *gs, const Ctl *ctls,
                                                                 const int4 *items, int nitems) {
    extern __shared__ __align__(128) uint8_t dyn_smem[];
    __shared__ BatchGraph sg;
    __shared__ int s_flag;
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        tma::mbar_init(&bar, 1);
        tma::mbar_init_fence();
    }
    uint32_t phase = 0;
    int4 tn = blockIdx.x < nitems ? items[blockIdx.x] : make_int4(0, 0, 0, 0);
    for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
        const int4 t = tn;
        if (it + (int)gridDim.x < nitems) tn = items[it + gridDim.x];  // the next item, in flight meanwhile
        if (!load_graph_done(gs, ctls, t.x, sg, &s_flag)) {
            const DevOps &ops = sg.ops;
            const int J = t.y, r = t.z, np = ops.np;
            // 128-byte aligned for the tensor loads (the plan's size leaves the slack)
            const uint32_t s0 = tma::smem_u32(dyn_smem);
            uint8_t *base = dyn_smem + (((s0 + 127) & ~127u) - s0);
            float *sD = reinterpret_cast<float *>(base);
            int2 *sKH = reinterpret_cast<int2 *>(base + (size_t)np * cols::kRowFloats * 4);
            int4 *sP = reinterpret_cast<int4 *>(base + ops.col_p_off);
            const int q_base = ops.col_q[2 * r], q_end = ops.col_q[2 * r + 1];
            const int p_base = ops.col_sb[r], p_end = ops.col_sb[r + 1];
            if (threadIdx.x < 32) {
                // the previous item's reads of these buffers came through the generic proxy
                asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
                const uint32_t kh_bytes = (uint32_t)((q_end - q_base) * 8);
                const uint32_t p_bytes = (uint32_t)((p_end - p_base) * 16 * cols::kBundleInt4);
                const uint32_t d_bytes = (uint32_t)np * cols::kRowFloats * 4;
                if (threadIdx.x == 0) {
                    tma::mbar_expect_tx(&bar, kh_bytes + p_bytes + d_bytes);
                    if (kh_bytes) tma::load_bulk(sKH, ops.col_kh + q_base, kh_bytes, &bar);
                    if (p_bytes)
                        tma::load_bulk(sP, ops.col_pieces + cols::kBundleInt4 * (size_t)p_base, p_bytes, &bar);
                    // the stage input's map: D (stage 1), da (stages 2 and 4), db (stage 3)
                    const CUtensorMap *tm = &sg.dmaps->d[STAGE == 1 ? 0 : (STAGE == 3 ? 2 : 1)];
                    for (int b = 0; b < np; b += cols::kBoxRows)
                        tma::load_3d(sD + (size_t)b * cols::kRowFloats, tm, &bar, J * cols::kCW, 0, b);
                }
            }
            const int ncb = np / cols::kCW;
            cols::cta_gain(ops, sg.mw, r * ncb + J, ncb * ops.col_splits,
                           reinterpret_cast<float *>(base + ops.col_sp_off));
            const bool ok = tma::mbar_wait(&bar, phase & 1);
            ++phase;
            if (__syncthreads_or(!ok)) {
                if (threadIdx.x == 0) atomicExch(&sg.mw.ctl->err_timeout, 1);
                tma::mbar_wait(&bar, (phase - 1) & 1);
                return;
            }
            const int warp = threadIdx.x >> 5;
            float *parts = reinterpret_cast<float *>(base + ops.col_part_off);
            cols::warp_bundles(sD, sKH, sP, p_base, ops.col_wb[r * cols::kAWarps + warp],
                               ops.col_wb[r * cols::kAWarps + warp + 1], J, np, sg.mw.X, parts);
            const int cb0 = ops.col_cutb[r], cb1 = ops.col_cutb[r + 1];
            if (cb1 > cb0) {
                __syncthreads();
                cols::combine_cuts(ops.col_cut + cb0, cb1 - cb0, parts, J, np, sg.mw.X);
            }
        }
        __syncthreads();
    }
}

// Column-block form: the epilogue over (problem, I, J, pair) items.
template <int STAGE>
__global__ void __launch_bounds__(cols::kENT, 3) b_cols_epi_kernel(const BatchGraph *gs, const Ctl *ctls,
                                                                 const int4 *items, int nitems) {
    __shared__ __align__(16) float sX1[mixed::TS * mixed::LDX];
    __shared__ __align__(16) float sX2[mixed::TS * mixed::LDX];
    __shared__ __align__(16) float sO[4 * mixed::TS * mixed::LDO];
    __shared__ float sg32[mixed::TS];
    __shared__ BatchGraph sg;
    __shared__ int s_flag;
    int4 tn = blockIdx.x < nitems ? items[blockIdx.x] : make_int4(0, 0, 0, 0);
    for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
        const int4 t = tn;
        if (it + (int)gridDim.x < nitems) tn = items[it + gridDim.x];  // the next item, in flight meanwhile
        if (!load_graph_done(gs, ctls, t.x, sg, &s_flag))
            cols::epilogue_pair<STAGE>(sg.ops, sg.mw, t.y, t.z, t.w, t.w == 0, sg.mw.npairs, sX1, sX2, sg32, sO);
        __syncthreads();
    }
}

template <int STAGE>
cudaError_t set_bcols_attr(int bytes) {
    return raise_smem_limit_t(b_cols_spmm_kernel<STAGE>, bytes);
}

template <int STAGE>
cudaError_t set_b_attr() {
    return cudaFuncSetAttribute(b_stage_mixed_kernel<STAGE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                mixed::kMixedDynSmem);
}

// Size classes of the column-block SpMM: problems whose padded edge is at
// most kClassNp[c] share one launch whose dynamic shared memory is the
// largest plan of the class, so small problems are not held to the shared
// memory (and the one CTA per SM) of the largest: up to np = 512 two CTAs fit
// an SM. Within a launch the units go largest problem first (the grid-stride
// loop then ends on short units).
constexpr int kClasses = 2;
constexpr int kClassNp[kClasses] = {512, 1 << 30};
int np_class(int np) {
    int c = 0;
    while (c + 1 < kClasses && np > kClassNp[c]) ++c;
    return c;
}

struct Lists {
    int *act;      // device, active problem indices
    int4 *items;   // device, (problem, I, J, pair index) of the active problems
    int nact, nitems;
    // per stage: column-block SpMM items (problem, J, split) per size class,
    // the pairs of the column-form problems and the pairs of the tile-form
    // problems
    int4 *items_a[kClasses];
    int na[kClasses], smem_a[kClasses], grid_a[kClasses];
    int4 *items_b, *items_t;
    int nb, nt;
};

// Device buffers one set of lists is uploaded into.
struct ListBufs {
    int *act = nullptr;
    int4 *items = nullptr, *items_a = nullptr, *items_b = nullptr, *items_t = nullptr;
};

int elem_chunks(int np) {
    const size_t tot = 2 * (size_t)np * np;
    size_t c = (tot + 256 * 8 - 1) / (256 * 8);
    return (int)std::min<size_t>(std::max<size_t>(c, 1), 64);
}

void launch_refresh(const BatchGraph *gs, const Lists &L, int max_np, cudaStream_t s, int64_t &launches,
                    const uint8_t *due = nullptr) {
    if (L.nact == 0) return;
    const dim3 eg(elem_chunks(max_np), L.nact);
    b_trace_kernel<<<L.nact, 256, 0, s>>>(gs, L.act, due);
    b_normalize_kernel<<<eg, 256, 0, s>>>(gs, L.act, due);
    b_gain64_kernel<<<L.nact, 256, 0, s>>>(gs, L.act, due);
    b_sparse64_kernel<<<std::min(L.nitems, 152 * 3), sparse64::NTHREADS, sparse64::SMEM_BYTES, s>>>(gs, L.items,
                                                                                                     L.nitems, due);
    b_post_kernel<<<eg, 256, 0, s>>>(gs, L.act, due);
    launches += 5;
}

template <int STAGE>
void launch_stage_b(const BatchGraph *gs, const Ctl *ctls, const Lists &L, cudaStream_t s, int64_t &launches) {
    bool any = false;
    for (int c = 0; c < kClasses; ++c)
        if (L.na[c]) {
            b_cols_spmm_kernel<STAGE><<<L.grid_a[c], cols::kANT, L.smem_a[c], s>>>(gs, ctls, L.items_a[c], L.na[c]);
            launches += 1;
            any = true;
        }
    if (any) {
        b_cols_epi_kernel<STAGE><<<std::min(L.nb, 152 * 3), cols::kENT, 0, s>>>(gs, ctls, L.items_b, L.nb);
        launches += 1;
    }
    if (L.nt) {
        b_stage_mixed_kernel<STAGE><<<std::min(L.nt, 152 * 3), kStageNT, mixed::kMixedDynSmem, s>>>(gs, L.items_t,
                                                                                                 L.nt);
        launches += 1;
    }
}

void launch_step(const BatchGraph *gs, const Ctl *ctls, const Lists &L, cudaStream_t s, int64_t &launches) {
    launch_stage_b<1>(gs, ctls, L, s, launches);
    launch_stage_b<2>(gs, ctls, L, s, launches);
    launch_stage_b<3>(gs, ctls, L, s, launches);
    launch_stage_b<4>(gs, ctls, L, s, launches);
}

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

bool is_device_ptr_b(const void *p) {
    cudaPointerAttributes attr;
    if (cudaPointerGetAttributes(&attr, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return attr.type == cudaMemoryTypeDevice || attr.type == cudaMemoryTypeManaged;
}

// RAII owner of every device/pinned allocation of one batched call.
struct BatchMem {
    std::vector<void *> dev;
    void *pinned = nullptr;
    cudaStream_t stream = nullptr;
    cudaEvent_t ev = nullptr;
    ~BatchMem() {
        if (stream) cudaStreamSynchronize(stream);
        for (void *p : dev) cudaFree(p);
        if (pinned) cudaFreeHost(pinned);
        if (ev) cudaEventDestroy(ev);
        if (stream) cudaStreamDestroy(stream);
        cudaGetLastError();
    }
    template <class T>
    cudaError_t alloc(T **p, size_t count) {
        void *q = nullptr;
        cudaError_t e = cudaMalloc(&q, std::max<size_t>(count, 1) * sizeof(T));
        if (e == cudaSuccess) {
            dev.push_back(q);
            *p = (T *)q;
        }
        return e;
    }
};

}  // namespace

cudaError_t init_batch() {
    cudaError_t e = cudaFuncSetAttribute(b_sparse64_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         sparse64::SMEM_BYTES);
    if (e == cudaSuccess) e = set_b_attr<1>();
    if (e == cudaSuccess) e = set_b_attr<2>();
    if (e == cudaSuccess) e = set_b_attr<3>();
    if (e == cudaSuccess) e = set_b_attr<4>();
    if (e == cudaSuccess) e = init_stage_mixed();
    return e;
}

cudaError_t bcols_ctas_per_sm(int bytes, int *ctas) {
    int n = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, b_cols_spmm_kernel<1>, cols::kANT, bytes);
    *ctas = (e == cudaSuccess && n > 0) ? n : 1;
    return e;
}

cudaError_t set_bcols_smem(int bytes) {
    cudaError_t e = set_bcols_attr<1>(bytes);
    if (e == cudaSuccess) e = set_bcols_attr<2>(bytes);
    if (e == cudaSuccess) e = set_bcols_attr<3>(bytes);
    if (e == cudaSuccess) e = set_bcols_attr<4>(bytes);
    return e;
}

}  // namespace qpr

using qpr::BatchGraph;
using qpr::Ctl;

extern "C" qpr_status qpr_batch_steady_state(int64_t count, const qpr_problem *problems, double alpha, double dt,
                                             double tol, int64_t max_steps, const qpr_options *opt,
                                             qpr_stats *stats) {
    qpr::NvtxRange nvtx_range("qpr_batch_steady_state");
    auto t0 = std::chrono::steady_clock::now();
    auto err = [&](qpr_status st, const std::string &msg) {
        qpr::set_create_error(msg);
        return st;
    };
    if (count < 1 || !problems) return err(QPR_E_ARG, "count must be >= 1 and problems non-NULL");
    if (!(alpha >= 0.0 && alpha <= 1.0)) return err(QPR_E_ARG, "alpha must lie in [0, 1]");
    if (!(dt > 0.0) || !std::isfinite(dt)) return err(QPR_E_ARG, "dt must be positive and finite");
    if (!(tol > 0.0)) return err(QPR_E_ARG, "tol must be positive");
    if (max_steps < 0) return err(QPR_E_ARG, "max_steps must be non-negative");
    qpr_options o;
    qpr_default_options(&o);
    if (opt) o = *opt;
    if (o.ref_refresh < 1 || o.ref_refresh > 4096) return err(QPR_E_ARG, "ref_refresh outside [1, 4096]");
    if (o.h_diag != QPR_HDIAG_ZERO && o.h_diag != QPR_HDIAG_NEG_OUTDEG) return err(QPR_E_ARG, "unknown h_diag mode");
    if (o.dangling != QPR_DANGLING_F && o.dangling != QPR_DANGLING_UNIFORM)
        return err(QPR_E_ARG, "unknown dangling mode");

    // ---- host assembly, per problem ----
    const size_t G = (size_t)count;
    std::vector<qpr::HostOps> H(G);
    std::vector<int> np(G), T(G), npairs(G);
    std::vector<std::vector<int>> rowseg(G);
    std::vector<std::vector<int2>> segs(G);
    std::vector<double> hdt(G);
    std::vector<int64_t> msub(G);
    for (size_t g = 0; g < G; ++g) {
        const qpr_problem &p = problems[g];
        if (p.n < 2 || p.n > 65536) return err(QPR_E_ARG, "problem " + std::to_string(g) + ": n outside [2, 65536]");
        if (!(p.omega >= 0.0 && p.omega <= 1.0))
            return err(QPR_E_ARG, "problem " + std::to_string(g) + ": omega must lie in [0, 1]");
        if (!p.rho) return err(QPR_E_ARG, "problem " + std::to_string(g) + ": rho is NULL");
        if (p.m < 0 || (p.m > 0 && (!p.src || !p.dst)))
            return err(QPR_E_ARG, "problem " + std::to_string(g) + ": edge arrays missing");
        std::string aerr;
        const qpr_status ast = qpr::assemble_host(p.n, p.m, p.src, p.dst, p.w, o.h_diag, H[g], aerr);
        if (ast != QPR_OK) return err(ast, "problem " + std::to_string(g) + ": " + aerr);
        np[g] = (int)(((p.n + qpr::kPadFp64 - 1) / qpr::kPadFp64) * qpr::kPadFp64);
        qpr::row_segments(H[g], np[g], 32, rowseg[g], segs[g]);
        T[g] = np[g] / qpr::kTileFp64;
        npairs[g] = T[g] * (T[g] + 1) / 2;
        double cmax = 0.0;
        qpr::column_sums_G(H[g], alpha, np[g], &cmax);
        const double spread = qpr::estimate_spread(p.n, H[g].hptr, H[g].hcol, H[g].hval);
        const double rate = (1.0 - p.omega) * spread + 2.0 * p.omega * cmax;
        const double dmax = rate > 0.0 ? 2.5 / rate : INFINITY;
        msub[g] = (dt > dmax) ? (int64_t)ceil(dt / dmax) : 1;
        hdt[g] = dt / (double)msub[g];
    }

    // ---- arena layout (elements), every sub-array aligned to 64 elements ----
    std::vector<size_t> od(G), of(G), oi(G), ob(G);
    size_t nd = 0, nf = 0, ni = 0, nb = 0, max_nn = 0;
    int max_np = 0;
    for (size_t g = 0; g < G; ++g) {
        const size_t p2 = 2 * (size_t)np[g] * np[g];
        const size_t nh = H[g].hval.size(), ns = H[g].sval.size(), n = (size_t)problems[g].n;
        od[g] = nd;
        nd += qpr::align_up(2 * p2 + 2 * np[g] + nh + ns + npairs[g], 64);
        of[g] = nf;
        nf += qpr::align_up(7 * p2 + 3 * np[g] + qpr::align_up(nh, 64) + qpr::align_up(ns, 64) + npairs[g], 64) + 64;
        oi[g] = ni;
        ni += qpr::align_up(2 * (n + 1) + nh + ns, 64) + qpr::align_up((size_t)np[g] + 1, 64) + 2 * segs[g].size();
        ni = qpr::align_up(ni, 64);
        ob[g] = nb;
        nb += qpr::align_up(n, 64);
        max_nn = std::max(max_nn, n * n);
        max_np = std::max(max_np, np[g]);
    }

    int dev = o.device;
    if (dev < 0 && cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return err(QPR_E_CUDA, "no CUDA device available");
    }
    int prev_dev = -1;
    cudaGetDevice(&prev_dev);
    if (prev_dev != dev) cudaSetDevice(dev);
    struct Restore {
        int d;
        ~Restore() {
            if (d >= 0) cudaSetDevice(d);
        }
    } restore{prev_dev != dev ? prev_dev : -1};

    // ---- column-block plans: the same decision as a single-problem solve ----
    std::vector<qpr::ColPlan> plans(G);
    std::vector<char> colg(G, 0);
    std::vector<size_t> okh(G), oci(G), opc(G), oxc(G);
    size_t nkh = 0, nci = 0, npc = 0, nxc = 0, na_max = 0;
    int smem_a = 0;
    int smem_class[qpr::kClasses] = {};
    for (size_t g = 0; g < G; ++g) {
        // one split where it fits: the batch fills the SMs with many problems
        if (o.sparse_form == QPR_SPARSE_FORM_TILES || !qpr::plan_columns(H[g], np[g], dev, plans[g], 1)) {
            if (o.sparse_form == QPR_SPARSE_FORM_COLUMNS || o.sparse_form == QPR_SPARSE_FORM_COLUMNS_PERSISTENT)
                return err(QPR_E_ARG, "problem " + std::to_string(g) +
                                          ": sparse_form COLUMNS does not fit one CTA's shared memory");
            continue;
        }
        const qpr::ColPlan &pl = plans[g];
        colg[g] = 1;
        okh[g] = nkh;
        nkh += pl.kh.size();
        oci[g] = nci;
        nci += pl.q.size() + pl.sb.size() + pl.wb.size() + pl.cutb.size();
        opc[g] = npc;
        npc += pl.pieces.size() + pl.cuts.size();
        oxc[g] = nxc;
        nxc += qpr::align_up(2 * (size_t)np[g] * np[g], 64);
        na_max += (size_t)(np[g] / qpr::cols::kCW) * pl.splits;
        smem_a = std::max(smem_a, pl.smem);
        smem_class[qpr::np_class(np[g])] = std::max(smem_class[qpr::np_class(np[g])], pl.smem);
    }

    qpr::BatchMem mem;
    double *dD = nullptr;
    float *dF = nullptr;
    int *dI = nullptr;
    unsigned char *dB = nullptr;
    Ctl *dCtl = nullptr;
    BatchGraph *dG = nullptr;
    double *dIO = nullptr;
    size_t total_pairs = 0;
    for (size_t g = 0; g < G; ++g) total_pairs += npairs[g];
#define BCUDA(call)                                                                             \
    do {                                                                                        \
        cudaError_t e_ = (call);                                                                \
        if (e_ != cudaSuccess)                                                                  \
            return err(e_ == cudaErrorMemoryAllocation ? QPR_E_OOM : QPR_E_CUDA,                \
                       std::string(#call) + ": " + cudaGetErrorString(e_));                     \
    } while (0)
    BCUDA(qpr::init_stage_sparse());
    BCUDA(qpr::init_batch());
    BCUDA(mem.alloc(&dD, nd));
    BCUDA(mem.alloc(&dF, nf));
    BCUDA(mem.alloc(&dI, ni));
    BCUDA(mem.alloc(&dB, nb));
    BCUDA(mem.alloc(&dCtl, G));
    BCUDA(mem.alloc(&dG, G));
    qpr::ListBufs gbuf, abuf;  // lists of the captured graph; lists of ad-hoc launches (confirming refreshes)
    uint8_t *dDue = nullptr;
    BCUDA(mem.alloc(&gbuf.act, G));
    BCUDA(mem.alloc(&gbuf.items, total_pairs));
    BCUDA(mem.alloc(&abuf.act, G));
    BCUDA(mem.alloc(&abuf.items, total_pairs));
    BCUDA(mem.alloc(&dDue, G));
    BCUDA(mem.alloc(&dIO, 2 * max_nn));
    int2 *dKH = nullptr;
    int *dCI = nullptr;
    int4 *dPC = nullptr;
    float *dXC = nullptr;
    BCUDA(mem.alloc(&dKH, nkh));
    BCUDA(mem.alloc(&dCI, nci));
    BCUDA(mem.alloc(&dPC, npc));
    BCUDA(mem.alloc(&dXC, nxc));
    for (qpr::ListBufs *b : {&gbuf, &abuf}) {
        BCUDA(mem.alloc(&b->items_a, na_max));
        BCUDA(mem.alloc(&b->items_b, total_pairs));
        BCUDA(mem.alloc(&b->items_t, total_pairs));
    }
    // CTAs per SM of each class's SpMM launch (its dynamic shared memory)
    int sms = 0, class_ctas[qpr::kClasses];
    for (int &c : class_ctas) c = 1;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) sms = 1;
    if (nxc) BCUDA(cudaMemset(dXC, 0, nxc * sizeof(float)));
    if (smem_a > 0) {
        BCUDA(qpr::set_bcols_smem(smem_a));
        for (int c = 0; c < qpr::kClasses; ++c)
            if (smem_class[c] > 0) BCUDA(qpr::bcols_ctas_per_sm(smem_class[c], &class_ctas[c]));
    }
    for (size_t g = 0; g < G; ++g) {
        if (!colg[g]) continue;
        const qpr::ColPlan &pl = plans[g];
        std::vector<int> ints(pl.q);
        ints.insert(ints.end(), pl.sb.begin(), pl.sb.end());
        ints.insert(ints.end(), pl.wb.begin(), pl.wb.end());
        ints.insert(ints.end(), pl.cutb.begin(), pl.cutb.end());
        std::vector<int4> pcs(pl.pieces);
        pcs.insert(pcs.end(), pl.cuts.begin(), pl.cuts.end());
        BCUDA(cudaMemcpy(dKH + okh[g], pl.kh.data(), pl.kh.size() * sizeof(int2), cudaMemcpyHostToDevice));
        BCUDA(cudaMemcpy(dCI + oci[g], ints.data(), ints.size() * sizeof(int), cudaMemcpyHostToDevice));
        if (!pcs.empty())
            BCUDA(cudaMemcpy(dPC + opc[g], pcs.data(), pcs.size() * sizeof(int4), cudaMemcpyHostToDevice));
    }
    BCUDA(cudaMemset(dD, 0, nd * sizeof(double)));
    BCUDA(cudaMemset(dF, 0, nf * sizeof(float)));
    BCUDA(cudaStreamCreateWithFlags(&mem.stream, cudaStreamNonBlocking));
    BCUDA(cudaEventCreateWithFlags(&mem.ev, cudaEventDisableTiming));
    BCUDA(cudaMallocHost(&mem.pinned, G * sizeof(Ctl)));
    cudaStream_t s = mem.stream;
    BCUDA(cudaEventRecord(mem.ev, (cudaStream_t)o.cuda_stream));
    BCUDA(cudaStreamWaitEvent(s, mem.ev, 0));

    // ---- fill and upload the operators, build the descriptors ----
    std::vector<double> hD(nd, 0.0);
    std::vector<float> hF(nf, 0.0f);
    std::vector<int> hI(ni, 0);
    std::vector<unsigned char> hB(nb, 0);
    std::vector<BatchGraph> desc(G);
    Ctl *hCtl = (Ctl *)mem.pinned;
    memset(hCtl, 0, G * sizeof(Ctl));
    for (size_t g = 0; g < G; ++g) {
        const qpr::HostOps &h = H[g];
        const int n = (int)problems[g].n, p = np[g];
        const size_t p2 = 2 * (size_t)p * p, nh = h.hval.size(), ns = h.sval.size();
        double *bd = dD + od[g];
        float *bf = dF + of[g];
        int *bi = dI + oi[g];
        // double arena: R F | g64 c | hval sval | partials
        double *R = bd, *F = bd + p2, *g64 = bd + 2 * p2, *c = g64 + p;
        double *hval = c + p, *sval = hval + nh, *part = sval + ns;
        std::vector<double> cg = qpr::column_sums_G(h, alpha, p, nullptr);
        std::copy(cg.begin(), cg.end(), hD.begin() + (c - dD));
        std::copy(h.hval.begin(), h.hval.end(), hD.begin() + (hval - dD));
        std::copy(h.sval.begin(), h.sval.end(), hD.begin() + (sval - dD));
        // float arena: F32 D Dlo da db Ghi Glo | g32 pv32 c32 | hval32 | sval32 | partials32
        // (uploaded from zeros, so the delta D + Dlo starts at 0)
        float *F32 = bf, *Dp = bf + p2, *Dlo = bf + 2 * p2, *da = bf + 3 * p2, *db = bf + 4 * p2;
        float *Ghi = bf + 5 * p2, *Glo = bf + 6 * p2;
        float *g32 = bf + 7 * p2, *pv32 = g32 + p, *c32 = pv32 + p, *hv32 = c32 + p;
        float *sv32 = hv32 + qpr::align_up(nh, 64), *part32 = sv32 + qpr::align_up(ns, 64);
        for (int j = 0; j < p; ++j) hF[(c32 - dF) + j] = (float)cg[j];
        for (size_t q = 0; q < nh; ++q) hF[(hv32 - dF) + q] = (float)h.hval[q];
        for (size_t q = 0; q < ns; ++q) hF[(sv32 - dF) + q] = (float)h.sval[q];
        // int arena: hptr hcol sptr scol | rowseg | seg (pairs of ints)
        int *hptr = bi, *hcol = hptr + (n + 1), *sptr = hcol + nh, *scol = sptr + (n + 1);
        int *rseg = bi + qpr::align_up(2 * (size_t)(n + 1) + nh + ns, 64);
        int *sg = rseg + qpr::align_up((size_t)p + 1, 64);
        std::copy(rowseg[g].begin(), rowseg[g].end(), hI.begin() + (rseg - dI));
        for (size_t q = 0; q < segs[g].size(); ++q) {
            hI[(sg - dI) + 2 * q] = segs[g][q].x;
            hI[(sg - dI) + 2 * q + 1] = segs[g][q].y;
        }
        for (int i = 0; i <= n; ++i) hI[(hptr - dI) + i] = (int)h.hptr[i];
        std::copy(h.hcol.begin(), h.hcol.end(), hI.begin() + (hcol - dI));
        std::copy(h.sptr.begin(), h.sptr.end(), hI.begin() + (sptr - dI));
        std::copy(h.scol.begin(), h.scol.end(), hI.begin() + (scol - dI));
        std::copy(h.dang.begin(), h.dang.end(), hB.begin() + ob[g]);

        BatchGraph &d = desc[g];
        memset(&d, 0, sizeof(d));
        d.ops.n = n;
        d.ops.np = p;
        d.ops.alpha = alpha;
        d.ops.omega = problems[g].omega;
        d.ops.dangling = o.dangling;
        d.ops.H = nullptr;
        d.ops.h_ptr = hptr;
        d.ops.h_col = hcol;
        d.ops.h_val = hval;
        d.ops.h_val32 = hv32;
        d.ops.rowseg = rseg;
        d.ops.seg = reinterpret_cast<const int2 *>(sg);
        d.ops.s_ptr = sptr;
        d.ops.s_col = scol;
        d.ops.s_val = sval;
        d.ops.dang = dB + ob[g];
        d.ops.c = c;
        d.ops.c32 = c32;
        if (colg[g]) {
            const qpr::ColPlan &pl = plans[g];
            d.ops.col_kh = dKH + okh[g];
            d.ops.col_q = dCI + oci[g];
            d.ops.col_sb = dCI + oci[g] + pl.q.size();
            d.ops.col_wb = dCI + oci[g] + pl.q.size() + pl.sb.size();
            d.ops.col_pieces = dPC + opc[g];
            d.ops.col_cutb = dCI + oci[g] + pl.q.size() + pl.sb.size() + pl.wb.size();
            d.ops.col_cut = dPC + opc[g] + pl.pieces.size();
            d.ops.col_part_off = pl.part_off;
            d.ops.col_splits = pl.splits;
            d.ops.col_smem = pl.smem;
            d.ops.col_p_off = pl.p_off;
            d.ops.col_sp_off = pl.sp_off;
        }
        d.ops.s_val32 = sv32;
        d.ops.alpha32 = (float)alpha;
        d.ops.oma32 = (float)(1.0 - alpha);
        d.ops.omega32 = (float)problems[g].omega;
        d.ops.inv_nm1_32 = (float)(1.0 / (double)(n - 1));
        d.ops.inv_n32 = (float)(1.0 / (double)n);
        qpr::MixedWork &mw = d.mw;
        mw.R = R; mw.F = F;
        mw.F32 = F32; mw.D = Dp; mw.Dlo = Dlo; mw.da = da; mw.db = db; mw.Ghi = Ghi; mw.Glo = Glo;
        mw.g = g32; mw.pv = pv32; mw.g64 = g64; mw.partials = part; mw.partials32 = part32;
        mw.X = colg[g] ? dXC + oxc[g] : nullptr;
        mw.pairs = nullptr; mw.npairs = npairs[g]; mw.tiles = T[g];
        mw.ctl = dCtl + g;
        mw.nstage_partials = npairs[g];
        qpr::Work &w = d.w64;
        w.y = R; w.z = F; w.ya = R; w.yb = R; w.g = g64; w.partials = part;
        w.pairs = nullptr; w.npairs = npairs[g]; w.tiles = T[g]; w.ctl = dCtl + g;
        Ctl &k = hCtl[g];
        k.max_steps = max_steps;
        k.tol = tol;
        k.dt = hdt[g];
        k.scale = 1.0;
        k.resid_exact_step = -1;
    }
    BCUDA(cudaMemcpyAsync(dD, hD.data(), nd * sizeof(double), cudaMemcpyHostToDevice, s));
    BCUDA(cudaMemcpyAsync(dF, hF.data(), nf * sizeof(float), cudaMemcpyHostToDevice, s));
    BCUDA(cudaMemcpyAsync(dI, hI.data(), ni * sizeof(int), cudaMemcpyHostToDevice, s));
    BCUDA(cudaMemcpyAsync(dB, hB.data(), nb, cudaMemcpyHostToDevice, s));
    // the column form's tensor maps (D, da, db of each problem), read by the
    // SpMM kernels from device memory
    qpr::ColMaps *dMaps = nullptr;
    BCUDA(mem.alloc(&dMaps, G));
    std::vector<qpr::ColMaps> hMaps(G);
    memset(hMaps.data(), 0, G * sizeof(qpr::ColMaps));
    for (size_t g = 0; g < G; ++g) {
        if (!colg[g]) continue;
        const float *din[3] = {desc[g].mw.D, desc[g].mw.da, desc[g].mw.db};
        if (!qpr::make_col_maps(desc[g].ops, din, &hMaps[g])) return err(QPR_E_CUDA, "cuTensorMapEncodeTiled failed");
        desc[g].dmaps = dMaps + g;
    }
    BCUDA(cudaMemcpyAsync(dMaps, hMaps.data(), G * sizeof(qpr::ColMaps), cudaMemcpyHostToDevice, s));
    BCUDA(cudaMemcpyAsync(dG, desc.data(), G * sizeof(BatchGraph), cudaMemcpyHostToDevice, s));
    BCUDA(cudaMemcpyAsync(dCtl, hCtl, G * sizeof(Ctl), cudaMemcpyHostToDevice, s));
    int64_t launches = 0;
    // ---- initial states ----
    for (size_t g = 0; g < G; ++g) {
        const int n = (int)problems[g].n;
        const double *srcp = (const double *)problems[g].rho;
        if (!qpr::is_device_ptr_b(problems[g].rho)) {
            BCUDA(cudaMemcpyAsync(dIO, problems[g].rho, (size_t)n * n * 16, cudaMemcpyHostToDevice, s));
            srcp = dIO;
        }
        qpr::launch_import(srcp, n, np[g], desc[g].mw.R, s);
        ++launches;
    }
    BCUDA(cudaStreamSynchronize(s));  // hD, hF, ... and the staging buffer may be released / reused

    // ---- blocks of (exact refresh + ref_refresh delta steps) ----
    std::vector<int> active(G);
    for (size_t g = 0; g < G; ++g) active[g] = (int)g;
    std::vector<int4> items, items_b, items_t;
    items.reserve(total_pairs);
    std::vector<int4> items_cls[qpr::kClasses];
    auto make_lists = [&](const std::vector<int> &list, const qpr::ListBufs &bufs, qpr::Lists &L) -> cudaError_t {
        items.clear();
        for (int g : list) {
            int q = 0;
            for (int I = 0; I < T[g]; ++I)
                for (int J = I + 1; J < T[g]; ++J) items.push_back(make_int4(g, I, J, q++));
            for (int I = 0; I < T[g]; ++I) items.push_back(make_int4(g, I, I, q++));
        }
        items_b.clear();
        items_t.clear();
        for (int c = 0; c < qpr::kClasses; ++c) items_cls[c].clear();
        for (const int4 &t : items) (colg[t.x] ? items_b : items_t).push_back(t);
        std::vector<int> by_size(list);
        std::stable_sort(by_size.begin(), by_size.end(), [&](int a, int b) { return np[a] > np[b]; });
        for (int g : by_size)
            if (colg[g])
                for (int r = 0; r < plans[g].splits; ++r)
                    for (int J = 0; J < np[g] / qpr::cols::kCW; ++J)
                        items_cls[qpr::np_class(np[g])].push_back(make_int4(g, J, r, 0));
        L.act = bufs.act;
        L.items = bufs.items;
        L.nact = (int)list.size();
        L.nitems = (int)items.size();
        size_t off = 0;
        for (int c = 0; c < qpr::kClasses; ++c) {
            L.items_a[c] = bufs.items_a + off;
            L.na[c] = (int)items_cls[c].size();
            L.smem_a[c] = smem_class[c];
            L.grid_a[c] = std::max(1, std::min(L.na[c], sms * class_ctas[c]));
            off += items_cls[c].size();
        }
        L.items_b = bufs.items_b;
        L.items_t = bufs.items_t;
        L.nb = (int)items_b.size();
        L.nt = (int)items_t.size();
        cudaError_t e = cudaMemcpyAsync(bufs.act, list.data(), list.size() * sizeof(int), cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(bufs.items, items.data(), items.size() * sizeof(int4), cudaMemcpyHostToDevice, s);
        for (int c = 0; c < qpr::kClasses && e == cudaSuccess; ++c)
            if (!items_cls[c].empty())
                e = cudaMemcpyAsync(L.items_a[c], items_cls[c].data(), items_cls[c].size() * sizeof(int4),
                                    cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess && !items_b.empty())
            e = cudaMemcpyAsync(bufs.items_b, items_b.data(), items_b.size() * sizeof(int4), cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess && !items_t.empty())
            e = cudaMemcpyAsync(bufs.items_t, items_t.data(), items_t.size() * sizeof(int4), cudaMemcpyHostToDevice, s);
        // the host vectors are reused: wait until the copies have read them
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        return e;
    };
    bool timeout = false;
    // per problem, the refresh window of a single-problem steady-state solve
    // (adaptive_refresh: the same rule on the same residuals, so the same
    // refresh steps): refresh before the next block, steps since the last
    // refresh, residual estimate after the first block
    const int block = o.ref_refresh;
    const bool adaptive = o.adaptive_refresh != 0;
    std::vector<char> due(G, 1);
    std::vector<int64_t> since(G, 0);
    std::vector<double> r0(G, -1.0);
    // The captured block: the refresh kernels (a problem's refresh runs when
    // its due flag is set; the host writes the flags before each launch) and
    // `block` steps, over the lists of the active set at capture time.
    // Problems that stop later keep their items in the lists (their kernels
    // return at once, the device retires them) until the lists are rebuilt
    // and the graph recaptured, once the active set has shrunk by a quarter.
    qpr::Lists LG{};
    cudaGraphExec_t gexec = nullptr;
    struct GraphGuard {
        cudaGraphExec_t *g;
        ~GraphGuard() {
            if (*g) cudaGraphExecDestroy(*g);
        }
    } gguard{&gexec};
    int64_t graph_launches = 0;
    size_t captured = 0;
    std::vector<uint8_t> hDue(G, 0);
    auto recapture = [&]() -> cudaError_t {
        if (gexec) {
            cudaGraphExecDestroy(gexec);
            gexec = nullptr;
        }
        cudaError_t e = make_lists(active, gbuf, LG);
        if (e != cudaSuccess) return e;
        captured = active.size();
        graph_launches = 0;
        cudaGraph_t gr = nullptr;
        e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) return e;
        qpr::launch_refresh(dG, LG, max_np, s, graph_launches, dDue);
        for (int k = 0; k < block; ++k) qpr::launch_step(dG, dCtl, LG, s, graph_launches);
        e = cudaStreamEndCapture(s, &gr);
        if (e != cudaSuccess) return e;
        e = cudaGraphInstantiate(&gexec, gr, 0);
        cudaGraphDestroy(gr);
        if (e != cudaSuccess) gexec = nullptr;
        return e;
    };
    BCUDA(recapture());
    while (!active.empty()) {
        qpr::NvtxRange nvtx_block("batch block");
        for (int g : active) hDue[g] = due[g] ? 1 : 0;
        BCUDA(cudaMemcpyAsync(dDue, hDue.data(), G, cudaMemcpyHostToDevice, s));
        BCUDA(cudaGraphLaunch(gexec, s));
        launches += graph_launches;
        for (int g : active) since[g] = (due[g] ? 0 : since[g]) + block;
        BCUDA(cudaMemcpyAsync(hCtl, dCtl, G * sizeof(Ctl), cudaMemcpyDeviceToHost, s));
        BCUDA(cudaStreamSynchronize(s));
        BCUDA(cudaGetLastError());
        std::vector<int> keep, confirm;
        for (int g : active) {
            const Ctl &k = hCtl[g];
            if (k.err_timeout) timeout = true;
            if (!k.done) {
                keep.push_back(g);
                due[g] = 1;
                if (adaptive) {
                    const double r = k.resid;
                    if (r0[g] < 0.0) r0[g] = r;
                    const double next = (double)(since[g] + block);
                    due[g] = !(r > 0.0 && next <= (double)qpr::kMaxRefreshGrowth * block &&
                               next * next * r <= (double)block * block * r0[g]);
                }
            } else if (k.status == qpr::kCtlNonFinite) {
                continue;
            } else if (k.resid_exact_step == k.step) {
                continue;  // decided by an exact refresh
            } else {
                confirm.push_back(g);
            }
        }
        if (!confirm.empty()) {
            for (int g : confirm) {
                hCtl[g].done = 0;
                hCtl[g].status = qpr::kCtlRunning;
            }
            BCUDA(cudaMemcpyAsync(dCtl, hCtl, G * sizeof(Ctl), cudaMemcpyHostToDevice, s));
            qpr::Lists Lc{};
            BCUDA(make_lists(confirm, abuf, Lc));
            qpr::launch_refresh(dG, Lc, max_np, s, launches);
            BCUDA(cudaMemcpyAsync(hCtl, dCtl, G * sizeof(Ctl), cudaMemcpyDeviceToHost, s));
            BCUDA(cudaStreamSynchronize(s));
            BCUDA(cudaGetLastError());
            for (int g : confirm)
                if (!hCtl[g].done) {
                    keep.push_back(g);
                    due[g] = adaptive ? 0 : 1;  // stepping on from this refresh
                    since[g] = 0;
                }
        }
        std::sort(keep.begin(), keep.end());
        active.swap(keep);
        if (!active.empty() && 4 * active.size() <= 3 * captured) BCUDA(recapture());
    }

    // ---- results ----
    qpr_status ret = QPR_OK;
    for (size_t g = 0; g < G; ++g) {
        const int n = (int)problems[g].n;
        if (qpr::is_device_ptr_b(problems[g].rho)) {
            qpr::launch_export(desc[g].mw.R, n, np[g], dCtl + g, 0, (double *)problems[g].rho, s);
        } else {
            qpr::launch_export(desc[g].mw.R, n, np[g], dCtl + g, 0, dIO, s);
            BCUDA(cudaMemcpyAsync(problems[g].rho, dIO, (size_t)n * n * 16, cudaMemcpyDeviceToHost, s));
        }
        ++launches;
        BCUDA(cudaStreamSynchronize(s));
        const Ctl &k = hCtl[g];
        if (k.status == qpr::kCtlNonFinite) ret = QPR_E_NONFINITE;
        else if (k.status != qpr::kCtlConverged && ret == QPR_OK) ret = QPR_E_NOT_CONVERGED;
    }
    const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    if (stats) {
        for (size_t g = 0; g < G; ++g) {
            const Ctl &k = hCtl[g];
            qpr_stats &st = stats[g];
            memset(&st, 0, sizeof(st));
            st.steps = k.step;
            st.substeps_m = msub[g];
            st.t = (double)k.step * hdt[g];
            st.residual = k.resid_exact;
            st.trace_before = k.trace;
            st.seconds = secs;
            st.kernel_launches = launches;
            st.converged = (k.status == qpr::kCtlConverged) ? 1 : 0;
        }
    }
#undef BCUDA
    if (timeout) return err(QPR_E_TIMEOUT, "a device-side wait gave up");
    if (ret == QPR_E_NONFINITE) return err(ret, "a problem produced a non-finite trace or residual");
    if (ret == QPR_E_NOT_CONVERGED) return err(ret, "some problems reached max_steps");
    return QPR_OK;
}
