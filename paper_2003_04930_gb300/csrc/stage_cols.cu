// Column-block form of the sparse mixed stage for one problem (see
// cols_body.cuh): the SpMM kernel stages delta[:, J] with a 3-D TMA box
// (rows of 16 real then 16 imaginary values), its split's CSR entries and
// its work list with bulk copies, and forms X[:, J] = H delta[:, J] for its
// rows; the epilogue kernel applies the RK4 stage per tile pair. Each step
// is 8 launches (SpMM + epilogue per stage); the SpMM grid's leading CTAs
// form the gain G p of the stage input on the SMs the product leaves free.
//
// The SpMM reads each column block once per row split (about splits x 8 N^2
// bytes of L2 traffic per stage) instead of gathering a row slice of delta
// from L2 for every (nonzero, column tile) pair (nnz x 8 N bytes), and its
// inner loop is two shared-memory reads and four FMAs per nonzero.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <mutex>
#include <vector>

#include "cols_body.cuh"
#include "cols_spmm.cuh"
#include "qpr_internal.cuh"
#include "tma_util.cuh"

namespace qpr {
namespace {

using namespace cols;

// The SpMM kernels: the first ops.col_gain_ctas CTAs form the gain of the
// stage input (gain_role), the others one (column block, row split) unit of
// the product each (whole block: unit u = block u % ncb of split u / ncb;
// gather: the splits of a block side by side).
// (timeline::enter / leave and the body's marks record the kernel timeline
// in the diagnostic build only; they are empty otherwise)
template <int STAGE>
__global__ void __launch_bounds__(kANT) cols_spmm_kernel(const __grid_constant__ CUtensorMap tm, DevOps ops,
                                                         MixedWork w) {
    timeline::enter((STAGE - 1) * 2);
    const int b = blockIdx.x, ng = ops.col_gain_ctas;
    if (b < ng) {
        gain_role<STAGE == 2>(ops, w, b, ng, [&] { return w.pv; });
    } else {
        const int u = b - ng, ncb = ops.np / kCW;
        spmm_block_body<true>([&] { return &tm; }, ops, w, u % ncb, u / ncb);
    }
    timeline::leave();
}

template <int STAGE>
__global__ void __launch_bounds__(kANT, kGatherCtasPerSm) cols_gather_kernel(DevOps ops, MixedWork w) {
    timeline::enter((STAGE - 1) * 2);
    const int b = blockIdx.x, ng = ops.col_gain_ctas;
    if (b < ng) {
        gain_role<STAGE == 2>(ops, w, b, ng, [&] { return w.pv; });
    } else {
        const int u = b - ng;
        spmm_gather_body([&] { return stage_input<STAGE>(w); }, ops, w, u % ops.col_splits, u / ops.col_splits);
    }
    timeline::leave();
}

static_assert(kANT == kENT, "the stop decision sums the residual partials with the same block size in the "
                            "stage-2 SpMM grid as in a stage-1 epilogue CTA");

// Launched with programmatic dependent launch: the elementwise operands (the
// stage input, F32, D, S, ...: written two kernels back, complete once the
// SpMM kernel has passed its own dependency wait) are loaded before
// grid_dependency_wait; X, the gain and the stop flag after it, together.
template <int STAGE>
__global__ void __launch_bounds__(kENT, 3) cols_epi_kernel(DevOps ops, MixedWork w) {
    __shared__ __align__(16) float sX1[TS * LDX];
    __shared__ __align__(16) float sX2[TS * LDX];
    __shared__ __align__(16) float sO[4 * TS * LDO];
    __shared__ float sg[TS];
    __shared__ int s_done;
    timeline::enter((STAGE - 1) * 2 + 1);
    const int4 pr = w.epi_pairs[blockIdx.x];  // {I, J, partial slot}
    mixed::EpiIn<STAGE, kENT> in;
    mixed::epi_load<STAGE, kENT>(ops, w, pr.x, pr.y, in);
    tma::grid_dependency_wait();
    tma::launch_dependents();
    // the stop flag and the X tiles in one round trip (X is read whatever the
    // flag says; nothing is written unless the run goes on)
    const int done = (threadIdx.x == 0) ? *(volatile int *)&w.ctl->done : 0;
    epilogue_load_x(ops, w, pr.x, pr.y, sX1, sX2, sg);
    if (threadIdx.x == 0) s_done = done;
    __syncthreads();
    if (!s_done) {
        // no ticket: the stage-2 SpMM grid takes the stop decision (gain_role)
        epilogue_pair_staged<STAGE, false>(ops, w, pr.x, pr.y, pr.z, blockIdx.x == 0, w.npairs, sX1, sX2, sg, sO,
                                           in);
    }
    timeline::leave();
}

int max_smem_optin(int device) {
    int v = 0;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, device) != cudaSuccess) {
        cudaGetLastError();
        v = 0;
    }
    return v;
}


// The entries of row i (column relative to c0, FP32 value bits).
using RowEntries = std::vector<std::vector<int2>>;

// Bundles of one split's rows [r0, r1) with the entries ent[i - r0]: long
// rows alone, the others groups x rpg at a time by decreasing length; dealt
// to the warps longest first, each to the least loaded warp. Appends, per
// warp, the bundles' descriptors and their interleaved, zero-padded entries
// (relative offsets from `kh_base`), and the warps' first bundles.
// skip_empty: rows without entries get no bundle (their sums are kept
// elsewhere); otherwise they get zero rounds, which store zeros. part_max >
// 0: rows longer than part_max are cut into parts (bundles whose sums go to
// partial slots 0, 1, ... of this block); each cut row appends {row, first
// slot, parts, 0} to `cuts`. Returns the number of partial slots.
// groups x rpg: row slots per round of a bundle, 8 x 1 (the whole-block
// layout: one per lane quad) or 2 x kRPG (the gather layout: kRPG per group
// pair).
int split_bundles(int r0, int r1, const RowEntries &ent, size_t kh_base, std::vector<int2> &kh,
                  std::vector<int4> &pieces, std::vector<int> &wb, std::vector<int4> &cuts, int part_max,
                  bool skip_empty, int groups, int rpg) {
    constexpr int kMaxSlots = 4 * (kBundleInt4 - 1);
    const int kSlots = groups * rpg;
    if (kSlots > kMaxSlots) return -1;
    struct Bundle {
        int rows[kMaxSlots];
        int T;
        bool lng, part;
        int src, e0, e1;  // long rows and parts: the row and its entries [e0, e1)
        long long cost;
    };
    std::vector<Bundle> bs;
    std::vector<int> shortrows;
    int nslots = 0;
    auto row_len = [&](int i) { return (int)ent[i - r0].size(); };
    auto fresh = [&](int T, bool lng) {
        Bundle b;
        for (int j = 0; j < kMaxSlots; ++j) b.rows[j] = -1;
        b.T = T;
        b.lng = lng;
        b.part = false;
        b.src = -1;
        b.e0 = b.e1 = 0;
        b.cost = (long long)rpg * T + 8;
        return b;
    };
    for (int i = r0; i < r1; ++i) {
        const int len = row_len(i);
        if (part_max > 0 && len > part_max) {
            // parts [k len / P, (k + 1) len / P) of the row's entries, in order
            const int P = (len + part_max - 1) / part_max;
            cuts.push_back(make_int4(i, nslots, P, 0));
            for (int k = 0; k < P; ++k) {
                const int e0 = (int)((long long)k * len / P), e1 = (int)((long long)(k + 1) * len / P);
                Bundle b = fresh((e1 - e0 + kSlots - 1) / kSlots, true);
                b.part = true;
                b.rows[0] = nslots + k;
                b.src = i;
                b.e0 = e0;
                b.e1 = e1;
                bs.push_back(b);
            }
            nslots += P;
        } else if (len > kLongRow) {
            Bundle b = fresh((len + kSlots - 1) / kSlots, true);
            b.rows[0] = i;
            b.src = i;
            b.e1 = len;
            bs.push_back(b);
        } else if (len > 0 || !skip_empty) {
            shortrows.push_back(i);
        }
    }
    std::stable_sort(shortrows.begin(), shortrows.end(), [&](int a, int b) { return row_len(a) > row_len(b); });
    for (size_t k = 0; k < shortrows.size(); k += kSlots) {
        Bundle b = fresh(row_len(shortrows[k]), false);
        for (int j = 0; j < kSlots; ++j)
            if (k + j < shortrows.size()) b.rows[j] = shortrows[k + j];
        bs.push_back(b);
    }
    std::stable_sort(bs.begin(), bs.end(), [](const Bundle &a, const Bundle &b) { return a.cost > b.cost; });
    std::vector<std::vector<int>> per(kAWarps);
    std::vector<long long> load(kAWarps, 0);
    for (int k = 0; k < (int)bs.size(); ++k) {
        const int wmin = (int)(std::min_element(load.begin(), load.end()) - load.begin());
        per[wmin].push_back(k);
        load[wmin] += bs[k].cost;
    }
    for (int wi = 0; wi < kAWarps; ++wi) {
        wb.push_back((int)(pieces.size() / kBundleInt4));
        for (int k : per[wi]) {
            const Bundle &b = bs[k];
            pieces.push_back(make_int4((int)(kh.size() - kh_base), b.T,
                                       (b.lng ? kPieceLong : 0) | (b.part ? kPiecePart : 0), 0));
            // slot s of group g is rows[g + groups s]
            for (int j = 0; j < kMaxSlots; j += 4)
                pieces.push_back(make_int4(b.rows[j], b.rows[j + 1], b.rows[j + 2], b.rows[j + 3]));
            // round t, group g, slot s -> position kSlots t + rpg g + s
            for (int t = 0; t < b.T; ++t)
                for (int g = 0; g < groups; ++g)
                    for (int sl = 0; sl < rpg; ++sl) {
                        int2 v = make_int2(0, 0);
                        if (b.lng) {
                            const int e = b.e0 + kSlots * t + rpg * g + sl;
                            if (e < b.e1) v = ent[b.src - r0][e];
                        } else {
                            const int row = b.rows[g + groups * sl];
                            if (row >= 0 && t < row_len(row)) v = ent[row - r0][t];
                        }
                        kh.push_back(v);
                    }
        }
    }
    return nslots;
}

// Row i's entries with a column in [c0, c1), columns relative to c0, in CSR order.
std::vector<int2> row_entries(const HostOps &h, int i, int c0, int c1) {
    std::vector<int2> out;
    if (i >= (int)h.n) return out;
    for (int64_t q = h.hptr[i]; q < h.hptr[i + 1]; ++q) {
        const int k = h.hcol[q];
        if (k < c0 || k >= c1) continue;
        const float v = (float)h.hval[q];
        int bits;
        memcpy(&bits, &v, 4);
        out.push_back(make_int2(k - c0, bits));
    }
    return out;
}

}  // namespace

bool plan_columns(const HostOps &h, int np, int device, ColPlan &plan, int min_splits, bool gather) {
    if ((!gather && np > kColMaxNp) || np % kBoxRows != 0) return false;
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess || sms <= 0) {
        cudaGetLastError();
        return false;
    }
    const int smem_max = max_smem_optin(device);
    const int n = (int)h.n;
    const int ncb = np / (gather ? kCWWide : kCW);  // the gather form: 32-column blocks
    // cumulative row cost (nonzeros + a per-row overhead) for the splits
    std::vector<double> cum(np + 1, 0.0);
    for (int i = 0; i < np; ++i) {
        const double nz = (i < n) ? (double)(h.hptr[i + 1] - h.hptr[i]) : 0.0;
        cum[i + 1] = cum[i] + nz + 4.0;
    }
    // gather form: at least kGatherWaves waves of kGatherCtasPerSm CTAs per
    // SM, up to 64 splits
    const int s_max = gather ? 64 : 16;
    const int s0 = min_splits > 0 ? min_splits
                   : gather ? std::min(std::max(1, (kGatherWaves * kGatherCtasPerSm * sms + ncb - 1) / ncb), s_max)
                            : std::min(std::max(1, sms / ncb), 16);
    int sm_per_sm = 0;
    if (cudaDeviceGetAttribute(&sm_per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, device) != cudaSuccess) {
        cudaGetLastError();
        sm_per_sm = 0;
    }
    for (int s = s0; s <= s_max; ++s) {
        ColPlan pl;
        pl.splits = s;
        std::vector<int> rows(s + 1, 0);
        int i = 0;
        for (int k = 1; k < s; ++k) {
            const double target = cum[np] * (double)k / (double)s;
            while (i < np && cum[i] < target) ++i;
            rows[k] = std::max(rows[k - 1], i);
        }
        rows[s] = np;
        size_t kh_max = 0, p_max = 0;
        int slots_max = 0;
        // rows are cut into parts above the whole-block range when the grid
        // has few waves (many waves absorb a long CTA; measured: N = 2048, 3.4
        // waves, 15% faster with cuts; N = 4096, 10 waves, 3% faster; N = 8192,
        // 40 waves, 5% slower)
        const bool cut = np > kColMaxNp && (double)s * ncb < kCutMaxWaves * kGatherCtasPerSm * (double)sms;
        for (int k = 0; k < s; ++k) {
            const size_t kb = pl.kh.size();  // even: every split's block starts 16-byte aligned
            const int first = (int)(pl.pieces.size() / kBundleInt4);
            pl.sb.push_back(first);
            pl.cutb.push_back((int)pl.cuts.size());
            RowEntries ent;
            for (int i = rows[k]; i < rows[k + 1]; ++i) ent.push_back(row_entries(h, i, 0, np));
            const int ns = split_bundles(rows[k], rows[k + 1], ent, kb, pl.kh, pl.pieces, pl.wb, pl.cuts,
                                         cut ? kPartMax : 0, false, gather ? 2 : kNarrowRows, gather ? kRPG : 1);
            if (ns < 0) return false;
            slots_max = std::max(slots_max, ns);
            if (pl.kh.size() % 2) pl.kh.push_back(make_int2(0, 0));
            pl.q.push_back((int)kb);
            pl.q.push_back((int)pl.kh.size());
            kh_max = std::max(kh_max, (pl.kh.size() - kb) * 8);
            p_max = std::max(p_max, (size_t)((int)(pl.pieces.size() / kBundleInt4) - first) * 16 * kBundleInt4);
        }
        pl.sb.push_back((int)(pl.pieces.size() / kBundleInt4));
        pl.wb.push_back((int)(pl.pieces.size() / kBundleInt4));
        pl.cutb.push_back((int)pl.cuts.size());
        const size_t part_bytes = (size_t)slots_max * kRowFloats * 4 * (gather ? 2 : 1);
        size_t smem, cap;
        if (gather) {
            // entries, bundles, partial slots; small enough for kGatherCtasPerSm CTAs per SM
            pl.p_off = (int)kh_max;
            pl.sp_off = 0;
            pl.part_off = (int)(((size_t)pl.p_off + p_max + 15) / 16 * 16);
            smem = (size_t)pl.part_off + part_bytes + 128;
            // per CTA: its dynamic and static shared memory and the 1 KB the
            // system reserves (the 1 KB below covers the static part)
            cap = std::min({(size_t)smem_max, (size_t)sm_per_sm / kGatherCtasPerSm - 1024,
                            (size_t)kGatherSplitBytes + 1024});
        } else {
            // column block, entries, bundles, staged diagonal, partial slots
            pl.p_off = (int)((size_t)np * kRowFloats * 4 + kh_max);
            pl.sp_off = (int)((size_t)pl.p_off + p_max);
            pl.part_off = (int)(((size_t)pl.sp_off + (size_t)np * 4 + 15) / 16 * 16);
            smem = (size_t)pl.part_off + part_bytes + 128;
            cap = (size_t)smem_max;
        }
        // 1 KB left for the static shared memory of the kernels (the batched
        // kernel keeps its problem descriptor there)
        if (cap > 1024 && smem <= cap - 1024) {
            pl.smem = (int)smem;
            if (pl.kh.empty()) pl.kh.assign(2, make_int2(0, 0));
            plan = std::move(pl);
            return true;
        }
    }
    return false;
}

bool make_col_maps(const DevOps &ops, const float *const din[3], ColMaps *maps) {
    PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
    if (!enc) return false;
    const cuuint64_t np = (cuuint64_t)ops.np;
    for (int i = 0; i < 3; ++i) {
        // (column, plane, row): a box is kBoxRows rows of kCW real then kCW imaginary values
        cuuint64_t dims[3] = {np, 2, np};
        cuuint64_t strides[2] = {np * np * sizeof(float), np * sizeof(float)};
        cuuint32_t box[3] = {kCW, 2, kBoxRows};
        cuuint32_t es[3] = {1, 1, 1};
        if (enc(&maps->d[i], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, (void *)din[i], dims, strides, box, es,
                CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return false;
    }
    return true;
}

cudaError_t set_cols_smem(int bytes) {
    cudaError_t e = raise_smem_limit_t(cols_spmm_kernel<1>, bytes);
    if (e == cudaSuccess) e = raise_smem_limit_t(cols_spmm_kernel<2>, bytes);
    if (e == cudaSuccess) e = raise_smem_limit_t(cols_spmm_kernel<3>, bytes);
    if (e == cudaSuccess) e = raise_smem_limit_t(cols_spmm_kernel<4>, bytes);
    return e;
}

cudaError_t set_gather_smem(int bytes) {
    cudaError_t e = raise_smem_limit_t(cols_gather_kernel<1>, bytes);
    if (e == cudaSuccess) e = raise_smem_limit_t(cols_gather_kernel<2>, bytes);
    if (e == cudaSuccess) e = raise_smem_limit_t(cols_gather_kernel<3>, bytes);
    if (e == cudaSuccess) e = raise_smem_limit_t(cols_gather_kernel<4>, bytes);
    return e;
}

// Stage inputs: stage 1 D (map 0), stage 2 da (map 1), stage 3 db (map 2),
// stage 4 da (map 1). With pdl, the launch may start before the previous
// kernel in the stream has finished (programmatic dependent launch; the
// kernel waits with griddepcontrol.wait before it reads that kernel's
// output); without, it is an ordinary stream-ordered launch.
template <typename K, typename... A>
void launch_pdl(K kernel, dim3 grid, dim3 block, size_t smem, cudaStream_t s, bool pdl, A... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = pdl ? 1 : 0;
    cudaLaunchKernelEx(&cfg, kernel, args...);
}

void launch_cols_stage(int stage, const DevOps &ops, const MixedWork &w, cudaStream_t s, int parts, bool serial) {
    const ColMaps &m = *w.cmaps;
    const int units = ops.col_gather ? ops.col_splits * (ops.np / kCWWide) : (ops.np / kCW) * ops.col_splits;
    const dim3 ga(ops.col_gain_ctas + units);
    const size_t sm = (size_t)ops.col_launch_smem;
    const CUtensorMap &tm = m.d[stage == 1 ? 0 : (stage == 3 ? 2 : 1)];
    const bool pdl = !serial;
    if (parts & 1) {
        if (ops.col_gather) {
            switch (stage) {
                case 1: launch_pdl(cols_gather_kernel<1>, ga, dim3(kANT), sm, s, pdl, ops, w); break;
                case 2: launch_pdl(cols_gather_kernel<2>, ga, dim3(kANT), sm, s, pdl, ops, w); break;
                case 3: launch_pdl(cols_gather_kernel<3>, ga, dim3(kANT), sm, s, pdl, ops, w); break;
                default: launch_pdl(cols_gather_kernel<4>, ga, dim3(kANT), sm, s, pdl, ops, w); break;
            }
        } else {
            switch (stage) {
                case 1: launch_pdl(cols_spmm_kernel<1>, ga, dim3(kANT), sm, s, pdl, tm, ops, w); break;
                case 2: launch_pdl(cols_spmm_kernel<2>, ga, dim3(kANT), sm, s, pdl, tm, ops, w); break;
                case 3: launch_pdl(cols_spmm_kernel<3>, ga, dim3(kANT), sm, s, pdl, tm, ops, w); break;
                default: launch_pdl(cols_spmm_kernel<4>, ga, dim3(kANT), sm, s, pdl, tm, ops, w); break;
            }
        }
    }
    if (parts & 2) {
        const dim3 ge(w.npairs);
        switch (stage) {
            case 1: launch_pdl(cols_epi_kernel<1>, ge, dim3(kENT), 0, s, pdl, ops, w); break;
            case 2: launch_pdl(cols_epi_kernel<2>, ge, dim3(kENT), 0, s, pdl, ops, w); break;
            case 3: launch_pdl(cols_epi_kernel<3>, ge, dim3(kENT), 0, s, pdl, ops, w); break;
            default: launch_pdl(cols_epi_kernel<4>, ge, dim3(kENT), 0, s, pdl, ops, w); break;
        }
    }
}

cudaError_t raise_smem_limit(const void *kernel, int bytes) {
    static std::mutex mu;
    std::lock_guard<std::mutex> lock(mu);
    cudaFuncAttributes a;
    cudaError_t e = cudaFuncGetAttributes(&a, kernel);
    if (e != cudaSuccess) return e;
    if (a.maxDynamicSharedSizeBytes >= bytes) return cudaSuccess;
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

}  // namespace qpr

#ifdef QPR_TIMELINE
// Entry points of the diagnostic build (include/qpr_timeline.h).
extern "C" {
__attribute__((visibility("default"))) int qpr_timeline_reset(void) {
    using namespace qpr::timeline;
    static unsigned long long h[kKinds][kInst][2 * kFields];
    for (int k = 0; k < kKinds; ++k)
        for (int i = 0; i < kInst; ++i)
            for (int f = 0; f < kFields; ++f) {
                h[k][i][2 * f] = ~0ull;  // first: a minimum
                h[k][i][2 * f + 1] = 0;  // last: a maximum
            }
    const unsigned long long z[kKinds] = {0};
    if (cudaMemcpyToSymbol(g_stamp, h, sizeof(h)) != cudaSuccess) return 1;
    if (cudaMemcpyToSymbol(g_count, z, sizeof(z)) != cudaSuccess) return 1;
    return cudaDeviceSynchronize() == cudaSuccess ? 0 : 1;
}
__attribute__((visibility("default"))) int qpr_timeline_read(unsigned long long *stamps,
                                                            unsigned long long *counts) {
    using namespace qpr::timeline;
    if (cudaDeviceSynchronize() != cudaSuccess) return 1;
    if (cudaMemcpyFromSymbol(stamps, g_stamp, sizeof(g_stamp)) != cudaSuccess) return 1;
    return cudaMemcpyFromSymbol(counts, g_count, sizeof(g_count)) == cudaSuccess ? 0 : 1;
}
}
#endif
