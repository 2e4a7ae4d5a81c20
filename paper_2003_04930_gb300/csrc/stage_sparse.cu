// Sparse FP64 RK4 stage kernel: X = H Y with H in CSR (exact FP64, O(nnz N)
// work per stage) and the same fused Lindblad/RK4 epilogue as the dense
// DMMA kernel.
//
// H of Eq. S6 has one nonzero per link (symmetrised) plus an optional
// diagonal, so H Y costs 4 nnz(H) N flops against 4 N^3 for the dense GEMM;
// the kernel is bound by L2/HBM bandwidth, not by arithmetic. One CTA owns
// the tile pair (I, J): every warp takes rows a of tile I and gathers, for
// each nonzero H_ak, the 32 columns J of row k of Re Y and Im Y (two
// coalesced 256-byte loads), so X_IJ(a, b) = sum_k H_ak Y_kb is formed in
// registers, one column per lane. X_JI is formed the same way.
#include "qpr_internal.cuh"
#include "stage_epilogue.cuh"

namespace qpr {
namespace {

constexpr int TS = kEpiTS;
constexpr int NTHREADS = kEpiThreads;
constexpr int LDX = 2 * TS + 1;
constexpr int LDO = kEpiLDO;
constexpr int SMEM_BYTES = (2 * TS * LDX + 4 * TS * LDO) * (int)sizeof(double);

// rows `rowtile` of H times columns `coltile` of Y into sX ([TS][LDX]).
__device__ __forceinline__ void spmm_tile(const DevOps &ops, const double *__restrict__ yin, size_t plane,
                                          int rowtile, int coltile, double *sX) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int np = ops.np, n = ops.n;
    const int col = coltile * TS + lane;
    const double *__restrict__ yre = yin + col;
    const double *__restrict__ yim = yin + plane + col;
    for (int a = warp; a < TS; a += NTHREADS / 32) {
        const int ga = rowtile * TS + a;
        double xr = 0.0, xi = 0.0;
        if (ga < n) {
            const int q1 = ops.h_ptr[ga + 1];
            int q = ops.h_ptr[ga];
            for (; q + 4 <= q1; q += 4) {
                const int k0 = ops.h_col[q], k1 = ops.h_col[q + 1], k2 = ops.h_col[q + 2], k3 = ops.h_col[q + 3];
                const double h0 = ops.h_val[q], h1 = ops.h_val[q + 1], h2 = ops.h_val[q + 2], h3 = ops.h_val[q + 3];
                const double r0 = yre[(size_t)k0 * np], r1 = yre[(size_t)k1 * np];
                const double r2 = yre[(size_t)k2 * np], r3 = yre[(size_t)k3 * np];
                const double i0 = yim[(size_t)k0 * np], i1 = yim[(size_t)k1 * np];
                const double i2 = yim[(size_t)k2 * np], i3 = yim[(size_t)k3 * np];
                xr += h0 * r0; xi += h0 * i0;
                xr += h1 * r1; xi += h1 * i1;
                xr += h2 * r2; xi += h2 * i2;
                xr += h3 * r3; xi += h3 * i3;
            }
            for (; q < q1; ++q) {
                const int k = ops.h_col[q];
                const double h = ops.h_val[q];
                xr += h * yre[(size_t)k * np];
                xi += h * yim[(size_t)k * np];
            }
        }
        sX[a * LDX + lane] = xr;
        sX[a * LDX + TS + lane] = -xi;
    }
}

template <int STAGE>
__global__ void __launch_bounds__(NTHREADS)
stage_sparse_kernel(DevOps ops, Work w) {
    extern __shared__ __align__(16) double smem[];
    __shared__ double red[NTHREADS / 32];
    __shared__ int s_done;
    if (threadIdx.x == 0) s_done = *(volatile int *)&w.ctl->done;
    __syncthreads();
    if (s_done) return;

    const int I = w.pairs[blockIdx.x].x;
    const int J = w.pairs[blockIdx.x].y;
    const bool diag = (I == J);
    const size_t plane = (size_t)ops.np * ops.np;
    const double *__restrict__ yin = (STAGE <= 1) ? w.y : (STAGE == 3 ? w.yb : w.ya);
    double *sX1 = smem;
    double *sX2 = smem + TS * LDX;
    double *sO = smem + 2 * TS * LDX;
    spmm_tile(ops, yin, plane, I, J, sX1);
    if (!diag) spmm_tile(ops, yin, plane, J, I, sX2);
    __syncthreads();
    stage_epilogue<STAGE>(ops, w, I, J, diag, sX1, sX2, LDX, sO, red);
}

template <int STAGE>
cudaError_t set_attr() {
    return cudaFuncSetAttribute(stage_sparse_kernel<STAGE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                SMEM_BYTES);
}

}  // namespace

cudaError_t init_stage_sparse() {
    cudaError_t e = set_attr<0>();
    if (e == cudaSuccess) e = set_attr<1>();
    if (e == cudaSuccess) e = set_attr<2>();
    if (e == cudaSuccess) e = set_attr<3>();
    if (e == cudaSuccess) e = set_attr<4>();
    return e;
}

void launch_stage_sparse(int stage, const DevOps &ops, const Work &w, cudaStream_t s) {
    switch (stage) {
        case 0: stage_sparse_kernel<0><<<w.npairs, NTHREADS, SMEM_BYTES, s>>>(ops, w); break;
        case 1: stage_sparse_kernel<1><<<w.npairs, NTHREADS, SMEM_BYTES, s>>>(ops, w); break;
        case 2: stage_sparse_kernel<2><<<w.npairs, NTHREADS, SMEM_BYTES, s>>>(ops, w); break;
        case 3: stage_sparse_kernel<3><<<w.npairs, NTHREADS, SMEM_BYTES, s>>>(ops, w); break;
        default: stage_sparse_kernel<4><<<w.npairs, NTHREADS, SMEM_BYTES, s>>>(ops, w); break;
    }
}

}  // namespace qpr
