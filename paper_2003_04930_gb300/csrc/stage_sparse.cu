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
#include "sparse_body.cuh"

namespace qpr {
namespace {

using namespace sparse64;

template <int STAGE>
__global__ void __launch_bounds__(NTHREADS)
stage_sparse_kernel(DevOps ops, Work w) {
    extern __shared__ __align__(16) double smem[];
    __shared__ int s_done;
    if (threadIdx.x == 0) s_done = *(volatile int *)&w.ctl->done;
    __syncthreads();
    if (s_done) return;
    tile<STAGE>(ops, w, w.pairs[blockIdx.x].x, w.pairs[blockIdx.x].y, blockIdx.x, blockIdx.x == 0, smem);
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
