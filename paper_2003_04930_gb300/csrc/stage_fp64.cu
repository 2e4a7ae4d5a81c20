// FP64 RK4 stage kernel: tile-pair DMMA GEMM X = H [Re Y | Im Y] with the
// Lindblad right-hand side and the RK4 stage update fused into its epilogue.
//
// Why one GEMM is enough (Eq. 1 / Eq. S7): H is real symmetric and every
// stage input Y is Hermitian, so rho H = (H rho)^dag. With X = H Y = A + iB
// (A = H Re Y, B = H Im Y) the commutator term is
//     -(1-omega) i (X - X^dag) = (1-omega) [ (B + B^T) - i (A - A^T) ].
// The dissipator with L_ij = sqrt(G_ij)|i><j| is diagonal-plus-Hadamard:
//     omega [ diag(g) - 1/2 (c_a + c_b) Y_ab ],  g = G p,  p_a = Y_aa,
// with c the column sums of G. So the only O(N^3) work is the real GEMM.
//
// One CTA owns the tile pair (I, J), I <= J, of the Hermitian output: it
// computes X_IJ and X_JI (the second only when I != J), combines them, writes
// tile (I, J) and its conjugate transpose as tile (J, I). Because the
// operands are Hermitian the GEMM is an "NT" product of row panels:
//     X_IJ(a, b) = sum_k H(a, k) Re Y(b, k) - i sum_k H(a, k) Im Y(b, k),
// since Re Y(k, b) = Re Y(b, k) and Im Y(k, b) = -Im Y(b, k).
//
// Classical RK4 (Supplementary Note 2): with Y1 = y / tr(y)
//   stage 1: k1 = f(Y1); Z = Y1 + dt/6 k1; Ya = Y1 + dt/2 k1 (and ||k1||^2)
//   stage 2: k2 = f(Ya); Z += dt/3 k2;     Yb = Y1 + dt/2 k2
//   stage 3: k3 = f(Yb); Z += dt/3 k3;     Ya = Y1 + dt k3
//   stage 4: k4 = f(Ya); y = Z + dt/6 k4
// Stage 1 reads the unnormalised y and multiplies by 1/tr(y) in the
// epilogue (f is linear), which is the per-step trace renormalisation.
//
// The FP64 tensor path is mma.sync m8n8k4 (DMMA): tcgen05 has no f64 kind.
#include "qpr_internal.cuh"
#include "stage_epilogue.cuh"

namespace qpr {
namespace {

constexpr int TS = kTileFp64;          // 32 complex rows / columns per tile
constexpr int KC = 32;                 // k extent of one pipeline chunk
constexpr int LDS = KC + 4;            // padded shared-memory row (doubles)
constexpr int PANEL = TS * LDS;        // doubles per staged 32 x 32 panel
constexpr int NPANEL = 6;              // H_I, ReY_I, ImY_I, H_J, ReY_J, ImY_J
constexpr int STAGE_DBL = NPANEL * PANEL;
constexpr int SMEM_BYTES = 2 * STAGE_DBL * (int)sizeof(double);
constexpr int LDX = 2 * TS + 1;        // epilogue X tile row (odd: conflict-free transpose)
constexpr int LDO = TS + 1;
constexpr int NTHREADS = 128;

static_assert(TS == kEpiTS && NTHREADS == kEpiThreads && LDO == kEpiLDO, "epilogue geometry");
static_assert(2 * TS * LDX + 4 * TS * LDO <= 2 * STAGE_DBL, "epilogue must fit in the pipeline buffers");

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
    unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
__device__ __forceinline__ void cp_async_wait1() { asm volatile("cp.async.wait_group 1;\n" ::); }

// D += A * B for one 8x8x4 FP64 tile. Fragments: a = A[lane/4][lane%4],
// b = B[lane%4][lane/4], d = D[lane/4][2*(lane%4) + {0,1}].
__device__ __forceinline__ void dmma(double (&d)[2], double a, double b) {
    asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};\n"
                 : "+d"(d[0]), "+d"(d[1])
                 : "d"(a), "d"(b));
}

// Stage one k-chunk of the six row panels into shared memory.
__device__ __forceinline__ void load_chunk(double *st, const double *__restrict__ H,
                                           const double *__restrict__ Y, size_t plane, int np,
                                           int I, int J, int kc, bool diag) {
    const int npan = diag ? 3 : 6;
    const int segs = KC / 2;  // 16-byte segments per row
    const int total = npan * TS * segs;
    for (int idx = threadIdx.x; idx < total; idx += NTHREADS) {
        const int p = idx / (TS * segs);
        const int rem = idx - p * (TS * segs);
        const int r = rem / segs;
        const int sg = rem - r * segs;
        const int tile = (p < 3) ? I : J;
        const int kind = p % 3;
        const double *base = (kind == 0) ? H : (kind == 1 ? Y : Y + plane);
        const double *src = base + (size_t)(tile * TS + r) * np + (size_t)kc * KC + sg * 2;
        cp_async16(st + p * PANEL + r * LDS + sg * 2, src);
    }
}

template <int STAGE>
__global__ void __launch_bounds__(NTHREADS, 2)
stage_fp64_kernel(DevOps ops, Work w) {
    extern __shared__ __align__(16) double smem[];
    __shared__ int s_done;
    Ctl *ctl = w.ctl;
    if (threadIdx.x == 0) s_done = *(volatile int *)&ctl->done;
    __syncthreads();
    if (s_done) return;

    const int I = w.pairs[blockIdx.x].x;
    const int J = w.pairs[blockIdx.x].y;
    const bool diag = (I == J);
    const int np = ops.np;
    const size_t plane = (size_t)np * np;
    // GEMM operand and dissipator input of this stage
    const double *__restrict__ yin = (STAGE <= 1) ? w.y : (STAGE == 3 ? w.yb : w.ya);

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int m0 = (warp & 1) * 16;  // rows of the warp's 16 x 32 sub-tile
    const int half = warp >> 1;      // 0: real-part columns, 1: imaginary-part columns

    double acc1[2][4][2], acc2[2][4][2];
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
        for (int nt = 0; nt < 4; ++nt) {
            acc1[mt][nt][0] = acc1[mt][nt][1] = 0.0;
            acc2[mt][nt][0] = acc2[mt][nt][1] = 0.0;
        }

    const int nchunks = np / KC;
    load_chunk(smem, ops.H, yin, plane, np, I, J, 0, diag);
    cp_async_commit();
    for (int kc = 0; kc < nchunks; ++kc) {
        const double *cur = smem + (kc & 1) * STAGE_DBL;
        if (kc + 1 < nchunks)
            load_chunk(smem + ((kc + 1) & 1) * STAGE_DBL, ops.H, yin, plane, np, I, J, kc + 1, diag);
        cp_async_commit();
        cp_async_wait1();
        __syncthreads();
        const double *sHI = cur;
        const double *sBI = cur + (1 + half) * PANEL;
        const double *sHJ = cur + 3 * PANEL;
        const double *sBJ = diag ? sBI : cur + (4 + half) * PANEL;
        const int ro = lane >> 2;
#pragma unroll
        for (int kk = 0; kk < KC; kk += 4) {
            const int ko = kk + (lane & 3);
            double a1[2], b1[4];
            a1[0] = sHI[(m0 + ro) * LDS + ko];
            a1[1] = sHI[(m0 + 8 + ro) * LDS + ko];
#pragma unroll
            for (int nt = 0; nt < 4; ++nt) b1[nt] = sBJ[(nt * 8 + ro) * LDS + ko];
#pragma unroll
            for (int mt = 0; mt < 2; ++mt)
#pragma unroll
                for (int nt = 0; nt < 4; ++nt) dmma(acc1[mt][nt], a1[mt], b1[nt]);
            if (!diag) {
                double a2[2], b2[4];
                a2[0] = sHJ[(m0 + ro) * LDS + ko];
                a2[1] = sHJ[(m0 + 8 + ro) * LDS + ko];
#pragma unroll
                for (int nt = 0; nt < 4; ++nt) b2[nt] = sBI[(nt * 8 + ro) * LDS + ko];
#pragma unroll
                for (int mt = 0; mt < 2; ++mt)
#pragma unroll
                    for (int nt = 0; nt < 4; ++nt) dmma(acc2[mt][nt], a2[mt], b2[nt]);
            }
        }
        __syncthreads();
    }

    // ---- epilogue ----
    double *sX1 = smem;                 // X_IJ: [TS][LDX], columns 0..TS-1 real, TS..2TS-1 imaginary
    double *sX2 = smem + TS * LDX;      // X_JI
    double *sO = smem + 2 * TS * LDX;   // outputs of tile (I, J) kept for the mirrored write
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
        for (int nt = 0; nt < 4; ++nt)
#pragma unroll
            for (int i = 0; i < 2; ++i) {
                const int r = m0 + mt * 8 + (lane >> 2);
                const int cidx = half * TS + nt * 8 + (lane & 3) * 2 + i;
                sX1[r * LDX + cidx] = acc1[mt][nt][i];
                if (!diag) sX2[r * LDX + cidx] = acc2[mt][nt][i];
            }
    __syncthreads();
    __shared__ double red[NTHREADS / 32];
    stage_epilogue<STAGE>(ops, w, I, J, diag, sX1, sX2, LDX, sO, red, blockIdx.x, blockIdx.x == 0);
}

template <int STAGE>
void launch_t(const DevOps &ops, const Work &w, cudaStream_t s) {
    stage_fp64_kernel<STAGE><<<w.npairs, NTHREADS, SMEM_BYTES, s>>>(ops, w);
}

template <int STAGE>
cudaError_t set_attr() {
    return cudaFuncSetAttribute(stage_fp64_kernel<STAGE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                SMEM_BYTES);
}

}  // namespace

cudaError_t init_stage_fp64() {
    cudaError_t e = set_attr<0>();
    if (e == cudaSuccess) e = set_attr<1>();
    if (e == cudaSuccess) e = set_attr<2>();
    if (e == cudaSuccess) e = set_attr<3>();
    if (e == cudaSuccess) e = set_attr<4>();
    return e;
}

void launch_stage_fp64(int stage, const DevOps &ops, const Work &w, cudaStream_t s) {
    switch (stage) {
        case 0: launch_t<0>(ops, w, s); break;
        case 1: launch_t<1>(ops, w, s); break;
        case 2: launch_t<2>(ops, w, s); break;
        case 3: launch_t<3>(ops, w, s); break;
        default: launch_t<4>(ops, w, s); break;
    }
}

}  // namespace qpr
