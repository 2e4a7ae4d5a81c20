// qpr_rhs_noalloc: one evaluation of the Lindblad right-hand side for
// callers that cannot allocate device memory.
//
// Every other entry point works through a context whose buffers qpr_create
// obtains with cudaMalloc. Some callers cannot allow that: hosts that hand
// out all device memory from their own pool or arena and forbid libraries
// from allocating behind their back, services that run under a fixed device
// memory budget, and code that must not allocate once it is past start-up.
// This entry point takes every input and output from the caller and keeps
// its scratch (the two Hermitian planes of rho and of f(rho), the gain G p,
// the column sums of G, the tile-pair table, the residual partials and the
// control block) in one file-scope __device__ array of fixed size, sized for
// N <= QPR_NOALLOC_MAX_N. It calls no cudaMalloc, cudaFree or other
// allocating routine.
//
// The array exists once per device that loads the library and stays
// resident until the process exits. All calls on a device share it and it
// keeps the last call's contents; each call rewrites every part it reads
// before reading it. Calls whose work overlaps on the GPU (different streams,
// or different host threads) race on the array and must be serialised by the
// caller.
#include <mutex>

#include "qpr_internal.cuh"

namespace {

constexpr int kMaxN = QPR_NOALLOC_MAX_N;
constexpr int kMaxNp = ((kMaxN + qpr::kPadFp64 - 1) / qpr::kPadFp64) * qpr::kPadFp64;
constexpr int kMaxTiles = kMaxNp / qpr::kTileFp64;
constexpr int kMaxPairs = kMaxTiles * (kMaxTiles + 1) / 2;
constexpr size_t kPlane = (size_t)kMaxNp * kMaxNp;
// layout of the scratch array, in doubles
constexpr size_t kOffY = 0;                       // 2 planes: Hermitised rho
constexpr size_t kOffZ = 2 * kPlane;              // 2 planes: f(rho)
constexpr size_t kOffG = 4 * kPlane;              // gain, kMaxNp
constexpr size_t kOffC = kOffG + kMaxNp;          // column sums of G, kMaxNp
constexpr size_t kOffPart = kOffC + kMaxNp;       // residual partials, kMaxPairs
constexpr size_t kOffPairs = kOffPart + kMaxPairs;  // int2 table, one double each
constexpr size_t kOffCtl = kOffPairs + kMaxPairs;
constexpr size_t kCtlDoubles = (sizeof(qpr::Ctl) + sizeof(double) - 1) / sizeof(double);
constexpr size_t kScratchDoubles = kOffCtl + kCtlDoubles;
static_assert(sizeof(int2) == sizeof(double), "one pair per double slot");

// The scratch array. In host code its name is only a host-side stand-in:
// the device address comes from cudaGetSymbolAddress (see scratch_base).
static __device__ __align__(256) double g_noalloc_scratch[kScratchDoubles];

std::mutex g_setup_mu;
constexpr int kMaxDevices = 64;
double *g_base[kMaxDevices] = {};

// Per-call set-up on the device: control block, tile-pair table (the order
// qpr_create uses) and the column sums of G = alpha S + (1 - alpha) F,
// summed in the same order as the host assembly.
__global__ void noalloc_setup_kernel(qpr::DevOps ops, qpr::Work w, double *c) {
    const int np = ops.np, n = ops.n;
    const int T = np / qpr::kTileFp64;
    if (threadIdx.x == 0) {
        qpr::Ctl *ctl = w.ctl;
        ctl->done = 0;
        ctl->status = qpr::kCtlRunning;
        ctl->step = 0;
        ctl->max_steps = 0;
        ctl->tol = 0.0;
        ctl->dt = 0.0;
        ctl->scale = 1.0;
        ctl->trace = 0.0;
        ctl->resid = 0.0;
        ctl->resid_step = 0;
        int q = 0;
        for (int I = 0; I < T; ++I)
            for (int J = I + 1; J < T; ++J) w.pairs[q++] = make_int2(I, J);
        for (int I = 0; I < T; ++I) w.pairs[q++] = make_int2(I, I);
    }
    const int nnz = ops.s_ptr[n];
    for (int j = threadIdx.x; j < np; j += blockDim.x) {
        double cj = 0.0;
        if (j < n) {
            double sj = 0.0;
            if (ops.dang[j]) {
                sj = 1.0;
            } else {
                for (int q = 0; q < nnz; ++q)
                    if (ops.s_col[q] == j) sj += ops.s_val[q];
            }
            cj = ops.alpha * sj + (1.0 - ops.alpha) * 1.0;
        }
        c[j] = cj;
    }
}

// Device address of the scratch array on the current device, found once per
// device with that device current.
cudaError_t scratch_base(int dev, double **out) {
    std::lock_guard<std::mutex> lk(g_setup_mu);
    if (!g_base[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        e = qpr::init_stage_sparse();
        if (e != cudaSuccess) return e;
        g_base[dev] = (double *)p;
    }
    *out = g_base[dev];
    return cudaSuccess;
}

}  // namespace

extern "C" qpr_status qpr_rhs_noalloc(int64_t n, const int32_t *h_ptr, const int32_t *h_col, const double *h_val,
                                      const int32_t *s_ptr, const int32_t *s_col, const double *s_val,
                                      const uint8_t *dangling_flags, double alpha, double omega,
                                      int32_t dangling_mode, const void *rho, void *out, void *cuda_stream) {
    if (n < 2 || n > kMaxN) return QPR_E_ARG;
    if (!h_ptr || !h_col || !h_val || !s_ptr || !s_col || !s_val || !dangling_flags || !rho || !out)
        return QPR_E_ARG;
    if (!(alpha >= 0.0 && alpha <= 1.0) || !(omega >= 0.0 && omega <= 1.0)) return QPR_E_ARG;
    if (dangling_mode != QPR_DANGLING_F && dangling_mode != QPR_DANGLING_UNIFORM) return QPR_E_ARG;
    // an error left on this thread by earlier work is not ours to clear: report
    // it before queuing anything, so the check after the launches below sees
    // only this call's own launch errors
    if (cudaPeekAtLastError() != cudaSuccess) return QPR_E_CUDA;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        return QPR_E_CUDA;
    }
    double *base = nullptr;
    if (scratch_base(dev, &base) != cudaSuccess) {
        cudaGetLastError();
        return QPR_E_CUDA;
    }
    cudaStream_t s = (cudaStream_t)cuda_stream;
    const int np = (int)(((n + qpr::kPadFp64 - 1) / qpr::kPadFp64) * qpr::kPadFp64);
    const int T = np / qpr::kTileFp64;

    qpr::DevOps ops{};
    ops.n = (int)n;
    ops.np = np;
    ops.alpha = alpha;
    ops.omega = omega;
    ops.dangling = dangling_mode;
    ops.H = nullptr;  // the sparse stage kernel reads H only through its CSR
    ops.h_ptr = h_ptr;
    ops.h_col = h_col;
    ops.h_val = h_val;
    ops.s_ptr = s_ptr;
    ops.s_col = s_col;
    ops.s_val = s_val;
    ops.dang = dangling_flags;
    ops.c = base + kOffC;

    qpr::Work w{};
    w.y = base + kOffY;
    w.z = base + kOffZ;
    w.ya = w.y;  // stage 0 reads only y and writes only z
    w.yb = w.y;
    w.g = base + kOffG;
    w.partials = base + kOffPart;
    w.pairs = reinterpret_cast<int2 *>(base + kOffPairs);
    w.npairs = T * (T + 1) / 2;
    w.tiles = T;
    w.ctl = reinterpret_cast<qpr::Ctl *>(base + kOffCtl);

    noalloc_setup_kernel<<<1, 256, 0, s>>>(ops, w, base + kOffC);
    qpr::launch_import((const double *)rho, (int)n, np, w.y, s);
    qpr::launch_gain(0, ops, w.y, w, s);
    qpr::launch_stage_sparse(0, ops, w, s);
    qpr::launch_export(w.z, (int)n, np, w.ctl, 0, (double *)out, s);
    return cudaGetLastError() == cudaSuccess ? QPR_OK : QPR_E_CUDA;
}
