// Warm-start network: a 4-layer message-passing network (width 64, BF16
// weights, FP32 accumulation) that predicts the steady-state populations p
// from the graph, so that rho0 = diag(p_hat) starts RK4 near its fixed point.
// Forward, backward and Adam are hand-written kernels; the network is
// trained on steady states the solver itself produces.
//
// Definition (identical to the CPU oracle's, written independently):
//   features x_i = [1, omega, log1p(in-strength), log1p(out-strength),
//                   log1p(in-degree), log1p(out-degree), log(N pi_i), dangles]
//   with A_ij = w for the link j -> i, pi the classical PageRank (stationary
//   vector of G = alpha S + (1 - alpha) F, 200 power-iteration steps from
//   uniform, the omega = 1 limit of the method);
//   P_ij = (A_ij + A_ji) / s_i, s_i = sum_j (A_ij + A_ji);
//   z_l = h_{l-1} Ws_l + (P h_{l-1}) Wn_l + b_l, h_l = relu(z_l), h_0 = x;
//   s = h_4 wo + bo, p_hat = softmax(s), L = -sum_i p_i log p_hat_i.
// The layers are (N x 128) x (128 x 64) products: far too small for tensor
// cores to matter, so they run on the FP32 pipe with the BF16-rounded weights
// staged in shared memory; every reduction (weight gradients, softmax) is in
// fixed order, so training is bitwise reproducible.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <cstdint>
#include <string>
#include <vector>

#include "qpr_internal.cuh"

namespace qpr {
namespace {

constexpr int FIN = 8, W = 64, LAYERS = 4;
constexpr int kParams = 2 * FIN * W + W + 3 * (2 * W * W + W) + W + 1;  // 25921
constexpr int kRowsWG = 128;  // rows per partial weight-gradient block

// offsets of the flat parameter layout
__host__ __device__ constexpr int off_ws(int l) { return l == 1 ? 0 : 2 * FIN * W + W + (l - 2) * (2 * W * W + W); }
__host__ __device__ constexpr int din_of(int l) { return l == 1 ? FIN : W; }
__host__ __device__ constexpr int off_wn(int l) { return off_ws(l) + din_of(l) * W; }
__host__ __device__ constexpr int off_b(int l) { return off_wn(l) + din_of(l) * W; }
constexpr int OFF_WO = 2 * FIN * W + W + 3 * (2 * W * W + W);
constexpr int OFF_BO = OFF_WO + W;
static_assert(OFF_BO + 1 == kParams, "parameter layout");

// ---------------------------------------------------------------- kernels
// Y[i][:] (+)= sum_q val[q] X[col[q]][:], d <= 64 columns, one warp per row.
__global__ void spmm_rows_kernel(const int *__restrict__ ptr, const int *__restrict__ col,
                                 const float *__restrict__ val, const float *__restrict__ X, float *__restrict__ Y,
                                 int n, int d, int accumulate) {
    const int lane = threadIdx.x & 31;
    const int i = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (i >= n) return;
    float a0 = 0.f, a1 = 0.f;
    for (int q = ptr[i]; q < ptr[i + 1]; ++q) {
        const float v = val[q];
        const float *x = X + (size_t)col[q] * d;
        if (lane < d) a0 = __fmaf_rn(v, x[lane], a0);
        if (lane + 32 < d) a1 = __fmaf_rn(v, x[lane + 32], a1);
    }
    float *y = Y + (size_t)i * d;
    if (lane < d) y[lane] = accumulate ? __fadd_rn(y[lane], a0) : a0;
    if (lane + 32 < d) y[lane + 32] = accumulate ? __fadd_rn(y[lane + 32], a1) : a1;
}

// Z = H Ws + M Wn + b, Hout = relu(Z): 32 rows per CTA, 256 threads.
__global__ void __launch_bounds__(256) dense_fwd_kernel(const float *__restrict__ H, const float *__restrict__ M,
                                                        const float *__restrict__ prm, int l, int n,
                                                        float *__restrict__ Z, float *__restrict__ Hout) {
    __shared__ float sW[2 * W * W];
    __shared__ float sH[32 * W], sM[32 * W];
    const int din = din_of(l);
    for (int t = threadIdx.x; t < 2 * din * W; t += blockDim.x) sW[t] = prm[off_ws(l) + t];  // Ws then Wn
    const int r0 = blockIdx.x * 32;
    for (int t = threadIdx.x; t < 32 * din; t += blockDim.x) {
        const int r = r0 + t / din;
        sH[t] = r < n ? H[(size_t)r * din + t % din] : 0.f;
        sM[t] = r < n ? M[(size_t)r * din + t % din] : 0.f;
    }
    __syncthreads();
    const int f = threadIdx.x & (W - 1);
    const float bf = prm[off_b(l) + f];
    for (int rr = threadIdx.x >> 6; rr < 32; rr += 4) {
        const int r = r0 + rr;
        if (r >= n) break;
        float z = bf;
        for (int k = 0; k < din; ++k) {
            z = __fmaf_rn(sH[rr * din + k], sW[k * W + f], z);
            z = __fmaf_rn(sM[rr * din + k], sW[din * W + k * W + f], z);
        }
        Z[(size_t)r * W + f] = z;
        Hout[(size_t)r * W + f] = z > 0.f ? z : 0.f;
    }
}

// Logits, softmax and loss of one graph (one CTA of 256 threads):
// s_i = h4_i . wo + bo; p_hat = softmax(s); L = -sum p_i log p_hat_i;
// ds_i = p_hat_i sum(p) - p_i. Fixed-order reductions.
__global__ void __launch_bounds__(256) softmax_loss_kernel(const float *__restrict__ H4, const float *__restrict__ prm,
                                                           const double *__restrict__ p, int n,
                                                           double *__restrict__ p_hat, float *__restrict__ ds,
                                                           double *__restrict__ loss_acc, float *__restrict__ s_buf) {
    __shared__ double red[8];
    __shared__ double bc;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int i = tid; i < n; i += blockDim.x) {
        float s = prm[OFF_BO];
        for (int k = 0; k < W; ++k) s = __fmaf_rn(H4[(size_t)i * W + k], prm[OFF_WO + k], s);
        s_buf[i] = s;
    }
    __syncthreads();
    auto bsum = [&](double v, bool is_max) {
        for (int o = 16; o > 0; o >>= 1) {
            const double u = __shfl_xor_sync(0xffffffffu, v, o);
            v = is_max ? fmax(v, u) : v + u;
        }
        __syncthreads();
        if (lane == 0) red[warp] = v;
        __syncthreads();
        if (tid == 0) {
            double t = red[0];
            for (int q = 1; q < 8; ++q) t = is_max ? fmax(t, red[q]) : t + red[q];
            bc = t;
        }
        __syncthreads();
        return bc;
    };
    double mx = -INFINITY;
    for (int i = tid; i < n; i += blockDim.x) mx = fmax(mx, (double)s_buf[i]);
    mx = bsum(mx, true);
    double se = 0.0, sp = 0.0;
    for (int i = tid; i < n; i += blockDim.x) {
        se += exp((double)s_buf[i] - mx);
        sp += p ? p[i] : 0.0;
    }
    se = bsum(se, false);
    sp = bsum(sp, false);
    const double lse = mx + log(se);
    double ls = 0.0;
    for (int i = tid; i < n; i += blockDim.x) {
        const double lp = (double)s_buf[i] - lse;
        const double ph = exp(lp);
        if (p_hat) p_hat[i] = ph;
        if (p) {
            ls -= p[i] * lp;
            if (ds) ds[i] = (float)(ph * sp - p[i]);
        }
    }
    if (p) {
        ls = bsum(ls, false);
        if (tid == 0 && loss_acc) *loss_acc += ls;
    }
}

// dH4 = ds wo^T (n x 64), and the partial sums of dwo = H4^T ds, dbo = sum ds
// per block of kRowsWG rows.
__global__ void __launch_bounds__(W) readout_bwd_kernel(const float *__restrict__ H4, const float *__restrict__ ds,
                                                        const float *__restrict__ prm, int n, float *__restrict__ dH,
                                                        float *__restrict__ part) {
    const int f = threadIdx.x;
    const int r0 = blockIdx.x * kRowsWG, r1 = min(n, r0 + kRowsWG);
    float gw = 0.f, gb = 0.f;
    const float wo = prm[OFF_WO + f];
    for (int r = r0; r < r1; ++r) {
        const float d = ds[r];
        gw = __fmaf_rn(H4[(size_t)r * W + f], d, gw);
        gb = __fadd_rn(gb, d);
        dH[(size_t)r * W + f] = __fmul_rn(d, wo);
    }
    part[(size_t)blockIdx.x * (W + 1) + f] = gw;
    if (f == 0) part[(size_t)blockIdx.x * (W + 1) + W] = gb;
}

// dZ = dH * [Z > 0] in place in dH; partial sums of dWs = H^T dZ,
// dWn = M^T dZ, db = sum dZ per block of kRowsWG rows (din x 64 each).
__global__ void __launch_bounds__(256) wgrad_kernel(const float *__restrict__ H, const float *__restrict__ M,
                                                    const float *__restrict__ Z, float *__restrict__ dH, int n,
                                                    int din, float *__restrict__ part) {
    __shared__ float sdz[32 * W];
    __shared__ float sH[32 * W], sM[32 * W];
    const int per = 2 * din * W + W;
    const int r0 = blockIdx.x * kRowsWG, r1 = min(n, r0 + kRowsWG);
    // each thread owns 2*din*W/256 weight outputs (+ one bias for threads < W)
    float acc[2 * W * W / 256];
    const int nown = (2 * din * W) / 256;
    for (int q = 0; q < nown; ++q) acc[q] = 0.f;
    float accb = 0.f;
    for (int rb = r0; rb < r1; rb += 32) {
        const int rows = min(32, r1 - rb);
        __syncthreads();
        for (int t = threadIdx.x; t < 32 * W; t += blockDim.x) {
            const int rr = t / W, f = t % W, r = rb + rr;
            float dz = 0.f;
            if (rr < rows) {
                const size_t o = (size_t)r * W + f;
                dz = Z[o] > 0.f ? dH[o] : 0.f;
                dH[o] = dz;
            }
            sdz[t] = dz;
        }
        for (int t = threadIdx.x; t < 32 * din; t += blockDim.x) {
            const int rr = t / din, k = t % din, r = rb + rr;
            sH[t] = rr < rows ? H[(size_t)r * din + k] : 0.f;
            sM[t] = rr < rows ? M[(size_t)r * din + k] : 0.f;
        }
        __syncthreads();
        for (int q = 0; q < nown; ++q) {
            const int idx = threadIdx.x + q * 256;  // 0 .. 2*din*W-1
            const int which = idx / (din * W), rem = idx % (din * W), k = rem / W, f = rem % W;
            const float *src = which == 0 ? sH : sM;
            float a = acc[q];
            for (int rr = 0; rr < rows; ++rr) a = __fmaf_rn(src[rr * din + k], sdz[rr * W + f], a);
            acc[q] = a;
        }
        if (threadIdx.x < W)
            for (int rr = 0; rr < rows; ++rr) accb = __fadd_rn(accb, sdz[rr * W + threadIdx.x]);
    }
    float *out = part + (size_t)blockIdx.x * per;
    for (int q = 0; q < nown; ++q) out[threadIdx.x + q * 256] = acc[q];
    if (threadIdx.x < W) out[2 * din * W + threadIdx.x] = accb;
}

// grad[dst + t] += sum over blocks of part[b * per + t], in block order.
__global__ void reduce_parts_kernel(const float *__restrict__ part, int nblocks, int per, float *__restrict__ grad) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= per) return;
    float s = 0.f;
    for (int b = 0; b < nblocks; ++b) s = __fadd_rn(s, part[(size_t)b * per + t]);
    grad[t] = __fadd_rn(grad[t], s);
}

// dHs = dZ Ws^T, dT = dZ Wn^T (n x din): one thread per (row, k).
__global__ void dense_bwd_kernel(const float *__restrict__ dZ, const float *__restrict__ prm, int l, int n,
                                 float *__restrict__ dHs, float *__restrict__ dT) {
    const int din = din_of(l);
    const size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (t >= (size_t)n * din) return;
    const int r = (int)(t / din), k = (int)(t % din);
    const float *ws = prm + off_ws(l) + k * W, *wn = prm + off_wn(l) + k * W;
    const float *dz = dZ + (size_t)r * W;
    float a = 0.f, b = 0.f;
    for (int f = 0; f < W; ++f) {
        a = __fmaf_rn(dz[f], ws[f], a);
        b = __fmaf_rn(dz[f], wn[f], b);
    }
    dHs[t] = a;
    dT[t] = b;
}

// Adam (bias-corrected) on the FP32 master weights; the forward copy keeps
// the weight matrices rounded to BF16 and the biases as stored.
__global__ void adam_kernel(float *__restrict__ theta, float *__restrict__ fwd, const float *__restrict__ grad,
                            float *__restrict__ m, float *__restrict__ v, float inv_batch, float lr, float b1,
                            float b2, float eps, float c1, float c2, int n) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    const float g = grad[t] * inv_batch;
    const float mt = b1 * m[t] + (1.f - b1) * g;
    const float vt = b2 * v[t] + (1.f - b2) * g * g;
    m[t] = mt;
    v[t] = vt;
    const float th = theta[t] - lr * (mt / c1) / (sqrtf(vt / c2) + eps);
    theta[t] = th;
    bool is_w = false;
    for (int l = 1; l <= LAYERS; ++l)
        if (t >= off_ws(l) && t < off_b(l)) is_w = true;
    fwd[t] = is_w ? __bfloat162float(__float2bfloat16_rn(th)) : th;
}

__global__ void round_params_kernel(const float *__restrict__ theta, float *__restrict__ fwd, int n) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    bool is_w = false;
    for (int l = 1; l <= LAYERS; ++l)
        if (t >= off_ws(l) && t < off_b(l)) is_w = true;
    fwd[t] = is_w ? __bfloat162float(__float2bfloat16_rn(theta[t])) : theta[t];
}

// ---------------------------------------------------------------- host side
struct HostGraph {
    int n = 0;
    std::vector<float> x;                        // n x FIN
    std::vector<int> pptr, pcol, tptr, tcol;     // P and P^T in CSR
    std::vector<float> pval, tval;
};

// Features and aggregation of one graph (see the file header).
qpr_status build_graph(int64_t n, int64_t m, const int64_t *src, const int64_t *dst, const double *w, double alpha,
                       double omega, HostGraph &out, std::string &err) {
    HostOps h;
    const qpr_status st = assemble_host(n, m, src, dst, w, QPR_HDIAG_ZERO, h, err);
    if (st != QPR_OK) return st;
    // A entries (i, j, a) from the CSR of S: A_ij = S_ij outDeg(j)
    struct E { int i, j; double a; };
    std::vector<E> ents;
    for (int64_t i = 0; i < n; ++i)
        for (int q = h.sptr[i]; q < h.sptr[i + 1]; ++q) ents.push_back({(int)i, h.scol[q], h.sval[q] * h.outdeg[h.scol[q]]});
    std::vector<double> instr(n, 0.0);
    std::vector<int> indeg(n, 0), outdeg_cnt(n, 0);
    for (const E &e : ents) {
        instr[e.i] += e.a;
        indeg[e.i] += 1;
        outdeg_cnt[e.j] += 1;
    }
    // classical PageRank: pi <- G pi, renormalised, 200 steps from uniform
    std::vector<double> pi(n, 1.0 / (double)n), nx(n);
    const double inv_nm1 = 1.0 / (double)(n - 1);
    for (int it = 0; it < 200; ++it) {
        double P = 0.0, D = 0.0;
        for (int64_t j = 0; j < n; ++j) {
            P += pi[j];
            if (h.dang[j]) D += pi[j];
        }
        double tot = 0.0;
        for (int64_t i = 0; i < n; ++i) {
            double s = 0.0;
            for (int q = h.sptr[i]; q < h.sptr[i + 1]; ++q) s += h.sval[q] * pi[h.scol[q]];
            const double dterm = (D - (h.dang[i] ? pi[i] : 0.0)) * inv_nm1;
            nx[i] = alpha * (s + dterm) + (1.0 - alpha) * (P - pi[i]) * inv_nm1;
            tot += nx[i];
        }
        for (int64_t i = 0; i < n; ++i) pi[i] = nx[i] / tot;
    }
    out.n = (int)n;
    out.x.assign((size_t)n * FIN, 0.f);
    for (int64_t i = 0; i < n; ++i) {
        float *x = &out.x[(size_t)i * FIN];
        x[0] = 1.f;
        x[1] = (float)omega;
        x[2] = (float)log1p(instr[i]);
        x[3] = (float)log1p(h.outdeg[i]);
        x[4] = (float)log1p((double)indeg[i]);
        x[5] = (float)log1p((double)outdeg_cnt[i]);
        x[6] = (float)log((double)n * pi[i]);
        x[7] = h.dang[i] ? 1.f : 0.f;
    }
    // B = A + A^T, P = B row-normalised, and its transpose
    std::vector<E> b;
    for (const E &e : ents) {
        b.push_back({e.i, e.j, e.a});
        b.push_back({e.j, e.i, e.a});
    }
    std::sort(b.begin(), b.end(), [](const E &x, const E &y) { return x.i != y.i ? x.i < y.i : x.j < y.j; });
    std::vector<E> bu;
    for (const E &e : b) {
        if (!bu.empty() && bu.back().i == e.i && bu.back().j == e.j) bu.back().a += e.a;
        else bu.push_back(e);
    }
    std::vector<double> rs(n, 0.0);
    for (const E &e : bu) rs[e.i] += e.a;
    out.pptr.assign(n + 1, 0);
    for (const E &e : bu) {
        out.pcol.push_back(e.j);
        out.pval.push_back((float)(e.a / rs[e.i]));
        out.pptr[e.i + 1]++;
    }
    for (int64_t i = 0; i < n; ++i) out.pptr[i + 1] += out.pptr[i];
    std::vector<E> t;
    for (size_t q = 0; q < bu.size(); ++q) t.push_back({bu[q].j, bu[q].i, (double)out.pval[q]});
    std::sort(t.begin(), t.end(), [](const E &x, const E &y) { return x.i != y.i ? x.i < y.i : x.j < y.j; });
    out.tptr.assign(n + 1, 0);
    for (const E &e : t) {
        out.tcol.push_back(e.j);
        out.tval.push_back((float)e.a);
        out.tptr[e.i + 1]++;
    }
    for (int64_t i = 0; i < n; ++i) out.tptr[i + 1] += out.tptr[i];
    return QPR_OK;
}

uint64_t splitmix(uint64_t &s) {
    uint64_t z = (s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

}  // namespace
}  // namespace qpr

struct qpr_gnn {
    int device = 0;
    cudaStream_t stream = nullptr;
    float *theta = nullptr, *fwd = nullptr, *grad = nullptr, *m = nullptr, *v = nullptr;
    int64_t adam_t = 0;
    // per-graph device workspace (grown on demand)
    int cap_n = 0, cap_nnz = 0;
    float *x = nullptr, *H[5] = {}, *M[5] = {}, *Z[5] = {}, *dH = nullptr, *dHs = nullptr, *dT = nullptr;
    float *ds = nullptr, *sbuf = nullptr, *part = nullptr;
    int *pptr = nullptr, *pcol = nullptr, *tptr = nullptr, *tcol = nullptr;
    float *pval = nullptr, *tval = nullptr;
    double *p = nullptr, *p_hat = nullptr, *loss = nullptr;
    std::vector<void *> bufs;
    std::string err;
};

namespace {

using qpr::FIN;
using qpr::W;

qpr_status gnn_fail(qpr_gnn *g, qpr_status st, const std::string &msg) {
    if (g) g->err = msg;
    qpr::set_create_error(msg);
    return st;
}

#define GCUDA(g, call)                                                                                     \
    do {                                                                                                   \
        cudaError_t e_ = (call);                                                                           \
        if (e_ != cudaSuccess)                                                                             \
            return gnn_fail(g, e_ == cudaErrorMemoryAllocation ? QPR_E_OOM : QPR_E_CUDA,                   \
                            std::string(#call) + ": " + cudaGetErrorString(e_));                           \
    } while (0)

template <class T>
cudaError_t galloc(qpr_gnn *g, T **p, size_t count) {
    void *q = nullptr;
    cudaError_t e = cudaMalloc(&q, std::max<size_t>(count, 1) * sizeof(T));
    if (e == cudaSuccess) {
        g->bufs.push_back(q);
        *p = (T *)q;
    }
    return e;
}

void free_ws(qpr_gnn *g) {
    // workspace buffers are those allocated after the five parameter arrays
    while (g->bufs.size() > 5) {
        cudaFree(g->bufs.back());
        g->bufs.pop_back();
    }
    g->cap_n = g->cap_nnz = 0;
}

qpr_status ensure_ws(qpr_gnn *g, int n, int nnz) {
    if (n <= g->cap_n && nnz <= g->cap_nnz) return QPR_OK;
    free_ws(g);
    const int cn = std::max(n, g->cap_n), cz = std::max(nnz, g->cap_nnz);
    GCUDA(g, galloc(g, &g->x, (size_t)cn * FIN));
    for (int l = 1; l <= qpr::LAYERS; ++l) {
        GCUDA(g, galloc(g, &g->H[l], (size_t)cn * W));
        GCUDA(g, galloc(g, &g->M[l], (size_t)cn * W));
        GCUDA(g, galloc(g, &g->Z[l], (size_t)cn * W));
    }
    GCUDA(g, galloc(g, &g->dH, (size_t)cn * W));
    GCUDA(g, galloc(g, &g->dHs, (size_t)cn * W));
    GCUDA(g, galloc(g, &g->dT, (size_t)cn * W));
    GCUDA(g, galloc(g, &g->ds, cn));
    GCUDA(g, galloc(g, &g->sbuf, cn));
    const int nblk = (cn + qpr::kRowsWG - 1) / qpr::kRowsWG;
    GCUDA(g, galloc(g, &g->part, (size_t)nblk * (2 * W * W + W)));
    GCUDA(g, galloc(g, &g->pptr, cn + 1));
    GCUDA(g, galloc(g, &g->tptr, cn + 1));
    GCUDA(g, galloc(g, &g->pcol, cz));
    GCUDA(g, galloc(g, &g->tcol, cz));
    GCUDA(g, galloc(g, &g->pval, cz));
    GCUDA(g, galloc(g, &g->tval, cz));
    GCUDA(g, galloc(g, &g->p, cn));
    GCUDA(g, galloc(g, &g->p_hat, cn));
    GCUDA(g, galloc(g, &g->loss, 1));
    g->cap_n = cn;
    g->cap_nnz = cz;
    return QPR_OK;
}

qpr_status upload_graph(qpr_gnn *g, const qpr::HostGraph &hg, const double *p) {
    const int n = hg.n, nnz = (int)hg.pcol.size();
    qpr_status st = ensure_ws(g, n, std::max(nnz, 1));
    if (st != QPR_OK) return st;
    cudaStream_t s = g->stream;
    GCUDA(g, cudaMemcpyAsync(g->x, hg.x.data(), hg.x.size() * sizeof(float), cudaMemcpyHostToDevice, s));
    GCUDA(g, cudaMemcpyAsync(g->pptr, hg.pptr.data(), (n + 1) * sizeof(int), cudaMemcpyHostToDevice, s));
    GCUDA(g, cudaMemcpyAsync(g->tptr, hg.tptr.data(), (n + 1) * sizeof(int), cudaMemcpyHostToDevice, s));
    if (nnz > 0) {
        GCUDA(g, cudaMemcpyAsync(g->pcol, hg.pcol.data(), nnz * sizeof(int), cudaMemcpyHostToDevice, s));
        GCUDA(g, cudaMemcpyAsync(g->tcol, hg.tcol.data(), nnz * sizeof(int), cudaMemcpyHostToDevice, s));
        GCUDA(g, cudaMemcpyAsync(g->pval, hg.pval.data(), nnz * sizeof(float), cudaMemcpyHostToDevice, s));
        GCUDA(g, cudaMemcpyAsync(g->tval, hg.tval.data(), nnz * sizeof(float), cudaMemcpyHostToDevice, s));
    }
    if (p) GCUDA(g, cudaMemcpyAsync(g->p, p, n * sizeof(double), cudaMemcpyHostToDevice, s));
    // the host vectors die with the caller: finish the copies now
    GCUDA(g, cudaStreamSynchronize(s));
    return QPR_OK;
}

// Forward pass (and, with a target, loss and backward into g->grad).
void enqueue_pass(qpr_gnn *g, int n, bool with_target, bool backward) {
    cudaStream_t s = g->stream;
    const int wpb = 8, rows_blocks = (n + wpb - 1) / wpb;
    const float *h = g->x;
    g->H[0] = g->x;
    for (int l = 1; l <= qpr::LAYERS; ++l) {
        const int din = qpr::din_of(l);
        qpr::spmm_rows_kernel<<<rows_blocks, 256, 0, s>>>(g->pptr, g->pcol, g->pval, h, g->M[l], n, din, 0);
        qpr::dense_fwd_kernel<<<(n + 31) / 32, 256, 0, s>>>(h, g->M[l], g->fwd, l, n, g->Z[l], g->H[l]);
        h = g->H[l];
    }
    qpr::softmax_loss_kernel<<<1, 256, 0, s>>>(g->H[qpr::LAYERS], g->fwd, with_target ? g->p : nullptr, n, g->p_hat,
                                             g->ds, g->loss, g->sbuf);
    if (!backward) return;
    const int nblk = (n + qpr::kRowsWG - 1) / qpr::kRowsWG;
    qpr::readout_bwd_kernel<<<nblk, W, 0, s>>>(g->H[qpr::LAYERS], g->ds, g->fwd, n, g->dH, g->part);
    qpr::reduce_parts_kernel<<<1, 128, 0, s>>>(g->part, nblk, W + 1, g->grad + qpr::OFF_WO);
    for (int l = qpr::LAYERS; l >= 1; --l) {
        const int din = qpr::din_of(l);
        const float *hin = (l == 1) ? g->x : g->H[l - 1];
        qpr::wgrad_kernel<<<nblk, 256, 0, s>>>(hin, g->M[l], g->Z[l], g->dH, n, din, g->part);
        const int per = 2 * din * W + W;
        qpr::reduce_parts_kernel<<<(per + 255) / 256, 256, 0, s>>>(g->part, nblk, per, g->grad + qpr::off_ws(l));
        if (l > 1) {
            const size_t tot = (size_t)n * din;
            qpr::dense_bwd_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(g->dH, g->fwd, l, n, g->dHs, g->dT);
            // dH_{l-1} = dHs + P^T dT
            qpr::spmm_rows_kernel<<<rows_blocks, 256, 0, s>>>(g->tptr, g->tcol, g->tval, g->dT, g->dHs, n, din, 1);
            std::swap(g->dH, g->dHs);
        }
    }
}

}  // namespace

extern "C" {

int64_t qpr_gnn_param_count(void) { return qpr::kParams; }

void qpr_gnn_destroy(qpr_gnn *g) {
    if (!g) return;
    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(g->device);
    if (g->stream) cudaStreamSynchronize(g->stream);
    for (void *p : g->bufs) cudaFree(p);
    if (g->stream) cudaStreamDestroy(g->stream);
    cudaGetLastError();
    if (prev >= 0) cudaSetDevice(prev);
    delete g;
}

qpr_status qpr_gnn_create(qpr_gnn **out, uint64_t seed, int32_t device) {
    if (!out) return QPR_E_ARG;
    *out = nullptr;
    qpr_gnn *g = new (std::nothrow) qpr_gnn();
    if (!g) return gnn_fail(nullptr, QPR_E_OOM, "host allocation failed");
    if (device < 0) {
        if (cudaGetDevice(&g->device) != cudaSuccess) {
            cudaGetLastError();
            delete g;
            return gnn_fail(nullptr, QPR_E_CUDA, "no CUDA device available");
        }
    } else {
        g->device = device;
    }
    cudaSetDevice(g->device);
    auto bail = [&](qpr_status st) {
        qpr_gnn_destroy(g);
        return st;
    };
    const int P = qpr::kParams;
    if (galloc(g, &g->theta, P) != cudaSuccess || galloc(g, &g->fwd, P) != cudaSuccess ||
        galloc(g, &g->grad, P) != cudaSuccess || galloc(g, &g->m, P) != cudaSuccess ||
        galloc(g, &g->v, P) != cudaSuccess || cudaStreamCreateWithFlags(&g->stream, cudaStreamNonBlocking) != cudaSuccess)
        return bail(gnn_fail(nullptr, QPR_E_OOM, "device allocation failed"));
    // Glorot-uniform weights from splitmix64(seed), zero biases
    std::vector<float> th(P, 0.f);
    uint64_t st = seed;
    for (int l = 1; l <= qpr::LAYERS; ++l) {
        const int din = qpr::din_of(l);
        const double lim = sqrt(6.0 / (double)(2 * din + W));
        for (int t = qpr::off_ws(l); t < qpr::off_b(l); ++t)
            th[t] = (float)(lim * (2.0 * ((double)(qpr::splitmix(st) >> 11) * (1.0 / 9007199254740992.0)) - 1.0));
    }
    const double limo = sqrt(6.0 / (double)(W + 1));
    for (int t = qpr::OFF_WO; t < qpr::OFF_BO; ++t)
        th[t] = (float)(limo * (2.0 * ((double)(qpr::splitmix(st) >> 11) * (1.0 / 9007199254740992.0)) - 1.0));
    if (cudaMemcpy(g->theta, th.data(), P * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemset(g->m, 0, P * sizeof(float)) != cudaSuccess || cudaMemset(g->v, 0, P * sizeof(float)) != cudaSuccess)
        return bail(gnn_fail(nullptr, QPR_E_CUDA, "parameter upload failed"));
    qpr::round_params_kernel<<<(P + 255) / 256, 256, 0, g->stream>>>(g->theta, g->fwd, P);
    if (cudaStreamSynchronize(g->stream) != cudaSuccess) return bail(gnn_fail(nullptr, QPR_E_CUDA, "init failed"));
    *out = g;
    return QPR_OK;
}

qpr_status qpr_gnn_get_params(qpr_gnn *g, float *host) {
    if (!g || !host) return QPR_E_ARG;
    cudaSetDevice(g->device);
    GCUDA(g, cudaMemcpy(host, g->theta, qpr::kParams * sizeof(float), cudaMemcpyDeviceToHost));
    return QPR_OK;
}

qpr_status qpr_gnn_set_params(qpr_gnn *g, const float *host) {
    if (!g || !host) return QPR_E_ARG;
    cudaSetDevice(g->device);
    GCUDA(g, cudaMemcpy(g->theta, host, qpr::kParams * sizeof(float), cudaMemcpyHostToDevice));
    qpr::round_params_kernel<<<(qpr::kParams + 255) / 256, 256, 0, g->stream>>>(g->theta, g->fwd, qpr::kParams);
    GCUDA(g, cudaMemset(g->m, 0, qpr::kParams * sizeof(float)));
    GCUDA(g, cudaMemset(g->v, 0, qpr::kParams * sizeof(float)));
    g->adam_t = 0;
    GCUDA(g, cudaStreamSynchronize(g->stream));
    return QPR_OK;
}

qpr_status qpr_gnn_predict(qpr_gnn *g, int64_t n, int64_t m, const int64_t *src, const int64_t *dst, const double *w,
                           double alpha, double omega, double *p_hat) {
    if (!g || !p_hat) return QPR_E_ARG;
    if (n < 2 || !(alpha >= 0.0 && alpha <= 1.0) || !(omega >= 0.0 && omega <= 1.0))
        return gnn_fail(g, QPR_E_ARG, "n < 2 or alpha/omega outside [0, 1]");
    cudaSetDevice(g->device);
    qpr::HostGraph hg;
    std::string e;
    qpr_status st = qpr::build_graph(n, m, src, dst, w, alpha, omega, hg, e);
    if (st != QPR_OK) return gnn_fail(g, st, e);
    st = upload_graph(g, hg, nullptr);
    if (st != QPR_OK) return st;
    enqueue_pass(g, (int)n, false, false);
    GCUDA(g, cudaMemcpyAsync(p_hat, g->p_hat, n * sizeof(double), cudaMemcpyDefault, g->stream));
    GCUDA(g, cudaStreamSynchronize(g->stream));
    GCUDA(g, cudaGetLastError());
    return QPR_OK;
}

qpr_status qpr_gnn_loss_grad(qpr_gnn *g, const qpr_gnn_sample *smp, double alpha, double *loss, float *grad) {
    if (!g || !smp || !smp->p) return QPR_E_ARG;
    cudaSetDevice(g->device);
    qpr::HostGraph hg;
    std::string e;
    qpr_status st = qpr::build_graph(smp->n, smp->m, smp->src, smp->dst, smp->w, alpha, smp->omega, hg, e);
    if (st != QPR_OK) return gnn_fail(g, st, e);
    st = upload_graph(g, hg, smp->p);
    if (st != QPR_OK) return st;
    GCUDA(g, cudaMemsetAsync(g->grad, 0, qpr::kParams * sizeof(float), g->stream));
    GCUDA(g, cudaMemsetAsync(g->loss, 0, sizeof(double), g->stream));
    enqueue_pass(g, (int)smp->n, true, true);
    if (loss) GCUDA(g, cudaMemcpyAsync(loss, g->loss, sizeof(double), cudaMemcpyDeviceToHost, g->stream));
    if (grad) GCUDA(g, cudaMemcpyAsync(grad, g->grad, qpr::kParams * sizeof(float), cudaMemcpyDeviceToHost, g->stream));
    GCUDA(g, cudaStreamSynchronize(g->stream));
    GCUDA(g, cudaGetLastError());
    return QPR_OK;
}

qpr_status qpr_gnn_train(qpr_gnn *g, int64_t count, const qpr_gnn_sample *samples, double alpha, int32_t epochs,
                         int32_t batch, double lr, uint64_t seed, double *epoch_loss) {
    if (!g || count < 1 || !samples || epochs < 1 || batch < 1 || !(lr > 0.0)) return QPR_E_ARG;
    cudaSetDevice(g->device);
    std::vector<qpr::HostGraph> hg((size_t)count);
    for (int64_t i = 0; i < count; ++i) {
        if (!samples[i].p) return gnn_fail(g, QPR_E_ARG, "sample without target populations");
        std::string e;
        const qpr_status st = qpr::build_graph(samples[i].n, samples[i].m, samples[i].src, samples[i].dst,
                                               samples[i].w, alpha, samples[i].omega, hg[i], e);
        if (st != QPR_OK) return gnn_fail(g, st, "sample " + std::to_string(i) + ": " + e);
    }
    {
        int maxn = 2, maxz = 1;
        for (const qpr::HostGraph &h : hg) {
            maxn = std::max(maxn, h.n);
            maxz = std::max(maxz, (int)h.pcol.size());
        }
        const qpr_status st = ensure_ws(g, maxn, maxz);
        if (st != QPR_OK) return st;
    }
    std::vector<int64_t> order((size_t)count);
    for (int64_t i = 0; i < count; ++i) order[i] = i;
    uint64_t rs = seed;
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    for (int ep = 0; ep < epochs; ++ep) {
        for (int64_t i = count - 1; i > 0; --i) std::swap(order[i], order[qpr::splitmix(rs) % (uint64_t)(i + 1)]);
        GCUDA(g, cudaMemsetAsync(g->loss, 0, sizeof(double), g->stream));
        for (int64_t b0 = 0; b0 < count; b0 += batch) {
            const int64_t b1i = std::min<int64_t>(count, b0 + batch);
            GCUDA(g, cudaMemsetAsync(g->grad, 0, qpr::kParams * sizeof(float), g->stream));
            for (int64_t k = b0; k < b1i; ++k) {
                const int64_t i = order[k];
                qpr_status st = upload_graph(g, hg[i], samples[i].p);
                if (st != QPR_OK) return st;
                enqueue_pass(g, hg[i].n, true, true);
            }
            ++g->adam_t;
            const float c1 = 1.f - powf(b1, (float)g->adam_t), c2 = 1.f - powf(b2, (float)g->adam_t);
            qpr::adam_kernel<<<(qpr::kParams + 255) / 256, 256, 0, g->stream>>>(
                g->theta, g->fwd, g->grad, g->m, g->v, 1.f / (float)(b1i - b0), (float)lr, b1, b2, eps, c1, c2,
                qpr::kParams);
        }
        double l = 0.0;
        GCUDA(g, cudaMemcpyAsync(&l, g->loss, sizeof(double), cudaMemcpyDeviceToHost, g->stream));
        GCUDA(g, cudaStreamSynchronize(g->stream));
        GCUDA(g, cudaGetLastError());
        if (epoch_loss) epoch_loss[ep] = l / (double)count;
    }
    return QPR_OK;
}

}  // extern "C"
