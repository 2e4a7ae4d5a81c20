// Dense mixed-form RK4 stage on the 5th-generation tensor cores (tcgen05).
//
// X = H delta for an FP32 stage delta is formed as a 3-term split-BF16
// product with FP32 accumulation: H = H0 + H1 + H2 and delta = d0 + d1 + d2
// (each term the BF16 rounding of what the previous terms left), and
//     X = sum over i + j <= 2 of H_i d_j
// (six BF16 products, concatenated along K into one GEMM of depth 6 N; the
// dropped terms are below 2^-24 relative). Because delta is Hermitian the
// B operand of output tile J is K-major with rows [Re delta_J ; -Im delta_J],
// so one MMA with M = 128 (rows of tile I) and N = 256 yields both the real
// part (columns 0..127) and the imaginary part (128..255) of X_IJ.
//
// One CTA owns the tile pair (I, J), I <= J, of 128 x 128 complex tiles and
// accumulates X_IJ and X_JI in TMEM (2 x 256 FP32 columns = all 512). Warp 0
// (one thread) streams operand tiles with TMA (128-byte swizzle, four stages),
// warp 1 (one thread) issues tcgen05.mma and commits to mbarriers, and all
// eight warps run the fused epilogue: X_JI is staged in shared memory for
// the transposed read, the Lindblad right-hand side of the delta and the RK4
// stage update are formed as in the sparse mixed kernel, tile (I, J) and its
// conjugate transpose are written, together with the BF16 split of the next
// stage's delta (the B operand of the next GEMM).
//
// Every mbarrier wait gives up after a bounded number of polls, sets
// ctl->err_timeout and skips the rest of the work; TMEM is always released.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>
#include <math.h>

#include "mixed_body.cuh"
#include "qpr_internal.cuh"
#include "tma_util.cuh"

namespace qpr {
namespace {

constexpr int TB = kTileTc;             // 128
constexpr int BK = 64;                  // BF16 K per stage: one 128-byte swizzle row
constexpr int NSTAGE = 4;
constexpr int A_BYTES = TB * BK * 2;        // 16 KB
constexpr int B_BYTES = 2 * TB * BK * 2;    // 32 KB (Re rows then -Im rows)
constexpr int OFF_A = 0, OFF_B = A_BYTES;
constexpr int STAGE_BYTES = A_BYTES + B_BYTES;  // 48 KB
constexpr int NTHREADS = 256;
// Epilogue, per chunk of EC columns b of tile (I, J): X_JI rows b staged as
// [EC][LDX2] (A 128 | B 128), X_IJ columns b as [TB][LDY] (A EC | B EC), and
// the chunk's outputs transposed as 4 x [EC][LDO2] for the mirrored write;
// the paddings make every access pattern below bank-conflict free.
constexpr int EC = 32;
constexpr int LDX2 = 2 * TB + 1;
constexpr int LDY = 2 * EC + 1;
constexpr int LDO2 = TB + 1;
constexpr int SMEM_PIPE = NSTAGE * STAGE_BYTES;
constexpr int SMEM_EPI = (EC * LDX2 + TB * LDY + 4 * EC * LDO2) * 4;
constexpr int SMEM_BYTES = (SMEM_PIPE > SMEM_EPI ? SMEM_PIPE : SMEM_EPI) + 1024;  // + alignment slack
constexpr uint32_t TMEM_COLS = 512;

static_assert(SMEM_BYTES <= 227 * 1024, "shared memory");

using tma::mbar_expect_tx;
using tma::mbar_init;
using tma::mbar_wait;
using tma::smem_u32;
using tma::load_3d;
using tma::load_4d;

// Shared-memory matrix descriptor: K-major operand in the canonical 128-byte
// swizzled layout written by TMA (8 rows x 128 B atoms, 1024 B between
// 8-row groups).
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFF);          // start address
    d |= (uint64_t)1 << 16;                          // leading byte offset (unused for swizzled K-major)
    d |= (uint64_t)((1024 >> 4) & 0x3FFF) << 32;     // stride byte offset: 8 rows x 128 B
    d |= (uint64_t)1 << 46;                          // descriptor version
    d |= (uint64_t)2 << 61;                          // 128-byte swizzle
    return d;
}

// Instruction descriptor, kind::f16: BF16 A and B (K-major), FP32 D, M = 128, N = 256.
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(256 >> 3) << 17) |
                            ((uint32_t)(128 >> 4) << 24);

__device__ __forceinline__ void umma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t accumulate) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(kIdesc), "r"(accumulate));
}
__device__ __forceinline__ void umma_commit(uint64_t *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                     smem_u32(bar))
                 : "memory");
}
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,"
        "%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]),
          "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]),
          "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void split3(float x, __nv_bfloat16 &h0, __nv_bfloat16 &h1, __nv_bfloat16 &h2) {
    h0 = __float2bfloat16_rn(x);
    const float r1 = x - __bfloat162float(h0);
    h1 = __float2bfloat16_rn(r1);
    const float r2 = r1 - __bfloat162float(h1);
    h2 = __float2bfloat16_rn(r2);
}

// Write the split of one delta entry (re, im) at offset o of the B-operand
// planes [level][plane][row][k]: plane 0 holds Re delta (symmetric), plane 1
// holds -Im delta (so the mirrored entry, conj, stores +im there).
__device__ __forceinline__ void put_split(__nv_bfloat16 *sp, size_t plane, size_t o, float re, float im) {
    __nv_bfloat16 r0, r1, r2, i0, i1, i2;
    split3(re, r0, r1, r2);
    split3(-im, i0, i1, i2);
    sp[0 * plane + o] = r0; sp[2 * plane + o] = r1; sp[4 * plane + o] = r2;
    sp[1 * plane + o] = i0; sp[3 * plane + o] = i1; sp[5 * plane + o] = i2;
}

template <int STAGE>
__global__ void __launch_bounds__(NTHREADS, 1)
stage_mixed_tc_kernel(DevOps ops, MixedWork w, const __grid_constant__ CUtensorMap tmH,
                      const __grid_constant__ CUtensorMap tmIn) {
    extern __shared__ uint8_t smem_raw[];
    __shared__ uint64_t full_bar[NSTAGE], empty_bar[NSTAGE], accum_bar;
    __shared__ uint32_t tmem_base_sh;
    __shared__ int s_done, s_fail;
    __shared__ float red[NTHREADS / 32];
    uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);

    Ctl *ctl = w.ctl;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) {
        s_done = *(volatile int *)&ctl->done;
        s_fail = 0;
    }
    __syncthreads();
    if (s_done) return;

    const int I = w.pairs_tc[blockIdx.x].x, J = w.pairs_tc[blockIdx.x].y;
    const bool diag = (I == J);
    const int np = ops.np;
    const size_t plane = (size_t)np * np;
    const int kb_per_seg = np / BK;
    const int nkb = 6 * kb_per_seg;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(
                         smem_u32(&tmem_base_sh)),
                     "r"(TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::);
    }
    if (tid == 32) {
        for (int s = 0; s < NSTAGE; ++s) {
            mbar_init(&full_bar[s], 1);
            mbar_init(&empty_bar[s], 1);
        }
        mbar_init(&accum_bar, 1);
        tma::mbar_init_fence();
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    const uint32_t tmem = tmem_base_sh;
    const uint32_t tm_ij = tmem, tm_ji = tmem + 256;

    // split segments s = 0..5: A level i and B level j with i + j <= 2, in the
    // order (0,2) (1,1) (2,0) (0,1) (1,0) (0,0), one hex digit per segment.
    // The tensor core's FP32 accumulation does not round to nearest, so its
    // error grows with every K-step added to a large accumulator: the small
    // correction products go first and the dominant H0 d0 product last.
    constexpr uint32_t kSegI = 0x010210u, kSegJ = 0x001012u;

    // Two passes over K: X_IJ = H_I. delta_.J, then (off the diagonal) X_JI =
    // H_J. delta_.I, each K block one stage of A (16 KB) and B (32 KB), so
    // NSTAGE = 4 stages keep three loads in flight behind the MMAs.
    const int nit = diag ? nkb : 2 * nkb;
    if (warp == 0 && lane == 0) {
        // TMA producer
        for (int it = 0; it < nit; ++it) {
            const int st = it % NSTAGE;
            if (it >= NSTAGE && !mbar_wait(&empty_bar[st], ((it / NSTAGE) - 1) & 1)) {
                atomicExch(&s_fail, 1);
                break;
            }
            const int pass = it / nkb, kb = it - pass * nkb;
            const int rt = pass ? J : I, ct = pass ? I : J;  // row tile of H, column tile of delta
            const int seg = kb / kb_per_seg;
            const int k0 = (kb - seg * kb_per_seg) * BK;
            const int li = (int)((kSegI >> (4 * seg)) & 0xFu), lj = (int)((kSegJ >> (4 * seg)) & 0xFu);
            uint8_t *sb = smem + st * STAGE_BYTES;
            mbar_expect_tx(&full_bar[st], (uint32_t)STAGE_BYTES);
            load_3d(sb + OFF_A, &tmH, &full_bar[st], k0, rt * TB, li);
            load_4d(sb + OFF_B, &tmIn, &full_bar[st], k0, ct * TB, 0, lj);
            load_4d(sb + OFF_B + B_BYTES / 2, &tmIn, &full_bar[st], k0, ct * TB, 1, lj);
        }
    } else if (warp == 1 && lane == 0) {
        // MMA issuer
        for (int it = 0; it < nit; ++it) {
            const int st = it % NSTAGE;
            if (!mbar_wait(&full_bar[st], (it / NSTAGE) & 1)) {
                atomicExch(&s_fail, 1);
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
            const int pass = it / nkb, kb = it - pass * nkb;
            const uint32_t sb = smem_u32(smem + st * STAGE_BYTES);
            const uint64_t dA = sw128_desc(sb + OFF_A), dB = sw128_desc(sb + OFF_B);
            const uint32_t tm_d = pass ? tm_ji : tm_ij;
#pragma unroll
            for (int kk = 0; kk < BK / 16; ++kk) {
                const uint64_t adv = (uint64_t)((kk * 32) >> 4);  // 16 BF16 = 32 bytes along K
                const uint32_t acc = (kb > 0 || kk > 0) ? 1u : 0u;
                umma_bf16(tm_d, dA + adv, dB + adv, acc);
            }
            umma_commit(&empty_bar[st]);
        }
        umma_commit(&accum_bar);
    }
    __syncwarp();

    // ---- epilogue (all warps) ----
    const bool ok_acc = mbar_wait(&accum_bar, 0);
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    __syncthreads();
    if (!ok_acc || s_fail) {
        if (tid == 0) atomicExch(&ctl->err_timeout, 1);
    } else {
        const int q = warp & 3;             // TMEM lane quarter this warp may read
        const int h = warp >> 2;            // A (0) or B (1) columns
        const uint32_t lane_off = (uint32_t)(q * 32) << 16;
        // aliases the pipeline buffers (every MMA has completed)
        float *sX = reinterpret_cast<float *>(smem);
        float *sY = sX + EC * LDX2;
        float *sO = sY + TB * LDY;
        const uint32_t src_ji = diag ? tm_ij : tm_ji;  // X_JI (X_IJ on the diagonal)

        const float om = ops.omega32, cm = 1.0f - om;
        const float dtf = ctl->dtf, dtl = ctl->dtl;
        // c_s dt of the next stage input (dt / 4 and dt / 2 exact from fl(dt); fl(dt / 3))
        const float cst = (STAGE == 1) ? 0.25f * dtf : (STAGE == 2 ? ctl->dt3 : 0.5f * dtf);
        const float *__restrict__ din = (STAGE == 1) ? w.D : (STAGE == 3 ? w.db : w.da);
        float *dnext = (STAGE == 2) ? w.db : w.da;
        __nv_bfloat16 *snext = (STAGE == 2) ? w.splitB : (STAGE == 4 ? w.splitD : w.splitA);
        float nrm = 0.f;
        for (int cb = 0; cb < TB / EC; ++cb) {
            // X_IJ[a][cb EC ..] (A or B) for every row a; X_JI rows b of this chunk
            {
                float v[32];
                tmem_ld32(tm_ij + lane_off + (uint32_t)(h * TB + cb * EC), v);
                const int a = q * 32 + lane;
#pragma unroll
                for (int i = 0; i < 32; ++i) sY[a * LDY + h * EC + i] = v[i];
            }
            if (q == cb) {
                for (int c = 0; c < TB; c += 32) {
                    float v[32];
                    tmem_ld32(src_ji + lane_off + (uint32_t)(h * TB + c), v);
#pragma unroll
                    for (int i = 0; i < 32; ++i) sX[lane * LDX2 + h * TB + c + i] = v[i];
                }
            }
            __syncthreads();
            // elements (a, b) of tile (I, J), lanes along b: the direct accesses are coalesced
            const int c = lane, b = cb * EC + c, gb = J * TB + b;
            const float cb32 = ops.c32[gb];
            for (int a = warp; a < TB; a += NTHREADS / 32) {
                const int ga = I * TB + a;
                const size_t off = (size_t)ga * np + gb;
                const float Aab = sY[a * LDY + c], Bab = sY[a * LDY + EC + c];
                const float Aba = sX[c * LDX2 + a], Bba = sX[c * LDX2 + TB + a];
                const float dr = din[off], di = din[plane + off];
                const float hc = 0.5f * (ops.c32[ga] + cb32);
                float kdr = cm * (Bab + Bba) - om * hc * dr;
                const float kdi = -cm * (Aab - Aba) - om * hc * di;
                if (ga == gb) kdr += om * w.g[ga];
                float o0, o1, o2, o3;  // the outputs the mirrored write needs
                if (STAGE <= 3) {
                    // the nested RK4 form: the next input D + c dt (F + f(delta))
                    const float kr = kdr + w.F32[off], ki = kdi + w.F32[plane + off];
                    if (STAGE == 1) nrm += kr * kr + ki * ki;
                    const float Dr = (STAGE == 1) ? dr : w.D[off], Di = (STAGE == 1) ? di : w.D[plane + off];
                    const float nr = Dr + cst * kr, ni = Di + cst * ki;
                    dnext[off] = nr; dnext[plane + off] = ni;
                    put_split(snext, plane, off, nr, ni);
                    o0 = 0.f; o1 = 0.f; o2 = nr; o3 = ni;
                } else {
                    // delta += dt F + dt f(delta_4) in float-float
                    const mixed::ff vr =
                        mixed::delta_update(w.D[off], w.Dlo[off], w.Ghi[off], w.Glo[off], dtf, dtl, kdr);
                    const mixed::ff vi = mixed::delta_update(w.D[plane + off], w.Dlo[plane + off], w.Ghi[plane + off],
                                                             w.Glo[plane + off], dtf, dtl, kdi);
                    w.D[off] = vr.hi; w.D[plane + off] = vi.hi;
                    w.Dlo[off] = vr.lo; w.Dlo[plane + off] = vi.lo;
                    put_split(snext, plane, off, vr.hi, vi.hi);
                    o0 = vr.lo; o1 = vi.lo; o2 = vr.hi; o3 = vi.hi;
                }
                if (!diag) {
                    sO[(0 * EC + c) * LDO2 + a] = o0;
                    sO[(1 * EC + c) * LDO2 + a] = o1;
                    sO[(2 * EC + c) * LDO2 + a] = o2;
                    sO[(3 * EC + c) * LDO2 + a] = o3;
                }
            }
            __syncthreads();
            if (!diag) {
                // the conjugate of the chunk at (b, a) of tile (J, I), lanes along a: coalesced
                for (int e = warp; e < EC * (TB / 32); e += NTHREADS / 32) {
                    const int cc = e >> 2, a = (e & 3) * 32 + lane;
                    const int gb2 = J * TB + cb * EC + cc, ga2 = I * TB + a;
                    const size_t moff = (size_t)gb2 * np + ga2;
                    const float o0 = sO[(0 * EC + cc) * LDO2 + a], o1 = sO[(1 * EC + cc) * LDO2 + a];
                    const float o2 = sO[(2 * EC + cc) * LDO2 + a], o3 = sO[(3 * EC + cc) * LDO2 + a];
                    if (STAGE <= 3) {
                        dnext[moff] = o2; dnext[plane + moff] = -o3;
                    } else {
                        w.Dlo[moff] = o0; w.Dlo[plane + moff] = -o1;
                        w.D[moff] = o2; w.D[plane + moff] = -o3;
                    }
                    put_split(snext, plane, moff, o2, -o3);
                }
            }
            __syncthreads();  // the chunk's buffers are reused by the next
        }
        if (STAGE == 1) {
            nrm = mixed::warp_sum_f(nrm);
            if (lane == 0) red[warp] = nrm;
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    if (STAGE == 1 && tid == 0 && ok_acc && !s_fail) {
        float s = 0.f;
        for (int i = 0; i < NTHREADS / 32; ++i) s += red[i];
        w.partials32[blockIdx.x] = diag ? s : 2.0f * s;
    }
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(TMEM_COLS));
    }
    if (STAGE == 4 && blockIdx.x == 0 && tid == 0) ctl->step += 1;
}

template <int STAGE>
cudaError_t set_attr() {
    return cudaFuncSetAttribute(stage_mixed_tc_kernel<STAGE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                SMEM_BYTES);
}

PFN_cuTensorMapEncodeTiled_v12000 get_encode_impl() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        cudaDriverEntryPointQueryResult q;
        void *p = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
    }
    return fn;
}

}  // namespace

PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() { return get_encode_impl(); }

cudaError_t init_mixed_tc() {
    cudaError_t e = set_attr<1>();
    if (e == cudaSuccess) e = set_attr<2>();
    if (e == cudaSuccess) e = set_attr<3>();
    if (e == cudaSuccess) e = set_attr<4>();
    return e;
}

// Tensor maps: H planes [3][np][np] and delta-split planes [3][2][np][np],
// BF16, boxes of 64 (K) x 128 rows, 128-byte swizzle.
bool make_tc_maps(const DevOps &ops, const __nv_bfloat16 *hsplit, const __nv_bfloat16 *const dsplit[3],
                  TcMaps *maps) {
    PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
    if (!enc) return false;
    const cuuint64_t np = (cuuint64_t)ops.np;
    {
        cuuint64_t dims[3] = {np, np, 3};
        cuuint64_t strides[2] = {np * 2, np * np * 2};
        cuuint32_t box[3] = {BK, TB, 1};
        cuuint32_t es[3] = {1, 1, 1};
        if (enc(&maps->h, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, (void *)hsplit, dims, strides, box, es,
                CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return false;
    }
    for (int i = 0; i < 3; ++i) {
        cuuint64_t dims[4] = {np, np, 2, 3};
        cuuint64_t strides[3] = {np * 2, np * np * 2, 2 * np * np * 2};
        cuuint32_t box[4] = {BK, TB, 1, 1};
        cuuint32_t es[4] = {1, 1, 1, 1};
        if (enc(&maps->d[i], CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, (void *)dsplit[i], dims, strides, box, es,
                CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return false;
    }
    return true;
}

// Stage input split planes: stage 1 D (map 0), stage 2 da (map 1), stage 3
// db (map 2), stage 4 da (map 1).
void launch_mixed_tc(int stage, const DevOps &ops, const MixedWork &w, const TcMaps &m, cudaStream_t s) {
    switch (stage) {
        case 1: stage_mixed_tc_kernel<1><<<w.npairs_tc, NTHREADS, SMEM_BYTES, s>>>(ops, w, m.h, m.d[0]); break;
        case 2: stage_mixed_tc_kernel<2><<<w.npairs_tc, NTHREADS, SMEM_BYTES, s>>>(ops, w, m.h, m.d[1]); break;
        case 3: stage_mixed_tc_kernel<3><<<w.npairs_tc, NTHREADS, SMEM_BYTES, s>>>(ops, w, m.h, m.d[2]); break;
        default: stage_mixed_tc_kernel<4><<<w.npairs_tc, NTHREADS, SMEM_BYTES, s>>>(ops, w, m.h, m.d[1]); break;
    }
}

}  // namespace qpr
