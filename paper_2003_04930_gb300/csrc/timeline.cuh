// Kernel timeline of the column-block RK4 stage, for the diagnostic build
// only (compiled with -DQPR_TIMELINE into libqpr_timeline.so; the product
// library has none of it). For every launch of the SpMM grid and of the
// epilogue, per stage, it records on the global nanosecond timer the first
// and last CTA to enter and to leave, and for the whole-block SpMM the first
// and last product CTA to have its column block staged and to finish its
// rows. Differences between consecutive kernels' exits give the critical
// path of a step inside a captured graph with programmatic dependent launch,
// which profilers, serialising the launches, do not show.
#pragma once

#include "tma_util.cuh"

namespace qpr {
namespace timeline {

constexpr int kKinds = 8;    // (stage - 1) * 2 + {0: SpMM grid, 1: epilogue}
constexpr int kInst = 2048;  // launches kept per kind (a ring)
constexpr int kFields = 4;   // {entered, left, staged, product rows done}, each as (first, last)

#ifdef QPR_TIMELINE
// internal linkage: the instrumented kernels and the exports live in one
// translation unit (stage_cols.cu), which reads its own copy
static __device__ unsigned long long g_stamp[kKinds][kInst][2 * kFields];
static __device__ unsigned long long g_count[kKinds];

__device__ __forceinline__ int &slot() {
    __shared__ int s;
    return s;
}
__device__ __forceinline__ int &kind() {
    __shared__ int s;
    return s;
}
__device__ __forceinline__ void put(int k, int i, int f, unsigned long long t) {
    atomicMin(&g_stamp[k][i][2 * f], t);
    atomicMax(&g_stamp[k][i][2 * f + 1], t);
}
#endif

// Called by every thread at kernel entry (ends with a barrier).
__device__ __forceinline__ void enter(int k) {
#ifdef QPR_TIMELINE
    if (threadIdx.x == 0) {
        const unsigned long long t = tma::global_ns();
        const int i = (int)((atomicAdd(&g_count[k], 1ull) / gridDim.x) % kInst);
        slot() = i;
        kind() = k;
        put(k, i, 0, t);
    }
    __syncthreads();
#endif
}

// Called by every thread when the CTA is done (starts with a barrier).
__device__ __forceinline__ void leave() {
#ifdef QPR_TIMELINE
    __syncthreads();
    if (threadIdx.x == 0) put(kind(), slot(), 1, tma::global_ns());
#endif
}

// Field f (2: staged, 3: rows done) of an instrumented kernel (ON); thread 0.
template <bool ON>
__device__ __forceinline__ void mark(int f) {
#ifdef QPR_TIMELINE
    if (ON && threadIdx.x == 0) put(kind(), slot(), f, tma::global_ns());
#endif
}

// The same once every thread of the CTA has reached it (a barrier first).
template <bool ON>
__device__ __forceinline__ void mark_all(int f) {
#ifdef QPR_TIMELINE
    if (ON) {
        __syncthreads();
        mark<ON>(f);
    }
#endif
}

}  // namespace timeline
}  // namespace qpr
