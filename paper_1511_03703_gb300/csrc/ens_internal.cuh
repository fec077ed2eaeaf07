// ens_internal.cuh -- shared device/host helpers of the CUDA library (not the oracle).
#pragma once
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>
#include <stdio.h>

#include "../../include/ens.h"

namespace ens {

// ------------------------------------------------------------ error state
void set_error(const char *fmt, ...);
int fail(int status, const char *fmt, ...);
int cuda_fail(cudaError_t err, const char *what);

#define ENS_CUDA_TRY(expr)                                        \
    do {                                                          \
        cudaError_t _e = (expr);                                  \
        if (_e != cudaSuccess) return ::ens::cuda_fail(_e, #expr); \
    } while (0)

#define ENS_LAUNCH_CHECK(what)                                     \
    do {                                                           \
        cudaError_t _e = cudaGetLastError();                       \
        if (_e != cudaSuccess) return ::ens::cuda_fail(_e, what);  \
    } while (0)

inline cudaStream_t as_stream(void *s) { return reinterpret_cast<cudaStream_t>(s); }
inline bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }
inline bool supported_s(int s) { return s == 1 || s == 4 || s == 8 || s == 16 || s == 32; }

int check_graph(const ens_graph *g);

// Device-side convergence loop of the Krylov solvers: an instantiated CUDA
// graph whose while node replays a body (the caller's capture callback, run
// on a capture stream: one block of iterations) followed by a one-thread
// control kernel.  The control kernel counts blocks in *blocks and continues
// while (flags[0] | flags[1]) != 0 and fewer than max_blocks blocks ran, so
// the host synchronises once per solve instead of once per block.  The body
// runs at least once.  Returns ENS_OK, or an error (graph objects released;
// callers then fall back to the host-polled loop).  use_device_loop(): the
// ENS_DEVICE_LOOP environment variable (0 or 1, default 1).
using LoopBodyFn = int (*)(void *ctx, cudaStream_t cap);
int while_graph(LoopBodyFn body, void *ctx, const int32_t *flags, int32_t *blocks, int max_blocks,
                cudaGraph_t *graph_out, cudaGraphExec_t *exec_out);
bool use_device_loop();
// while_graph with a callable body(cudaStream_t cap) (a lambda with captures)
template <typename F>
inline int while_graph_fn(F &body, const int32_t *flags, int32_t *blocks, int max_blocks, cudaGraph_t *graph_out,
                          cudaGraphExec_t *exec_out) {
    LoopBodyFn fn = [](void *c, cudaStream_t cap) -> int {
        (*static_cast<F *>(c))(cap);
        return ENS_OK;
    };
    return while_graph(fn, &body, flags, blocks, max_blocks, graph_out, exec_out);
}
// launch an instantiated device-loop graph on st and release it (it stays
// alive until its replay completes)
inline int launch_while_graph(cudaGraph_t graph, cudaGraphExec_t exec, cudaStream_t st) {
    const cudaError_t ce = cudaGraphLaunch(exec, st);
    cudaGraphExecDestroy(exec);
    cudaGraphDestroy(graph);
    return ce == cudaSuccess ? ENS_OK : cuda_fail(ce, "device loop graph launch");
}

// -------------------------------------------------------- cache-hinted loads
// streaming loads for data read exactly once (matrix values): evict-first
__device__ __forceinline__ double2 ld_stream(const double2 *p) {
    double2 v;
    asm volatile("ld.global.cs.v2.f64 {%0, %1}, [%2];" : "=d"(v.x), "=d"(v.y) : "l"(p));
    return v;
}
__device__ __forceinline__ double ld_stream(const double *p) {
    double v;
    asm volatile("ld.global.cs.f64 %0, [%1];" : "=d"(v) : "l"(p));
    return v;
}
__device__ __forceinline__ float2 ld_stream(const float2 *p) {
    float2 v;
    asm volatile("ld.global.cs.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "l"(p));
    return v;
}
__device__ __forceinline__ float4 ld_stream(const float4 *p) {
    float4 v;
    asm volatile("ld.global.cs.v4.f32 {%0, %1, %2, %3}, [%4];"
                 : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "l"(p));
    return v;
}
__device__ __forceinline__ float ld_stream(const float *p) {
    float v;
    asm volatile("ld.global.cs.f32 %0, [%1];" : "=f"(v) : "l"(p));
    return v;
}
__device__ __forceinline__ uint32_t ld_stream_u32(const void *p) {
    uint32_t v;
    asm volatile("ld.global.cs.u32 %0, [%1];" : "=r"(v) : "l"(p));
    return v;
}
__device__ __forceinline__ uint16_t ld_stream_u16(const void *p) {
    uint16_t v;
    asm volatile("ld.global.cs.u16 %0, [%1];" : "=h"(v) : "l"(p));
    return v;
}
// the same load with the default cache policy (allocates in L1 and L2 at
// normal priority), for a line that the same warp reads again a few
// instructions later
__device__ __forceinline__ float4 ld_normal(const float4 *p) {
    float4 v;
    asm volatile("ld.global.v4.f32 {%0, %1, %2, %3}, [%4];"
                 : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "l"(p));
    return v;
}
// L2-coherent load that bypasses L1 (reads data written by other CTAs of the
// same kernel after a fence)
__device__ __forceinline__ double ld_cg(const double *p) {
    double v;
    asm volatile("ld.global.cg.f64 %0, [%1];" : "=d"(v) : "l"(p));
    return v;
}
__device__ __forceinline__ int ld_cg(const int *p) {
    int v;
    asm volatile("ld.global.cg.s32 %0, [%1];" : "=r"(v) : "l"(p));
    return v;
}

// ------------------------------------------------ deterministic dot trees
// Canonical per-member reduction shared by every dot product of the library
// (ens_dot and the CG kernels).  Level 0: one product per row.  Level 1: the
// 32 rows of a chunk [32c, 32c+32) are combined by the butterfly
//     t_i <- t_i + t_{i^16}, then ^8, ^4, ^2, ^1
// (rows past the end contribute 0).  Level l+1 combines 32 consecutive level-l
// results the same way, until one value per member remains.  The order
// depends only on the row index, never on s or on the launch shape, so a
// member's dot is bitwise the same at every ensemble size.
constexpr int kTreeMaxLevels = 8;

template <typename T>
struct DotTreeT {
    int levels;                       // number of levels above level 0 (>= 1)
    int width;                        // values per item = ndots * s
    int64_t count[kTreeMaxLevels];    // items at level l (level 1 = chunks)
    T *buf[kTreeMaxLevels];           // buf[l][item*width + w]
    int *counter[kTreeMaxLevels];     // counter[l][g]: arrivals of level-l items in group g
};
using DotTree = DotTreeT<double>;

template <typename T>
__device__ __forceinline__ T warp_tree32(T v) {
    v += __shfl_xor_sync(0xffffffffu, v, 16);
    v += __shfl_xor_sync(0xffffffffu, v, 8);
    v += __shfl_xor_sync(0xffffffffu, v, 4);
    v += __shfl_xor_sync(0xffffffffu, v, 2);
    v += __shfl_xor_sync(0xffffffffu, v, 1);
    return v;
}

__device__ __forceinline__ float ld_cg(const float *p) {
    float v;
    asm volatile("ld.global.cg.f32 %0, [%1];" : "=f"(v) : "l"(p));
    return v;
}

// Host: lay a tree out in caller scratch; returns bytes used (align 256).
size_t dot_tree_bytes(int64_t n_rows, int width, size_t elem = sizeof(double));
void dot_tree_layout_raw(int *levels, int64_t *count, void **buf, int **counter, int64_t n_rows,
                         int width, size_t elem, void *base);
template <typename T>
inline void dot_tree_layout(DotTreeT<T> *t, int64_t n_rows, int width, void *base) {
    void *bufs[kTreeMaxLevels] = {nullptr};
    t->width = width;
    for (int l = 0; l < kTreeMaxLevels; ++l) { t->count[l] = 0; t->buf[l] = nullptr; t->counter[l] = nullptr; }
    dot_tree_layout_raw(&t->levels, t->count, bufs, t->counter, n_rows, width, sizeof(T), base);
    for (int l = 0; l < kTreeMaxLevels; ++l) t->buf[l] = static_cast<T *>(bufs[l]);
}
// zero all arrival counters of a tree (the tree's kernels self-reset them)
int dot_tree_clear_raw(int levels, const int64_t *count, int *const *counter, cudaStream_t st);
template <typename T>
inline int dot_tree_clear(const DotTreeT<T> &t, cudaStream_t st) {
    return dot_tree_clear_raw(t.levels, t.count, t.counter, st);
}

// Device: called by all threads of a CTA after the CTA wrote the level-1
// items [item0, item0 + nitems) (buf[1][item*width ...], plain stores, all
// items inside one level-2 group, i.e. item0/32 == (item0+nitems-1)/32).
// Propagates through the levels; returns true in the single CTA that produced
// the top value (buf[levels][0..width)).  Release: the barrier orders the
// CTA's stores before thread 0's gpu-scope fence and arrival atomic (fences
// are cumulative); acquire: the last arriver fences after its atomic and the
// barrier orders the other threads' L2 reads after it.
// dot_tree_propagate_from starts at level `level` (its items [item0,
// item0 + nitems) written there); dot_tree_propagate is level 1.
template <typename T>
__device__ __forceinline__ bool dot_tree_propagate_from(const DotTreeT<T> &t, int level, int64_t item0, int nitems) {
    __shared__ int s_last;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;
    int64_t item = item0;
    int add = nitems;
    __syncthreads();
    for (int l = level; l < t.levels; ++l) {
        const int64_t g = item >> 5;
        const int cnt = (int)min((int64_t)32, t.count[l] - (g << 5));
        if (tid == 0) {
            __threadfence();
            const int old = atomicAdd(&t.counter[l][g], add);
            s_last = (old + add == cnt);
            if (s_last) {
                t.counter[l][g] = 0;  // self-reset for the next launch
                __threadfence();
            }
        }
        __syncthreads();
        if (!s_last) return false;
        const T *src = t.buf[l];
        T *dst = t.buf[l + 1];
        for (int w = warp; w < t.width; w += nwarps) {
            T v = (lane < cnt) ? ld_cg(src + ((g << 5) + lane) * t.width + w) : T(0);
            v = warp_tree32<T>(v);
            if (lane == 0) dst[g * t.width + w] = v;
        }
        __syncthreads();
        item = g;
        add = 1;
    }
    if (tid == 0) __threadfence();
    __syncthreads();
    return true;
}

template <typename T>
__device__ __forceinline__ bool dot_tree_propagate(const DotTreeT<T> &t, int64_t item0, int nitems) {
    return dot_tree_propagate_from(t, 1, item0, nitems);
}

// Level-1 group g of a tree whose level-1 items are complete (written by an
// earlier kernel): its 32 items reduced into level-2 item g exactly as the
// group's last arriver does in dot_tree_propagate; all threads of the CTA.
template <typename T>
__device__ __forceinline__ void dot_tree_reduce_group(const DotTreeT<T> &t, int64_t g) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const int cnt = (int)min((int64_t)32, t.count[1] - (g << 5));
    for (int w = warp; w < t.width; w += nwarps) {
        T v = (lane < cnt) ? ld_cg(t.buf[1] + ((g << 5) + lane) * t.width + w) : T(0);
        v = warp_tree32<T>(v);
        if (lane == 0) t.buf[2][g * t.width + w] = v;
    }
}

}  // namespace ens
