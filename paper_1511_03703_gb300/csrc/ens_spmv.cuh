// ens_spmv.cuh -- device building blocks of the ensemble SpMV (Fig. 5 semantics).
//
// Mapping (GB300-first, not the paper's Kokkos warp mapping): a CTA owns one
// chunk of 32 consecutive rows.  For s >= 2 each row gets G = s/2 threads and
// thread g owns members 2g and 2g+1, so one entry's s values are read as one
// contiguous run of 16-byte loads (s*8 bytes) and x[col*s + 2g..] as one
// coalesced 16-byte gather; the column index is one broadcast load per row.
// For s = 1 each row gets 4 threads that stride over the row's entries.
//
// Summation order (identical for every s, so member e's result does not
// depend on the ensemble it is solved in): entry j of a row goes to partial
// j mod 4, each partial accumulates with FMA in increasing j, and the row
// value is (p0 + p1) + (p2 + p3).
#pragma once
#include "ens_internal.cuh"

namespace ens {

template <int S>
struct RowMap {
    static constexpr int G = (S == 1) ? 4 : S / 2;  // threads per row
    static constexpr int THREADS = 32 * G;          // one 32-row chunk per CTA
};

// -------------------------------------------------- value loads (2 members)
template <typename V>
struct ValLoad;

template <>
struct ValLoad<double> {
    __device__ __forceinline__ static double2 two(const double *v, int64_t i) {
        return ld_stream(reinterpret_cast<const double2 *>(v + i));
    }
    __device__ __forceinline__ static double one(const double *v, int64_t i) { return ld_stream(v + i); }
};

template <>
struct ValLoad<float> {
    __device__ __forceinline__ static double2 two(const float *v, int64_t i) {
        float2 f = ld_stream(reinterpret_cast<const float2 *>(v + i));
        return make_double2((double)f.x, (double)f.y);
    }
    __device__ __forceinline__ static double one(const float *v, int64_t i) { return (double)ld_stream(v + i); }
};

template <>
struct ValLoad<__nv_bfloat16> {
    __device__ __forceinline__ static double2 two(const __nv_bfloat16 *v, int64_t i) {
        uint32_t u = ld_stream_u32(v + i);
        float lo = __uint_as_float(u << 16), hi = __uint_as_float(u & 0xffff0000u);
        return make_double2((double)lo, (double)hi);
    }
    __device__ __forceinline__ static double one(const __nv_bfloat16 *v, int64_t i) {
        uint16_t u = ld_stream_u16(v + i);
        return (double)__uint_as_float(((uint32_t)u) << 16);
    }
};

__device__ __forceinline__ double2 ld_x2(const double *x, int64_t i) {
    return __ldg(reinterpret_cast<const double2 *>(x + i));
}

// y for members (2g, 2g+1) of row R, s >= 2, FP64 accumulation
template <int S, typename V>
__device__ __forceinline__ double2 row_spmv2(const int32_t *__restrict__ row_map,
                                             const int32_t *__restrict__ col,
                                             const V *__restrict__ vals,
                                             const double *__restrict__ x, int64_t R, int g) {
    const int rs = __ldg(row_map + R), re = __ldg(row_map + R + 1);
    double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;  // member 2g, partials 0..3
    double b0 = 0.0, b1 = 0.0, b2 = 0.0, b3 = 0.0;  // member 2g+1
    const int m = 2 * g;
    int j = rs;
    for (; j + 4 <= re; j += 4) {
        const int c0 = __ldg(col + j), c1 = __ldg(col + j + 1), c2 = __ldg(col + j + 2),
                  c3 = __ldg(col + j + 3);
        const double2 v0 = ValLoad<V>::two(vals, (int64_t)j * S + m);
        const double2 v1 = ValLoad<V>::two(vals, (int64_t)(j + 1) * S + m);
        const double2 v2 = ValLoad<V>::two(vals, (int64_t)(j + 2) * S + m);
        const double2 v3 = ValLoad<V>::two(vals, (int64_t)(j + 3) * S + m);
        const double2 x0 = ld_x2(x, (int64_t)c0 * S + m);
        const double2 x1 = ld_x2(x, (int64_t)c1 * S + m);
        const double2 x2 = ld_x2(x, (int64_t)c2 * S + m);
        const double2 x3 = ld_x2(x, (int64_t)c3 * S + m);
        a0 = fma(v0.x, x0.x, a0); b0 = fma(v0.y, x0.y, b0);
        a1 = fma(v1.x, x1.x, a1); b1 = fma(v1.y, x1.y, b1);
        a2 = fma(v2.x, x2.x, a2); b2 = fma(v2.y, x2.y, b2);
        a3 = fma(v3.x, x3.x, a3); b3 = fma(v3.y, x3.y, b3);
    }
    if (j < re) {
        const double2 v = ValLoad<V>::two(vals, (int64_t)j * S + m);
        const double2 xv = ld_x2(x, (int64_t)__ldg(col + j) * S + m);
        a0 = fma(v.x, xv.x, a0); b0 = fma(v.y, xv.y, b0);
    }
    if (j + 1 < re) {
        const double2 v = ValLoad<V>::two(vals, (int64_t)(j + 1) * S + m);
        const double2 xv = ld_x2(x, (int64_t)__ldg(col + j + 1) * S + m);
        a1 = fma(v.x, xv.x, a1); b1 = fma(v.y, xv.y, b1);
    }
    if (j + 2 < re) {
        const double2 v = ValLoad<V>::two(vals, (int64_t)(j + 2) * S + m);
        const double2 xv = ld_x2(x, (int64_t)__ldg(col + j + 2) * S + m);
        a2 = fma(v.x, xv.x, a2); b2 = fma(v.y, xv.y, b2);
    }
    return make_double2((a0 + a1) + (a2 + a3), (b0 + b1) + (b2 + b3));
}

// y of row R for s = 1: 4 threads (g = 0..3, consecutive lanes) per row; the
// result is returned on all 4 lanes.  Must be called by full warps.
template <typename V>
__device__ __forceinline__ double row_spmv1(const int32_t *__restrict__ row_map,
                                            const int32_t *__restrict__ col,
                                            const V *__restrict__ vals,
                                            const double *__restrict__ x, int64_t R, int g,
                                            bool valid) {
    double a = 0.0;
    if (valid) {
        const int rs = __ldg(row_map + R), re = __ldg(row_map + R + 1);
        for (int j = rs + g; j < re; j += 4) a = fma(ValLoad<V>::one(vals, j), __ldg(x + __ldg(col + j)), a);
    }
    a += __shfl_xor_sync(0xffffffffu, a, 1);   // p0+p1 | p2+p3
    a += __shfl_xor_sync(0xffffffffu, a, 2);   // (p0+p1)+(p2+p3)
    return a;
}

// Level-1 tree step: every thread of the CTA holds the per-row products of its
// (row r, members 2g, 2g+1) [s >= 2] or (row r) [s = 1, value on all G lanes].
// Writes the chunk's per-member partials to t.buf[1][chunk*width + off + e].
template <int S>
__device__ __forceinline__ void chunk_tree(double (*sm)[S + 1], double v0, double v1, int r,
                                           int g, const DotTree &t, int64_t chunk, int off) {
    if constexpr (S == 1) {
        if (g == 0) sm[r][0] = v0;
    } else {
        sm[r][2 * g] = v0;
        sm[r][2 * g + 1] = v1;
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int e = warp; e < S; e += nw) {
        double v = warp_tree32(sm[lane][e]);
        if (lane == 0) t.buf[1][chunk * t.width + off + e] = v;
    }
    __syncthreads();
}

}  // namespace ens
