// ens_spmv_f32.cuh -- the FP32-accumulated ensemble SpMV on FP32 or BF16
// values (the inner solver of the mixed-precision CG and the FP32 V-cycle of
// the multigrid): per row the same 2-partial entry order as the FP64 SpMV.
#pragma once
#include "ens_spmv.cuh"

namespace ens {

// streaming 8-byte load (4 BF16 values) for data read exactly once
__device__ __forceinline__ uint2 ld_stream_u2(const void *p) {
    uint2 v;
    asm volatile("ld.global.cs.v2.u32 {%0, %1}, [%2];" : "=r"(v.x), "=r"(v.y) : "l"(p));
    return v;
}

// --------------------------------------------------- FP32 SpMV row evaluation
template <typename V>
struct ValLoad32;
template <>
struct ValLoad32<float> {
    __device__ __forceinline__ static float2 two(const float *v, int64_t i) {
        return ld_stream(reinterpret_cast<const float2 *>(v + i));
    }
    __device__ __forceinline__ static float4 four(const float *v, int64_t i) {
        return ld_stream(reinterpret_cast<const float4 *>(v + i));
    }
    __device__ __forceinline__ static float one(const float *v, int64_t i) { return ld_stream(v + i); }
};
template <>
struct ValLoad32<__nv_bfloat16> {
    __device__ __forceinline__ static float2 two(const __nv_bfloat16 *v, int64_t i) {
        const uint32_t u = ld_stream_u32(v + i);
        return make_float2(__uint_as_float(u << 16), __uint_as_float(u & 0xffff0000u));
    }
    __device__ __forceinline__ static float4 four(const __nv_bfloat16 *v, int64_t i) {
        const uint2 u = ld_stream_u2(v + i);
        return make_float4(__uint_as_float(u.x << 16), __uint_as_float(u.x & 0xffff0000u),
                           __uint_as_float(u.y << 16), __uint_as_float(u.y & 0xffff0000u));
    }
    __device__ __forceinline__ static float one(const __nv_bfloat16 *v, int64_t i) {
        return __uint_as_float(((uint32_t)ld_stream_u16(v + i)) << 16);
    }
};

// members (2g, 2g+1); same 2-partial order as the FP64 SpMV; + diag * x_row
template <int S, typename V, typename CA>
__device__ __forceinline__ float2 row_spmv2_f32(CA colf, int rs, int re, const V *__restrict__ vals,
                                                const float *__restrict__ x, int g) {
    float a0 = 0.f, a1 = 0.f, b0 = 0.f, b1 = 0.f;
    const int m = 2 * g;
    int j = rs;
    for (; j + 4 <= re; j += 4) {
        const int c0 = colf(j), c1 = colf(j + 1), c2 = colf(j + 2), c3 = colf(j + 3);
        const float2 v0 = ValLoad32<V>::two(vals, (int64_t)j * S + m);
        const float2 v1 = ValLoad32<V>::two(vals, (int64_t)(j + 1) * S + m);
        const float2 v2 = ValLoad32<V>::two(vals, (int64_t)(j + 2) * S + m);
        const float2 v3 = ValLoad32<V>::two(vals, (int64_t)(j + 3) * S + m);
        const float2 x0 = __ldg(reinterpret_cast<const float2 *>(x + (int64_t)c0 * S + m));
        const float2 x1 = __ldg(reinterpret_cast<const float2 *>(x + (int64_t)c1 * S + m));
        const float2 x2 = __ldg(reinterpret_cast<const float2 *>(x + (int64_t)c2 * S + m));
        const float2 x3 = __ldg(reinterpret_cast<const float2 *>(x + (int64_t)c3 * S + m));
        a0 = __fmaf_rn(v0.x, x0.x, a0); b0 = __fmaf_rn(v0.y, x0.y, b0);
        a1 = __fmaf_rn(v1.x, x1.x, a1); b1 = __fmaf_rn(v1.y, x1.y, b1);
        a0 = __fmaf_rn(v2.x, x2.x, a0); b0 = __fmaf_rn(v2.y, x2.y, b0);
        a1 = __fmaf_rn(v3.x, x3.x, a1); b1 = __fmaf_rn(v3.y, x3.y, b1);
    }
    for (; j < re; ++j) {
        const float2 v = ValLoad32<V>::two(vals, (int64_t)j * S + m);
        const float2 xv = __ldg(reinterpret_cast<const float2 *>(x + (int64_t)colf(j) * S + m));
        if ((j - rs) & 1) { a1 = __fmaf_rn(v.x, xv.x, a1); b1 = __fmaf_rn(v.y, xv.y, b1); }
        else { a0 = __fmaf_rn(v.x, xv.x, a0); b0 = __fmaf_rn(v.y, xv.y, b0); }
    }
    return make_float2(__fadd_rn(a0, a1), __fadd_rn(b0, b1));
}

// members 4g .. 4g+3 from 16-byte (FP32) or 8-byte (BF16) loads: per member
// the same two partials over alternate entries as row_spmv2_f32, so the
// result is bitwise that of the 2-member form
__device__ __forceinline__ void fma4(float4 &a, const float4 v, const float4 x) {
    a.x = __fmaf_rn(v.x, x.x, a.x);
    a.y = __fmaf_rn(v.y, x.y, a.y);
    a.z = __fmaf_rn(v.z, x.z, a.z);
    a.w = __fmaf_rn(v.w, x.w, a.w);
}
template <int S, typename V, typename CA>
__device__ __forceinline__ float4 row_spmv4_f32(CA colf, int rs, int re, const V *__restrict__ vals,
                                                const float *__restrict__ x, int g) {
    float4 a = make_float4(0.f, 0.f, 0.f, 0.f), b = a;  // even / odd entry offsets
    const int m = 4 * g;
    int j = rs;
    for (; j + 4 <= re; j += 4) {
        const int c0 = colf(j), c1 = colf(j + 1), c2 = colf(j + 2), c3 = colf(j + 3);
        const float4 v0 = ValLoad32<V>::four(vals, (int64_t)j * S + m);
        const float4 v1 = ValLoad32<V>::four(vals, (int64_t)(j + 1) * S + m);
        const float4 v2 = ValLoad32<V>::four(vals, (int64_t)(j + 2) * S + m);
        const float4 v3 = ValLoad32<V>::four(vals, (int64_t)(j + 3) * S + m);
        const float4 x0 = __ldg(reinterpret_cast<const float4 *>(x + (int64_t)c0 * S + m));
        const float4 x1 = __ldg(reinterpret_cast<const float4 *>(x + (int64_t)c1 * S + m));
        const float4 x2 = __ldg(reinterpret_cast<const float4 *>(x + (int64_t)c2 * S + m));
        const float4 x3 = __ldg(reinterpret_cast<const float4 *>(x + (int64_t)c3 * S + m));
        fma4(a, v0, x0);
        fma4(b, v1, x1);
        fma4(a, v2, x2);
        fma4(b, v3, x3);
    }
    for (; j < re; ++j) {
        const float4 v = ValLoad32<V>::four(vals, (int64_t)j * S + m);
        const float4 xv = __ldg(reinterpret_cast<const float4 *>(x + (int64_t)colf(j) * S + m));
        if ((j - rs) & 1) fma4(b, v, xv);
        else fma4(a, v, xv);
    }
    return make_float4(__fadd_rn(a.x, b.x), __fadd_rn(a.y, b.y), __fadd_rn(a.z, b.z), __fadd_rn(a.w, b.w));
}

template <typename V, typename CA>
__device__ __forceinline__ float row_spmv1_f32(CA colf, int rs, int re, const V *__restrict__ vals,
                                               const float *__restrict__ x, int g, bool valid) {
    float a = 0.f;
    if (valid)
        for (int j = rs + g; j < re; j += 2) a = __fmaf_rn(ValLoad32<V>::one(vals, j), __ldg(x + colf(j)), a);
    const float o = __shfl_xor_sync(0xffffffffu, a, 1);
    return (g == 0) ? __fadd_rn(a, o) : __fadd_rn(o, a);
}

template <int S, typename V>
__device__ __forceinline__ float2 chunk_spmv_f32(const ChunkCols &cc, bool staged,
                                                 const int32_t *__restrict__ col,
                                                 const V *__restrict__ vals,
                                                 const float *__restrict__ diag,
                                                 const float *__restrict__ x, int r, int g,
                                                 int64_t R, bool valid) {
    const int rs = valid ? cc.rm[r] : 0, re = valid ? cc.rm[r + 1] : 0;
    float2 y;
    if constexpr (S == 1) {
        const float v = staged ? row_spmv1_f32<V>(ColShared{cc.col, cc.base}, rs, re, vals, x, g, valid)
                               : row_spmv1_f32<V>(ColGlobal{col}, rs, re, vals, x, g, valid);
        y = make_float2(v, 0.f);
        if (diag && valid) y.x = __fmaf_rn(diag[R], x[R], y.x);
    } else {
        if (!valid) return make_float2(0.f, 0.f);
        y = staged ? row_spmv2_f32<S, V>(ColShared{cc.col, cc.base}, rs, re, vals, x, g)
                   : row_spmv2_f32<S, V>(ColGlobal{col}, rs, re, vals, x, g);
        if (diag) {
            const float2 d = reinterpret_cast<const float2 *>(diag)[R * (S / 2) + g];
            const float2 xr = reinterpret_cast<const float2 *>(x)[R * (S / 2) + g];
            y.x = __fmaf_rn(d.x, xr.x, y.x);
            y.y = __fmaf_rn(d.y, xr.y, y.y);
        }
    }
    return y;
}

// 4 members per thread (S >= 8: S/4 threads per row); + diag * x_row
template <int S, typename V>
__device__ __forceinline__ float4 chunk_spmv4_f32(const ChunkCols &cc, bool staged,
                                                  const int32_t *__restrict__ col,
                                                  const V *__restrict__ vals,
                                                  const float *__restrict__ diag,
                                                  const float *__restrict__ x, int r, int g,
                                                  int64_t R, bool valid) {
    static_assert(S % 4 == 0, "4 members per thread");
    if (!valid) return make_float4(0.f, 0.f, 0.f, 0.f);
    const int rs = cc.rm[r], re = cc.rm[r + 1];
    float4 y = staged ? row_spmv4_f32<S, V>(ColShared{cc.col, cc.base}, rs, re, vals, x, g)
                      : row_spmv4_f32<S, V>(ColGlobal{col}, rs, re, vals, x, g);
    if (diag) {
        const float4 d = reinterpret_cast<const float4 *>(diag)[R * (S / 4) + g];
        const float4 xr = reinterpret_cast<const float4 *>(x)[R * (S / 4) + g];
        y.x = __fmaf_rn(d.x, xr.x, y.x);
        y.y = __fmaf_rn(d.y, xr.y, y.y);
        y.z = __fmaf_rn(d.z, xr.z, y.z);
        y.w = __fmaf_rn(d.w, xr.w, y.w);
    }
    return y;
}

}  // namespace ens
