// ens_spmv.cuh -- device building blocks of the ensemble SpMV (Fig. 5 semantics).
//
// Mapping (GB300-first, not the paper's Kokkos warp mapping): a CTA owns one
// chunk of 32 consecutive rows.  For s >= 2 each row gets G = s/2 threads and
// thread g owns members 2g and 2g+1, so one entry's s values are read as one
// contiguous run of 16-byte loads (s*8 bytes) and x[col*s + 2g..] as one
// coalesced 16-byte gather; the column index is one broadcast load per row.
// For s = 1 each row gets 2 threads that take alternate entries.
//
// Summation order (identical for every s, so member e's result does not
// depend on the ensemble it is solved in): entry j of a row goes to partial
// j mod 2, each partial accumulates in increasing j, and the row value is
// p0 + p1.
//
// Two arithmetic forms of the FP64 product:
//  - native: IEEE FP64 FMA.  GB300 issues 2 DFMA per cycle per SM (1/64 of
//    its FP32 rate) and the ensemble SpMV needs one FMA per 8 bytes, so this
//    form is bound by the FP64 pipe near 60-65 % of the HBM bandwidth.
//  - double-float ("df"): each FP64 value is split into two floats (hi + lo,
//    truncation, 47 bits), x arrives pre-split, products are formed exactly
//    (hi*hi by FMA error recovery, cross terms in FP32) and sums carried as an
//    unevaluated float pair by TwoSum (Knuth; Dekker's double-float
//    arithmetic, 1971).  About 27 FP32/INT ops per term on the 128/cycle/SM
//    pipes; error per term <= ~6*2^-48 |a x|, so a row is within
//    ~1.2e-13 * sum |a_j x_j| of the exact value.  Values outside
//    [2^-103, 2^128) and non-finite values take an FP64 FMA instead.  The
//    float-pair error terms are exact only while the products stay in FP32's
//    normal range, so each member also tracks max |a_j x_j| (in FP32); a
//    member whose largest product lies in (0, 2^-96) is recomputed with FP64
//    FMAs (rows where every product is below 2^-149 return 0, an absolute
//    error below 27 * 2^-149).
#pragma once
#include <stddef.h>

#include "ens_internal.cuh"

namespace ens {

template <int S>
struct RowMap {
    static constexpr int G = (S == 1) ? 2 : S / 2;  // threads per row
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

// ------------------------------------------------------ column staging
// A CTA stages the row offsets and column indices of its 32-row chunk in
// shared memory, so each x gather waits for one shared load instead of a
// dependent global load.  The columns are copied with 16-byte loads, every
// load of a thread issued before its first shared store, starting at the
// chunk's first entry rounded down to a multiple of 4 (col[base] holds entry
// `base`).  Chunks with more than kColCap entries (not produced by the hex
// mesh, whose rows hold at most 27) read their columns from global memory.
constexpr int kColCap = 1024;

struct __align__(16) ChunkCols {
    int rm[33];
    int base;      // entry index of col[0]: the chunk's first entry rounded down to a multiple of 4
    int pad[2];
    int col[kColCap];
};
static_assert(offsetof(ChunkCols, col) % 16 == 0, "staged columns must be 16-byte aligned");

struct ColShared {
    const int *s;
    int base;
    __device__ __forceinline__ int operator()(int j) const { return s[j - base]; }
};
struct ColGlobal {
    const int32_t *p;
    __device__ __forceinline__ int operator()(int j) const { return __ldg(p + j); }
};

// columns [e0, e1) into cc.col (threads tid = 0..nthr-1 of the caller's group);
// reads only whole 16-byte groups inside [base, e1) plus at most 3 single
// entries before e1, so nothing past the chunk's last entry is touched.
// VEC = false: one entry per load.  U: 16-byte loads a thread issues before
// its first store -- 4 for groups of at most 128 threads (a hex-mesh chunk has
// up to 216 groups of 16 bytes), 1 for groups of 256 or more, where one pass
// covers the chunk and 4 in flight would only hold 16 more registers (the FP32
// power step went from 40 to 62 registers and 3 to 2 CTAs per SM with it).
template <bool VEC = true, int U = 1>
__device__ __forceinline__ void stage_cols(ChunkCols &cc, const int32_t *__restrict__ col, int e0, int e1,
                                           int tid, int nthr) {
    const int base = e0 & ~3;
    if (!VEC || (reinterpret_cast<uintptr_t>(col) & 15u)) {   // column array not 16-byte aligned: one entry per load
        for (int i = base + tid; i < e1; i += nthr) cc.col[i - base] = __ldg(col + i);
        if (tid == 0) cc.base = base;
        return;
    }
    const int v0 = base >> 2, v1 = e1 >> 2;
    const int nv = v1 - v0;
    const int4 *c4 = reinterpret_cast<const int4 *>(col) + v0;
    int4 *d4 = reinterpret_cast<int4 *>(cc.col);
    for (int k0 = tid; k0 < nv; k0 += U * nthr) {
        int4 t[U];
#pragma unroll
        for (int u = 0; u < U; ++u)
            if (k0 + u * nthr < nv) t[u] = __ldg(c4 + k0 + u * nthr);
#pragma unroll
        for (int u = 0; u < U; ++u)
            if (k0 + u * nthr < nv) d4[k0 + u * nthr] = t[u];
    }
    for (int i = 4 * max(v1, v0) + tid; i < e1; i += nthr) cc.col[i - base] = __ldg(col + i);
    if (tid == 0) cc.base = base;
}

__device__ __forceinline__ bool chunk_fits(int e0, int e1) { return e1 - (e0 & ~3) <= kColCap; }

// stage_cols' loads in flight per thread for a group of `threads` threads per chunk
constexpr int stage_unroll(int threads) { return threads <= 128 ? 4 : 1; }

// all threads of the CTA; returns true when the columns are staged
__device__ __forceinline__ bool stage_chunk(ChunkCols &cc, const int32_t *__restrict__ row_map,
                                            const int32_t *__restrict__ col, int64_t chunk,
                                            int32_t n) {
    const int64_t r0 = chunk * 32;
    const int nr = (int)min((int64_t)32, (int64_t)n - r0);
    for (int i = threadIdx.x; i <= nr; i += blockDim.x) cc.rm[i] = __ldg(row_map + r0 + i);
    __syncthreads();
    const int e0 = cc.rm[0], e1 = cc.rm[nr];
    const bool staged = chunk_fits(e0, e1);
    if (staged) stage_cols(cc, col, e0, e1, threadIdx.x, blockDim.x);
    __syncthreads();
    return staged;
}

// Staging with an L2 prefetch of the chunk's value block: once the row
// offsets are known, thread 0 asks the copy engine to bring up to cap bytes
// of the block [e0*bpe, e1*bpe) (16-byte aligned, clamped to the array of
// total_bytes) into L2 with evict-first priority, so the row loops' value
// loads hit L2 while the column indices are still being staged.
__device__ __forceinline__ void l2_prefetch_bulk(const void *base, uint64_t begin, uint64_t end,
                                                 uint64_t total_bytes, uint32_t cap) {
    begin &= ~(uint64_t)15;
    end = min((end + 15) & ~(uint64_t)15, total_bytes & ~(uint64_t)15);
    if (end > begin + cap) end = begin + cap;
    if (end <= begin) return;
    const char *p = static_cast<const char *>(base) + begin;
    uint64_t policy;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(policy));
    asm volatile("cp.async.bulk.prefetch.L2.global.L2::cache_hint [%0], %1, %2;"
                 :: "l"(p), "r"((uint32_t)(end - begin)), "l"(policy) : "memory");
}

// L2 prefetch of [begin, end) bytes of an array (rounded inward to 16-byte
// boundaries; normal eviction priority), for data a kernel reads soon
__device__ __forceinline__ void l2_prefetch_span(const void *base, uint64_t begin, uint64_t end) {
    begin = (begin + 15) & ~(uint64_t)15;
    end &= ~(uint64_t)15;
    if (end <= begin) return;
    const char *p = static_cast<const char *>(base) + begin;
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"((uint32_t)(end - begin)) : "memory");
}

template <bool VEC = true, int U = 1>
__device__ __forceinline__ bool stage_chunk_pf(ChunkCols &cc, const int32_t *__restrict__ row_map,
                                               const int32_t *__restrict__ col, int64_t chunk, int32_t n,
                                               const void *vbase, uint32_t bytes_per_entry,
                                               uint64_t total_bytes, uint32_t cap) {
    const int64_t r0 = chunk * 32;
    const int nr = (int)min((int64_t)32, (int64_t)n - r0);
    for (int i = threadIdx.x; i <= nr; i += blockDim.x) cc.rm[i] = __ldg(row_map + r0 + i);
    __syncthreads();
    const int e0 = cc.rm[0], e1 = cc.rm[nr];
    if (threadIdx.x == 0 && cap > 0)
        l2_prefetch_bulk(vbase, (uint64_t)e0 * bytes_per_entry, (uint64_t)e1 * bytes_per_entry, total_bytes, cap);
    const bool staged = chunk_fits(e0, e1);
    if (staged) stage_cols<VEC, U>(cc, col, e0, e1, threadIdx.x, blockDim.x);
    __syncthreads();
    return staged;
}

// Subset form used when one CTA works on NSUB chunks at once (nthr threads
// per chunk, ltid the thread's index inside its chunk): the same copy, with
// chunks past the end of the matrix left empty, and (cap > 0) each chunk's
// value block prefetched into L2 as in stage_chunk_pf.  All threads of the
// CTA call it.  U: see stage_cols.
template <int U = 1>
__device__ __forceinline__ bool stage_chunk_sub(ChunkCols &cc, const int32_t *__restrict__ row_map,
                                                const int32_t *__restrict__ col, int64_t chunk,
                                                int32_t n, int ltid, int nthr, const void *vbase = nullptr,
                                                uint32_t bytes_per_entry = 0, uint64_t total_bytes = 0,
                                                uint32_t cap = 0) {
    const int64_t r0 = chunk * 32;
    const int nr = (int)max((int64_t)0, min((int64_t)32, (int64_t)n - r0));
    if (nr > 0)
        for (int i = ltid; i <= nr; i += nthr) cc.rm[i] = __ldg(row_map + r0 + i);
    else if (ltid == 0)
        cc.rm[0] = 0;
    __syncthreads();
    const int e0 = cc.rm[0], e1 = (nr > 0) ? cc.rm[nr] : e0;
    if (ltid == 0 && cap > 0 && e1 > e0)
        l2_prefetch_bulk(vbase, (uint64_t)e0 * bytes_per_entry, (uint64_t)e1 * bytes_per_entry, total_bytes, cap);
    const bool staged = chunk_fits(e0, e1);
    if (staged) stage_cols<true, U>(cc, col, e0, e1, ltid, nthr);
    __syncthreads();
    return staged;
}

// ------------------------------------------------------------ native FP64
// y for members (2g, 2g+1) of a row with entries [rs, re), s >= 2
template <int S, typename V, typename CA>
__device__ __forceinline__ double2 row_spmv2(CA colf, int rs, int re, const V *__restrict__ vals,
                                             const double *__restrict__ x, int g) {
    double a0 = 0.0, a1 = 0.0;  // member 2g, partials 0 / 1
    double b0 = 0.0, b1 = 0.0;  // member 2g+1
    const int m = 2 * g;
    int j = rs;
    for (; j + 4 <= re; j += 4) {
        const int c0 = colf(j), c1 = colf(j + 1), c2 = colf(j + 2), c3 = colf(j + 3);
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
        a0 = fma(v2.x, x2.x, a0); b0 = fma(v2.y, x2.y, b0);
        a1 = fma(v3.x, x3.x, a1); b1 = fma(v3.y, x3.y, b1);
    }
    for (; j < re; ++j) {
        const double2 v = ValLoad<V>::two(vals, (int64_t)j * S + m);
        const double2 xv = ld_x2(x, (int64_t)colf(j) * S + m);
        if ((j - rs) & 1) { a1 = fma(v.x, xv.x, a1); b1 = fma(v.y, xv.y, b1); }
        else { a0 = fma(v.x, xv.x, a0); b0 = fma(v.y, xv.y, b0); }
    }
    return make_double2(a0 + a1, b0 + b1);
}

// y of a row for s = 1: 2 threads (g = 0, 1, adjacent lanes) per row; the
// result is returned on both lanes.  Must be called by full warps.
template <typename V, typename CA>
__device__ __forceinline__ double row_spmv1(CA colf, int rs, int re, const V *__restrict__ vals,
                                            const double *__restrict__ x, int g, bool valid) {
    double a = 0.0;
    if (valid)
        for (int j = rs + g; j < re; j += 2) a = fma(ValLoad<V>::one(vals, j), __ldg(x + colf(j)), a);
    a += __shfl_xor_sync(0xffffffffu, a, 1);   // p0 + p1 (commutative: same on both lanes)
    return a;
}

// --------------------------------------------------------- double-float
struct DfAcc {
    float s, c;   // unevaluated sum s + c
};

__device__ __forceinline__ DfAcc df_zero() { return DfAcc{0.0f, 0.0f}; }

// Knuth's TwoSum: s + e == a + b exactly, s = fl(a + b)
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// Split of a double into hi + lo floats by truncation of its fraction:
// hi keeps the sign, the exponent and the top 23 fraction bits, lo the next 23.
// Returns false (hi = lo = 0) when |a| is outside [2^-103, 2^128) or not
// finite; exact zero gives hi = lo = 0 and true.
__device__ __forceinline__ bool df_split_trunc(double a, float &hi, float &lo) {
    const uint32_t uh = (uint32_t)__double2hiint(a), ul = (uint32_t)__double2loint(a);
    const uint32_t e = (uh >> 20) & 0x7ffu;
    const uint32_t sgn = uh & 0x80000000u;
    const bool zero = (e == 0u);
    const bool ok = (e - 920u) <= 230u;  // 2^-103 <= |a| < 2^128
    const uint32_t frac_hi = __funnelshift_l(ul, uh, 3) & 0x7fffffu;
    const uint32_t hb = sgn | ((e - 896u) << 23) | frac_hi;
    const float one_f = __uint_as_float(0x3f800000u | ((ul & 0x1fffffffu) >> 6));
    const float scale = __uint_as_float(sgn | ((e - 919u) << 23));
    hi = ok ? __uint_as_float(hb) : 0.0f;
    lo = ok ? __fmul_rn(__fsub_rn(one_f, 1.0f), scale) : 0.0f;
    return ok || zero;
}

// Split of a vector element for the pre-split x: the same truncating split,
// integer and FP32 instructions only.  ok = false when v is non-zero and
// outside [2^-103, 2^128) (the caller then falls back to FP64 products).
__device__ __forceinline__ float2 df_split_vec(double v, bool &ok) {
    float hi, lo;
    const bool in = df_split_trunc(v, hi, lo);
    ok = in;
    return make_float2(hi, lo);
}

// Exact float -> double by moving the bit fields (no FP64-pipe conversion);
// zero, infinity and NaN by bits as well, subnormal floats (rare) out of
// line by the hardware conversion.
static __device__ __noinline__ double f2d_subnormal(float f) { return (double)f; }

__device__ __forceinline__ double f2d_exact(float f) {
    const uint32_t u = __float_as_uint(f);
    const uint32_t e = (u >> 23) & 0xffu, man = u & 0x7fffffu;
    if (e == 0u && man != 0u) return f2d_subnormal(f);
    const uint32_t de = (e == 0u) ? 0u : ((e == 0xffu) ? 0x7ffu : e + 896u);
    const uint32_t hi = (u & 0x80000000u) | (de << 20) | (man >> 3);
    const uint32_t lo = man << 29;
    return __hiloint2double((int)hi, (int)lo);
}

// one term (ah + al)*(xh + xl) of already split operands into A
__device__ __forceinline__ void df_term_pre(DfAcc &A, float ah, float al, float xh, float xl) {
    const float p = __fmul_rn(ah, xh);
    float e = __fmaf_rn(ah, xh, -p);        // exact: ah*xh = p + e
    e = __fmaf_rn(ah, xl, e);
    e = __fmaf_rn(al, xh, e);
    float s, t;
    two_sum(A.s, p, s, t);
    A.s = s;
    A.c = __fadd_rn(A.c, __fadd_rn(t, e));
}

// df_term_pre that also keeps mx = max |ah*xh| of the member's terms
__device__ __forceinline__ void df_term_pm(DfAcc &A, float &mx, float ah, float al, float xh, float xl) {
    const float p = __fmul_rn(ah, xh);
    mx = fmaxf(mx, fabsf(p));
    float e = __fmaf_rn(ah, xh, -p);
    e = __fmaf_rn(ah, xl, e);
    e = __fmaf_rn(al, xh, e);
    float s, t;
    two_sum(A.s, p, s, t);
    A.s = s;
    A.c = __fadd_rn(A.c, __fadd_rn(t, e));
}

// a member's float-pair products reached below FP32's normal range: its
// largest |a_j x_j| is positive but under 2^-96 (then every error term may
// have lost bits to underflow)
__device__ __forceinline__ bool df_tiny(float mx) { return mx > 0.0f && mx < 0x1p-96f; }

// one term a*(xh + xl) into A; returns false when a needs the FP64 path
// (the term then contributes nothing here and is added by df_fixup)
__device__ __forceinline__ bool df_term(DfAcc &A, float &mx, double a, float xh, float xl) {
    float ah, al;
    const bool ok = df_split_trunc(a, ah, al);
    df_term_pm(A, mx, ah, al, xh, xl);
    return ok;
}

// true when the double is neither infinite nor NaN (exponent field test on
// the integer pipe)
__device__ __forceinline__ bool finite_bits(double v) {
    return ((uint32_t)__double2hiint(v) & 0x7ff00000u) != 0x7ff00000u;
}

// p0 + p1 with the same operation order on every lane and every s; fb (the
// FP64 sum of out-of-range terms) is added only when non-zero
__device__ __forceinline__ double df_finish(const DfAcc &A0, const DfAcc &A1, double fb) {
    float s, t;
    two_sum(A0.s, A1.s, s, t);
    const float c = __fadd_rn(__fadd_rn(A0.c, A1.c), t);
    const double y = f2d_exact(s) + f2d_exact(c);
    return (fb != 0.0) ? y + fb : y;
}

// Sources of the pre-split x: XPre reads the float pairs written by the CG
// kernels; XSplit reads FP64 x and splits it on the fly with the same
// rounding (used by ens_spmv, where x arrives in FP64).
struct XPre {
    using ptr = const float2 *;
    __device__ __forceinline__ static float4 two(ptr x, int64_t i) {
        return __ldg(reinterpret_cast<const float4 *>(x + i));
    }
    __device__ __forceinline__ static float2 one(ptr x, int64_t i) { return __ldg(x + i); }
    // hi + lo of element i, exact in FP64
    __device__ __forceinline__ static double dbl(ptr x, int64_t i) {
        const float2 h = __ldg(x + i);
        return (double)h.x + (double)h.y;
    }
};
// An x outside the split range (or not finite) is returned with a NaN leading
// part, so that its products make the row's sum non-finite and the row falls
// back to FP64 (row_fp64_member / split_odd_fp64 read the FP64 x).
struct XSplit {
    using ptr = const double *;
    __device__ __forceinline__ static float4 two(ptr x, int64_t i) {
        const double2 v = ld_x2(x, i);
        bool ok0, ok1;
        const float2 a = df_split_vec(v.x, ok0), b = df_split_vec(v.y, ok1);
        const float qnan = __int_as_float(0x7fc00000);
        return make_float4(ok0 ? a.x : qnan, a.y, ok1 ? b.x : qnan, b.y);
    }
    __device__ __forceinline__ static float2 one(ptr x, int64_t i) {
        bool ok;
        const float2 a = df_split_vec(__ldg(x + i), ok);
        return make_float2(ok ? a.x : __int_as_float(0x7fc00000), a.y);
    }
    __device__ __forceinline__ static double dbl(ptr x, int64_t i) {
        bool ok;
        const float2 h = df_split_vec(__ldg(x + i), ok);
        return ok ? (double)h.x + (double)h.y : __ldg(x + i);
    }
};

// FP64 value of member mm of a row with entries [rs, re) against the split x
// (hi + lo, exact in FP64; FP64 x where the split is out of range): entry j to
// partial (j - rs) mod 2, each partial in increasing j, row value p0 + p1 --
// the order of every other form.  Used for members whose float-pair products
// fell below FP32's normal range (rare).
template <int S, typename XS, typename CA>
__device__ __noinline__ double row_fp64_member(CA colf, int rs, int re, const double *__restrict__ vals,
                                               typename XS::ptr x, int mm) {
    double p0 = 0.0, p1 = 0.0;
    for (int j = rs; j < re; ++j) {
        const double t = ValLoad<double>::one(vals, (int64_t)j * S + mm);
        const double xv = XS::dbl(x, (int64_t)colf(j) * S + mm);
        if ((j - rs) & 1) p1 = fma(t, xv, p1);
        else p0 = fma(t, xv, p0);
    }
    return p0 + p1;
}

// FP64 sum, in entry order, of the terms whose value is outside the split
// range (rare: run only by rows that met one)
template <int S, typename XS, typename CA>
__device__ __noinline__ double2 df_fixup2(CA colf, int rs, int re, const double *__restrict__ vals,
                                          typename XS::ptr x, int m) {
    double f0[2] = {0.0, 0.0}, f1[2] = {0.0, 0.0};  // entries of even / odd position
    for (int j = rs; j < re; ++j) {
        const double2 v = ValLoad<double>::two(vals, (int64_t)j * S + m);
        float h, l;
        const bool ok0 = df_split_trunc(v.x, h, l), ok1 = df_split_trunc(v.y, h, l);
        if (ok0 && ok1) continue;
        const float4 xv = XS::two(x, (int64_t)colf(j) * S + m);
        const int par = (j - rs) & 1;
        if (!ok0) f0[par] = fma(v.x, (double)xv.x + (double)xv.y, f0[par]);
        if (!ok1) f1[par] = fma(v.y, (double)xv.z + (double)xv.w, f1[par]);
    }
    return make_double2(f0[0] + f0[1], f1[0] + f1[1]);
}

// df form of row_spmv2 (members 2g, 2g+1 of a row with entries [rs, re))
template <int S, typename XS, typename CA>
__device__ __forceinline__ double2 row_spmv2_df(CA colf, int rs, int re,
                                                const double *__restrict__ vals,
                                                typename XS::ptr __restrict__ x, int g) {
    DfAcc a0 = df_zero(), a1 = df_zero(), b0 = df_zero(), b1 = df_zero();
    float ma = 0.0f, mb = 0.0f;  // max |product| of members m, m+1
    bool ok = true;
    const int m = 2 * g;
    int j = rs;
    for (; j + 4 <= re; j += 4) {
        const int c0 = colf(j), c1 = colf(j + 1), c2 = colf(j + 2), c3 = colf(j + 3);
        const double2 v0 = ValLoad<double>::two(vals, (int64_t)j * S + m);
        const double2 v1 = ValLoad<double>::two(vals, (int64_t)(j + 1) * S + m);
        const double2 v2 = ValLoad<double>::two(vals, (int64_t)(j + 2) * S + m);
        const double2 v3 = ValLoad<double>::two(vals, (int64_t)(j + 3) * S + m);
        const float4 x0 = XS::two(x, (int64_t)c0 * S + m);
        const float4 x1 = XS::two(x, (int64_t)c1 * S + m);
        const float4 x2 = XS::two(x, (int64_t)c2 * S + m);
        const float4 x3 = XS::two(x, (int64_t)c3 * S + m);
        ok &= df_term(a0, ma, v0.x, x0.x, x0.y); ok &= df_term(b0, mb, v0.y, x0.z, x0.w);
        ok &= df_term(a1, ma, v1.x, x1.x, x1.y); ok &= df_term(b1, mb, v1.y, x1.z, x1.w);
        ok &= df_term(a0, ma, v2.x, x2.x, x2.y); ok &= df_term(b0, mb, v2.y, x2.z, x2.w);
        ok &= df_term(a1, ma, v3.x, x3.x, x3.y); ok &= df_term(b1, mb, v3.y, x3.z, x3.w);
    }
    for (; j < re; ++j) {
        const double2 v = ValLoad<double>::two(vals, (int64_t)j * S + m);
        const float4 xv = XS::two(x, (int64_t)colf(j) * S + m);
        if ((j - rs) & 1) { ok &= df_term(a1, ma, v.x, xv.x, xv.y); ok &= df_term(b1, mb, v.y, xv.z, xv.w); }
        else { ok &= df_term(a0, ma, v.x, xv.x, xv.y); ok &= df_term(b0, mb, v.y, xv.z, xv.w); }
    }
    double2 fb = make_double2(0.0, 0.0);
    if (!ok) fb = df_fixup2<S, XS, CA>(colf, rs, re, vals, x, m);
    double2 y = make_double2(df_finish(a0, a1, fb.x), df_finish(b0, b1, fb.y));
    // FP64 for members with tiny products or a non-finite sum (an x outside
    // the split range, or non-finite data)
    if (df_tiny(ma) || !finite_bits(y.x)) y.x = row_fp64_member<S, XS, CA>(colf, rs, re, vals, x, m);
    if (df_tiny(mb) || !finite_bits(y.y)) y.y = row_fp64_member<S, XS, CA>(colf, rs, re, vals, x, m + 1);
    return y;
}

// df form of row_spmv1 (s = 1, 2 threads per row, result on both lanes)
template <typename XS, typename CA>
__device__ __forceinline__ double row_spmv1_df(CA colf, int rs, int re,
                                               const double *__restrict__ vals,
                                               typename XS::ptr __restrict__ x, int g, bool valid) {
    DfAcc a = df_zero();
    float mx = 0.0f;
    bool ok = true;
    if (valid)
        for (int j = rs + g; j < re; j += 2) {
            const float2 xv = XS::one(x, colf(j));
            ok &= df_term(a, mx, ValLoad<double>::one(vals, j), xv.x, xv.y);
        }
    double fb = 0.0;
    if (!ok)
        for (int j = rs + g; j < re; j += 2) {
            const double v = ValLoad<double>::one(vals, j);
            float h, l;
            if (df_split_trunc(v, h, l)) continue;
            const float2 xv = XS::one(x, colf(j));
            fb = fma(v, (double)xv.x + (double)xv.y, fb);
        }
    DfAcc o;
    o.s = __shfl_xor_sync(0xffffffffu, a.s, 1);
    o.c = __shfl_xor_sync(0xffffffffu, a.c, 1);
    const double ofb = __shfl_xor_sync(0xffffffffu, fb, 1);
    const double y = (g == 0) ? df_finish(a, o, fb + ofb) : df_finish(o, a, ofb + fb);
    mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, 1));
    const bool redo = valid && (df_tiny(mx) || !finite_bits(y));
    if (!__any_sync(0xffffffffu, redo)) return y;
    // FP64 partial of this lane's entries, then p0 + p1 (both lanes of a pair agree)
    double p = 0.0;
    if (valid)
        for (int j = rs + g; j < re; j += 2) p = fma(ValLoad<double>::one(vals, j), XS::dbl(x, colf(j)), p);
    const double po = __shfl_xor_sync(0xffffffffu, p, 1);
    const double yd = (g == 0) ? p + po : po + p;
    return redo ? yd : y;
}

// --------------------------------------------- double-float, pre-split values
// The df form with the values split once per ensemble (ens_convert_values,
// ENS_F64_DF: float pairs (hi, lo) by the same truncating split; a value
// outside the split range is stored as (NaN, 0)).  The terms are the same
// operations as row_spmv2_df without the per-term split, so every row whose
// result is finite equals row_spmv2_df bitwise; a non-finite result (a marked
// value, or a non-finite x or sum) is recomputed by row_spmv2_df from the
// FP64 values, which keeps the equality in every case.
template <int S, typename XS, typename CA>
__device__ __noinline__ double2 row_spmv2_df_redo(CA colf, int rs, int re, const double *__restrict__ vals,
                                                  typename XS::ptr x, int g) {
    return row_spmv2_df<S, XS, CA>(colf, rs, re, vals, x, g);
}

// XS: the source of the split x (XPre: the CG's split vectors; XSplit: FP64 x
// split on the fly with the same rounding, as in ens_spmv_df)
template <int S, typename XS, typename CA>
__device__ __forceinline__ double2 row_spmv2_dfv(CA colf, int rs, int re, const float2 *__restrict__ vdf,
                                                 const double *__restrict__ vals,
                                                 typename XS::ptr __restrict__ x, int g) {
    DfAcc a0 = df_zero(), a1 = df_zero(), b0 = df_zero(), b1 = df_zero();
    float ma = 0.0f, mb = 0.0f;  // max |product| of members m, m+1
    const int m = 2 * g;
    int j = rs;
    for (; j + 4 <= re; j += 4) {
        const int c0 = colf(j), c1 = colf(j + 1), c2 = colf(j + 2), c3 = colf(j + 3);
        const float4 v0 = ld_stream(reinterpret_cast<const float4 *>(vdf + (int64_t)j * S + m));
        const float4 v1 = ld_stream(reinterpret_cast<const float4 *>(vdf + (int64_t)(j + 1) * S + m));
        const float4 v2 = ld_stream(reinterpret_cast<const float4 *>(vdf + (int64_t)(j + 2) * S + m));
        const float4 v3 = ld_stream(reinterpret_cast<const float4 *>(vdf + (int64_t)(j + 3) * S + m));
        const float4 x0 = XS::two(x, (int64_t)c0 * S + m);
        const float4 x1 = XS::two(x, (int64_t)c1 * S + m);
        const float4 x2 = XS::two(x, (int64_t)c2 * S + m);
        const float4 x3 = XS::two(x, (int64_t)c3 * S + m);
        df_term_pm(a0, ma, v0.x, v0.y, x0.x, x0.y); df_term_pm(b0, mb, v0.z, v0.w, x0.z, x0.w);
        df_term_pm(a1, ma, v1.x, v1.y, x1.x, x1.y); df_term_pm(b1, mb, v1.z, v1.w, x1.z, x1.w);
        df_term_pm(a0, ma, v2.x, v2.y, x2.x, x2.y); df_term_pm(b0, mb, v2.z, v2.w, x2.z, x2.w);
        df_term_pm(a1, ma, v3.x, v3.y, x3.x, x3.y); df_term_pm(b1, mb, v3.z, v3.w, x3.z, x3.w);
    }
    for (; j < re; ++j) {
        const float4 v = ld_stream(reinterpret_cast<const float4 *>(vdf + (int64_t)j * S + m));
        const float4 xv = XS::two(x, (int64_t)colf(j) * S + m);
        if ((j - rs) & 1) { df_term_pm(a1, ma, v.x, v.y, xv.x, xv.y); df_term_pm(b1, mb, v.z, v.w, xv.z, xv.w); }
        else { df_term_pm(a0, ma, v.x, v.y, xv.x, xv.y); df_term_pm(b0, mb, v.z, v.w, xv.z, xv.w); }
    }
    const double2 y = make_double2(df_finish(a0, a1, 0.0), df_finish(b0, b1, 0.0));
    if (finite_bits(y.x) && finite_bits(y.y) && !df_tiny(ma) && !df_tiny(mb)) return y;
    return row_spmv2_df_redo<S, XS, CA>(colf, rs, re, vals, x, g);
}

// row_spmv2_dfv with the value loads in the default cache policy, for s < 16.
// From s = 16 the threads of a row read whole 128-byte lines of values at each
// entry, once: streaming loads (evict-first, row_spmv2_dfv).  Below s = 16 a
// line holds 16 / s consecutive entries of a row, which the same warp reads
// over as many steps of its row loop: normal loads keep the line in L1 between
// them (64^3 mesh: s = 8 140.9 -> 115.9 us, s = 4 90.9 -> 79 us per launch;
// at s = 16 streaming loads are faster, 205.5 against 219.4 us).  A separate
// function rather than a load chosen by s inside row_spmv2_dfv: routing the
// s = 32 loads through a shared helper changed that kernel's register
// allocation and cost 6 % (354.5 -> 376.9 us per launch).
template <int S, typename XS, typename CA>
__device__ __forceinline__ double2 row_spmv2_dfv_l1(CA colf, int rs, int re, const float2 *__restrict__ vdf,
                                                 const double *__restrict__ vals,
                                                 typename XS::ptr __restrict__ x, int g) {
    DfAcc a0 = df_zero(), a1 = df_zero(), b0 = df_zero(), b1 = df_zero();
    float ma = 0.0f, mb = 0.0f;  // max |product| of members m, m+1
    const int m = 2 * g;
    int j = rs;
    for (; j + 4 <= re; j += 4) {
        const int c0 = colf(j), c1 = colf(j + 1), c2 = colf(j + 2), c3 = colf(j + 3);
        const float4 v0 = ld_normal(reinterpret_cast<const float4 *>(vdf + (int64_t)j * S + m));
        const float4 v1 = ld_normal(reinterpret_cast<const float4 *>(vdf + (int64_t)(j + 1) * S + m));
        const float4 v2 = ld_normal(reinterpret_cast<const float4 *>(vdf + (int64_t)(j + 2) * S + m));
        const float4 v3 = ld_normal(reinterpret_cast<const float4 *>(vdf + (int64_t)(j + 3) * S + m));
        const float4 x0 = XS::two(x, (int64_t)c0 * S + m);
        const float4 x1 = XS::two(x, (int64_t)c1 * S + m);
        const float4 x2 = XS::two(x, (int64_t)c2 * S + m);
        const float4 x3 = XS::two(x, (int64_t)c3 * S + m);
        df_term_pm(a0, ma, v0.x, v0.y, x0.x, x0.y); df_term_pm(b0, mb, v0.z, v0.w, x0.z, x0.w);
        df_term_pm(a1, ma, v1.x, v1.y, x1.x, x1.y); df_term_pm(b1, mb, v1.z, v1.w, x1.z, x1.w);
        df_term_pm(a0, ma, v2.x, v2.y, x2.x, x2.y); df_term_pm(b0, mb, v2.z, v2.w, x2.z, x2.w);
        df_term_pm(a1, ma, v3.x, v3.y, x3.x, x3.y); df_term_pm(b1, mb, v3.z, v3.w, x3.z, x3.w);
    }
    for (; j < re; ++j) {
        const float4 v = ld_normal(reinterpret_cast<const float4 *>(vdf + (int64_t)j * S + m));
        const float4 xv = XS::two(x, (int64_t)colf(j) * S + m);
        if ((j - rs) & 1) { df_term_pm(a1, ma, v.x, v.y, xv.x, xv.y); df_term_pm(b1, mb, v.z, v.w, xv.z, xv.w); }
        else { df_term_pm(a0, ma, v.x, v.y, xv.x, xv.y); df_term_pm(b0, mb, v.z, v.w, xv.z, xv.w); }
    }
    const double2 y = make_double2(df_finish(a0, a1, 0.0), df_finish(b0, b1, 0.0));
    if (finite_bits(y.x) && finite_bits(y.y) && !df_tiny(ma) && !df_tiny(mb)) return y;
    return row_spmv2_df_redo<S, XS, CA>(colf, rs, re, vals, x, g);
}

// s = 1 (2 threads per row, full warps): the recomputation is taken by the
// whole warp when any of its rows needs it (row_spmv1_df shuffles)
template <typename XS, typename CA>
__device__ __forceinline__ double row_spmv1_dfv(CA colf, int rs, int re, const float2 *__restrict__ vdf,
                                                const double *__restrict__ vals,
                                                typename XS::ptr __restrict__ x, int g, bool valid) {
    DfAcc a = df_zero();
    float mx = 0.0f;
    if (valid)
        for (int j = rs + g; j < re; j += 2) {
            const float2 xv = XS::one(x, colf(j));
            const float2 v = ld_stream(vdf + j);
            df_term_pm(a, mx, v.x, v.y, xv.x, xv.y);
        }
    DfAcc o;
    o.s = __shfl_xor_sync(0xffffffffu, a.s, 1);
    o.c = __shfl_xor_sync(0xffffffffu, a.c, 1);
    const double y = (g == 0) ? df_finish(a, o, 0.0) : df_finish(o, a, 0.0);
    mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, 1));
    if (!__any_sync(0xffffffffu, !finite_bits(y) || (valid && df_tiny(mx)))) return y;
    return row_spmv1_df<XS, CA>(colf, rs, re, vals, x, g, valid);
}

// ------------------------------------------------- split FP64 / double-float
// Both pipes at once: entries at even positions of a row (partial 0) use the
// FP64 FMA with x in FP64, entries at odd positions (partial 1) use the
// double-float product with x pre-split; row value = p0 + double(p1).
// GB300 retires 2 DFMA and ~3 double-float terms per cycle per SM, so half of
// the terms on each pipe keeps the SpMV under the HBM time.
// FP64 sum, in increasing j, of the odd-position terms of member mm (the
// split form's double-float partial), used when its products were tiny
template <int S, typename CA>
__device__ __noinline__ double split_odd_fp64(CA colf, int rs, int re, const double *__restrict__ vals,
                                              const double *__restrict__ x, int mm) {
    double p = 0.0;
    for (int j = rs + 1; j < re; j += 2)
        p = fma(ValLoad<double>::one(vals, (int64_t)j * S + mm), __ldg(x + (int64_t)colf(j) * S + mm), p);
    return p;
}

template <int S, typename XS, typename CA>
__device__ __forceinline__ double2 row_spmv2_split(CA colf, int rs, int re,
                                                   const double *__restrict__ vals,
                                                   const double *__restrict__ x,
                                                   typename XS::ptr __restrict__ xdf, int g) {
    double a0 = 0.0, b0 = 0.0;          // FP64 partial, members m, m+1
    DfAcc a1 = df_zero(), b1 = df_zero();  // double-float partial
    float ma = 0.0f, mb = 0.0f;            // max |product| of the double-float partials
    bool ok = true;
    const int m = 2 * g;
    int j = rs;
    for (; j + 4 <= re; j += 4) {
        const int c0 = colf(j), c1 = colf(j + 1), c2 = colf(j + 2), c3 = colf(j + 3);
        const double2 v0 = ValLoad<double>::two(vals, (int64_t)j * S + m);
        const double2 v1 = ValLoad<double>::two(vals, (int64_t)(j + 1) * S + m);
        const double2 v2 = ValLoad<double>::two(vals, (int64_t)(j + 2) * S + m);
        const double2 v3 = ValLoad<double>::two(vals, (int64_t)(j + 3) * S + m);
        const double2 x0 = ld_x2(x, (int64_t)c0 * S + m);
        const float4 d1 = XS::two(xdf, (int64_t)c1 * S + m);
        const double2 x2 = ld_x2(x, (int64_t)c2 * S + m);
        const float4 d3 = XS::two(xdf, (int64_t)c3 * S + m);
        a0 = fma(v0.x, x0.x, a0); b0 = fma(v0.y, x0.y, b0);
        ok &= df_term(a1, ma, v1.x, d1.x, d1.y); ok &= df_term(b1, mb, v1.y, d1.z, d1.w);
        a0 = fma(v2.x, x2.x, a0); b0 = fma(v2.y, x2.y, b0);
        ok &= df_term(a1, ma, v3.x, d3.x, d3.y); ok &= df_term(b1, mb, v3.y, d3.z, d3.w);
    }
    for (; j < re; ++j) {
        const double2 v = ValLoad<double>::two(vals, (int64_t)j * S + m);
        const int c = colf(j);
        if ((j - rs) & 1) {
            const float4 d = XS::two(xdf, (int64_t)c * S + m);
            ok &= df_term(a1, ma, v.x, d.x, d.y); ok &= df_term(b1, mb, v.y, d.z, d.w);
        } else {
            const double2 xv = ld_x2(x, (int64_t)c * S + m);
            a0 = fma(v.x, xv.x, a0); b0 = fma(v.y, xv.y, b0);
        }
    }
    double f0 = 0.0, f1 = 0.0;  // odd-position terms outside the split range, FP64, in order
    if (!ok)
        for (int jj = rs + 1; jj < re; jj += 2) {
            const double2 v = ValLoad<double>::two(vals, (int64_t)jj * S + m);
            float h, l;
            const bool ok0 = df_split_trunc(v.x, h, l), ok1 = df_split_trunc(v.y, h, l);
            if (ok0 && ok1) continue;
            const double2 xv = ld_x2(x, (int64_t)colf(jj) * S + m);
            if (!ok0) f0 = fma(v.x, xv.x, f0);
            if (!ok1) f1 = fma(v.y, xv.y, f1);
        }
    double p1a = f2d_exact(a1.s) + f2d_exact(a1.c), p1b = f2d_exact(b1.s) + f2d_exact(b1.c);
    if (f0 != 0.0) p1a += f0;
    if (f1 != 0.0) p1b += f1;
    // odd-position partials whose products fell below FP32's normal range, or
    // whose sum is not finite (an x outside the split range): FP64
    if (df_tiny(ma) || !finite_bits(p1a)) p1a = split_odd_fp64<S, CA>(colf, rs, re, vals, x, m);
    if (df_tiny(mb) || !finite_bits(p1b)) p1b = split_odd_fp64<S, CA>(colf, rs, re, vals, x, m + 1);
    return make_double2(a0 + p1a, b0 + p1b);
}

// s = 1: lane g = 0 sums the even positions in FP64, lane 1 the odd ones in
// double-float; the row value is returned on both lanes
template <typename XS, typename CA>
__device__ __forceinline__ double row_spmv1_split(CA colf, int rs, int re,
                                                  const double *__restrict__ vals,
                                                  const double *__restrict__ x,
                                                  typename XS::ptr __restrict__ xdf, int g,
                                                  bool valid) {
    double p = 0.0;
    if (valid) {
        if (g == 0) {
            for (int j = rs; j < re; j += 2) p = fma(ValLoad<double>::one(vals, j), __ldg(x + colf(j)), p);
        } else {
            DfAcc a = df_zero();
            float mx = 0.0f;
            bool ok = true;
            for (int j = rs + 1; j < re; j += 2) {
                const float2 d = XS::one(xdf, colf(j));
                ok &= df_term(a, mx, ValLoad<double>::one(vals, j), d.x, d.y);
            }
            double f = 0.0;
            if (!ok)
                for (int j = rs + 1; j < re; j += 2) {
                    const double v = ValLoad<double>::one(vals, j);
                    float h, l;
                    if (df_split_trunc(v, h, l)) continue;
                    f = fma(v, __ldg(x + colf(j)), f);
                }
            const double p1 = f2d_exact(a.s) + f2d_exact(a.c);
            p = (f != 0.0) ? p1 + f : p1;
            if (df_tiny(mx) || !finite_bits(p)) p = split_odd_fp64<1, CA>(colf, rs, re, vals, x, 0);
        }
    }
    const double o = __shfl_xor_sync(0xffffffffu, p, 1);
    return (g == 0) ? p + o : o + p;
}

// ------------------------------------------- chunk-level row evaluation
// Value(s) of the calling thread's row r (members 2g, 2g+1; s = 1: the row,
// in .x) inside a staged 32-row chunk.  valid = the row exists.
template <int S, typename V>
__device__ __forceinline__ double2 chunk_spmv(const ChunkCols &cc, bool staged,
                                              const int32_t *__restrict__ col,
                                              const V *__restrict__ vals,
                                              const double *__restrict__ x, int r, int g,
                                              bool valid) {
    const int rs = valid ? cc.rm[r] : 0, re = valid ? cc.rm[r + 1] : 0;
    if constexpr (S == 1) {
        const double v = staged ? row_spmv1<V>(ColShared{cc.col, cc.base}, rs, re, vals, x, g, valid)
                                : row_spmv1<V>(ColGlobal{col}, rs, re, vals, x, g, valid);
        return make_double2(v, 0.0);
    } else {
        if (!valid) return make_double2(0.0, 0.0);
        return staged ? row_spmv2<S, V>(ColShared{cc.col, cc.base}, rs, re, vals, x, g)
                      : row_spmv2<S, V>(ColGlobal{col}, rs, re, vals, x, g);
    }
}

template <int S, typename XS>
__device__ __forceinline__ double2 chunk_spmv_df(const ChunkCols &cc, bool staged,
                                                 const int32_t *__restrict__ col,
                                                 const double *__restrict__ vals,
                                                 typename XS::ptr __restrict__ x, int r, int g,
                                                 bool valid) {
    const int rs = valid ? cc.rm[r] : 0, re = valid ? cc.rm[r + 1] : 0;
    if constexpr (S == 1) {
        const double v = staged ? row_spmv1_df<XS>(ColShared{cc.col, cc.base}, rs, re, vals, x, g, valid)
                                : row_spmv1_df<XS>(ColGlobal{col}, rs, re, vals, x, g, valid);
        return make_double2(v, 0.0);
    } else {
        if (!valid) return make_double2(0.0, 0.0);
        return staged ? row_spmv2_df<S, XS>(ColShared{cc.col, cc.base}, rs, re, vals, x, g)
                      : row_spmv2_df<S, XS>(ColGlobal{col}, rs, re, vals, x, g);
    }
}

template <int S, typename XS = XPre>
__device__ __forceinline__ double2 chunk_spmv_dfv(const ChunkCols &cc, bool staged,
                                                  const int32_t *__restrict__ col,
                                                  const float2 *__restrict__ vdf,
                                                  const double *__restrict__ vals,
                                                  typename XS::ptr __restrict__ x, int r, int g, bool valid) {
    const int rs = valid ? cc.rm[r] : 0, re = valid ? cc.rm[r + 1] : 0;
    if constexpr (S == 1) {
        const double v = staged ? row_spmv1_dfv<XS>(ColShared{cc.col, cc.base}, rs, re, vdf, vals, x, g, valid)
                                : row_spmv1_dfv<XS>(ColGlobal{col}, rs, re, vdf, vals, x, g, valid);
        return make_double2(v, 0.0);
    } else {
        if (!valid) return make_double2(0.0, 0.0);
        if constexpr (S >= 16)
            return staged ? row_spmv2_dfv<S, XS>(ColShared{cc.col, cc.base}, rs, re, vdf, vals, x, g)
                          : row_spmv2_dfv<S, XS>(ColGlobal{col}, rs, re, vdf, vals, x, g);
        else
            return staged ? row_spmv2_dfv_l1<S, XS>(ColShared{cc.col, cc.base}, rs, re, vdf, vals, x, g)
                          : row_spmv2_dfv_l1<S, XS>(ColGlobal{col}, rs, re, vdf, vals, x, g);
    }
}

template <int S, typename XS>
__device__ __forceinline__ double2 chunk_spmv_split(const ChunkCols &cc, bool staged,
                                                    const int32_t *__restrict__ col,
                                                    const double *__restrict__ vals,
                                                    const double *__restrict__ x,
                                                    typename XS::ptr __restrict__ xdf, int r,
                                                    int g, bool valid) {
    const int rs = valid ? cc.rm[r] : 0, re = valid ? cc.rm[r + 1] : 0;
    if constexpr (S == 1) {
        const double v = staged ? row_spmv1_split<XS>(ColShared{cc.col, cc.base}, rs, re, vals, x, xdf, g, valid)
                                : row_spmv1_split<XS>(ColGlobal{col}, rs, re, vals, x, xdf, g, valid);
        return make_double2(v, 0.0);
    } else {
        if (!valid) return make_double2(0.0, 0.0);
        return staged ? row_spmv2_split<S, XS>(ColShared{cc.col, cc.base}, rs, re, vals, x, xdf, g)
                      : row_spmv2_split<S, XS>(ColGlobal{col}, rs, re, vals, x, xdf, g);
    }
}

// Level-1 tree step: every thread of the CTA holds the per-row products of its
// (row r, members 2g, 2g+1) [s >= 2] or (row r) [s = 1, value on both lanes].
// Writes the chunk's per-member partials to t.buf[1][chunk*width + off + e].
// The 32 rows are combined by the halving tree v[i] += v[i + h], h = 16..1,
// in shared memory, the adds of all members packed into full warps (31 S adds
// per chunk, one barrier per level).  WARP = true: the same sums in the
// butterfly order of warp_tree32 (lane 0's value, operand for operand the
// halving tree) after one shared-memory transpose, one warp per member
// column: two barriers instead of six, but every lane adds at every level,
// 5 x 32 adds per member where the halving tree issues 31 -- on GB300's FP64
// pipe (one 32-lane FP64 instruction per 16 cycles per SM) that costs the
// FP64-bound SpMV forms 13 % at s = 32.  The default takes the butterfly only
// at s = 1, where both issue the same FP64 instructions.
template <int S, bool WARP = (S == 1)>
__device__ __forceinline__ void chunk_tree(double (*sm)[S + 1], double v0, double v1, int r, int g,
                                           const DotTree &t, int64_t chunk, int off) {
    if constexpr (S == 1) {
        if (g == 0) sm[r][0] = v0;
    } else {
        sm[r][2 * g] = v0;
        sm[r][2 * g + 1] = v1;
    }
    __syncthreads();
    if constexpr (WARP) {
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
        for (int e = warp; e < S; e += nw) {
            const double v = warp_tree32<double>(sm[lane][e]);
            if (lane == 0) t.buf[1][chunk * t.width + off + e] = v;
        }
    } else {
#pragma unroll
        for (int h = 16; h >= 1; h >>= 1) {
            for (int it = threadIdx.x; it < h * S; it += blockDim.x) {
                const int i = it / S, e = it % S;
                sm[i][e] += sm[i + h][e];
            }
            __syncthreads();
        }
        for (int e = threadIdx.x; e < S; e += blockDim.x) t.buf[1][chunk * t.width + off + e] = sm[0][e];
    }
    __syncthreads();
}

// Subset form of chunk_tree (halving tree): the chunk's threads are
// [ltid = 0, nthr); all threads of the CTA call it (its barriers are
// CTA-wide); writes only when the chunk exists.
template <int S>
__device__ __forceinline__ void chunk_tree_sub(double (*sm)[S + 1], double v0, double v1, int r,
                                               int g, const DotTree &t, int64_t chunk, int off,
                                               int ltid, int nthr) {
    if constexpr (S == 1) {
        if (g == 0) sm[r][0] = v0;
    } else {
        sm[r][2 * g] = v0;
        sm[r][2 * g + 1] = v1;
    }
    __syncthreads();
#pragma unroll
    for (int h = 16; h >= 1; h >>= 1) {
        for (int it = ltid; it < h * S; it += nthr) {
            const int i = it / S, e = it % S;
            sm[i][e] += sm[i + h][e];
        }
        __syncthreads();
    }
    if (chunk < t.count[1])
        for (int e = ltid; e < S; e += nthr) t.buf[1][chunk * t.width + off + e] = sm[0][e];
    __syncthreads();
}

}  // namespace ens
