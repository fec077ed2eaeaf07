// ens_cg_mixed.cu -- mixed-precision ensemble CG: FP64 iterative refinement
// around an FP32 inner CG on FP32 or BF16 matrix values.
//
// Refinement (per member e, member-wise masks as in ens_cg):
//   r = b - A x            FP64 values, FP64 arithmetic (the true residual)
//   stop when |r| <= tol |b|
//   solve A_lo d = r/|r|   FP32 CG on the low-precision copy of A (FP32 vectors,
//                          FP32 accumulation) to |r_in| <= inner_tol
//   x += |r| d             FP64 update
// The low-precision copy is made by ens_convert_values.  BF16 keeps 8
// significand bits, which perturbs the zero row sums of the diffusion stencil
// by about as much as its smallest eigenvalue; the converter can therefore
// keep the diagonal in FP32, chosen so that every row of A_lo sums to the FP64
// row sum (the smooth modes that carry the small eigenvalues are preserved).
#include <algorithm>
#include <vector>

#include "ens_spmv_f32.cuh"

namespace ens {

// ------------------------------------------------------------ conversion
template <typename V>
__device__ __forceinline__ V to_lo(double v);
template <>
__device__ __forceinline__ float to_lo<float>(double v) { return __double2float_rn(v); }
template <>
__device__ __forceinline__ __nv_bfloat16 to_lo<__nv_bfloat16>(double v) {
    return __float2bfloat16_rn(__double2float_rn(v));
}
template <typename V>
__device__ __forceinline__ double lo_to_double(V v);
template <>
__device__ __forceinline__ double lo_to_double<float>(float v) { return (double)v; }
template <>
__device__ __forceinline__ double lo_to_double<__nv_bfloat16>(__nv_bfloat16 v) {
    return (double)__bfloat162float(v);
}

// thread per (row, member)
template <typename V>
__global__ void convert_values_kernel(int32_t n, int s, const int32_t *__restrict__ row_map,
                                      const int32_t *__restrict__ col,
                                      const double *__restrict__ v64, V *__restrict__ vlo,
                                      float *__restrict__ diag) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t I = t / s;
    const int e = (int)(t % s);
    if (I >= n) return;
    const int rs = row_map[I], re = row_map[I + 1];
    double rowsum = 0.0, offsum = 0.0;
    for (int j = rs; j < re; ++j) {
        const double a = v64[(int64_t)j * s + e];
        V lo = to_lo<V>(a);
        if (diag) {
            rowsum += a;
            if (col[j] == I) lo = to_lo<V>(0.0);
            else offsum += lo_to_double<V>(lo);
        }
        vlo[(int64_t)j * s + e] = lo;
    }
    if (diag) diag[I * s + e] = __double2float_rn(rowsum - offsum);
}

// float chunk tree: 32-row halving tree, members packed (same pairing as
// warp_tree32); sm[r][e] holds row r's value of member e on entry
template <int S>
__device__ __forceinline__ void chunk_tree_f_sum(float (*sm)[S + 1], const DotTreeT<float> &t, int64_t chunk) {
    __syncthreads();
#pragma unroll
    for (int h = 16; h >= 1; h >>= 1) {
        for (int it = threadIdx.x; it < h * S; it += blockDim.x) {
            const int i = it / S, e = it % S;
            sm[i][e] = __fadd_rn(sm[i][e], sm[i + h][e]);
        }
        __syncthreads();
    }
    for (int e = threadIdx.x; e < S; e += blockDim.x) t.buf[1][chunk * t.width + e] = sm[0][e];
    __syncthreads();
}

template <int S>
__device__ __forceinline__ void chunk_tree_f(float (*sm)[S + 1], float v0, float v1, int r, int g,
                                             const DotTreeT<float> &t, int64_t chunk) {
    if constexpr (S == 1) {
        if (g == 0) sm[r][0] = v0;
    } else {
        sm[r][2 * g] = v0;
        sm[r][2 * g + 1] = v1;
    }
    chunk_tree_f_sum<S>(sm, t, chunk);
}

// the same tree with 4 members per thread (members 4g .. 4g+3 of row r)
template <int S>
__device__ __forceinline__ void chunk_tree_f4(float (*sm)[S + 1], const float4 v, int r, int g,
                                              const DotTreeT<float> &t, int64_t chunk) {
    sm[r][4 * g] = v.x;
    sm[r][4 * g + 1] = v.y;
    sm[r][4 * g + 2] = v.z;
    sm[r][4 * g + 3] = v.w;
    chunk_tree_f_sum<S>(sm, t, chunk);
}

// ------------------------------------------------------------ state
struct MxState {
    double rn[32], bnorm[32];
    float rho0[32], rho[32], alpha[32], beta[32];
    int active_out[32], active_in[32], updd[32], outer_it[32], inner_it[32], inner_total[32];
    int status[32], inner_break[32], zerox[32];
    int active_out_count, active_in_count, updd_any, zero_any;
    int spmv_real, pad0, pad1, pad2;
};

struct MxArgs {
    int32_t n;
    const int32_t *row_map, *col;
    const double *v64;
    const void *vlo;
    const float *diag;
    const double *b;
    double *x;
    float *r32, *rf, *pf, *qf, *d;
    MxState *st;
    DotTreeT<double> t64;  // width 2s: r.r and b.b
    DotTreeT<float> t32;   // width s
    double tol;
    float inner_tol;
    int max_outer, max_inner;
    uint64_t vlo_bytes;  // size of the low-precision value array (L2 prefetch bound)
};

// ------------------------------------------------------------------ MR
// r = b - A x in FP64 (split SpMV, x split on the fly); r32 = float(r); norms
template <int S>
__global__ void __launch_bounds__(RowMap<S>::THREADS, 1024 / RowMap<S>::THREADS) mx_resid_kernel(MxArgs a, int first) {
    constexpr int G = RowMap<S>::G;
    __shared__ ChunkCols cc;
    __shared__ double sm[32][S + 1];
    const int r = threadIdx.x / G, g = threadIdx.x % G;
    const int64_t R = (int64_t)blockIdx.x * 32 + r;
    const bool staged = stage_chunk(cc, a.row_map, a.col, blockIdx.x, a.n);
    const double2 ax = chunk_spmv_split<S, XSplit>(cc, staged, a.col, a.v64, a.x, a.x, r, g, R < a.n);
    double rr0 = 0.0, rr1 = 0.0, bb0 = 0.0, bb1 = 0.0;
    if (R < a.n) {
        if constexpr (S == 1) {
            const double bv = a.b[R], res = bv - ax.x;
            if (g == 0) a.r32[R] = __double2float_rn(res);
            rr0 = res * res;
            bb0 = bv * bv;
        } else {
            const double2 bv = reinterpret_cast<const double2 *>(a.b)[R * G + g];
            const double rx = bv.x - ax.x, ry = bv.y - ax.y;
            reinterpret_cast<float2 *>(a.r32)[R * G + g] = make_float2(__double2float_rn(rx), __double2float_rn(ry));
            rr0 = rx * rx; rr1 = ry * ry;
            bb0 = bv.x * bv.x; bb1 = bv.y * bv.y;
        }
    }
    chunk_tree<S>(sm, rr0, rr1, r, g, a.t64, blockIdx.x, 0);
    chunk_tree<S>(sm, bb0, bb1, r, g, a.t64, blockIdx.x, S);
    if (!dot_tree_propagate(a.t64, blockIdx.x, 1)) return;
    if (threadIdx.x >= 32) return;
    const unsigned FULL = 0xffffffffu;
    const int e = threadIdx.x;
    MxState *st = a.st;
    const double *top = a.t64.buf[a.t64.levels];
    int act = 0;
    if (e < S) {
        const double rn = sqrt(ld_cg(top + e));
        const double bn = first ? sqrt(ld_cg(top + S + e)) : st->bnorm[e];
        st->rn[e] = rn;
        if (first) {
            st->bnorm[e] = bn;
            st->outer_it[e] = 0;
            st->inner_total[e] = 0;
            st->inner_break[e] = 0;
            st->status[e] = ENS_OK;
            act = 1;
        } else {
            act = st->active_out[e];
        }
        int zx = 0;
        if (act) {
            if (bn == 0.0) { act = 0; zx = first; st->status[e] = ENS_OK; st->rn[e] = 0.0; }  // b = 0: x = 0
            else if (rn <= a.tol * bn) { act = 0; st->status[e] = ENS_OK; }
            else if (st->outer_it[e] >= a.max_outer) { act = 0; st->status[e] = ENS_ERR_NOT_CONVERGED; }
        }
        st->active_out[e] = act;
        if (first) st->zerox[e] = zx;
    }
    const int ac = __popc(__ballot_sync(FULL, act));
    const int zany = __popc(__ballot_sync(FULL, (e < S && first) ? st->zerox[e] : 0));
    if (e == 0) {
        st->active_out_count = ac;
        if (first) st->zero_any = zany;
    }
    __threadfence();
}

// ------------------------------------------------------------------ MI0
template <int S>
__global__ void __launch_bounds__(RowMap<S>::THREADS) mx_inner_init_kernel(MxArgs a) {
    if (ld_cg(&a.st->active_out_count) == 0) return;
    constexpr int G = RowMap<S>::G;
    __shared__ float sm[32][S + 1];
    const int r = threadIdx.x / G, g = threadIdx.x % G;
    const int64_t R = (int64_t)blockIdx.x * 32 + r;
    const MxState *cs = a.st;
    float v0 = 0.f, v1 = 0.f;
    if (R < a.n) {
        if constexpr (S == 1) {
            if (g == 0) {
                const float inv = cs->rn[0] > 0.0 ? (float)(1.0 / cs->rn[0]) : 0.f;
                const float rv = a.r32[R] * inv;
                a.rf[R] = rv; a.pf[R] = rv; a.d[R] = 0.f;
                v0 = rv * rv;
            }
        } else {
            const int m = 2 * g;
            const float i0 = cs->rn[m] > 0.0 ? (float)(1.0 / cs->rn[m]) : 0.f;
            const float i1 = cs->rn[m + 1] > 0.0 ? (float)(1.0 / cs->rn[m + 1]) : 0.f;
            const float2 rv0 = reinterpret_cast<const float2 *>(a.r32)[R * G + g];
            const float2 rv = make_float2(rv0.x * i0, rv0.y * i1);
            reinterpret_cast<float2 *>(a.rf)[R * G + g] = rv;
            reinterpret_cast<float2 *>(a.pf)[R * G + g] = rv;
            reinterpret_cast<float2 *>(a.d)[R * G + g] = make_float2(0.f, 0.f);
            v0 = rv.x * rv.x;
            v1 = rv.y * rv.y;
        }
    }
    chunk_tree_f<S>(sm, v0, v1, r, g, a.t32, blockIdx.x);
    if (!dot_tree_propagate(a.t32, blockIdx.x, 1)) return;
    if (threadIdx.x >= 32) return;
    const unsigned FULL = 0xffffffffu;
    const int e = threadIdx.x;
    MxState *st = a.st;
    int act = 0;
    if (e < S) {
        const float rho = ld_cg(a.t32.buf[a.t32.levels] + e);
        st->rho0[e] = rho;
        st->rho[e] = rho;
        st->inner_it[e] = 0;
        st->updd[e] = 0;
        act = st->active_out[e] && rho > 0.f;
        st->active_in[e] = act;
    }
    const int ac = __popc(__ballot_sync(FULL, act));
    if (e == 0) { st->active_in_count = ac; st->updd_any = 0; }
    __threadfence();
}

// ------------------------------------------------------------------ MI1
// alpha = rho / (p.q) per member, after the chunk trees of p.q (warp 0 of the
// CTA that finishes the tree)
template <int S>
__device__ __forceinline__ void mx_inner_alpha(MxArgs &a) {
    if (!dot_tree_propagate(a.t32, blockIdx.x, 1)) return;
    if (threadIdx.x >= 32) return;
    MxState *st = a.st;
    const unsigned FULL = 0xffffffffu;
    const int e = threadIdx.x;
    int act = 0;
    if (e < S) {
        act = st->active_in[e];
        const float pi = ld_cg(a.t32.buf[a.t32.levels] + e);
        if (act) {
            if (!(pi > 0.f) || !isfinite(pi)) { act = 0; st->inner_break[e] += 1; }
            else st->alpha[e] = st->rho[e] / pi;
        }
        st->active_in[e] = act;
        st->updd[e] = 0;
    }
    const int ac = __popc(__ballot_sync(FULL, act));
    if (e == 0) { st->active_in_count = ac; st->updd_any = 0; st->spmv_real += 1; }
    __threadfence();
}

// an inner solve that has finished leaves the remaining launches of its
// block with nothing to do (clears the update flags once)
__device__ __forceinline__ bool mx_inner_idle(MxArgs &a, int S) {
    MxState *st = a.st;
    if (ld_cg(&st->active_in_count) != 0) return false;
    if (blockIdx.x == 0 && threadIdx.x == 0 && st->updd_any) {
        for (int e = 0; e < S; ++e) st->updd[e] = 0;
        st->updd_any = 0;
    }
    return true;
}

// q = A_lo p and p.q; 2 members per thread (s <= 4)
template <int S, typename V>
__global__ void __launch_bounds__(RowMap<S>::THREADS, 1536 / RowMap<S>::THREADS) mx_inner_spmv_kernel(MxArgs a) {
    if (mx_inner_idle(a, S)) return;
    constexpr int G = RowMap<S>::G;
    __shared__ ChunkCols cc;
    __shared__ float sm[32][S + 1];
    const int r = threadIdx.x / G, g = threadIdx.x % G;
    const int64_t R = (int64_t)blockIdx.x * 32 + r;
    // the chunk's value block is prefetched into L2 while its columns are staged
    const bool staged = stage_chunk_pf(cc, a.row_map, a.col, blockIdx.x, a.n, a.vlo, S * (uint32_t)sizeof(V),
                                       a.vlo_bytes, 0xffffffffu);
    const float2 ap = chunk_spmv_f32<S, V>(cc, staged, a.col, static_cast<const V *>(a.vlo), a.diag,
                                           a.pf, r, g, R, R < a.n);
    float v0 = 0.f, v1 = 0.f;
    if (R < a.n) {
        if constexpr (S == 1) {
            if (g == 0) a.qf[R] = ap.x;
            v0 = ap.x * a.pf[R];
        } else {
            reinterpret_cast<float2 *>(a.qf)[R * G + g] = ap;
            const float2 pv = reinterpret_cast<const float2 *>(a.pf)[R * G + g];
            v0 = ap.x * pv.x;
            v1 = ap.y * pv.y;
        }
    }
    chunk_tree_f<S>(sm, v0, v1, r, g, a.t32, blockIdx.x);
    mx_inner_alpha<S>(a);
}

// the same with 4 members per thread (s >= 8): 16-byte value and p loads;
// every member's sums are bitwise those of the 2-member form
template <int S>
struct RowMap4 {
    static constexpr int G = S / 4;
    static constexpr int THREADS = 32 * G;
};
template <int S, typename V>
__global__ void __launch_bounds__(RowMap4<S>::THREADS, 1280 / RowMap4<S>::THREADS) mx_inner_spmv4_kernel(MxArgs a) {
    if (mx_inner_idle(a, S)) return;
    constexpr int G = RowMap4<S>::G;
    __shared__ ChunkCols cc;
    __shared__ float sm[32][S + 1];
    const int r = threadIdx.x / G, g = threadIdx.x % G;
    const int64_t R = (int64_t)blockIdx.x * 32 + r;
    const bool staged = stage_chunk_pf(cc, a.row_map, a.col, blockIdx.x, a.n, a.vlo, S * (uint32_t)sizeof(V),
                                       a.vlo_bytes, 0xffffffffu);
    const float4 ap = chunk_spmv4_f32<S, V>(cc, staged, a.col, static_cast<const V *>(a.vlo), a.diag,
                                            a.pf, r, g, R, R < a.n);
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    if (R < a.n) {
        reinterpret_cast<float4 *>(a.qf)[R * G + g] = ap;
        const float4 pv = reinterpret_cast<const float4 *>(a.pf)[R * G + g];
        v = make_float4(ap.x * pv.x, ap.y * pv.y, ap.z * pv.z, ap.w * pv.w);
    }
    chunk_tree_f4<S>(sm, v, r, g, a.t32, blockIdx.x);
    mx_inner_alpha<S>(a);
}

// ------------------------------------------------------------------ MI2
template <int S>
__global__ void __launch_bounds__(RowMap<S>::THREADS) mx_inner_resid_kernel(MxArgs a) {
    if (ld_cg(&a.st->active_in_count) == 0) return;
    constexpr int G = RowMap<S>::G;
    __shared__ float sm[32][S + 1];
    const int r = threadIdx.x / G, g = threadIdx.x % G;
    const int64_t R = (int64_t)blockIdx.x * 32 + r;
    const MxState *cs = a.st;
    float v0 = 0.f, v1 = 0.f;
    if (R < a.n) {
        if constexpr (S == 1) {
            if (g == 0) {
                float rv = a.rf[R];
                if (cs->active_in[0]) { rv = __fmaf_rn(-cs->alpha[0], a.qf[R], rv); a.rf[R] = rv; }
                v0 = rv * rv;
            }
        } else {
            const int m = 2 * g;
            float2 rv = reinterpret_cast<const float2 *>(a.rf)[R * G + g];
            const float2 qv = reinterpret_cast<const float2 *>(a.qf)[R * G + g];
            const bool a0 = cs->active_in[m], a1 = cs->active_in[m + 1];
            if (a0) rv.x = __fmaf_rn(-cs->alpha[m], qv.x, rv.x);
            if (a1) rv.y = __fmaf_rn(-cs->alpha[m + 1], qv.y, rv.y);
            if (a0 || a1) reinterpret_cast<float2 *>(a.rf)[R * G + g] = rv;
            v0 = rv.x * rv.x;
            v1 = rv.y * rv.y;
        }
    }
    chunk_tree_f<S>(sm, v0, v1, r, g, a.t32, blockIdx.x);
    if (!dot_tree_propagate(a.t32, blockIdx.x, 1)) return;
    if (threadIdx.x >= 32) return;
    const unsigned FULL = 0xffffffffu;
    const int e = threadIdx.x;
    MxState *st = a.st;
    int act = 0, ux = 0;
    if (e < S) {
        act = st->active_in[e];
        const float rn = ld_cg(a.t32.buf[a.t32.levels] + e);
        if (act) {
            ux = 1;
            const int it = st->inner_it[e] + 1;
            st->inner_it[e] = it;
            st->inner_total[e] += 1;
            if (sqrtf(rn) <= a.inner_tol * sqrtf(st->rho0[e]) || it >= a.max_inner) act = 0;
            else st->beta[e] = rn / st->rho[e];
            st->rho[e] = rn;
        }
        st->active_in[e] = act;
        st->updd[e] = ux;
    }
    const int ac = __popc(__ballot_sync(FULL, act)), uany = __popc(__ballot_sync(FULL, ux));
    if (e == 0) { st->active_in_count = ac; st->updd_any = uany; }
    __threadfence();
}

// ------------------------------------------------------------------ MI3
template <int S>
__global__ void __launch_bounds__(RowMap<S>::THREADS) mx_inner_update_kernel(MxArgs a) {
    const MxState *st = a.st;
    if (ld_cg(&st->updd_any) == 0) return;
    constexpr int G = RowMap<S>::G;
    const int r = threadIdx.x / G, g = threadIdx.x % G;
    const int64_t R = (int64_t)blockIdx.x * 32 + r;
    if (R >= a.n) return;
    if constexpr (S == 1) {
        if (g != 0) return;
        const float pv = a.pf[R];
        if (st->updd[0]) a.d[R] = __fmaf_rn(st->alpha[0], pv, a.d[R]);
        if (st->active_in[0]) a.pf[R] = __fmaf_rn(st->beta[0], pv, a.rf[R]);
    } else {
        const int m = 2 * g;
        const float2 pv = reinterpret_cast<const float2 *>(a.pf)[R * G + g];
        const bool u0 = st->updd[m], u1 = st->updd[m + 1];
        const bool c0 = st->active_in[m], c1 = st->active_in[m + 1];
        if (u0 || u1) {
            float2 dv = reinterpret_cast<const float2 *>(a.d)[R * G + g];
            if (u0) dv.x = __fmaf_rn(st->alpha[m], pv.x, dv.x);
            if (u1) dv.y = __fmaf_rn(st->alpha[m + 1], pv.y, dv.y);
            reinterpret_cast<float2 *>(a.d)[R * G + g] = dv;
        }
        if (c0 || c1) {
            const float2 rv = reinterpret_cast<const float2 *>(a.rf)[R * G + g];
            float2 pn = pv;
            if (c0) pn.x = __fmaf_rn(st->beta[m], pv.x, rv.x);
            if (c1) pn.y = __fmaf_rn(st->beta[m + 1], pv.y, rv.y);
            reinterpret_cast<float2 *>(a.pf)[R * G + g] = pn;
        }
    }
}

// x = 0 for members with b = 0 (one-shot, after the first residual)
template <int S>
__global__ void mx_zero_kernel(MxArgs a) {
    if (ld_cg(&a.st->zero_any) == 0) return;
    const int64_t total = (int64_t)a.n * S;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x)
        if (a.st->zerox[i % S]) a.x[i] = 0.0;
}

// ------------------------------------------------------------------ MU
// x += |r| d (FP64) for members still refining; counts the refinement step
template <int S>
__global__ void mx_update_x_kernel(MxArgs a) {
    const MxState *st = a.st;
    if (ld_cg(&st->active_out_count) == 0) return;
    const int64_t total = (int64_t)a.n * S;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int e = (int)(i % S);
        if (st->active_out[e]) a.x[i] = fma(st->rn[e], (double)a.d[i], a.x[i]);
    }
    if (blockIdx.x == 0 && threadIdx.x < S && st->active_out[threadIdx.x])
        a.st->outer_it[threadIdx.x] += 1;
}

// ------------------------------------------------------------ host side
static size_t al256(size_t x) { return (x + 255) / 256 * 256; }

static size_t mx_bytes(int64_t n, int s) {
    return al256(sizeof(MxState)) + 5 * al256(sizeof(float) * (size_t)n * s) +
           dot_tree_bytes(n, 2 * s, sizeof(double)) + dot_tree_bytes(n, s, sizeof(float));
}

struct MxOut {
    int32_t *outer, *inner;
    double *relres;
    int32_t *status;
    ens_cg_stats *stats;
};

template <int S, typename V>
static int mx_run(const ens_graph *g, const double *v64, const void *vlo, const float *diag,
                  const double *b, double *x, double tol, int max_outer, double inner_tol,
                  int max_inner, int check_every, int flags, void *work, MxOut out, cudaStream_t st) {
    const int64_t n = g->num_rows;
    char *w = static_cast<char *>(work);
    MxArgs a;
    a.n = g->num_rows;
    a.row_map = g->row_map;
    a.col = g->col_entry;
    a.v64 = v64;
    a.vlo = vlo;
    a.diag = diag;
    a.b = b;
    a.x = x;
    a.st = reinterpret_cast<MxState *>(w);
    w += al256(sizeof(MxState));
    float **vecs[5] = {&a.r32, &a.rf, &a.pf, &a.qf, &a.d};
    for (auto v : vecs) { *v = reinterpret_cast<float *>(w); w += al256(sizeof(float) * (size_t)n * S); }
    dot_tree_layout(&a.t64, n, 2 * S, w);
    w += dot_tree_bytes(n, 2 * S, sizeof(double));
    dot_tree_layout(&a.t32, n, S, w);
    a.tol = tol;
    a.inner_tol = (float)inner_tol;
    a.max_outer = max_outer;
    a.max_inner = max_inner;
    a.vlo_bytes = (uint64_t)g->num_entries * S * sizeof(V);
    const unsigned grid = (unsigned)a.t32.count[1];
    int rc;
    if ((rc = dot_tree_clear(a.t64, st))) return rc;
    if ((rc = dot_tree_clear(a.t32, st))) return rc;
    ENS_CUDA_TRY(cudaMemsetAsync(a.st, 0, sizeof(MxState), st));
    int launches = 0, polls = 0;
    const bool timing = (flags & ENS_CG_TIME_SPMV) != 0;
    std::vector<cudaEvent_t> ev;
    std::vector<float> spmv_ms;
    if (timing) {
        ev.resize(2 * (size_t)check_every);
        for (auto &x_ev : ev) ENS_CUDA_TRY(cudaEventCreate(&x_ev));
    }
    struct EvGuard {
        std::vector<cudaEvent_t> &v;
        ~EvGuard() { for (auto &x_ev : v) cudaEventDestroy(x_ev); }
    } ev_guard{ev};
    int32_t hflag[2];
    auto poll = [&](const int *dev, int cnt) -> int {
        ENS_CUDA_TRY(cudaMemcpyAsync(hflag, dev, cnt * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
        ENS_CUDA_TRY(cudaStreamSynchronize(st));
        ++polls;
        return ENS_OK;
    };
    mx_resid_kernel<S><<<grid, RowMap<S>::THREADS, 0, st>>>(a, 1);
    mx_zero_kernel<S><<<152 * 2, 256, 0, st>>>(a);
    launches += 2;
    ENS_LAUNCH_CHECK("mx_resid_kernel");
    if ((rc = poll(&a.st->active_out_count, 1))) return rc;
    for (int outer = 0; outer < max_outer + 1 && hflag[0] > 0; ++outer) {
        mx_inner_init_kernel<S><<<grid, RowMap<S>::THREADS, 0, st>>>(a);
        ++launches;
        const int max_blocks = max_inner / check_every + 2;
        for (int blk = 0; blk < max_blocks; ++blk) {
            for (int i = 0; i < check_every; ++i) {
                if (timing) cudaEventRecord(ev[2 * i], st);
                if constexpr (S >= 8) mx_inner_spmv4_kernel<S, V><<<grid, RowMap4<S>::THREADS, 0, st>>>(a);
                else mx_inner_spmv_kernel<S, V><<<grid, RowMap<S>::THREADS, 0, st>>>(a);
                if (timing) cudaEventRecord(ev[2 * i + 1], st);
                mx_inner_resid_kernel<S><<<grid, RowMap<S>::THREADS, 0, st>>>(a);
                mx_inner_update_kernel<S><<<grid, RowMap<S>::THREADS, 0, st>>>(a);
            }
            launches += 3 * check_every;
            ENS_LAUNCH_CHECK("mixed inner CG launch");
            if ((rc = poll(&a.st->active_in_count, 2))) return rc;
            if (timing)
                for (int i = 0; i < check_every; ++i) {
                    float ms = 0.f;
                    cudaEventElapsedTime(&ms, ev[2 * i], ev[2 * i + 1]);
                    spmv_ms.push_back(ms);
                }
            if (hflag[0] == 0 && hflag[1] == 0) break;
        }
        mx_update_x_kernel<S><<<152 * 4, 256, 0, st>>>(a);
        mx_resid_kernel<S><<<grid, RowMap<S>::THREADS, 0, st>>>(a, 0);
        launches += 2;
        ENS_LAUNCH_CHECK("mixed refinement launch");
        if ((rc = poll(&a.st->active_out_count, 1))) return rc;
    }
    MxState hs;
    ENS_CUDA_TRY(cudaMemcpyAsync(&hs, a.st, sizeof(MxState), cudaMemcpyDeviceToHost, st));
    ENS_CUDA_TRY(cudaStreamSynchronize(st));
    int first_bad = ENS_OK, maxit = 0;
    for (int e = 0; e < S; ++e) {
        if (out.outer) out.outer[e] = hs.outer_it[e];
        if (out.inner) out.inner[e] = hs.inner_total[e];
        if (out.relres) out.relres[e] = hs.bnorm[e] > 0.0 ? hs.rn[e] / hs.bnorm[e] : 0.0;
        int stt = hs.status[e];
        if (hs.active_out[e]) stt = ENS_ERR_NOT_CONVERGED;
        if (out.status) out.status[e] = stt;
        if (stt != ENS_OK && first_bad == ENS_OK) first_bad = stt;
        maxit = hs.inner_total[e] > maxit ? hs.inner_total[e] : maxit;
    }
    if (out.stats) {
        out.stats->spmv_ms = 0.0;
        out.stats->spmv_launches = 0;
        if (timing) {
            // inner SpMV launches run in order; the first spmv_real of each
            // inner solve did work, the rest exited early: keep the longest ones
            std::vector<float> sorted = spmv_ms;
            std::sort(sorted.begin(), sorted.end(), [](float u, float v) { return u > v; });
            const int real = hs.spmv_real < (int)sorted.size() ? hs.spmv_real : (int)sorted.size();
            double tot = 0.0;
            for (int i = 0; i < real; ++i) tot += sorted[i];
            out.stats->spmv_launches = real;
            out.stats->spmv_ms = tot;
        }
        out.stats->kernel_launches = launches;
        out.stats->iterations = maxit;
        out.stats->host_checks = polls;
        out.stats->guess_fallbacks = 0;
        out.stats->reserved = 0;
    }
    if (first_bad != ENS_OK)
        set_error("ens_cg_mixed: member status %d (%s)", first_bad, ens_status_string(first_bad));
    return first_bad;
}

template <typename V>
static int mx_dispatch(int s, const ens_graph *g, const double *v64, const void *vlo,
                       const float *diag, const double *b, double *x, double tol, int max_outer,
                       double inner_tol, int max_inner, int check_every, int flags, void *work, MxOut out,
                       cudaStream_t st) {
    switch (s) {
        case 1: return mx_run<1, V>(g, v64, vlo, diag, b, x, tol, max_outer, inner_tol, max_inner, check_every, flags, work, out, st);
        case 4: return mx_run<4, V>(g, v64, vlo, diag, b, x, tol, max_outer, inner_tol, max_inner, check_every, flags, work, out, st);
        case 8: return mx_run<8, V>(g, v64, vlo, diag, b, x, tol, max_outer, inner_tol, max_inner, check_every, flags, work, out, st);
        case 16: return mx_run<16, V>(g, v64, vlo, diag, b, x, tol, max_outer, inner_tol, max_inner, check_every, flags, work, out, st);
        default: return mx_run<32, V>(g, v64, vlo, diag, b, x, tol, max_outer, inner_tol, max_inner, check_every, flags, work, out, st);
    }
}

}  // namespace ens

using namespace ens;

// values -> float pairs (hi, lo) by the truncating split of the double-float
// SpMV; values outside the split range (or not finite) become (NaN, 0)
__global__ void split_values_kernel(int64_t count, const double *__restrict__ values,
                                    float2 *__restrict__ out) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count;
         i += (int64_t)gridDim.x * blockDim.x) {
        float hi, lo;
        const bool ok = df_split_trunc(ld_stream(values + i), hi, lo);
        out[i] = ok ? make_float2(hi, lo) : make_float2(__int_as_float(0x7fc00000), 0.0f);
    }
}

extern "C" int ens_convert_values(const ens_graph *graph, int s, const double *values,
                                  int dtype, void *values_lo, float *diag_lo, void *stream) {
    int rc = check_graph(graph);
    if (rc) return rc;
    if (!supported_s(s)) return fail(ENS_ERR_UNSUPPORTED, "ensemble size s=%d not in {1,4,8,16,32}", s);
    if (!values || !values_lo) return fail(ENS_ERR_ARG, "NULL values / values_lo");
    if (s > 1 && (!aligned16(values_lo) || (diag_lo && !aligned16(diag_lo))))
        return fail(ENS_ERR_ALIGN, "values_lo / diag_lo must be 16-byte aligned");
    const int64_t nt = (int64_t)graph->num_rows * s;
    if (nt == 0) return ENS_OK;
    cudaStream_t st = as_stream(stream);
    const unsigned grid = (unsigned)((nt + 255) / 256);
    if (dtype == ENS_F64_DF) {
        if (diag_lo) return fail(ENS_ERR_ARG, "convert to ENS_F64_DF takes no diag_lo");
        const int64_t count = graph->num_entries * s;
        const int64_t blocks = std::min<int64_t>((count + 255) / 256, 152 * 16);
        split_values_kernel<<<(unsigned)blocks, 256, 0, st>>>(count, values, static_cast<float2 *>(values_lo));
        ENS_LAUNCH_CHECK("split_values_kernel");
        return ENS_OK;
    }
    if (dtype == ENS_F32)
        convert_values_kernel<float><<<grid, 256, 0, st>>>(graph->num_rows, s, graph->row_map, graph->col_entry,
                                                           values, static_cast<float *>(values_lo), diag_lo);
    else if (dtype == ENS_BF16)
        convert_values_kernel<__nv_bfloat16><<<grid, 256, 0, st>>>(graph->num_rows, s, graph->row_map,
                                                                   graph->col_entry, values,
                                                                   static_cast<__nv_bfloat16 *>(values_lo), diag_lo);
    else
        return fail(ENS_ERR_UNSUPPORTED, "convert to dtype %d (ENS_F32, ENS_BF16 or ENS_F64_DF only)", dtype);
    ENS_LAUNCH_CHECK("convert_values_kernel");
    return ENS_OK;
}

extern "C" int ens_cg_mixed_workspace_size(int32_t num_rows, int s, size_t *bytes) {
    if (num_rows < 0) return fail(ENS_ERR_ARG, "num_rows < 0");
    if (!supported_s(s)) return fail(ENS_ERR_UNSUPPORTED, "ensemble size s=%d not in {1,4,8,16,32}", s);
    if (!bytes) return fail(ENS_ERR_ARG, "bytes is NULL");
    *bytes = mx_bytes(num_rows, s);
    return ENS_OK;
}

extern "C" int ens_cg_mixed(const ens_graph *graph, int s, const double *values,
                            const void *values_lo, int dtype_lo, const float *diag_lo,
                            const double *b, double *x, double tol, int max_outer,
                            double inner_tol, int max_inner, int check_every, int flags, void *work,
                            size_t work_bytes, int32_t *outer_iters_host,
                            int32_t *inner_iters_host, double *relres_host,
                            int32_t *status_host, ens_cg_stats *stats_host, void *stream) {
    int rc = check_graph(graph);
    if (rc) return rc;
    if (!supported_s(s)) return fail(ENS_ERR_UNSUPPORTED, "ensemble size s=%d not in {1,4,8,16,32}", s);
    if (graph->num_rows == 0) return fail(ENS_ERR_ARG, "empty graph");
    if (!values || !values_lo || !b || !x || !work) return fail(ENS_ERR_ARG, "NULL pointer argument");
    if (dtype_lo != ENS_F32 && dtype_lo != ENS_BF16)
        return fail(ENS_ERR_UNSUPPORTED, "inner dtype %d (ENS_F32 or ENS_BF16 only)", dtype_lo);
    if (!(tol >= 0.0) || !(inner_tol > 0.0) || max_outer < 0 || max_inner < 1 || check_every < 1)
        return fail(ENS_ERR_ARG, "tol=%g inner_tol=%g max_outer=%d max_inner=%d check_every=%d",
                    tol, inner_tol, max_outer, max_inner, check_every);
    if (!aligned16(work) || (s > 1 && (!aligned16(values) || !aligned16(values_lo) || !aligned16(b) ||
                                       !aligned16(x) || (diag_lo && !aligned16(diag_lo)))))
        return fail(ENS_ERR_ALIGN, "arrays must be 16-byte aligned");
    const size_t need = mx_bytes(graph->num_rows, s);
    if (work_bytes < need) return fail(ENS_ERR_WORKSPACE, "mixed workspace %zu < %zu bytes", work_bytes, need);
    MxOut out{outer_iters_host, inner_iters_host, relres_host, status_host, stats_host};
    cudaStream_t st = as_stream(stream);
    if (dtype_lo == ENS_F32)
        return mx_dispatch<float>(s, graph, values, values_lo, diag_lo, b, x, tol, max_outer, inner_tol,
                                  max_inner, check_every, flags, work, out, st);
    return mx_dispatch<__nv_bfloat16>(s, graph, values, values_lo, diag_lo, b, x, tol, max_outer,
                                      inner_tol, max_inner, check_every, flags, work, out, st);
}
