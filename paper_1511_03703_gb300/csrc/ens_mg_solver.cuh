// ens_mg_solver.cuh -- the ensemble multigrid V-cycle (the paper's
// preconditioner, Sect. 3.5 and Algorithm 1, in its geometric form on nested
// hex meshes), shared by the multigrid-preconditioned CG (ens_mg.cu) and the
// preconditioned GMRES of the Newton solver (ens_newton.cu).
//
// Levels l = 0 (finest) .. L: the ensemble's matrix on the (N/2^l)^3-cell
// mesh, assembled by the caller from the same KL coefficient.  Per member:
//   P_l   trilinear interpolation from the interior nodes of level l+1 to the
//         interior nodes of level l (fine index 2i <- coarse i, weight 1;
//         2i+1 <- coarse i and i+1, weight 1/2 each, per axis); R_l = P_l^T
//   S_l   Chebyshev smoother: x += p(D^-1 A) D^-1 (b - A x), `degree` steps
//         on [lam/ratio, lam], lam from the power iteration of ens_pcg
//   V_L   x = A_L^-1 b with the inverse of the coarsest matrix, formed once per
//         solve by Gauss-Jordan elimination (the matrix is SPD; <= 125 rows)
//   V_l   x = S(b, 0); r = b - A x; x += P V_{l+1}(R r); x = S(b, x)
// FP64 vectors; a level's SpMVs are FP64 or, on a level with pre-split values,
// double-float (as the pre-split CG SpMV).  Every V-cycle kernel exits at
// entry once the calling solver's
// active-member count is 0, so launches queued past convergence cost nothing.
#pragma once

#include <stdlib.h>
#include <string.h>

#include <vector>

#include "ens_pcg_kernels.cuh"
#include "ens_spmv_f32.cuh"

namespace ens {

constexpr int kMgMaxLevels = 8;
constexpr int kMgMaxCoarse = 125;  // rows of the coarsest level (N <= 4)

// ------------------------------------------------------------ transfers
// node index of (i, j, k) on an N^3-cell mesh
__device__ __forceinline__ int64_t node_id(int i, int j, int k, int n1) {
    return (int64_t)i + (int64_t)n1 * ((int64_t)j + (int64_t)n1 * k);
}

// b_c = R r_f on the interior coarse nodes, 0 on the coarse boundary
// (thread per coarse node and member)
template <int S, typename T = double>
__global__ void mg_restrict_kernel(const int *active, int Nc, const T *__restrict__ rf, T *__restrict__ bc) {
    if (ld_cg(active) == 0) return;
    const int nc1 = Nc + 1, nf1 = 2 * Nc + 1;
    const uint32_t plane = (uint32_t)nc1 * nc1;
    const int64_t total = (int64_t)nc1 * nc1 * nc1 * S;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int e = (int)(t % S);
        // node coordinates in 32-bit arithmetic (a level has fewer than 2^32 nodes)
        const uint32_t I = (uint32_t)(t / S), rem = I % plane;
        const int ck = (int)(I / plane), cj = (int)(rem / nc1), ci = (int)(rem % nc1);
        T acc = T(0);
        if (ci > 0 && ci < Nc && cj > 0 && cj < Nc && ck > 0 && ck < Nc) {
            for (int dk = -1; dk <= 1; ++dk)
                for (int dj = -1; dj <= 1; ++dj)
                    for (int di = -1; di <= 1; ++di) {
                        const int fi = 2 * ci + di, fj = 2 * cj + dj, fk = 2 * ck + dk;
                        // fine boundary nodes are not in the range of P
                        if (fi <= 0 || fi >= 2 * Nc || fj <= 0 || fj >= 2 * Nc || fk <= 0 || fk >= 2 * Nc) continue;
                        const T w = T((di ? 0.5 : 1.0) * (dj ? 0.5 : 1.0) * (dk ? 0.5 : 1.0));
                        acc = fma(w, rf[node_id(fi, fj, fk, nf1) * S + e], acc);
                    }
        }
        bc[t] = acc;
    }
}

// x_f += P x_c on the interior fine nodes (thread per fine node and member);
// xfs != NULL: also the double-float split of the new x_f
template <int S, typename T = double>
__global__ void mg_prolong_kernel(const int *active, int Nc, const T *__restrict__ xc, T *__restrict__ xf,
                                  float2 *__restrict__ xfs, int *split_bad) {
    if (ld_cg(active) == 0) return;
    const int nc1 = Nc + 1, Nf = 2 * Nc, nf1 = Nf + 1;
    const uint32_t plane = (uint32_t)nf1 * nf1;
    const int64_t total = (int64_t)nf1 * nf1 * nf1 * S;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int e = (int)(t % S);
        // node coordinates in 32-bit arithmetic (a level has fewer than 2^32 nodes)
        const uint32_t I = (uint32_t)(t / S), rem = I % plane;
        const int k = (int)(I / plane), j = (int)(rem / nf1), i = (int)(rem % nf1);
        if (i <= 0 || i >= Nf || j <= 0 || j >= Nf || k <= 0 || k >= Nf) continue;
        T acc = T(0);
        const int i0 = i >> 1, j0 = j >> 1, k0 = k >> 1;
        const int ni = (i & 1) ? 2 : 1, nj = (j & 1) ? 2 : 1, nk = (k & 1) ? 2 : 1;
        // the weight 2^-(number of odd coordinates), exact in T (no arithmetic)
        const int odd = (i & 1) + (j & 1) + (k & 1);
        const T w = odd == 0 ? T(1) : odd == 1 ? T(0.5) : odd == 2 ? T(0.25) : T(0.125);
        for (int a = 0; a < nk; ++a)
            for (int bq = 0; bq < nj; ++bq)
                for (int c = 0; c < ni; ++c) {
                    const int ci = i0 + c, cj = j0 + bq, ck = k0 + a;
                    if (ci <= 0 || ci >= Nc || cj <= 0 || cj >= Nc || ck <= 0 || ck >= Nc) continue;
                    acc = fma(w, xc[node_id(ci, cj, ck, nc1) * S + e], acc);
                }
        const T xn = xf[t] + acc;
        xf[t] = xn;
        if (xfs) store_split1(xfs, t, (double)xn, split_bad);
    }
}

// ------------------------------------------------------------ smoother
// Level SpMVs in two forms: MODE 0 FP64; MODE 3 double-float from the
// level's pre-split values and the pre-split input vector (the form of the
// pre-split CG SpMV, values prefetched into L2), falling back to FP64 once a
// producer met a value outside the split range (*split_bad).  Producers
// write the split copy next to every FP64 vector that an SpMV reads.
struct MgSpmv {
    const int32_t *row_map, *col;
    const double *vals;
    const float2 *vdf;   // MODE 3: pre-split values
    uint64_t val_bytes;  // MODE 3: bytes of the pre-split values (prefetch bound)
    int *split_bad;
};

template <int S, int MODE>
__device__ __forceinline__ double2 mg_chunk_spmv(const MgSpmv &A, ChunkCols &cc, int32_t n, const double *x,
                                                 const float2 *xs, int r, int g, bool valid) {
    if constexpr (MODE == 3) {
        const bool staged =
            stage_chunk_pf(cc, A.row_map, A.col, blockIdx.x, n, A.vdf, S * 8u, A.val_bytes, 0xffffffffu);
        if (ld_cg(A.split_bad) == 0) return chunk_spmv_dfv<S>(cc, staged, A.col, A.vdf, A.vals, xs, r, g, valid);
        return chunk_spmv<S, double>(cc, staged, A.col, A.vals, x, r, g, valid);
    } else {
        const bool staged = stage_chunk(cc, A.row_map, A.col, blockIdx.x, n);
        return chunk_spmv<S, double>(cc, staged, A.col, A.vals, x, r, g, valid);
    }
}

// write a pair of members' values (and their split when vs != NULL)
template <int S>
__device__ __forceinline__ void mg_put2(double *v, float2 *vs, int64_t R, int g, double a0, double a1, int *bad) {
    if constexpr (S == 1) {
        v[R] = a0;
        if (vs) store_split1(vs, R, a0, bad);
    } else {
        const int64_t i = R * S + 2 * g;
        reinterpret_cast<double2 *>(v)[i >> 1] = make_double2(a0, a1);
        if (vs) store_split(vs, i, a0, a1, bad);
    }
}

// first Chebyshev step from z = 0: z = d = D^-1 res / theta; with x (degree 1)
// x = z (set) or x += z (add); zs / xs: the split copies (NULL: none)
template <int S>
__global__ void mg_cheb_first_kernel(const int *active, int64_t n, const double *__restrict__ res,
                                     const double *__restrict__ dinv, const PcgState *__restrict__ ps,
                                     double *__restrict__ z, float2 *__restrict__ zs, double *__restrict__ d,
                                     double *__restrict__ x, float2 *__restrict__ xs, int add, int *split_bad) {
    if (ld_cg(active) == 0) return;
    const int64_t total = n * S;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int e = (int)(t % S);
        const double zv = res[t] * dinv[t] * ps->inv_theta[e];
        z[t] = zv;
        d[t] = zv;
        if (zs) store_split1(zs, t, zv, split_bad);
        if (x) {
            const double xv = add ? x[t] + zv : zv;
            x[t] = xv;
            if (xs) store_split1(xs, t, xv, split_bad);
        }
    }
}

// Chebyshev step k: w = res - A z_in, d = rho_k rho_{k-1} d + (2 rho_k/delta) D^-1 w,
// z_out = z_in + d; on the last step x = z_out (set) or x += z_out (add)
template <int S, int MODE>
__global__ void __launch_bounds__(RowMap<S>::THREADS, 1024 / RowMap<S>::THREADS)
    mg_cheb_step_kernel(const int *active, int32_t n, MgSpmv A, const double *__restrict__ res,
                        const double *__restrict__ dinv, const PcgState *__restrict__ ps, int k,
                        const double *__restrict__ zin, const float2 *__restrict__ zins, double *__restrict__ zout,
                        float2 *__restrict__ zouts, double *__restrict__ d, double *__restrict__ x,
                        float2 *__restrict__ xs, int add) {
    if (ld_cg(active) == 0) return;
    constexpr int G = RowMap<S>::G;
    __shared__ ChunkCols cc;
    const int r = threadIdx.x / G, g = threadIdx.x % G;
    const int64_t R = (int64_t)blockIdx.x * 32 + r;
    const double2 az = mg_chunk_spmv<S, MODE>(A, cc, n, zin, zins, r, g, R < n);
    if (R >= n || (S == 1 && g != 0)) return;
    const int w = (S == 1) ? 1 : 2;
    const int64_t i0 = (S == 1) ? R : R * S + 2 * g;
    double zo[2] = {0.0, 0.0}, xo[2] = {0.0, 0.0};
    for (int j = 0; j < w; ++j) {
        const int64_t i = i0 + j;
        const int e = (S == 1) ? 0 : 2 * g + j;
        const double rk = ps->rhoc[k][e], rk1 = ps->rhoc[k - 1][e];
        const double dv = rk * rk1 * d[i] + ps->c2[k][e] * (dinv[i] * (res[i] - (j == 0 ? az.x : az.y)));
        zo[j] = zin[i] + dv;
        d[i] = dv;
        if (x) xo[j] = add ? x[i] + zo[j] : zo[j];
    }
    mg_put2<S>(zout, zouts, R, g, zo[0], zo[1], A.split_bad);
    if (x) mg_put2<S>(x, xs, R, g, xo[0], xo[1], A.split_bad);
}

// r = b - A x
template <int S, int MODE>
__global__ void __launch_bounds__(RowMap<S>::THREADS, 1024 / RowMap<S>::THREADS)
    mg_residual_kernel(const int *active, int32_t n, MgSpmv A, const double *__restrict__ b,
                       const double *__restrict__ x, const float2 *__restrict__ xs, double *__restrict__ r) {
    if (ld_cg(active) == 0) return;
    constexpr int G = RowMap<S>::G;
    __shared__ ChunkCols cc;
    const int rr = threadIdx.x / G, g = threadIdx.x % G;
    const int64_t R = (int64_t)blockIdx.x * 32 + rr;
    const double2 ax = mg_chunk_spmv<S, MODE>(A, cc, n, x, xs, rr, g, R < n);
    if (R >= n) return;
    if constexpr (S == 1) {
        if (g == 0) r[R] = b[R] - ax.x;
    } else {
        const double2 bv = reinterpret_cast<const double2 *>(b)[R * G + g];
        reinterpret_cast<double2 *>(r)[R * G + g] = make_double2(bv.x - ax.x, bv.y - ax.y);
    }
}

// ------------------------------------------------------------ FP32 V-cycle
// The same smoother and residual with FP32 values, vectors and arithmetic
// (a mixed-precision preconditioner: the CG around it stays FP64).  TR is the
// type of the right-hand side read (FP64 at the finest level, where it is the
// CG residual).  x64: FP64 copy of the result (the finest level's output).
template <int S, typename TR>
__global__ void mg32_cheb_first_kernel(const int *active, int64_t n, const TR *__restrict__ res,
                                       const float *__restrict__ dinv, const PcgState *__restrict__ ps,
                                       float *__restrict__ z, float *__restrict__ d, float *__restrict__ x,
                                       double *__restrict__ x64, int add) {
    if (ld_cg(active) == 0) return;
    const int64_t total = n * S;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int e = (int)(t % S);
        const float zv = __fmul_rn(__fmul_rn((float)res[t], dinv[t]), (float)ps->inv_theta[e]);
        z[t] = zv;
        d[t] = zv;
        if (x) {
            const float xv = add ? __fadd_rn(x[t], zv) : zv;
            x[t] = xv;
            if (x64) x64[t] = (double)xv;
        }
    }
}

// thread map of the FP32 V-cycle kernels: W members per thread (4 from s = 8,
// with 16-byte loads; the per-member sums are those of the 2-member SpMV)
template <int S>
struct Map32 {
    static constexpr int W = (S >= 8) ? 4 : (S == 1 ? 1 : 2);
    static constexpr int G = (S == 1) ? 2 : S / W;
    static constexpr int THREADS = 32 * G;
};
template <int S, typename V>
__device__ __forceinline__ float4 mg32_spmv(const ChunkCols &cc, bool staged, const int32_t *__restrict__ col,
                                            const V *__restrict__ vals, const float *__restrict__ x, int r,
                                            int g, int64_t R, bool valid) {
    if constexpr (Map32<S>::W == 4) {
        return chunk_spmv4_f32<S, V>(cc, staged, col, vals, nullptr, x, r, g, R, valid);
    } else {
        const float2 t = chunk_spmv_f32<S, V>(cc, staged, col, vals, nullptr, x, r, g, R, valid);
        return make_float4(t.x, t.y, 0.f, 0.f);
    }
}

template <int S, typename TR>
__global__ void __launch_bounds__(Map32<S>::THREADS, 1024 / Map32<S>::THREADS)
    mg32_cheb_step_kernel(const int *active, int32_t n, const int32_t *__restrict__ row_map,
                          const int32_t *__restrict__ col, const float *__restrict__ vals, uint64_t val_bytes,
                          const TR *__restrict__ res, const float *__restrict__ dinv,
                          const PcgState *__restrict__ ps, int k, const float *__restrict__ zin,
                          float *__restrict__ zout, float *__restrict__ d, float *__restrict__ x,
                          double *__restrict__ x64, int add) {
    if (ld_cg(active) == 0) return;
    constexpr int G = Map32<S>::G, W = Map32<S>::W;
    __shared__ ChunkCols cc;
    const int r = threadIdx.x / G, g = threadIdx.x % G;
    const int64_t R = (int64_t)blockIdx.x * 32 + r;
    const bool staged = stage_chunk_pf(cc, row_map, col, blockIdx.x, n, vals, S * 4u, val_bytes, 0xffffffffu);
    const float4 az4 = mg32_spmv<S, float>(cc, staged, col, vals, zin, r, g, R, R < n);
    if (R >= n || (S == 1 && g != 0)) return;
    const float az[4] = {az4.x, az4.y, az4.z, az4.w};
    const int64_t i0 = (S == 1) ? R : R * S + W * g;
#pragma unroll
    for (int j = 0; j < W; ++j) {
        const int64_t i = i0 + j;
        const int e = (S == 1) ? 0 : W * g + j;
        const float rk = (float)ps->rhoc[k][e], rk1 = (float)ps->rhoc[k - 1][e], c2 = (float)ps->c2[k][e];
        const float wv = __fsub_rn((float)res[i], az[j]);
        const float dv = __fmaf_rn(__fmul_rn(rk, rk1), d[i], __fmul_rn(c2, __fmul_rn(dinv[i], wv)));
        const float zv = __fadd_rn(zin[i], dv);
        d[i] = dv;
        zout[i] = zv;
        if (x) {
            const float xv = add ? __fadd_rn(x[i], zv) : zv;
            x[i] = xv;
            if (x64) x64[i] = (double)xv;
        }
    }
}

template <int S, typename TR>
__global__ void __launch_bounds__(Map32<S>::THREADS, 1024 / Map32<S>::THREADS)
    mg32_residual_kernel(const int *active, int32_t n, const int32_t *__restrict__ row_map,
                         const int32_t *__restrict__ col, const float *__restrict__ vals, uint64_t val_bytes,
                         const TR *__restrict__ b, const float *__restrict__ x, float *__restrict__ r) {
    if (ld_cg(active) == 0) return;
    constexpr int G = Map32<S>::G, W = Map32<S>::W;
    __shared__ ChunkCols cc;
    const int rr = threadIdx.x / G, g = threadIdx.x % G;
    const int64_t R = (int64_t)blockIdx.x * 32 + rr;
    const bool staged = stage_chunk_pf(cc, row_map, col, blockIdx.x, n, vals, S * 4u, val_bytes, 0xffffffffu);
    const float4 ax = mg32_spmv<S, float>(cc, staged, col, vals, x, rr, g, R, R < n);
    if (R >= n) return;
    if constexpr (S == 1) {
        if (g == 0) r[R] = __fsub_rn((float)b[R], ax.x);
    } else if constexpr (W == 2) {
        const int64_t i = R * S + 2 * g;
        reinterpret_cast<float2 *>(r)[i >> 1] =
            make_float2(__fsub_rn((float)b[i], ax.x), __fsub_rn((float)b[i + 1], ax.y));
    } else {
        const int64_t i = R * S + 4 * g;
        reinterpret_cast<float4 *>(r)[i >> 2] =
            make_float4(__fsub_rn((float)b[i], ax.x), __fsub_rn((float)b[i + 1], ax.y),
                        __fsub_rn((float)b[i + 2], ax.z), __fsub_rn((float)b[i + 3], ax.w));
    }
}

// D^-1 in FP32 for the FP32 V-cycle
static __global__ void mg32_to_f32_kernel(int64_t total, const double *__restrict__ v, float *__restrict__ out) {
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x)
        out[t] = __double2float_rn(v[t]);
}

// ------------------------------------------------------------ coarse level
// Ainv_e = A_e^-1 by in-place Gauss-Jordan elimination in shared memory
// (A_e SPD: no pivoting); one CTA per member.  The inverse is stored
// transposed (invT[j*n+i] = Ainv[i][j]) so that the solve reads it coalesced.
template <int S>
__global__ void __launch_bounds__(512) mg_coarse_inverse_kernel(int32_t n, const int32_t *__restrict__ row_map,
                                                                const int32_t *__restrict__ col,
                                                                const double *__restrict__ vals,
                                                                double *__restrict__ inv, int *bad) {
    extern __shared__ double A[];  // n x n, row-major
    const int e = blockIdx.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    for (int t = threadIdx.x; t < n * n; t += blockDim.x) A[t] = 0.0;
    __syncthreads();
    for (int I = threadIdx.x; I < n; I += blockDim.x)
        for (int32_t p = row_map[I]; p < row_map[I + 1]; ++p) A[I * n + col[p]] = vals[(int64_t)p * S + e];
    __syncthreads();
    __shared__ double piv;
    for (int k = 0; k < n; ++k) {
        if (threadIdx.x == 0) {
            const double a = A[k * n + k];
            if (!(a > 0.0)) *bad = 1;
            piv = 1.0 / a;
            A[k * n + k] = 1.0;
        }
        __syncthreads();
        for (int j = threadIdx.x; j < n; j += blockDim.x) A[k * n + j] *= piv;
        __syncthreads();
        // rows i != k, columns j != k: A[i][j] -= A[i][k] A[k][j] (row k and column k are not written)
        for (int i = warp; i < n; i += nwarps) {
            if (i == k) continue;
            const double f = A[i * n + k];
            for (int j = lane; j < n; j += 32)
                if (j != k) A[i * n + j] = fma(-f, A[k * n + j], A[i * n + j]);
        }
        __syncthreads();
        for (int i = threadIdx.x; i < n; i += blockDim.x)
            if (i != k) A[i * n + k] = -A[i * n + k] * piv;
        __syncthreads();
    }
    double *out = inv + (int64_t)e * n * n;
    for (int t = threadIdx.x; t < n * n; t += blockDim.x) {
        const int i = t / n, j = t % n;
        out[j * n + i] = A[t];
    }
}

// x = Ainv_e b_e (one CTA per member; thread i reads column i of invT)
template <int S, typename T = double>
__global__ void mg_coarse_solve_kernel(const int *active, int32_t n, const double *__restrict__ inv,
                                       const T *__restrict__ b, T *__restrict__ x) {
    if (ld_cg(active) == 0) return;
    const int e = blockIdx.x;
    __shared__ double bs[kMgMaxCoarse];
    for (int i = threadIdx.x; i < n; i += blockDim.x) bs[i] = (double)b[(int64_t)i * S + e];
    __syncthreads();
    const double *invT = inv + (int64_t)e * n * n;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        double acc = 0.0;
        for (int j = 0; j < n; ++j) acc = fma(invT[(int64_t)j * n + i], bs[j], acc);
        x[(int64_t)i * S + e] = (T)acc;
    }
}

// ------------------------------------------------------------ host side
static size_t mg_align(size_t x) { return (x + 255) / 256 * 256; }

struct MgLevel {
    int32_t n, N;
    const int32_t *row_map, *col;
    const double *vals;
    const float2 *vdf;    // pre-split values (the level's SpMVs in MODE 3), or NULL
    uint64_t val_bytes;   // 8 bytes per value and member
    PcgArgs pa;           // per-level set-up (power iteration) and Chebyshev state
    double *b, *x, *r, *z[2], *d;
    float2 *xs, *zs[2];   // split copies of x, z0, z1 (MODE 3 levels)
    int *split_bad;       // shared by all levels
    const float *v32;     // FP32 values (the FP32 V-cycle), or NULL
    uint64_t v32_bytes;
    float *b32, *x32, *r32, *z32[2], *d32, *dinv32;  // the FP32 V-cycle's vectors
};

// Scratch of the hierarchy from `base` (NULL: only count the bytes): per
// level the Chebyshev state, ten vectors (D, D^-1, two power-iteration
// vectors, b, x, r, z0, z1, d) and two dot trees, plus four split copies
// (x, z0, z1, v) on levels with pre-split values; then the coarsest level's
// inverses and two status words.  Returns the bytes (a multiple of 256).
static size_t mg_layout(int nl, const ens_mg_level *lv, int s, std::vector<MgLevel> *out, char *base,
                        double **coarse_inv, int **bad) {
    size_t off = 0;
    auto take = [&](size_t bytes) -> char * {
        char *p = base ? base + off : nullptr;
        off += mg_align(bytes);
        return p;
    };
    if (out) out->resize(nl);
    for (int l = 0; l < nl; ++l) {
        const int64_t n = lv[l].graph.num_rows;
        const size_t vb = sizeof(double) * (size_t)n * s;
        PcgState *ps = reinterpret_cast<PcgState *>(take(sizeof(PcgState)));
        double *vec[10];
        for (int i = 0; i < 10; ++i) vec[i] = reinterpret_cast<double *>(take(vb));
        char *t1 = take(dot_tree_bytes(n, s));
        char *t2 = take(dot_tree_bytes(n, 2 * s));
        float2 *sv[4] = {nullptr, nullptr, nullptr, nullptr};
        if (lv[l].values_df)
            for (int i = 0; i < 4; ++i) sv[i] = reinterpret_cast<float2 *>(take(vb));
        float *fv[8] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
        if (lv[l].values_f32)
            for (int i = 0; i < 8; ++i) fv[i] = reinterpret_cast<float *>(take(vb / 2));
        if (out && base) {
            MgLevel &m = (*out)[l];
            m.n = (int32_t)n;
            m.N = lv[l].N;
            m.row_map = lv[l].graph.row_map;
            m.col = lv[l].graph.col_entry;
            m.vals = lv[l].values;
            m.vdf = reinterpret_cast<const float2 *>(lv[l].values_df);
            m.val_bytes = (uint64_t)lv[l].graph.num_entries * s * 8u;
            memset(&m.pa, 0, sizeof(m.pa));
            CgArgs &c = m.pa.c;
            c.n = (int32_t)n;
            c.row_map = m.row_map;
            c.col = m.col;
            c.vals = m.vals;
            c.vdf = m.vdf;
            c.pdf = sv[3];
            c.val_bytes = m.val_bytes;
            m.xs = sv[0];
            m.zs[0] = sv[1];
            m.zs[1] = sv[2];
            m.v32 = lv[l].values_f32;
            m.v32_bytes = (uint64_t)lv[l].graph.num_entries * s * 4u;
            m.b32 = fv[0];
            m.x32 = fv[1];
            m.r32 = fv[2];
            m.z32[0] = fv[3];
            m.z32[1] = fv[4];
            m.d32 = fv[5];
            m.dinv32 = fv[6];
            m.pa.vals32 = m.v32;
            m.pa.v32 = fv[7];
            m.pa.vals32_bytes = m.v32_bytes;
            dot_tree_layout(&c.t1, n, s, t1);
            dot_tree_layout(&c.t2, n, 2 * s, t2);
            m.pa.ps = ps;
            m.pa.dg = vec[0];
            m.pa.dinv = vec[1];
            m.pa.v = vec[2];
            m.pa.y = vec[3];
            m.b = vec[4];
            m.x = vec[5];
            m.r = vec[6];
            m.z[0] = vec[7];
            m.z[1] = vec[8];
            m.d = vec[9];
        }
    }
    const int64_t nc = lv[nl - 1].graph.num_rows;
    double *inv = reinterpret_cast<double *>(take(sizeof(double) * (size_t)nc * nc * s));
    int *badp = reinterpret_cast<int *>(take(sizeof(int)));
    int *split_bad = reinterpret_cast<int *>(take(sizeof(int)));
    if (base) {
        *coarse_inv = inv;
        *bad = badp;
        if (out)
            for (int l = 0; l < nl; ++l) {
                (*out)[l].split_bad = split_bad;
                (*out)[l].pa.split_bad = split_bad;
            }
    }
    return off;
}

template <int S>
struct MgSolver {
    std::vector<MgLevel> lv;
    double *inv;
    const int *active;  // CG active-member count: every V-cycle kernel exits at entry once it is 0
    int degree;
    bool f32 = false;   // the FP32 V-cycle (every level has FP32 values)
    unsigned eg;  // grid of the elementwise kernels

    static unsigned chunks(int64_t n) { return (unsigned)((n + 31) / 32); }

    static MgSpmv spmv_of(const MgLevel &m) {
        MgSpmv A;
        A.row_map = m.row_map;
        A.col = m.col;
        A.vals = m.vals;
        A.vdf = m.vdf;
        A.val_bytes = m.val_bytes;
        A.split_bad = m.split_bad;
        return A;
    }

    // x = S(res, x) (add) or S(res, 0); xs: the split copy of x to write (NULL: none)
    void smooth(int l, const double *res, double *x, float2 *xs, int add, cudaStream_t st) {
        MgLevel &m = lv[l];
        const bool pre = m.vdf != nullptr;
        mg_cheb_first_kernel<S><<<eg, 256, 0, st>>>(active, m.n, res, m.pa.dinv, m.pa.ps, m.z[0],
                                                    (pre && degree > 1) ? m.zs[0] : nullptr, m.d,
                                                    degree == 1 ? x : nullptr, degree == 1 ? xs : nullptr, add,
                                                    m.split_bad);
        const MgSpmv A = spmv_of(m);
        for (int k = 1; k < degree; ++k) {
            const bool last = (k == degree - 1);
            const double *zin = m.z[(k - 1) & 1];
            const float2 *zins = m.zs[(k - 1) & 1];
            double *zout = m.z[k & 1];
            float2 *zouts = (pre && !last) ? m.zs[k & 1] : nullptr;
            double *xo = last ? x : nullptr;
            float2 *xso = last ? xs : nullptr;
            if (pre)
                mg_cheb_step_kernel<S, 3><<<chunks(m.n), RowMap<S>::THREADS, 0, st>>>(
                    active, m.n, A, res, m.pa.dinv, m.pa.ps, k, zin, zins, zout, zouts, m.d, xo, xso, add);
            else
                mg_cheb_step_kernel<S, 0><<<chunks(m.n), RowMap<S>::THREADS, 0, st>>>(
                    active, m.n, A, res, m.pa.dinv, m.pa.ps, k, zin, nullptr, zout, nullptr, m.d, xo, nullptr, add);
        }
    }

    void residual(int l, const double *b, const double *x, cudaStream_t st) {
        MgLevel &m = lv[l];
        const MgSpmv A = spmv_of(m);
        if (m.vdf)
            mg_residual_kernel<S, 3><<<chunks(m.n), RowMap<S>::THREADS, 0, st>>>(active, m.n, A, b, x, m.xs, m.r);
        else
            mg_residual_kernel<S, 0><<<chunks(m.n), RowMap<S>::THREADS, 0, st>>>(active, m.n, A, b, x, nullptr, m.r);
    }

    // x = V_l(b); out_split: on a pre-split level, also leave the split copy of
    // the result in the level's xs (for a caller's pre-split SpMV of x)
    void vcycle(int l, const double *b, double *x, cudaStream_t st, bool out_split = false) {
        const int L = (int)lv.size() - 1;
        if (l == L) {
            mg_coarse_solve_kernel<S><<<S, 128, 0, st>>>(active, lv[L].n, inv, b, x);
            return;
        }
        MgLevel &m = lv[l], &mc = lv[l + 1];
        float2 *xs = m.vdf ? m.xs : nullptr;  // x's split copy: read by this level's residuals
        smooth(l, b, x, xs, 0, st);                                                 // x = S(b, 0)
        residual(l, b, x, st);
        mg_restrict_kernel<S><<<eg, 256, 0, st>>>(active, mc.N, m.r, mc.b);
        vcycle(l + 1, mc.b, mc.x, st);
        mg_prolong_kernel<S><<<eg, 256, 0, st>>>(active, mc.N, mc.x, x, xs, m.split_bad);  // x += P x_c
        residual(l, b, x, st);
        smooth(l, m.r, x, out_split ? xs : nullptr, 1, st);                         // x = S(b, x)
    }

    // ---- the FP32 V-cycle (f32): res64 / b64 are read at the finest level
    // (the CG residual), res32 / b32 below; x64 receives the finest level's
    // result in FP64 (the CG's z)
    void smooth32(int l, const double *res64, const float *res32, float *x, double *x64, int add,
                  cudaStream_t st) {
        MgLevel &m = lv[l];
        const PcgState *ps = m.pa.ps;
        if (res64)
            mg32_cheb_first_kernel<S, double><<<eg, 256, 0, st>>>(active, m.n, res64, m.dinv32, ps, m.z32[0], m.d32,
                                                                 degree == 1 ? x : nullptr,
                                                                 degree == 1 ? x64 : nullptr, add);
        else
            mg32_cheb_first_kernel<S, float><<<eg, 256, 0, st>>>(active, m.n, res32, m.dinv32, ps, m.z32[0], m.d32,
                                                                degree == 1 ? x : nullptr,
                                                                degree == 1 ? x64 : nullptr, add);
        for (int k = 1; k < degree; ++k) {
            const bool last = (k == degree - 1);
            float *xo = last ? x : nullptr;
            double *x64o = last ? x64 : nullptr;
            if (res64)
                mg32_cheb_step_kernel<S, double><<<chunks(m.n), Map32<S>::THREADS, 0, st>>>(
                    active, m.n, m.row_map, m.col, m.v32, m.v32_bytes, res64, m.dinv32, ps, k, m.z32[(k - 1) & 1],
                    m.z32[k & 1], m.d32, xo, x64o, add);
            else
                mg32_cheb_step_kernel<S, float><<<chunks(m.n), Map32<S>::THREADS, 0, st>>>(
                    active, m.n, m.row_map, m.col, m.v32, m.v32_bytes, res32, m.dinv32, ps, k, m.z32[(k - 1) & 1],
                    m.z32[k & 1], m.d32, xo, x64o, add);
        }
    }

    void residual32(int l, const double *b64, const float *b32, const float *x, cudaStream_t st) {
        MgLevel &m = lv[l];
        if (b64)
            mg32_residual_kernel<S, double><<<chunks(m.n), Map32<S>::THREADS, 0, st>>>(
                active, m.n, m.row_map, m.col, m.v32, m.v32_bytes, b64, x, m.r32);
        else
            mg32_residual_kernel<S, float><<<chunks(m.n), Map32<S>::THREADS, 0, st>>>(
                active, m.n, m.row_map, m.col, m.v32, m.v32_bytes, b32, x, m.r32);
    }

    // x = V_l(b) in FP32 (b64 at l = 0, b32 below); x64: FP64 copy of the result
    void vcycle32(int l, const double *b64, const float *b32, float *x, double *x64, cudaStream_t st) {
        const int L = (int)lv.size() - 1;
        if (l == L) {  // L >= 1: the coarsest level is never the finest
            mg_coarse_solve_kernel<S, float><<<S, 128, 0, st>>>(active, lv[L].n, inv, b32, x);
            return;
        }
        MgLevel &m = lv[l], &mc = lv[l + 1];
        smooth32(l, b64, b32, x, nullptr, 0, st);                                  // x = S(b, 0)
        residual32(l, b64, b32, x, st);
        mg_restrict_kernel<S, float><<<eg, 256, 0, st>>>(active, mc.N, m.r32, mc.b32);
        vcycle32(l + 1, nullptr, mc.b32, mc.x32, nullptr, st);
        mg_prolong_kernel<S, float><<<eg, 256, 0, st>>>(active, mc.N, mc.x32, x, nullptr, m.split_bad);
        residual32(l, b64, b32, x, st);
        smooth32(l, nullptr, m.r32, x, x64, 1, st);                                // x = S(b, x)
    }

    // Per level: D and D^-1, the power estimate of the largest eigenvalue of
    // D^-1 A from the caller's start vectors, the Chebyshev parameters; then
    // the inverse of the coarsest matrix (*bad = 1 if it is not positive
    // definite; the caller reads it).  All asynchronous on st.
    // the set-up of level l on stream st (diagonal, eigenvalue bound, Chebyshev parameters)
    int setup_level(int l, const ens_mg_level *levels, double ratio, double boost, int power_iters,
                    bool lanczos, cudaStream_t st, int *launches) {
        MgLevel &m = lv[l];
        PcgArgs &a = m.pa;
        int rc;
        a.degree = degree;
        a.boost = boost;
        a.ratio = ratio;
        if ((rc = dot_tree_clear(a.c.t1, st))) return rc;
        if ((rc = dot_tree_clear(a.c.t2, st))) return rc;
        ENS_CUDA_TRY(cudaMemsetAsync(a.ps, 0, sizeof(PcgState), st));
        const int64_t nt = (int64_t)m.n * S;
        pc_diag_kernel<S><<<(unsigned)((nt + 255) / 256), 256, 0, st>>>(m.n, m.row_map, m.col, m.vals,
                                                                     const_cast<double *>(a.dg),
                                                                     const_cast<double *>(a.dinv));
        if (f32) mg32_to_f32_kernel<<<152 * 4, 256, 0, st>>>(nt, a.dinv, m.dinv32);
        ENS_CUDA_TRY(cudaMemcpyAsync(a.v, levels[l].power_start, sizeof(double) * (size_t)nt,
                                     cudaMemcpyDeviceToDevice, st));
        if (lanczos) {   // the level's r holds q_{j-1} (the set-up runs before any V-cycle)
            if (f32) *launches += lanczos_bound<S, 4>(a, m.r, chunks(m.n), power_iters, st);
            else if (m.vdf) *launches += lanczos_bound<S, 3>(a, m.r, chunks(m.n), power_iters, st);
            else *launches += lanczos_bound<S, 0>(a, m.r, chunks(m.n), power_iters, st);
        } else if (f32) {  // the FP32 V-cycle's bound: power iteration on its FP32 values
            mg32_to_f32_kernel<<<152 * 4, 256, 0, st>>>(nt, a.v, a.v32);
            for (int k = 0; k < power_iters; ++k) {
                pc_power_kernel<S, 4><<<chunks(m.n), RowMap<S>::THREADS, 0, st>>>(a);
                pc_scale_kernel<S, 4><<<152 * 4, 256, 0, st>>>(a);
            }
            pc_rayleigh_kernel<S, 4><<<chunks(m.n), RowMap<S>::THREADS, 0, st>>>(a);
            *launches += 4 + 2 * power_iters;
        } else if (m.vdf) {
            pc_split_kernel<S><<<152 * 4, 256, 0, st>>>(a);
            for (int k = 0; k < power_iters; ++k) {
                pc_power_kernel<S, 3><<<chunks(m.n), RowMap<S>::THREADS, 0, st>>>(a);
                pc_scale_kernel<S, 3><<<152 * 4, 256, 0, st>>>(a);
            }
            pc_rayleigh_kernel<S, 3><<<chunks(m.n), RowMap<S>::THREADS, 0, st>>>(a);
            *launches += 3 + 2 * power_iters;
        } else {
            for (int k = 0; k < power_iters; ++k) {
                pc_power_kernel<S><<<chunks(m.n), RowMap<S>::THREADS, 0, st>>>(a);
                pc_scale_kernel<S><<<152 * 4, 256, 0, st>>>(a);
            }
            pc_rayleigh_kernel<S><<<chunks(m.n), RowMap<S>::THREADS, 0, st>>>(a);
            *launches += 2 + 2 * power_iters;
        }
        return ENS_OK;
    }

    // Per level: D and D^-1, the power estimate of the largest eigenvalue of
    // D^-1 A from the caller's start vectors, the Chebyshev parameters; then
    // the inverse of the coarsest matrix (*bad = 1 if it is not positive
    // definite; the caller reads it).  Level 0 runs on st; the coarser levels
    // (short, latency-bound launches) and the coarsest inverse (one CTA per
    // member) on two forked streams that st then waits for.  Asynchronous.
    int setup(const ens_mg_level *levels, double ratio, double boost, int power_iters, int *bad,
              cudaStream_t st, int *launches, bool lanczos = false) {
        const int nl = (int)lv.size();
        int rc = ENS_OK;
        ENS_CUDA_TRY(cudaMemsetAsync(bad, 0, sizeof(int), st));
        ENS_CUDA_TRY(cudaMemsetAsync(lv[0].split_bad, 0, sizeof(int), st));
        MgLevel &mc = lv[nl - 1];
        const size_t smem = sizeof(double) * (size_t)mc.n * mc.n;
        ENS_CUDA_TRY(cudaFuncSetAttribute(mg_coarse_inverse_kernel<S>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)smem));
        cudaStream_t side[2] = {nullptr, nullptr};
        cudaEvent_t fork = nullptr, join[2] = {nullptr, nullptr};
        cudaError_t ce = cudaEventCreateWithFlags(&fork, cudaEventDisableTiming);
        for (int i = 0; i < 2 && ce == cudaSuccess; ++i) {
            ce = cudaStreamCreateWithFlags(&side[i], cudaStreamNonBlocking);
            if (ce == cudaSuccess) ce = cudaEventCreateWithFlags(&join[i], cudaEventDisableTiming);
        }
        if (ce == cudaSuccess) ce = cudaEventRecord(fork, st);
        for (int i = 0; i < 2 && ce == cudaSuccess; ++i) ce = cudaStreamWaitEvent(side[i], fork, 0);
        if (ce == cudaSuccess) {
            for (int l = 0; l < nl && rc == ENS_OK; ++l)
                rc = setup_level(l, levels, ratio, boost, power_iters, lanczos, l == 0 ? st : side[0], launches);
            mg_coarse_inverse_kernel<S><<<S, 512, smem, side[1]>>>(mc.n, mc.row_map, mc.col, mc.vals, inv, bad);
            ++*launches;
            for (int i = 0; i < 2 && ce == cudaSuccess; ++i) {
                ce = cudaEventRecord(join[i], side[i]);
                if (ce == cudaSuccess) ce = cudaStreamWaitEvent(st, join[i], 0);
            }
        }
        for (int i = 0; i < 2; ++i) {
            if (side[i]) cudaStreamDestroy(side[i]);  // released once their work is done
            if (join[i]) cudaEventDestroy(join[i]);
        }
        if (fork) cudaEventDestroy(fork);
        if (ce != cudaSuccess) return cuda_fail(ce, "ens_mg set-up streams");
        if (rc) return rc;
        ENS_LAUNCH_CHECK("ens_mg set-up");
        return ENS_OK;
    }

    int launches_per_vcycle() const {
        const int L = (int)lv.size() - 1;
        return L * (2 * degree + 4) + 1;
    }
};

static int mg_check(int nl, const ens_mg_level *lv, int s) {
    if (nl < 2 || nl > kMgMaxLevels || !lv) return fail(ENS_ERR_ARG, "ens_mg: 2 <= nlevels <= %d", kMgMaxLevels);
    if (!supported_s(s)) return fail(ENS_ERR_UNSUPPORTED, "ensemble size s=%d not in {1,4,8,16,32}", s);
    for (int l = 0; l < nl; ++l) {
        int rc = check_graph(&lv[l].graph);
        if (rc) return rc;
        const int64_t n1 = (int64_t)lv[l].N + 1;
        if (lv[l].N < 1 || lv[l].graph.num_rows != n1 * n1 * n1)
            return fail(ENS_ERR_ARG, "ens_mg: level %d: graph is not that of the %d^3-cell mesh", l, lv[l].N);
        if (l > 0 && 2 * lv[l].N != lv[l - 1].N)
            return fail(ENS_ERR_ARG, "ens_mg: level %d has N=%d, not half of %d", l, lv[l].N, lv[l - 1].N);
        if (!lv[l].values) return fail(ENS_ERR_ARG, "ens_mg: level %d: NULL values", l);
        if (s > 1 && !aligned16(lv[l].values)) return fail(ENS_ERR_ALIGN, "ens_mg: level %d values not aligned", l);
        if (lv[l].values_df && !aligned16(lv[l].values_df))
            return fail(ENS_ERR_ALIGN, "ens_mg: level %d values_df not aligned", l);
        if ((lv[l].values_f32 != nullptr) != (lv[0].values_f32 != nullptr))
            return fail(ENS_ERR_ARG, "ens_mg: values_f32 on every level or none (level %d)", l);
        if (lv[l].values_f32 && s > 1 && !aligned16(lv[l].values_f32))
            return fail(ENS_ERR_ALIGN, "ens_mg: level %d values_f32 not aligned", l);
    }
    if (lv[nl - 1].graph.num_rows > kMgMaxCoarse)
        return fail(ENS_ERR_UNSUPPORTED, "ens_mg: coarsest level has %d rows (at most %d: N <= 4)",
                    lv[nl - 1].graph.num_rows, kMgMaxCoarse);
    return ENS_OK;
}

}  // namespace ens
