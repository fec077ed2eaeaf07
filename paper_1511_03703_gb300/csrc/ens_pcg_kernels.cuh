// ens_pcg_kernels.cuh -- device pieces shared by the preconditioned CG
// (ens_pcg.cu) and the multigrid-preconditioned CG (ens_mg.cu): per-member
// Chebyshev parameters, the diagonal, the eigenvalue bound (power iteration or
// Lanczos) and the epilogue of the preconditioner stage.
#pragma once
#include <cfloat>
#include "ens_cg_kernels.cuh"
#include "ens_spmv_f32.cuh"

namespace ens {

constexpr int kPcMaxDegree = 8;
constexpr int kLzMaxSteps = 32;   // Lanczos steps of the eigenvalue bound

struct PcgState {
    double lam[32];                    // power-iteration estimate (before the boost)
    double theta[32], delta[32];       // Chebyshev interval centre and half width
    double rhoc[kPcMaxDegree][32];     // rho_k of the Chebyshev recurrence
    double rr[32];                     // r.r of the current iteration (stop test)
    double nrm[32];                    // power iteration: ||y||
    // per-member factors of the element-wise updates, formed once so that no
    // kernel divides per element (an FP64 division costs many FP64-pipe slots)
    double inv_nrm[32];                // 1 / ||y||
    double inv_theta[32];              // 1 / theta
    double c2[kPcMaxDegree][32];       // 2 rho_k / delta
    double lz_a[kLzMaxSteps][32];      // Lanczos: alpha_j (diagonal of T)
    double lz_b[kLzMaxSteps][32];      // Lanczos: beta_j (off-diagonal of T)
};

struct PcgArgs {
    CgArgs c;
    PcgState *ps;
    const double *dg, *dinv;  // diagonal and its inverse, commuted layout
    double *zk[2];            // Chebyshev iterates (ping-pong); zk[0] is z for Jacobi
    double *d;                // Chebyshev direction
    double *v, *y;            // power iteration; Lanczos: q_j and y = A q_j, then u
    double *vprev;            // Lanczos: q_{j-1} (NULL at the first step)
    int lz_step;              // Lanczos: j (0-based), or the step count for the finish
    int degree;               // 0: Jacobi, >= 1: Chebyshev steps
    double boost, ratio;
    int *split_bad;           // MODE 3 set-up kernels: a split copy met a value out of range
    const float *vals32;      // MODE 4 set-up kernels: FP32 values (the FP32 V-cycle's)
    float *v32;               // MODE 4: FP32 copy of v
    uint64_t vals32_bytes;
};

// the set-up SpMV of v: MODE 0 FP64; MODE 3 double-float from the pre-split
// values c.vdf and the split copy c.pdf of v (FP64 once *split_bad is set);
// MODE 4 FP32 from the FP32 values and the FP32 copy of v (the eigenvalue
// bound of an FP32 V-cycle)
template <int S, int MODE>
__device__ __forceinline__ double2 pc_setup_spmv(const PcgArgs &a, ChunkCols &cc, int r, int g, bool valid) {
    const CgArgs &c = a.c;
    if constexpr (MODE == 4) {   // one column per load: 40 registers, 3 CTAs of 512 threads per SM at s = 32
        const bool staged = stage_chunk_pf<false>(cc, c.row_map, c.col, blockIdx.x, c.n, a.vals32, S * 4u,
                                                  a.vals32_bytes, 0xffffffffu);
        const int64_t R = (int64_t)blockIdx.x * 32 + r;
        const float2 y = chunk_spmv_f32<S, float>(cc, staged, c.col, a.vals32, nullptr, a.v32, r, g, R, valid);
        return make_double2((double)y.x, (double)y.y);
    } else if constexpr (MODE == 3) {
        const bool staged = stage_chunk_pf(cc, c.row_map, c.col, blockIdx.x, c.n, c.vdf, S * 8u, c.val_bytes,
                                           0xffffffffu);
        if (ld_cg(a.split_bad) == 0) return chunk_spmv_dfv<S>(cc, staged, c.col, c.vdf, c.vals, c.pdf, r, g, valid);
        return chunk_spmv<S, double>(cc, staged, c.col, c.vals, a.v, r, g, valid);
    } else {
        const bool staged = stage_chunk(cc, c.row_map, c.col, blockIdx.x, c.n);
        return chunk_spmv<S, double>(cc, staged, c.col, c.vals, a.v, r, g, valid);
    }
}

// ------------------------------------------------------------ set-up kernels
// diagonal of every member and its inverse (thread per row and member)
template <int S>
__global__ void pc_diag_kernel(int32_t n, const int32_t *__restrict__ row_map, const int32_t *__restrict__ col,
                               const double *__restrict__ vals, double *__restrict__ dg, double *__restrict__ dinv) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= (int64_t)n * S) return;
    const int32_t I = (int32_t)(t / S);
    const int e = (int)(t % S);
    double dv = 0.0;
    for (int32_t p = row_map[I]; p < row_map[I + 1]; ++p)
        if (col[p] == I) dv = vals[(int64_t)p * S + e];
    dg[t] = dv;
    dinv[t] = 1.0 / dv;
}

// power step: y = D^-1 A v, ||y||_e  (chunk per CTA, tree t1)
template <int S, int MODE = 0>
__global__ void __launch_bounds__(RowMap<S>::THREADS, 1024 / RowMap<S>::THREADS) pc_power_kernel(PcgArgs a) {
    constexpr int G = RowMap<S>::G;
    __shared__ double sm[32][S + 1];
    __shared__ ChunkCols cc;
    const CgArgs &c = a.c;
    const int r = threadIdx.x / G, g = threadIdx.x % G;
    const int64_t R = (int64_t)blockIdx.x * 32 + r;
    const double2 av = pc_setup_spmv<S, MODE>(a, cc, r, g, R < c.n);
    double v0 = 0.0, v1 = 0.0;
    if (R < c.n) {
        if constexpr (S == 1) {
            const double yv = av.x * a.dinv[R];
            if (g == 0) a.y[R] = yv;
            v0 = yv * yv;
        } else {
            const double2 di = reinterpret_cast<const double2 *>(a.dinv)[R * G + g];
            const double2 yv = make_double2(av.x * di.x, av.y * di.y);
            reinterpret_cast<double2 *>(a.y)[R * G + g] = yv;
            v0 = yv.x * yv.x;
            v1 = yv.y * yv.y;
        }
    }
    chunk_tree<S>(sm, v0, v1, r, g, c.t1, blockIdx.x, 0);
    if (!dot_tree_propagate(c.t1, blockIdx.x, 1)) return;
    const int e = threadIdx.x;
    if (e < S) {
        const double nv = sqrt(ld_cg(c.t1.buf[c.t1.levels] + e));
        a.ps->nrm[e] = nv;
        a.ps->inv_nrm[e] = 1.0 / nv;
    }
    __threadfence();
}

// v = y / ||y||_e (as y * (1 / ||y||_e)); MODE 3 also its split copy
template <int S, int MODE = 0>
__global__ void pc_scale_kernel(PcgArgs a) {
    const int64_t total = (int64_t)a.c.n * S;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const double vv = a.y[t] * a.ps->inv_nrm[t % S];
        a.v[t] = vv;
        if (MODE == 3) store_split1(a.c.pdf, t, vv, a.split_bad);
        if (MODE == 4) a.v32[t] = __double2float_rn(vv);
    }
}

// the split copy of the start vector v (MODE 3 set-up)
template <int S>
__global__ void pc_split_kernel(PcgArgs a) {
    const int64_t total = (int64_t)a.c.n * S;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x)
        store_split1(a.c.pdf, t, a.v[t], a.split_bad);
}

// member e's eigenvalue estimate lam and its Chebyshev parameters: the
// interval [lmax / ratio, lmax], lmax = boost * lam (Saad, Sect. 12.3)
__device__ __forceinline__ void pc_set_chebyshev(const PcgArgs &a, int e, double lam) {
    PcgState *ps = a.ps;
    ps->lam[e] = lam;
    const double lmax = a.boost * lam, lmin = lmax / a.ratio;
    const double theta = 0.5 * (lmax + lmin), delta = 0.5 * (lmax - lmin), sigma = theta / delta;
    ps->theta[e] = theta;
    ps->delta[e] = delta;
    ps->inv_theta[e] = 1.0 / theta;
    double rho = 1.0 / sigma;
    ps->rhoc[0][e] = rho;
    ps->c2[0][e] = 2.0 * rho / delta;
    for (int k = 1; k < kPcMaxDegree; ++k) {
        rho = 1.0 / (2.0 * sigma - rho);
        ps->rhoc[k][e] = rho;
        ps->c2[k][e] = 2.0 * rho / delta;
    }
}

// lam_e = (v.Av) / (v.Dv) and the Chebyshev parameters of member e
template <int S, int MODE = 0>
__global__ void __launch_bounds__(RowMap<S>::THREADS, 1024 / RowMap<S>::THREADS) pc_rayleigh_kernel(PcgArgs a) {
    constexpr int G = RowMap<S>::G;
    __shared__ double sm[32][S + 1];
    __shared__ ChunkCols cc;
    const CgArgs &c = a.c;
    const int r = threadIdx.x / G, g = threadIdx.x % G;
    const int64_t R = (int64_t)blockIdx.x * 32 + r;
    const double2 av = pc_setup_spmv<S, MODE>(a, cc, r, g, R < c.n);
    double n0 = 0.0, n1 = 0.0, d0 = 0.0, d1 = 0.0;
    if (R < c.n) {
        if constexpr (S == 1) {
            const double vv = a.v[R];
            n0 = vv * av.x;
            d0 = vv * (a.dg[R] * vv);
        } else {
            const double2 vv = reinterpret_cast<const double2 *>(a.v)[R * G + g];
            const double2 dd = reinterpret_cast<const double2 *>(a.dg)[R * G + g];
            n0 = vv.x * av.x; n1 = vv.y * av.y;
            d0 = vv.x * (dd.x * vv.x); d1 = vv.y * (dd.y * vv.y);
        }
    }
    chunk_tree<S>(sm, n0, n1, r, g, c.t2, blockIdx.x, 0);
    chunk_tree<S>(sm, d0, d1, r, g, c.t2, blockIdx.x, S);
    if (!dot_tree_propagate(c.t2, blockIdx.x, 1)) return;
    const int e = threadIdx.x;
    if (e < S) {
        const double *top = c.t2.buf[c.t2.levels];
        pc_set_chebyshev(a, e, ld_cg(top + e) / ld_cg(top + S + e));
    }
    __threadfence();
}

// ----------------------------------------------- Lanczos eigenvalue bound
// The largest eigenvalue of D^-1 A by Lanczos steps in the D inner product
// <x, y> = x.D y, in which D^-1 A is self-adjoint (Lanczos 1950; Saad,
// Iterative Methods, Sect. 6.6): q_1 = v / ||v||_D; for j = 1, 2, ...
//   y = A q_j, alpha_j = q_j.y, u = D^-1 y - alpha_j q_j - beta_{j-1} q_{j-1},
//   beta_j = ||u||_D, q_{j+1} = u / beta_j (0 when beta_j = 0);
// then the largest eigenvalue of the tridiagonal T_k(alpha, beta).  One
// kernel per dot (each with the canonical tree); the scaling is
// pc_scale_kernel (with inv_nrm = 1 / beta_j), which also writes the split or
// FP32 copy of q_{j+1} that the next SpMV reads.

// ||v||_D of the start vector v: inv_nrm = 1 / ||v||_D (0 for v = 0)
template <int S>
__global__ void __launch_bounds__(RowMap<S>::THREADS, 1024 / RowMap<S>::THREADS) pc_lz_dnorm_kernel(PcgArgs a) {
    constexpr int G = RowMap<S>::G;
    __shared__ double sm[32][S + 1];
    const CgArgs &c = a.c;
    const int r = threadIdx.x / G, g = threadIdx.x % G;
    const int64_t R = (int64_t)blockIdx.x * 32 + r;
    double v0 = 0.0, v1 = 0.0;
    if (R < c.n) {
        if constexpr (S == 1) {
            const double vv = a.v[R];
            v0 = vv * (a.dg[R] * vv);
        } else {
            const double2 vv = reinterpret_cast<const double2 *>(a.v)[R * G + g];
            const double2 dd = reinterpret_cast<const double2 *>(a.dg)[R * G + g];
            v0 = vv.x * (dd.x * vv.x);
            v1 = vv.y * (dd.y * vv.y);
        }
    }
    chunk_tree<S>(sm, v0, v1, r, g, c.t1, blockIdx.x, 0);
    if (!dot_tree_propagate(c.t1, blockIdx.x, 1)) return;
    const int e = threadIdx.x;
    if (e < S) {
        const double nv = sqrt(ld_cg(c.t1.buf[c.t1.levels] + e));
        a.ps->nrm[e] = nv;
        a.ps->inv_nrm[e] = (nv > 0.0) ? 1.0 / nv : 0.0;
    }
    __threadfence();
}

// step j: y = A q_j (the SpMV of MODE, as the power iteration's) and
// alpha_j = q_j.y into lz_a[j]
template <int S, int MODE = 0>
__global__ void __launch_bounds__(RowMap<S>::THREADS, 1024 / RowMap<S>::THREADS) pc_lz_spmv_kernel(PcgArgs a) {
    constexpr int G = RowMap<S>::G;
    __shared__ double sm[32][S + 1];
    __shared__ ChunkCols cc;
    const CgArgs &c = a.c;
    const int r = threadIdx.x / G, g = threadIdx.x % G;
    const int64_t R = (int64_t)blockIdx.x * 32 + r;
    const double2 av = pc_setup_spmv<S, MODE>(a, cc, r, g, R < c.n);
    double v0 = 0.0, v1 = 0.0;
    if (R < c.n) {
        if constexpr (S == 1) {
            if (g == 0) a.y[R] = av.x;
            v0 = a.v[R] * av.x;
        } else {
            reinterpret_cast<double2 *>(a.y)[R * G + g] = av;
            const double2 qv = reinterpret_cast<const double2 *>(a.v)[R * G + g];
            v0 = qv.x * av.x;
            v1 = qv.y * av.y;
        }
    }
    chunk_tree<S>(sm, v0, v1, r, g, c.t1, blockIdx.x, 0);
    if (!dot_tree_propagate(c.t1, blockIdx.x, 1)) return;
    const int e = threadIdx.x;
    if (e < S) a.ps->lz_a[a.lz_step][e] = ld_cg(c.t1.buf[c.t1.levels] + e);
    __threadfence();
}

// step j: u = D^-1 y - alpha_j q_j - beta_{j-1} q_{j-1} (in place of y) and
// beta_j = ||u||_D into lz_b[j], inv_nrm = 1 / beta_j (0 when beta_j = 0)
template <int S>
__global__ void __launch_bounds__(RowMap<S>::THREADS, 1024 / RowMap<S>::THREADS) pc_lz_update_kernel(PcgArgs a) {
    constexpr int G = RowMap<S>::G;
    __shared__ double sm[32][S + 1];
    const CgArgs &c = a.c;
    const PcgState *ps = a.ps;
    const int j = a.lz_step;
    const int r = threadIdx.x / G, g = threadIdx.x % G;
    const int m = (S == 1) ? 0 : 2 * g;
    const int64_t R = (int64_t)blockIdx.x * 32 + r;
    const double al0 = ps->lz_a[j][m], al1 = (S == 1) ? 0.0 : ps->lz_a[j][m + 1];
    const double be0 = (j > 0) ? ps->lz_b[j - 1][m] : 0.0;
    const double be1 = (j > 0 && S > 1) ? ps->lz_b[j - 1][m + 1] : 0.0;
    double v0 = 0.0, v1 = 0.0;
    if (R < c.n) {
        if constexpr (S == 1) {
            double u = a.y[R] * a.dinv[R] - al0 * a.v[R];
            if (j > 0) u -= be0 * a.vprev[R];
            if (g == 0) a.y[R] = u;
            v0 = u * (a.dg[R] * u);
        } else {
            const int64_t i = R * G + g;
            const double2 yv = reinterpret_cast<const double2 *>(a.y)[i];
            const double2 di = reinterpret_cast<const double2 *>(a.dinv)[i];
            const double2 qv = reinterpret_cast<const double2 *>(a.v)[i];
            double2 u = make_double2(yv.x * di.x - al0 * qv.x, yv.y * di.y - al1 * qv.y);
            if (j > 0) {
                const double2 pv = reinterpret_cast<const double2 *>(a.vprev)[i];
                u.x -= be0 * pv.x;
                u.y -= be1 * pv.y;
            }
            reinterpret_cast<double2 *>(a.y)[i] = u;
            const double2 dd = reinterpret_cast<const double2 *>(a.dg)[i];
            v0 = u.x * (dd.x * u.x);
            v1 = u.y * (dd.y * u.y);
        }
    }
    chunk_tree<S>(sm, v0, v1, r, g, c.t1, blockIdx.x, 0);
    if (!dot_tree_propagate(c.t1, blockIdx.x, 1)) return;
    const int e = threadIdx.x;
    if (e < S) {
        const double be = sqrt(ld_cg(c.t1.buf[c.t1.levels] + e));
        a.ps->lz_b[j][e] = be;
        a.ps->nrm[e] = be;
        a.ps->inv_nrm[e] = (be > 0.0) ? 1.0 / be : 0.0;
    }
    __threadfence();
}

// Number of eigenvalues of the k x k symmetric tridiagonal T(al, be) below x,
// by the signs of the pivots of the LDL^T factorisation of T - x I (Sturm
// sequence count; Golub and Van Loan, Matrix Computations, Sect. 8.4.1); a
// pivot of magnitude below pivmin is replaced by -pivmin, as in LAPACK's
// bisection.
__device__ __forceinline__ int lz_sturm_count(const double *al, const double *be2, int k, double x,
                                              double pivmin) {
    int cnt = 0;
    double d = 1.0;
    for (int i = 0; i < k; ++i) {
        d = (al[i] - x) - ((i > 0) ? be2[i - 1] / d : 0.0);
        if (fabs(d) < pivmin) d = -pivmin;
        if (d < 0.0) ++cnt;
    }
    return cnt;
}

// after k = lz_step steps: lam = the largest eigenvalue of T_k by
// multisection between Gershgorin bounds.  One warp per member (CTA e for
// member e, T in shared memory): the lanes count the eigenvalues below 32
// equally spaced interior points of [lo, hi] at once and the warp keeps the
// sub-interval where the count reaches k, a 33-fold shrink per step (about 11
// steps to the last bit).  One CTA per member spreads the FP64 divisions of
// the counts over S SMs (on one SM, 32 warps of them took 279 us; one warp
// bisecting for all members, 139 us).
template <int S>
__global__ void __launch_bounds__(32) pc_lz_finish_kernel(PcgArgs a) {
    const unsigned FULL = 0xffffffffu;
    __shared__ double al[kLzMaxSteps], be2[kLzMaxSteps];
    const int e = blockIdx.x, lane = threadIdx.x;
    const int k = a.lz_step;
    double rlo = 0.0, rhi = 0.0, rb = 1.0;
    if (lane < k) {
        const double b = (lane + 1 < k) ? a.ps->lz_b[lane][e] : 0.0;
        al[lane] = a.ps->lz_a[lane][e];
        be2[lane] = b * b;
    }
    __syncwarp();
    if (lane < k) {   // Gershgorin interval of row `lane`
        const double rad = ((lane > 0) ? sqrt(be2[lane - 1]) : 0.0) + sqrt(be2[lane]);
        rlo = al[lane] - rad;
        rhi = al[lane] + rad;
        rb = fmax(1.0, be2[lane]);
    } else {
        rlo = al[0];
        rhi = al[0];
    }
    for (int o = 16; o >= 1; o >>= 1) {
        rlo = fmin(rlo, __shfl_xor_sync(FULL, rlo, o));
        rhi = fmax(rhi, __shfl_xor_sync(FULL, rhi, o));
        rb = fmax(rb, __shfl_xor_sync(FULL, rb, o));
    }
    const double pivmin = DBL_MIN * rb;
    // every eigenvalue lies in the Gershgorin interval; widened a little, the
    // count is k at hi and below k at lo, which every step keeps
    double lo = rlo - (1e-300 + fabs(rlo) * 1e-15);
    double hi = rhi + (1e-300 + fabs(rhi) * 1e-15);
    for (int it = 0; it < 24; ++it) {
        const double x = lo + (hi - lo) * ((double)(lane + 1) / 33.0);
        const unsigned full = __ballot_sync(FULL, lz_sturm_count(al, be2, k, x, pivmin) == k);
        const int f = full ? __ffs(full) - 1 : 32;   // first point with every eigenvalue below it
        const double xf = __shfl_sync(FULL, x, f & 31), xp = __shfl_sync(FULL, x, (f + 31) & 31);
        const double nlo = (f > 0) ? xp : lo, nhi = (f < 32) ? xf : hi;
        if (!(nlo > lo || nhi < hi)) break;   // the points no longer split the interval
        lo = nlo;
        hi = nhi;
    }
    if (lane == 0) pc_set_chebyshev(a, e, 0.5 * (lo + hi));
    __threadfence();
}

// Host: the Lanczos bound of the level or system in a (start vector in a.v,
// overwritten) with `steps` steps and the SpMV of MODE, on st; qp is a third
// vector of n*s doubles for q_{j-1}.  Returns the launches issued.
template <int S, int MODE>
static int lanczos_bound(const PcgArgs &a, double *qp, unsigned chunks, int steps, cudaStream_t st) {
    double *q = a.v, *u = a.y;
    pc_lz_dnorm_kernel<S><<<chunks, RowMap<S>::THREADS, 0, st>>>(a);
    PcgArgs b = a;
    b.y = q;   // q_1 = v / ||v||_D in place, with its split or FP32 copy
    pc_scale_kernel<S, MODE><<<152 * 4, 256, 0, st>>>(b);
    for (int j = 0; j < steps; ++j) {
        b = a;
        b.v = q;
        b.y = u;
        b.vprev = (j > 0) ? qp : nullptr;
        b.lz_step = j;
        pc_lz_spmv_kernel<S, MODE><<<chunks, RowMap<S>::THREADS, 0, st>>>(b);
        pc_lz_update_kernel<S><<<chunks, RowMap<S>::THREADS, 0, st>>>(b);
        if (j + 1 < steps) {   // q_{j+1} = u / beta_j over q_{j-1}
            b.v = qp;
            pc_scale_kernel<S, MODE><<<152 * 4, 256, 0, st>>>(b);
            double *t = qp;
            qp = q;
            q = t;
        }
    }
    b = a;
    b.lz_step = steps;
    pc_lz_finish_kernel<S><<<S, 32, 0, st>>>(b);
    return 3 + 3 * steps;
}

// ------------------------------------------------------------ CG kernels
// Last CTA of the preconditioner stage, one lane per member: the stop test
// on r.r, beta = r.z / rho, rho = r.z (init: rho = r.z, beta = 0, no x update)
template <int S>
__device__ __forceinline__ void pc_epilogue(const PcgArgs &a, double rr, double rz, bool init) {
    const unsigned FULL = 0xffffffffu;
    const int e = threadIdx.x;
    CgState *st = a.c.st;
    int act = (e < S) ? st->active[e] : 0, ux = 0;
    int it = (e < S) ? st->iters[e] : 0;
    if (e < S) {
        if (init) {
            if (act && !(rz > 0.0 && isfinite(rz))) { act = 0; st->status[e] = ENS_ERR_BREAKDOWN; }
            st->rho[e] = rz;
            st->beta[e] = 0.0;
        } else if (act) {
            it += 1;
            ux = 1;
            if (sqrt(rr) <= a.c.tol * st->bnorm[e]) { act = 0; st->status[e] = ENS_OK; }
            else if (it >= a.c.max_iter) { act = 0; st->status[e] = ENS_ERR_NOT_CONVERGED; }
            else if (!(rz > 0.0 && isfinite(rz))) { act = 0; st->status[e] = ENS_ERR_BREAKDOWN; }
            else { st->beta[e] = rz / st->rho[e]; st->rho[e] = rz; }
        }
        st->iters[e] = it;
        st->updx[e] = ux;
        st->active[e] = act;
    }
    const int ac = __popc(__ballot_sync(FULL, act)), uany = __popc(__ballot_sync(FULL, ux));
    if (e == 0) {
        st->active_count = ac;
        // K3 runs only when some flag is set: at init it must still set p = z
        // (no member updates x: every updx is 0); the next K1 clears the word
        st->updx_any = init ? 1 : uany;
    }
    __threadfence();
}

}  // namespace ens
