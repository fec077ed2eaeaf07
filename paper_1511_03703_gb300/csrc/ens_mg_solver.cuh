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
// All FP64.  Every V-cycle kernel exits at entry once the calling solver's
// active-member count is 0, so launches queued past convergence cost nothing.
#pragma once

#include <stdlib.h>
#include <string.h>

#include <vector>

#include "ens_pcg_kernels.cuh"

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
template <int S>
__global__ void mg_restrict_kernel(const int *active, int Nc, const double *__restrict__ rf,
                                   double *__restrict__ bc) {
    if (ld_cg(active) == 0) return;
    const int nc1 = Nc + 1, nf1 = 2 * Nc + 1;
    const int64_t total = (int64_t)nc1 * nc1 * nc1 * S;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int e = (int)(t % S);
        const int64_t I = t / S;
        const int ci = (int)(I % nc1), cj = (int)((I / nc1) % nc1), ck = (int)(I / ((int64_t)nc1 * nc1));
        double acc = 0.0;
        if (ci > 0 && ci < Nc && cj > 0 && cj < Nc && ck > 0 && ck < Nc) {
            for (int dk = -1; dk <= 1; ++dk)
                for (int dj = -1; dj <= 1; ++dj)
                    for (int di = -1; di <= 1; ++di) {
                        const int fi = 2 * ci + di, fj = 2 * cj + dj, fk = 2 * ck + dk;
                        // fine boundary nodes are not in the range of P
                        if (fi <= 0 || fi >= 2 * Nc || fj <= 0 || fj >= 2 * Nc || fk <= 0 || fk >= 2 * Nc) continue;
                        const double w = (di ? 0.5 : 1.0) * (dj ? 0.5 : 1.0) * (dk ? 0.5 : 1.0);
                        acc = fma(w, rf[node_id(fi, fj, fk, nf1) * S + e], acc);
                    }
        }
        bc[t] = acc;
    }
}

// x_f += P x_c on the interior fine nodes (thread per fine node and member)
template <int S>
__global__ void mg_prolong_kernel(const int *active, int Nc, const double *__restrict__ xc,
                                  double *__restrict__ xf) {
    if (ld_cg(active) == 0) return;
    const int nc1 = Nc + 1, Nf = 2 * Nc, nf1 = Nf + 1;
    const int64_t total = (int64_t)nf1 * nf1 * nf1 * S;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int e = (int)(t % S);
        const int64_t I = t / S;
        const int i = (int)(I % nf1), j = (int)((I / nf1) % nf1), k = (int)(I / ((int64_t)nf1 * nf1));
        if (i <= 0 || i >= Nf || j <= 0 || j >= Nf || k <= 0 || k >= Nf) continue;
        double acc = 0.0;
        const int i0 = i >> 1, j0 = j >> 1, k0 = k >> 1;
        const int ni = (i & 1) ? 2 : 1, nj = (j & 1) ? 2 : 1, nk = (k & 1) ? 2 : 1;
        for (int a = 0; a < nk; ++a)
            for (int bq = 0; bq < nj; ++bq)
                for (int c = 0; c < ni; ++c) {
                    const int ci = i0 + c, cj = j0 + bq, ck = k0 + a;
                    if (ci <= 0 || ci >= Nc || cj <= 0 || cj >= Nc || ck <= 0 || ck >= Nc) continue;
                    const double w = ((i & 1) ? 0.5 : 1.0) * ((j & 1) ? 0.5 : 1.0) * ((k & 1) ? 0.5 : 1.0);
                    acc = fma(w, xc[node_id(ci, cj, ck, nc1) * S + e], acc);
                }
        xf[t] += acc;
    }
}

// ------------------------------------------------------------ smoother
// first Chebyshev step from z = 0: z = d = D^-1 res / theta; with x (degree 1)
// x = z (set) or x += z (add)
template <int S>
__global__ void mg_cheb_first_kernel(const int *active, int64_t n, const double *__restrict__ res,
                                     const double *__restrict__ dinv, const PcgState *__restrict__ ps,
                                     double *__restrict__ z, double *__restrict__ d, double *__restrict__ x, int add) {
    if (ld_cg(active) == 0) return;
    const int64_t total = n * S;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int e = (int)(t % S);
        const double zv = res[t] * dinv[t] * ps->inv_theta[e];
        z[t] = zv;
        d[t] = zv;
        if (x) x[t] = add ? x[t] + zv : zv;
    }
}

// Chebyshev step k: w = res - A z_in, d = rho_k rho_{k-1} d + (2 rho_k/delta) D^-1 w,
// z_out = z_in + d; on the last step x = z_out (set) or x += z_out (add)
template <int S>
__global__ void __launch_bounds__(RowMap<S>::THREADS, 1024 / RowMap<S>::THREADS)
    mg_cheb_step_kernel(const int *active, int32_t n, const int32_t *__restrict__ row_map, const int32_t *__restrict__ col,
                        const double *__restrict__ vals, const double *__restrict__ res,
                        const double *__restrict__ dinv, const PcgState *__restrict__ ps, int k,
                        const double *__restrict__ zin, double *__restrict__ zout, double *__restrict__ d,
                        double *__restrict__ x, int add) {
    if (ld_cg(active) == 0) return;
    constexpr int G = RowMap<S>::G;
    __shared__ ChunkCols cc;
    const int r = threadIdx.x / G, g = threadIdx.x % G;
    const int64_t R = (int64_t)blockIdx.x * 32 + r;
    const bool staged = stage_chunk(cc, row_map, col, blockIdx.x, n);
    const double2 az = chunk_spmv<S, double>(cc, staged, col, vals, zin, r, g, R < n);
    if (R >= n || (S == 1 && g != 0)) return;
    const int w = (S == 1) ? 1 : 2;
    const int64_t i0 = (S == 1) ? R : R * S + 2 * g;
    for (int j = 0; j < w; ++j) {
        const int64_t i = i0 + j;
        const int e = (S == 1) ? 0 : 2 * g + j;
        const double rk = ps->rhoc[k][e], rk1 = ps->rhoc[k - 1][e];
        const double dv = rk * rk1 * d[i] + ps->c2[k][e] * (dinv[i] * (res[i] - (j == 0 ? az.x : az.y)));
        const double zv = zin[i] + dv;
        d[i] = dv;
        zout[i] = zv;
        if (x) x[i] = add ? x[i] + zv : zv;
    }
}

// r = b - A x
template <int S>
__global__ void __launch_bounds__(RowMap<S>::THREADS, 1024 / RowMap<S>::THREADS)
    mg_residual_kernel(const int *active, int32_t n, const int32_t *__restrict__ row_map,
                       const int32_t *__restrict__ col, const double *__restrict__ vals,
                       const double *__restrict__ b, const double *__restrict__ x, double *__restrict__ r) {
    if (ld_cg(active) == 0) return;
    constexpr int G = RowMap<S>::G;
    __shared__ ChunkCols cc;
    const int rr = threadIdx.x / G, g = threadIdx.x % G;
    const int64_t R = (int64_t)blockIdx.x * 32 + rr;
    const bool staged = stage_chunk(cc, row_map, col, blockIdx.x, n);
    const double2 ax = chunk_spmv<S, double>(cc, staged, col, vals, x, rr, g, R < n);
    if (R >= n) return;
    if constexpr (S == 1) {
        if (g == 0) r[R] = b[R] - ax.x;
    } else {
        const double2 bv = reinterpret_cast<const double2 *>(b)[R * G + g];
        reinterpret_cast<double2 *>(r)[R * G + g] = make_double2(bv.x - ax.x, bv.y - ax.y);
    }
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
template <int S>
__global__ void mg_coarse_solve_kernel(const int *active, int32_t n, const double *__restrict__ inv,
                                       const double *__restrict__ b, double *__restrict__ x) {
    if (ld_cg(active) == 0) return;
    const int e = blockIdx.x;
    __shared__ double bs[kMgMaxCoarse];
    for (int i = threadIdx.x; i < n; i += blockDim.x) bs[i] = b[(int64_t)i * S + e];
    __syncthreads();
    const double *invT = inv + (int64_t)e * n * n;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        double acc = 0.0;
        for (int j = 0; j < n; ++j) acc = fma(invT[(int64_t)j * n + i], bs[j], acc);
        x[(int64_t)i * S + e] = acc;
    }
}

// ------------------------------------------------------------ host side
static size_t mg_align(size_t x) { return (x + 255) / 256 * 256; }

struct MgLevel {
    int32_t n, N;
    const int32_t *row_map, *col;
    const double *vals;
    PcgArgs pa;      // per-level set-up (power iteration) and Chebyshev state
    double *b, *x, *r, *z[2], *d;
};

// workspace of the whole solve; with lv != NULL also lays the levels out

// Scratch of the hierarchy from `base` (NULL: only count the bytes): per
// level the Chebyshev state, ten vectors (D, D^-1, two power-iteration
// vectors, b, x, r, z0, z1, d) and two dot trees; then the coarsest level's
// inverses and a status word.  Returns the bytes (a multiple of 256).
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
        if (out && base) {
            MgLevel &m = (*out)[l];
            m.n = (int32_t)n;
            m.N = lv[l].N;
            m.row_map = lv[l].graph.row_map;
            m.col = lv[l].graph.col_entry;
            m.vals = lv[l].values;
            memset(&m.pa, 0, sizeof(m.pa));
            CgArgs &c = m.pa.c;
            c.n = (int32_t)n;
            c.row_map = m.row_map;
            c.col = m.col;
            c.vals = m.vals;
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
    if (base) {
        *coarse_inv = inv;
        *bad = badp;
    }
    return off;
}

template <int S>
struct MgSolver {
    std::vector<MgLevel> lv;
    double *inv;
    const int *active;  // CG active-member count: every V-cycle kernel exits at entry once it is 0
    int degree;
    unsigned eg;  // grid of the elementwise kernels

    static unsigned chunks(int64_t n) { return (unsigned)((n + 31) / 32); }

    void smooth(int l, const double *res, double *x, int add, cudaStream_t st) {
        MgLevel &m = lv[l];
        mg_cheb_first_kernel<S><<<eg, 256, 0, st>>>(active, m.n, res, m.pa.dinv, m.pa.ps, m.z[0], m.d,
                                                    degree == 1 ? x : nullptr, add);
        for (int k = 1; k < degree; ++k)
            mg_cheb_step_kernel<S><<<chunks(m.n), RowMap<S>::THREADS, 0, st>>>(
                active, m.n, m.row_map, m.col, m.vals, res, m.pa.dinv, m.pa.ps, k, m.z[(k - 1) & 1], m.z[k & 1], m.d,
                k == degree - 1 ? x : nullptr, add);
    }

    // x = V_l(b)
    void vcycle(int l, const double *b, double *x, cudaStream_t st) {
        const int L = (int)lv.size() - 1;
        if (l == L) {
            mg_coarse_solve_kernel<S><<<S, 128, 0, st>>>(active, lv[L].n, inv, b, x);
            return;
        }
        MgLevel &m = lv[l], &mc = lv[l + 1];
        smooth(l, b, x, 0, st);                                                     // x = S(b, 0)
        mg_residual_kernel<S><<<chunks(m.n), RowMap<S>::THREADS, 0, st>>>(active, m.n, m.row_map, m.col, m.vals, b, x, m.r);
        mg_restrict_kernel<S><<<eg, 256, 0, st>>>(active, mc.N, m.r, mc.b);
        vcycle(l + 1, mc.b, mc.x, st);
        mg_prolong_kernel<S><<<eg, 256, 0, st>>>(active, mc.N, mc.x, x);                     // x += P x_c
        mg_residual_kernel<S><<<chunks(m.n), RowMap<S>::THREADS, 0, st>>>(active, m.n, m.row_map, m.col, m.vals, b, x, m.r);
        smooth(l, m.r, x, 1, st);                                                   // x = S(b, x)
    }

    // Per level: D and D^-1, the power estimate of the largest eigenvalue of
    // D^-1 A from the caller's start vectors, the Chebyshev parameters; then
    // the inverse of the coarsest matrix (*bad = 1 if it is not positive
    // definite; the caller reads it).  All asynchronous on st.
    int setup(const ens_mg_level *levels, double ratio, double boost, int power_iters, int *bad,
              cudaStream_t st, int *launches) {
        const int nl = (int)lv.size();
        int rc;
        ENS_CUDA_TRY(cudaMemsetAsync(bad, 0, sizeof(int), st));
        for (int l = 0; l < nl; ++l) {
            MgLevel &m = lv[l];
            PcgArgs &a = m.pa;
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
            ENS_CUDA_TRY(cudaMemcpyAsync(a.v, levels[l].power_start, sizeof(double) * (size_t)nt,
                                         cudaMemcpyDeviceToDevice, st));
            for (int k = 0; k < power_iters; ++k) {
                pc_power_kernel<S><<<chunks(m.n), RowMap<S>::THREADS, 0, st>>>(a);
                pc_scale_kernel<S><<<152 * 4, 256, 0, st>>>(a);
            }
            pc_rayleigh_kernel<S><<<chunks(m.n), RowMap<S>::THREADS, 0, st>>>(a);
            *launches += 2 + 2 * power_iters;
        }
        MgLevel &mc = lv[nl - 1];
        const size_t smem = sizeof(double) * (size_t)mc.n * mc.n;
        ENS_CUDA_TRY(cudaFuncSetAttribute(mg_coarse_inverse_kernel<S>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)smem));
        mg_coarse_inverse_kernel<S><<<S, 512, smem, st>>>(mc.n, mc.row_map, mc.col, mc.vals, inv, bad);
        ++*launches;
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
    }
    if (lv[nl - 1].graph.num_rows > kMgMaxCoarse)
        return fail(ENS_ERR_UNSUPPORTED, "ens_mg: coarsest level has %d rows (at most %d: N <= 4)",
                    lv[nl - 1].graph.num_rows, kMgMaxCoarse);
    return ENS_OK;
}

}  // namespace ens
