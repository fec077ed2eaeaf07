/*
 * ens_oracle.c -- CPU oracle (TEST INFRASTRUCTURE ONLY; see ens_oracle.h).
 *
 * Plain sequential FP64 loops that follow the paper's definitions:
 *   - Fig. 2: CRS matrix and the row-by-row matrix-vector product.
 *   - Sect. 4, Eq. 9-10: KL expansion of the exponential covariance with the
 *     L1 norm, whose eigenfunctions are tensor products of 1D sines/cosines.
 *   - Algorithm 2: element loop, gather through NodeIndex, quadrature-point
 *     loop, scatter through ElemGraph (done sequentially, so no atomics).
 *   - Sect. 3.4: CG as run by the solver library; inner products per sample.
 * Compiled with -ffp-contract=off so every a*b+c rounds twice, as written.
 */
#include "ens_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------ mesh */

int64_t or_num_rows(int N) { return (int64_t)(N + 1) * (N + 1) * (N + 1); }
int64_t or_num_cells(int N) { return (int64_t)N * N * N; }

static int64_t node_of(int N, int i, int j, int k) {
    return (int64_t)i + (int64_t)(N + 1) * ((int64_t)j + (int64_t)(N + 1) * k);
}

void or_node_index(int N, int32_t *node_index) {
    for (int ck = 0; ck < N; ++ck)
        for (int cj = 0; cj < N; ++cj)
            for (int ci = 0; ci < N; ++ci) {
                int64_t c = ci + (int64_t)N * (cj + (int64_t)N * ck);
                for (int l = 0; l < 8; ++l)
                    node_index[c * 8 + l] = (int32_t)node_of(
                        N, ci + (l & 1), cj + ((l >> 1) & 1), ck + ((l >> 2) & 1));
            }
}

static int cmp_i32(const void *a, const void *b) {
    int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
    return (x > y) - (x < y);
}

/* columns of row I: union of the nodes of every cell that contains I */
static int row_columns(int N, int64_t I, int32_t out[64]) {
    int i = (int)(I % (N + 1)), j = (int)((I / (N + 1)) % (N + 1)),
        k = (int)(I / ((int64_t)(N + 1) * (N + 1)));
    int32_t cand[64];
    int nc = 0;
    for (int ck = k - 1; ck <= k; ++ck)
        for (int cj = j - 1; cj <= j; ++cj)
            for (int ci = i - 1; ci <= i; ++ci) {
                if (ci < 0 || cj < 0 || ck < 0 || ci >= N || cj >= N || ck >= N) continue;
                for (int l = 0; l < 8; ++l)
                    cand[nc++] = (int32_t)node_of(N, ci + (l & 1), cj + ((l >> 1) & 1),
                                                  ck + ((l >> 2) & 1));
            }
    qsort(cand, (size_t)nc, sizeof(int32_t), cmp_i32);
    int m = 0;
    for (int t = 0; t < nc; ++t)
        if (m == 0 || cand[t] != out[m - 1]) out[m++] = cand[t];
    return m;
}

int64_t or_graph(int N, int32_t *row_map, int32_t *col_entry) {
    int64_t n = or_num_rows(N);
    int32_t cols[64];
    row_map[0] = 0;
    for (int64_t I = 0; I < n; ++I) {
        int m = row_columns(N, I, cols);
        row_map[I + 1] = row_map[I] + m;
        if (col_entry)
            for (int t = 0; t < m; ++t) col_entry[row_map[I] + t] = cols[t];
    }
    return col_entry ? (int64_t)row_map[n] : -1;
}

static int64_t find_entry(const int32_t *row_map, const int32_t *col_entry, int64_t I,
                          int32_t J) {
    for (int64_t e = row_map[I]; e < row_map[I + 1]; ++e)
        if (col_entry[e] == J) return e;
    return -1;
}

int or_elem_graph(int N, const int32_t *row_map, const int32_t *col_entry,
                  int32_t *elem_graph) {
    int64_t nc = or_num_cells(N);
    int32_t *ni = (int32_t *)malloc(sizeof(int32_t) * (size_t)(nc * 8));
    if (!ni) return 1;
    or_node_index(N, ni);
    for (int64_t c = 0; c < nc; ++c)
        for (int a = 0; a < 8; ++a)
            for (int b = 0; b < 8; ++b) {
                int64_t e = find_entry(row_map, col_entry, ni[c * 8 + a], ni[c * 8 + b]);
                if (e < 0) { free(ni); return 2; }
                elem_graph[c * 64 + a * 8 + b] = (int32_t)e;
            }
    free(ni);
    return 0;
}

void or_bmask(int N, uint8_t *bmask) {
    for (int k = 0; k <= N; ++k)
        for (int j = 0; j <= N; ++j)
            for (int i = 0; i <= N; ++i)
                bmask[node_of(N, i, j, k)] =
                    (i == 0 || j == 0 || k == 0 || i == N || j == N || k == N) ? 1 : 0;
}

/* ------------------------------------------------------------------- KL */
/*
 * 1D problem: int_0^1 exp(-|x - x'| / L) f(x') dx' = lambda f(x).  With the
 * interval centred (t = x - 1/2, half-width a = 1/2) and c = 1/L the
 * eigenfunctions are cos(omega t) with c - omega tan(omega a) = 0 (even) or
 * sin(omega t) with omega + c tan(omega a) = 0 (odd), lambda = 2c/(omega^2+c^2)
 * (the classical solution quoted by the paper's KL reference, Ghanem and
 * Spanos, Sect. 2.3).  Mode p: even p -> n-th cosine root in
 * (n pi/a, (n+1/2) pi/a), odd p -> n-th sine root in ((n+1/2) pi/a, (n+1) pi/a),
 * n = p/2.  Roots by bisection on the tan-free forms below.
 */
static const double KL_A = 0.5;

static double kl_even_fn(double w, double c) { return c * cos(w * KL_A) - w * sin(w * KL_A); }
static double kl_odd_fn(double w, double c) { return w * cos(w * KL_A) + c * sin(w * KL_A); }

int or_kl_1d(int P, double L, double *omega, double *lambda) {
    const double c = 1.0 / L;
    for (int p = 0; p < P; ++p) {
        int n = p / 2, odd = p & 1;
        double lo = odd ? (n + 0.5) * M_PI / KL_A : n * M_PI / KL_A;
        double hi = odd ? (n + 1.0) * M_PI / KL_A : (n + 0.5) * M_PI / KL_A;
        double flo = odd ? kl_odd_fn(lo, c) : kl_even_fn(lo, c);
        for (int it = 0; it < 200; ++it) {
            double mid = 0.5 * (lo + hi);
            if (mid <= lo || mid >= hi) break;
            double fm = odd ? kl_odd_fn(mid, c) : kl_even_fn(mid, c);
            if (fm == 0.0) { lo = hi = mid; break; }
            if ((fm > 0) == (flo > 0)) { lo = mid; flo = fm; } else { hi = mid; }
        }
        double w = 0.5 * (lo + hi);
        omega[p] = w;
        lambda[p] = 2.0 * c / (w * w + c * c);
    }
    return 0;
}

double or_kl_phi1d(int p, double L, double omega, double x) {
    (void)L;
    double t = x - 0.5;
    double s2 = sin(2.0 * omega * KL_A) / (2.0 * omega);
    if (p & 1) return sin(omega * t) / sqrt(KL_A - s2);
    return cos(omega * t) / sqrt(KL_A + s2);
}

typedef struct { int p, q, r; double lam; } kl_mode3;

static int cmp_mode3(const void *a, const void *b) {
    const kl_mode3 *x = (const kl_mode3 *)a, *y = (const kl_mode3 *)b;
    if (x->lam != y->lam) return (x->lam < y->lam) ? 1 : -1; /* descending */
    if (x->p != y->p) return x->p - y->p;
    if (x->q != y->q) return x->q - y->q;
    return x->r - y->r;
}

/* 3D eigenvalue = product of the three 1D eigenvalues taken in ascending
 * index order, so that permuted triples give bitwise-equal products and tie
 * groups stay ties; ties broken by (p,q,r) ascending, p the x index. */
int or_kl_modes(int M, double L, int32_t *pqr, double *lambda3) {
    if (M <= 0) return 0;
    int P = M;
    double *om = (double *)malloc(sizeof(double) * P), *la = (double *)malloc(sizeof(double) * P);
    kl_mode3 *all = (kl_mode3 *)malloc(sizeof(kl_mode3) * (size_t)P * P * P);
    if (!om || !la || !all) { free(om); free(la); free(all); return 1; }
    or_kl_1d(P, L, om, la);
    int cnt = 0;
    for (int p = 0; p < P; ++p)
        for (int q = 0; q < P; ++q)
            for (int r = 0; r < P; ++r) {
                int s0 = p, s1 = q, s2 = r, t;
                if (s0 > s1) { t = s0; s0 = s1; s1 = t; }
                if (s1 > s2) { t = s1; s1 = s2; s2 = t; }
                if (s0 > s1) { t = s0; s0 = s1; s1 = t; }
                all[cnt].p = p; all[cnt].q = q; all[cnt].r = r;
                all[cnt].lam = (la[s0] * la[s1]) * la[s2];
                ++cnt;
            }
    qsort(all, (size_t)cnt, sizeof(kl_mode3), cmp_mode3);
    for (int k = 0; k < M; ++k) {
        pqr[3 * k] = all[k].p; pqr[3 * k + 1] = all[k].q; pqr[3 * k + 2] = all[k].r;
        lambda3[k] = all[k].lam;
    }
    free(om); free(la); free(all);
    return 0;
}

double or_kl_coeff_at(int M, double L, double sigma, double kappa0, const int32_t *pqr,
                      const double *lambda3, const double *omega1d, const double *xi,
                      const double x[3]) {
    double sum = 0.0;
    for (int k = 0; k < M; ++k) {
        int p = pqr[3 * k], q = pqr[3 * k + 1], r = pqr[3 * k + 2];
        double term = sqrt(lambda3[k]) * or_kl_phi1d(p, L, omega1d[p], x[0]) *
                      or_kl_phi1d(q, L, omega1d[q], x[1]) * or_kl_phi1d(r, L, omega1d[r], x[2]);
        sum += term * xi[k];
    }
    return kappa0 + sigma * sum;
}

/* 2-point Gauss-Legendre on [0,1]: (1 -+ 1/sqrt(3))/2, weight 1/2 each */
static double gauss_pt(int t) {
    double d = 0.5 / sqrt(3.0);
    return t ? 0.5 + d : 0.5 - d;
}

int or_kl_coeff_qp(int N, int M, double L, double sigma, double kappa0, const double *xi,
                   double *a_qp) {
    int32_t *pqr = (int32_t *)malloc(sizeof(int32_t) * 3 * (M > 0 ? M : 1));
    double *lam = (double *)malloc(sizeof(double) * (M > 0 ? M : 1));
    double *om = (double *)malloc(sizeof(double) * (M > 0 ? M : 1));
    double *la1 = (double *)malloc(sizeof(double) * (M > 0 ? M : 1));
    if (!pqr || !lam || !om || !la1) { free(pqr); free(lam); free(om); free(la1); return 1; }
    if (M > 0) { or_kl_modes(M, L, pqr, lam); or_kl_1d(M, L, om, la1); }
    double h = 1.0 / N;
    for (int ck = 0; ck < N; ++ck)
        for (int cj = 0; cj < N; ++cj)
            for (int ci = 0; ci < N; ++ci) {
                int64_t c = ci + (int64_t)N * (cj + (int64_t)N * ck);
                for (int q = 0; q < 8; ++q) {
                    double x[3] = {(ci + gauss_pt(q & 1)) * h, (cj + gauss_pt((q >> 1) & 1)) * h,
                                   (ck + gauss_pt((q >> 2) & 1)) * h};
                    a_qp[c * 8 + q] = or_kl_coeff_at(M, L, sigma, kappa0, pqr, lam, om, xi, x);
                }
            }
    free(pqr); free(lam); free(om); free(la1);
    return 0;
}

/* ------------------------------------------------------------- assembly */
/* trilinear basis on the reference cell [0,1]^3: phi_l(xi) = prod_d L_d,
 * L = xi_d if offset_d(l) = 1 else 1 - xi_d */
static double lin(int o, double t) { return o ? t : 1.0 - t; }
static double dlin(int o) { return o ? 1.0 : -1.0; }

static void ref_grad(int l, const double xi[3], double g[3]) {
    int o0 = l & 1, o1 = (l >> 1) & 1, o2 = (l >> 2) & 1;
    g[0] = dlin(o0) * lin(o1, xi[1]) * lin(o2, xi[2]);
    g[1] = lin(o0, xi[0]) * dlin(o1) * lin(o2, xi[2]);
    g[2] = lin(o0, xi[0]) * lin(o1, xi[1]) * dlin(o2);
}

/* K(a,b) = sum_q a_q * w_q * h^3 * (grad phi_a . grad phi_b)(x_q) with
 * physical gradients = reference gradients / h, w_q = 1/8; computed for
 * a <= b and mirrored so the element matrix is exactly symmetric */
void or_element_matrix(double h, const double a_q[8], double K[64]) {
    double g[8][8][3];
    for (int q = 0; q < 8; ++q) {
        double xi[3] = {gauss_pt(q & 1), gauss_pt((q >> 1) & 1), gauss_pt((q >> 2) & 1)};
        for (int l = 0; l < 8; ++l) ref_grad(l, xi, g[q][l]);
    }
    double scale = h * 0.125; /* w_q h^3 / h^2 */
    for (int a = 0; a < 8; ++a)
        for (int b = a; b < 8; ++b) {
            double sum = 0.0;
            for (int q = 0; q < 8; ++q) {
                double gg = g[q][a][0] * g[q][b][0] + g[q][a][1] * g[q][b][1] +
                            g[q][a][2] * g[q][b][2];
                sum += a_q[q] * (scale * gg);
            }
            K[a * 8 + b] = sum;
            K[b * 8 + a] = sum;
        }
}

/* f(a) = sum_q phi_a(x_q) * w_q * h^3 * source, source = 1 */
void or_element_load(double h, double f[8]) {
    double vol = h * h * h * 0.125;
    for (int a = 0; a < 8; ++a) {
        double sum = 0.0;
        for (int q = 0; q < 8; ++q) {
            double phi = lin(a & 1, gauss_pt(q & 1)) * lin((a >> 1) & 1, gauss_pt((q >> 1) & 1)) *
                         lin((a >> 2) & 1, gauss_pt((q >> 2) & 1));
            sum += phi * vol;
        }
        f[a] = sum;
    }
}

int or_assemble(int N, int M, double L, double sigma, double kappa0, const double *xi,
                const int32_t *row_map, const int32_t *col_entry, double *values, double *b) {
    int64_t n = or_num_rows(N), nc = or_num_cells(N);
    int64_t nnz = row_map[n];
    double h = 1.0 / N;
    int32_t *ni = (int32_t *)malloc(sizeof(int32_t) * (size_t)(nc * 8));
    int32_t *eg = (int32_t *)malloc(sizeof(int32_t) * (size_t)(nc * 64));
    double *a_qp = (double *)malloc(sizeof(double) * (size_t)(nc * 8));
    uint8_t *bm = (uint8_t *)malloc((size_t)n);
    if (!ni || !eg || !a_qp || !bm) { free(ni); free(eg); free(a_qp); free(bm); return 1; }
    or_node_index(N, ni);
    if (or_elem_graph(N, row_map, col_entry, eg)) { free(ni); free(eg); free(a_qp); free(bm); return 2; }
    or_kl_coeff_qp(N, M, L, sigma, kappa0, xi, a_qp);
    /* Sect. 4: the diffusion coefficient must be positive for the problem to
     * be elliptic (and the stiffness matrix SPD); report a(x_q) <= 0 or NaN */
    int nonpos = 0;
    for (int64_t i = 0; i < nc * 8; ++i)
        if (!(a_qp[i] > 0.0)) nonpos = 1;
    or_bmask(N, bm);
    memset(values, 0, sizeof(double) * (size_t)nnz);
    memset(b, 0, sizeof(double) * (size_t)n);
    double fe[8], Ke[64];
    or_element_load(h, fe);
    for (int64_t c = 0; c < nc; ++c) {           /* Algorithm 2 cell loop */
        or_element_matrix(h, &a_qp[c * 8], Ke);   /* quadrature-point loop */
        for (int a = 0; a < 8; ++a) {             /* scatter via NodeIndex / ElemGraph */
            b[ni[c * 8 + a]] += fe[a];
            for (int bb = 0; bb < 8; ++bb) values[eg[c * 64 + a * 8 + bb]] += Ke[a * 8 + bb];
        }
    }
    /* Dirichlet u = 0: boundary rows -> identity row, b = 0; interior rows
     * drop their boundary columns (stored zeros keep the graph intact) */
    for (int64_t I = 0; I < n; ++I) {
        for (int64_t e = row_map[I]; e < row_map[I + 1]; ++e) {
            int32_t J = col_entry[e];
            if (bm[I]) values[e] = (J == I) ? 1.0 : 0.0;
            else if (bm[J]) values[e] = 0.0;
        }
        if (bm[I]) b[I] = 0.0;
    }
    free(ni); free(eg); free(a_qp); free(bm);
    return nonpos ? OR_NONPOS_COEFF : 0;
}

/* --------------------------------------------------------- linear algebra */

void or_spmv(int64_t num_rows, const int32_t *row_map, const int32_t *col_entry,
             const double *values, const double *x, double *z) {
    for (int64_t row = 0; row < num_rows; ++row) {
        double sum = 0.0;
        for (int64_t e = row_map[row]; e < row_map[row + 1]; ++e)
            sum += values[e] * x[col_entry[e]];
        z[row] = sum;
    }
}

double or_dot(int64_t n, const double *u, const double *v) {
    double s = 0.0;
    for (int64_t i = 0; i < n; ++i) s += u[i] * v[i];
    return s;
}

int or_cg(int64_t n, const int32_t *row_map, const int32_t *col_entry, const double *values,
          const double *b, double *x, double tol, int max_iter, int32_t *iters, double *relres) {
    double *r = (double *)malloc(sizeof(double) * (size_t)n);
    double *p = (double *)malloc(sizeof(double) * (size_t)n);
    double *q = (double *)malloc(sizeof(double) * (size_t)n);
    if (!r || !p || !q) { free(r); free(p); free(q); return 1; }
    int status = 5;
    int k = 0;
    double bnorm = sqrt(or_dot(n, b, b));
    if (bnorm == 0.0) {            /* b = 0: the solution is x = 0 */
        for (int64_t i = 0; i < n; ++i) x[i] = 0.0;
        *iters = 0; *relres = 0.0;
        free(r); free(p); free(q);
        return 0;
    }
    or_spmv(n, row_map, col_entry, values, x, q);
    for (int64_t i = 0; i < n; ++i) { r[i] = b[i] - q[i]; p[i] = r[i]; }
    double rho = or_dot(n, r, r);
    if (sqrt(rho) <= tol * bnorm) status = 0;
    while (status != 0 && k < max_iter) {
        or_spmv(n, row_map, col_entry, values, p, q);
        double pi = or_dot(n, p, q);
        if (!(pi > 0.0) || !isfinite(pi)) { status = 6; break; }
        double alpha = rho / pi;
        for (int64_t i = 0; i < n; ++i) { x[i] += alpha * p[i]; r[i] -= alpha * q[i]; }
        double rho_new = or_dot(n, r, r);
        ++k;
        if (sqrt(rho_new) <= tol * bnorm) { status = 0; break; }
        double beta = rho_new / rho;
        for (int64_t i = 0; i < n; ++i) p[i] = r[i] + beta * p[i];
        rho = rho_new;
    }
    /* true residual of the returned iterate */
    or_spmv(n, row_map, col_entry, values, x, q);
    for (int64_t i = 0; i < n; ++i) r[i] = b[i] - q[i];
    *iters = k;
    *relres = sqrt(or_dot(n, r, r)) / bnorm;
    free(r); free(p); free(q);
    return status;
}

int or_max_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

int or_solve_samples(int N, int M, double L, double sigma, double kappa0, int num_samples,
                     const double *xi, double tol, int max_iter, int nthreads, double *x_out,
                     int32_t *iters, double *relres, int32_t *status) {
    int64_t n = or_num_rows(N);
    int32_t *row_map = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n + 1));
    if (!row_map) return 1;
    or_graph(N, row_map, NULL);
    int64_t nnz = row_map[n];
    int32_t *col = (int32_t *)malloc(sizeof(int32_t) * (size_t)nnz);
    if (!col) { free(row_map); return 1; }
    or_graph(N, row_map, col);
    int err = 0;
    (void)nthreads;
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads) reduction(| : err)
    for (int j = 0; j < num_samples; ++j) {
        double *vals = (double *)malloc(sizeof(double) * (size_t)nnz);
        double *b = (double *)malloc(sizeof(double) * (size_t)n);
        double *x = (double *)calloc((size_t)n, sizeof(double));
        if (!vals || !b || !x) { err |= 1; free(vals); free(b); free(x); continue; }
        const int ra = or_assemble(N, M, L, sigma, kappa0, xi + (int64_t)j * M, row_map, col, vals, b);
        if (ra == OR_NONPOS_COEFF) {   /* not an elliptic problem: no solve */
            status[j] = OR_NONPOS_COEFF;
            iters[j] = 0;
            relres[j] = 0.0;
        } else {
            err |= ra;
            status[j] = or_cg(n, row_map, col, vals, b, x, tol, max_iter, &iters[j], &relres[j]);
        }
        if (x_out) memcpy(x_out + (int64_t)j * n, x, sizeof(double) * (size_t)n);
        free(vals); free(b); free(x);
    }
    free(row_map); free(col);
    return err;
}
