/*
 * ens_oracle.h -- CPU oracle for the embedded-ensemble diffusion problem.
 *
 * TEST INFRASTRUCTURE ONLY.  This is a plain, slow, per-sample FP64
 * restatement of what the paper's method computes.  Only the tests, the
 * smoke check and the benchmark's CPU-baseline leg may load it; the CUDA
 * library shares no code, header, table or helper with it.
 *
 * Everything here is per sample (one value per matrix entry / node), the
 * "scalar" system f(u, y) = 0 of Sect. 2.  The ensemble system of Eq. 3
 * (commuted Kronecker ordering) is, member by member, exactly s copies of
 * this, which is why a per-sample oracle is the definition the ensemble
 * path must reproduce.
 *
 * Conventions (the paper is silent on them; these are the readings used):
 *   node (i,j,k), 0 <= i,j,k <= N      -> i + (N+1)*(j + (N+1)*k), x = (i,j,k)/N
 *   cell (ci,cj,ck), 0 <= ci,cj,ck < N -> ci + N*(cj + N*ck)
 *   local node l (0..7)                 -> offsets (l&1, (l>>1)&1, (l>>2)&1)
 *   quadrature point q (0..7)           -> 2x2x2 Gauss, same bit convention
 */
#ifndef ENS_ORACLE_H
#define ENS_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- mesh and CRS graph (Fig. 2 data structure, Algorithm 2 NodeIndex) ---- */
int64_t or_num_rows(int N);
int64_t or_num_cells(int N);
/* node_index[c*8 + l] = NodeIndex(c, l) */
void or_node_index(int N, int32_t *node_index);
/* CRS graph: row I's columns = every node sharing a cell with I, ascending.
 * row_map has num_rows+1 entries; returns num_entries, or -1 if col_entry is
 * NULL (then only row_map is filled). */
int64_t or_graph(int N, int32_t *row_map, int32_t *col_entry);
/* elem_graph[c*64 + a*8 + b] = CRS entry of (NodeIndex(c,a), NodeIndex(c,b)) */
int or_elem_graph(int N, const int32_t *row_map, const int32_t *col_entry,
                  int32_t *elem_graph);
/* bmask[I] = 1 on the boundary of the unit cube, else 0 */
void or_bmask(int N, uint8_t *bmask);

/* ---- Karhunen-Loeve expansion of exp(-|x-x'|_1 / L) on [0,1]^3 (Sect. 4) ---- */
/* first P one-dimensional eigenpairs: omega[p], lambda[p]; p even -> cosine
 * mode, p odd -> sine mode; returns 0 */
int or_kl_1d(int P, double L, double *omega, double *lambda);
/* normalised 1D eigenfunction p (frequency omega) at x in [0,1] */
double or_kl_phi1d(int p, double L, double omega, double x);
/* the M largest 3D modes: pqr[3k..3k+2] = (p,q,r), lambda3[k] */
int or_kl_modes(int M, double L, int32_t *pqr, double *lambda3);
/* coefficient a(x, xi) = kappa0 + sigma * sum_k sqrt(lambda_k) phi_k(x) xi_k */
double or_kl_coeff_at(int M, double L, double sigma, double kappa0,
                      const int32_t *pqr, const double *lambda3,
                      const double *omega1d, const double *xi, const double x[3]);
/* a at every quadrature point: a_qp[c*8 + q] */
int or_kl_coeff_qp(int N, int M, double L, double sigma, double kappa0,
                   const double *xi, double *a_qp);

/* ---- finite-element assembly (Algorithm 2, alpha = beta = 0, source 1) ---- */
/* element stiffness for coefficient values a_q at the 8 Gauss points */
void or_element_matrix(double h, const double a_q[8], double K[64]);
void or_element_load(double h, double f[8]);
/* full assembly of one sample, Dirichlet u = 0 applied by symmetric
 * elimination; values[num_entries], b[num_rows].  Returns 0, or
 * OR_NONPOS_COEFF when the coefficient is not positive (or NaN) at some
 * Gauss point (values and b are written all the same). */
#define OR_NONPOS_COEFF 7
int or_assemble(int N, int M, double L, double sigma, double kappa0,
                const double *xi, const int32_t *row_map, const int32_t *col_entry,
                double *values, double *b);

/* ---- sparse linear algebra (Fig. 2 SpMV, Sect. 3.4 inner products) ---- */
void or_spmv(int64_t num_rows, const int32_t *row_map, const int32_t *col_entry,
             const double *values, const double *x, double *z);
double or_dot(int64_t n, const double *u, const double *v);

/* Unpreconditioned CG (Hestenes-Stiefel).  Stops when ||r|| <= tol*||b||
 * (recursive residual).  x holds x0 on entry.  Returns 0 converged,
 * 5 not converged within max_iter, 6 breakdown (p'Ap <= 0 or not finite).
 * iters = iterations done; relres = true ||b - A x|| / ||b||. */
int or_cg(int64_t num_rows, const int32_t *row_map, const int32_t *col_entry,
          const double *values, const double *b, double *x, double tol,
          int max_iter, int32_t *iters, double *relres);

/* assemble + CG for num_samples independent samples, xi[j*M + k];
 * samples run in parallel over nthreads OpenMP threads (one sample per
 * thread at a time).  x_out[j*num_rows + I] may be NULL. */
int or_solve_samples(int N, int M, double L, double sigma, double kappa0,
                     int num_samples, const double *xi, double tol, int max_iter,
                     int nthreads, double *x_out, int32_t *iters, double *relres,
                     int32_t *status);
int or_max_threads(void);

#ifdef __cplusplus
}
#endif
#endif
