/*
 * ens.h -- C ABI of the embedded-ensemble (Phipps et al., "Embedded Ensemble
 * Propagation ...") diffusion hot path on one NVIDIA GB300 (sm_103a).
 *
 * Problem (Sect. 4): -div(a(x,xi) grad u) = 1 on [0,1]^3, u = 0 on the
 * boundary, trilinear hex finite elements on an N^3 cell mesh, coefficient a
 * a truncated Karhunen-Loeve expansion (Eq. 9-10).  s samples ("an ensemble")
 * share one CRS graph (Fig. 2) and are stored in the commuted Kronecker
 * ordering of Eq. 3: the s values that belong to one matrix entry, node or KL
 * variable are contiguous:
 *     values[entry*s + e], x[node*s + e], xi[k*s + e],  e = 0..s-1.
 *
 * Conventions shared by every call
 *   - Pointers are DEVICE pointers unless the name ends in _host.  The caller
 *     allocates every buffer (inputs, outputs and workspaces); the library
 *     never allocates device memory.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Calls are asynchronous on that stream unless documented as
 *     synchronising (those return host results).
 *   - Every call returns an ens_status.  On failure ens_last_error() gives a
 *     thread-local message.  No kernel traps; device-side failures (breakdown,
 *     non-convergence) are reported through per-member status words.
 *   - Supported ensemble sizes: s in {1, 4, 8, 16, 32} (s = 1 is the
 *     per-sample path the paper's speed-up s*T1/Ts is measured against).
 *   - Node numbering: (i,j,k) -> i + (N+1)(j + (N+1)k); cell (ci,cj,ck) ->
 *     ci + N(cj + N ck); local node / Gauss point l -> offsets
 *     (l&1, (l>>1)&1, (l>>2)&1).
 */
#ifndef ENS_H
#define ENS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum ens_status {
    ENS_OK = 0,
    ENS_ERR_ARG = 1,           /* bad size, NULL pointer or inconsistent argument */
    ENS_ERR_UNSUPPORTED = 2,   /* s not in {1,4,8,16,32}, dtype or mesh too large */
    ENS_ERR_ALIGN = 3,         /* a pointer is not 16-byte aligned */
    ENS_ERR_CUDA = 4,          /* a CUDA runtime call failed */
    ENS_ERR_NOT_CONVERGED = 5, /* CG hit max_iter before the tolerance */
    ENS_ERR_BREAKDOWN = 6,     /* p'Ap <= 0 or not finite (matrix not SPD) */
    ENS_ERR_NONPOS_COEFF = 7,  /* a member's coefficient a(x_q) <= 0 at a Gauss point (ens_assemble) */
    ENS_ERR_TIMEOUT = 8,       /* reserved: a bounded device wait gave up */
    ENS_ERR_WORKSPACE = 9      /* workspace smaller than the *_workspace_size value */
} ens_status;

/* Value types.  ENS_F64_DF: values and x are FP64 in memory, products and sums
 * are formed in double-float arithmetic on the FP32 pipe (each FP64 operand
 * split into two floats; error per term <= ~6*2^-48 |a x|, so a row is within
 * ~1.2e-13 * sum |a_j x_j|).  GB300 runs FP64 FMA at 1/64 of its FP32 rate,
 * which bounds the native form of the ensemble SpMV below the HBM roofline. */
/* ENS_F64_SPLIT: FP64 values and x; entries at even positions of a row are
 * multiplied with the FP64 FMA, entries at odd positions in double-float, so
 * both arithmetic pipes work at once; row value = p_even + p_odd. */
typedef enum ens_dtype {
    ENS_F64 = 0, ENS_F32 = 1, ENS_BF16 = 2, ENS_F64_DF = 3, ENS_F64_SPLIT = 4
} ens_dtype;

/* CRS graph (Fig. 2): row_map[num_rows+1], col_entry[num_entries] (device,
 * int32, columns ascending within a row).  Values live in a separate array in
 * the commuted layout, one block of s values per entry. */
typedef struct ens_graph {
    int32_t num_rows;
    int32_t reserved;
    int64_t num_entries;
    const int32_t *row_map;
    const int32_t *col_entry;
} ens_graph;

const char *ens_last_error(void);
const char *ens_status_string(int status);
int ens_version(void);

/* ---------------------------------------------------------------- A1 graph */
/* Host only.  Sizes of the Q1 mesh with N cells per side:
 * num_rows = (N+1)^3, num_entries = (3N+1)^3, num_cells = N^3.  1 <= N <= 400. */
int ens_mesh_sizes(int N, int32_t *num_rows, int64_t *num_entries, int64_t *num_cells);

/* Builds the CRS graph of the Q1 hex mesh (Fig. 2; Algorithm 2's NodeIndex and
 * ElemGraph): row I holds every node that shares a cell with I, ascending.
 *   row_map   int32[num_rows+1]     (out)
 *   col_entry int32[num_entries]    (out)
 *   elem_graph int32[num_cells*64]  (out, may be NULL): entry of
 *              (NodeIndex(c,a), NodeIndex(c,b)) at [c*64 + a*8 + b]
 *   bmask     uint8[num_rows]       (out, may be NULL): 1 on the boundary.
 * Integer work, bit-exact by construction. */
int ens_graph_build(int N, int32_t *row_map, int32_t *col_entry, int32_t *elem_graph,
                    uint8_t *bmask, void *stream);

/* ------------------------------------------------------------------- A2 KL */
/* KL of C(x,x') = exp(-|x-x'|_1 / L) on [0,1]^3 (Sect. 4, Eq. 9-10): the M
 * largest eigenpairs, each a product of 1D cosine/sine modes (ordering: by
 * eigenvalue, ties by (p,q,r) ascending with p the x index).  kl_table holds,
 * for the 2N Gauss coordinates per axis, kl_table[(d*M + k)*2N + t] =
 * phi_k,d(x_t) with sqrt(lambda_k) folded into d = 0, so
 * kappa_k(x_q) = T[0][k][tx] * T[1][k][ty] * T[2][k][tz].
 * ens_kl_table_size gives the length in doubles (3*M*2N).  The roots are
 * found on the device; lambda_host[M] and pqr_host[3M] may be NULL, if not the
 * call synchronises `stream` to fill them.  1 <= M <= 64. */
int ens_kl_table_size(int N, int M, int64_t *num_doubles);
int ens_kl_setup(int N, int M, double L, double *kl_table, double *lambda_host,
                 int32_t *pqr_host, void *stream);

/* Sample-independent part of the assembly (Algorithm 2 with the coefficient
 * split by linearity): for k = 0..M the stiffness matrix of coefficient
 * kappa_k (kappa_0 = 1) on the full graph,
 *   modes[k*num_entries + entry] = sum_{cells c} sum_q kappa_k(x_q) G_q(a,b),
 * where G_q is the Q1 gradient product at Gauss point q times w_q h (2x2x2
 * Gauss), summed over the cells shared by the entry's row and column nodes;
 * and load[num_rows] = the load vector of source 1 (zero on the boundary).
 * Boundary rows and columns are stored as zeros (ens_assemble applies the
 * Dirichlet rows).  modes: double[(M+1)*num_entries]. */
int ens_mode_matrices(int N, const ens_graph *graph, int M, const double *kl_table,
                      double *modes, double *load, void *stream);

/* ------------------------------------------------------------- A3 assembly */
/* Ensemble assembly of s samples: member e has coefficient
 *   a_e(x) = kappa0 + sigma * sum_k kappa_k(x) xi[k*s + e]
 * so its matrix is kappa0*modes_0 + sum_k (sigma*xi[k*s+e]) modes_k.  Output
 * in the commuted layout: values[entry*s + e], b[node*s + e].  Dirichlet
 * u = 0 by symmetric elimination: boundary rows become identity rows with
 * b = 0; interior rows keep stored zeros in boundary columns.
 * bmask from ens_graph_build; values and b must be 16-byte aligned for s>1.
 *
 * Coefficient check (Sect. 4: the KL coefficient must stay positive for the
 * stiffness matrix to be SPD).  kl_table may be NULL (no check); otherwise it
 * is the table ens_kl_setup wrote for this mesh and M, and before assembling
 * the call verifies for every member that a_e(x_q) > 0 at every Gauss point:
 * first by the bound kappa0 - |sigma| sum_k |xi_k^e| max_q |kappa_k(x_q)|
 * (exact maxima of the separable table), and for members that bound does not
 * clear by the exact minimum over all (2N)^3 Gauss coordinates.  With
 * kl_table the call synchronises `stream` (b, 16-byte aligned, is the check's
 * scratch before it is written).  The bounds reach the host through pinned,
 * device-mapped host memory that the kernel writes directly, so the wait is
 * not held up by copies on other streams; the library allocates that memory
 * once per device and CUDA context (64 slots of 256 bytes, released with the
 * context) and reads the bounds by a copy when no slot is free.  Thread-safe
 * across host threads and streams.  If a member fails, values and b are still
 * written for every member and the call returns ENS_ERR_NONPOS_COEFF (the
 * message names the member and its minimum); a NaN coefficient fails too. */
int ens_assemble(const ens_graph *graph, const uint8_t *bmask, int s, int M, const double *kl_table,
                 const double *modes, const double *load, const double *xi, double sigma,
                 double kappa0, double *values, double *b, void *stream);

/* ens_assemble with the KL terms in double-float arithmetic on the FP32
 * pipe: sum_k (sigma*xi_k) modes_k (k >= 1) is formed from float pairs as in
 * the ENS_F64_DF SpMV and summed as a float pair, and each value is
 * kappa0*modes_0 + that sum by one FP64 FMA (coefficients or mode values
 * outside [2^-103, 2^128) use the FP64 combination).  The KL terms carry a
 * relative error of about 2^-46 each, so values agree with ens_assemble to
 * within 1e-14 of their row's diagonal for sigma = 0.1 (measured 4e-15).
 * values_df (float2[nnz*s], may be NULL): also writes the ENS_F64_DF split
 * of values, bitwise what ens_convert_values(..., ENS_F64_DF, ...) would
 * write, for ens_cg_df.  16-byte aligned for s > 1.  kl_table: the
 * coefficient check of ens_assemble (NULL: none). */
int ens_assemble_df(const ens_graph *graph, const uint8_t *bmask, int s, int M, const double *kl_table,
                    const double *modes, const double *load, const double *xi, double sigma,
                    double kappa0, double *values, void *values_df, double *b, void *stream);

/* --------------------------------------------------------------- A4 SpMV */
/* y = A_c x for the commuted ensemble matrix (Fig. 5 semantics):
 *   y[I*s+e] = sum_{entry in row I} values[entry*s+e] * x[col_entry[entry]*s+e].
 * dtype = ENS_F64 (values double), ENS_F32 (float), ENS_BF16 (bfloat16),
 * ENS_F64_DF (double values, double-float arithmetic) or ENS_F64_SPLIT (double
 * values, alternate entries FP64 / double-float); x and y are double.  The per-member sum
 * order is fixed and independent of s: entry j goes to partial j mod 2 and
 * the row value is p0 + p1, so member e's result is bitwise the same for
 * every s.  x, y, values 16-byte aligned when s > 1. */
int ens_spmv(const ens_graph *graph, int s, int dtype, const void *values, const double *x,
             double *y, void *stream);

/* ens_spmv with the values also given pre-split: values_df is their
 * ENS_F64_DF copy (float2[nnz*s], written by ens_convert_values(...,
 * ENS_F64_DF, ...) or ens_assemble_df) and values the FP64 originals.  The
 * products and sums are the double-float terms of ENS_F64_DF without the
 * per-term split of the values (the arithmetic of ens_cg_df's SpMV), x split
 * on the fly; a row is bitwise the ENS_F64_DF result.  Rows that meet a value
 * or an x outside the split range, a non-finite sum, or products below
 * 2^-96 are recomputed from the FP64 values.  values_df 16-byte aligned
 * (values, x, y too for s > 1). */
int ens_spmv_df(const ens_graph *graph, int s, const double *values, const void *values_df,
                const double *x, double *y, void *stream);

/* ---------------------------------------------------------------- A5 dot */
/* Per-member inner products (Sect. 3.4: the ensemble inner product computed
 * first as sum_i u_i^T v_i (x) e_i):  out[e] = sum_I u[I*s+e] * v[I*s+e].
 * Deterministic, s-independent order: products are summed in a fixed tree
 * (the 32 rows of a chunk pairwise, v[i] += v[i + h] for h = 16, 8, 4, 2, 1;
 * then groups of 32 chunk sums the same way, and so on).
 * work: device scratch of ens_dot_workspace_size bytes (16-byte aligned);
 * its counters are cleared by the call.  out: device double[s]. */
int ens_dot_workspace_size(int64_t n, int s, size_t *bytes);
int ens_dot(int64_t n, int s, const double *u, const double *v, double *out, void *work,
            size_t work_bytes, void *stream);

/* Allocation-free ens_dot (the paper has no counterpart; this is a library
 * convenience).  For callers that cannot allocate device memory when they
 * need the product -- e.g. code running while an allocator is locked or owned
 * by another runtime -- it computes the same per-member dots as ens_dot,
 * bitwise identical, with its reduction scratch in a static device array of
 * ENS_DOT_STATIC_MAX_BYTES bytes that every GPU loading the library keeps
 * until the process exits.  It calls no allocator.
 *   Limit: ens_dot_workspace_size(n, s) must be <= ENS_DOT_STATIC_MAX_BYTES
 *   (about 2.3 MB for n = 274,625 rows at s = 32); larger sizes return
 *   ENS_ERR_UNSUPPORTED.
 *   Set-up: the first call with a device current looks up the array's device
 *   address (cudaGetSymbolAddress); make that first call before any stream
 *   capture.  The stream must belong to the current device.
 *   Sharing: all calls share the array and it keeps the last call's contents;
 *   the call clears the counters it needs, but calls that overlap on the GPU
 *   race with each other.  u, v, out: device pointers as for ens_dot. */
#define ENS_DOT_STATIC_MAX_BYTES (4u << 20)
int ens_dot_static(int64_t n, int s, const double *u, const double *v, double *out, void *stream);

/* ----------------------------------------------------------------- A6 CG */
/* Statistics of one ens_cg call (optional). */
typedef struct ens_cg_stats {
    double spmv_ms;          /* summed CUDA-event time of the CG SpMV launches (ENS_CG_TIME_SPMV) */
    int32_t spmv_launches;   /* SpMV launches timed */
    int32_t kernel_launches; /* all kernels launched by the call */
    int32_t iterations;      /* iterations run (max over members) */
    int32_t host_checks;     /* device->host convergence polls */
    int32_t guess_fallbacks; /* members restarted from x = 0 (ENS_CG_GUESS_FALLBACK) */
    int32_t reserved;        /* zero */
} ens_cg_stats;

enum {
    ENS_CG_COUPLED = 1,      /* paper's coupled ensemble CG (Sects. 3.4, 3.7): alpha, beta
                                from member-summed dots, one convergence test */
    ENS_CG_GRAPH = 2,        /* replay the iteration through a captured CUDA graph */
    ENS_CG_TIME_SPMV = 4,    /* record CUDA events around each CG SpMV (with ENS_CG_GRAPH
                                as event-record nodes of the graph; ens_cg only) */
    ENS_CG_DF64 = 8,         /* CG SpMV in double-float arithmetic (see ENS_F64_DF);
                                p is kept split as float pairs, all other vector
                                arithmetic and every dot stays FP64 */
    ENS_CG_SPLIT64 = 16,     /* CG SpMV with alternate entries FP64 FMA / double-float
                                (see ENS_F64_SPLIT); takes precedence over ENS_CG_DF64 */
    ENS_CG_GUESS_FALLBACK = 32, /* zero-guess fallback for a supplied start x0 (a learned
                                guess, not in the paper): a member whose ||b - A x0||
                                is not below ||b|| (or is not finite) restarts from
                                x = 0, so its iterates are exactly those of a zero-guess
                                solve; counted in ens_cg_stats.guess_fallbacks */
    ENS_CG_X0_ZERO = 64      /* the caller states that x holds zeros on entry: r0 = b is
                                taken without the initial SpMV (the result is the same,
                                bitwise, as computing b - A*0) */
};

/* Launch mapping of the CG's SpMV (a tuning knob; not in the paper): rows per
 * CTA of the SpMV kernel.  ENS_CG_K1_CHUNKS(k) in the flags of ens_cg /
 * ens_cg_df asks for 2^k chunks of 32 rows per CTA (k = 0..3), each chunk on
 * 32 * max(s/2, 2) threads; a CTA holds at most 1024 threads, so k <= 1 at
 * s = 32 and k <= 2 at s = 16 (ENS_ERR_ARG beyond).  Without the field the
 * library's default for s is used.  Every sum is ordered by row index, so
 * the mapping never changes a result bit.  Bits 16..18 of flags. */
#define ENS_CG_K1_CHUNKS_SHIFT 16
#define ENS_CG_K1_CHUNKS(k) (((k) + 1) << ENS_CG_K1_CHUNKS_SHIFT)
/* The batched SpMV's mapping (ens_cg_batched): CTAs of 512 threads (default)
 * or, with this flag, 1024, i.e. 512 / (32 max(s/2, 2)) chunks of 32 rows of
 * an item per CTA, or twice that; no effect on results either. */
#define ENS_CG_BATCH_K1_WIDE (1 << 19)
/* ens_cg / ens_cg_df: the SpMV's CTAs (one chunk each) write only their
 * chunks' partial p.q, and a second, small kernel reduces the upper levels of
 * the same tree, in the same order, so no SpMV CTA waits on the tree's fence
 * and arrival counter; pays off at small s, where a CTA's own work is short.
 * Results bitwise those of the default. */
#define ENS_CG_K1_DEFER (1 << 20)

/* Unpreconditioned CG (Hestenes-Stiefel) on each member of the ensemble
 * system, with per-member dots (default) or the paper's coupled form.
 * Member e stops when ||r_e|| <= tol*||b_e|| (recursive residual) and is
 * then frozen; the call returns when every member has stopped.
 *   values: A_c (double, commuted), b: rhs, x: in = x0, out = solution.
 *   work: ens_cg_workspace_size bytes of device scratch (16-byte aligned).
 *   iters_host[s], relres_host[s] (true ||b-Ax||/||b||), status_host[s]
 *   (ENS_OK / ENS_ERR_NOT_CONVERGED / ENS_ERR_BREAKDOWN) may be NULL.
 *   check_every: iterations between host polls of the convergence word (>=1).
 * Synchronises `stream`.  Returns ENS_OK if every member converged, else the
 * first member's failure status. */
int ens_cg_workspace_size(int32_t num_rows, int s, size_t *bytes);
int ens_cg(const ens_graph *graph, int s, const double *values, const double *b, double *x,
           double tol, int max_iter, int flags, int check_every, void *work, size_t work_bytes,
           int32_t *iters_host, double *relres_host, int32_t *status_host,
           ens_cg_stats *stats_host, void *stream);

/* ens_cg with the double-float CG SpMV reading pre-split values: values_df is
 * the ens_convert_values(..., ENS_F64_DF, ...) copy of `values` (float2[nnz*s]),
 * read by every iteration's SpMV instead of splitting each FP64 value again;
 * `values` (FP64) is still read by the initial and final residuals and by
 * rows whose double-float sum is not finite.  Every result is bitwise that of
 * ens_cg with ENS_CG_DF64 (the same operations in the same order).  flags:
 * ENS_CG_COUPLED, ENS_CG_GRAPH, ENS_CG_TIME_SPMV, ENS_CG_GUESS_FALLBACK
 * (ENS_CG_DF64 / ENS_CG_SPLIT64 are implied / ignored).  Same workspace. */
int ens_cg_df(const ens_graph *graph, int s, const double *values, const void *values_df, const double *b,
              double *x, double tol, int max_iter, int flags, int check_every, void *work, size_t work_bytes,
              int32_t *iters_host, double *relres_host, int32_t *status_host, ens_cg_stats *stats_host,
              void *stream);

/* ------------------------------------- preconditioned ensemble CG */
/* Not in the paper as a standalone solver: its CG is preconditioned by
 * multigrid whose smoothers are order-2 Chebyshev polynomials (Sect. 3.5).
 * Per member, PCG (Hestenes-Stiefel with z = M^-1 r, rho = r.z, stop when
 * ||r|| <= tol ||b||) with
 *   ENS_PC_JACOBI     z = D^-1 r (D the diagonal of A);
 *   ENS_PC_CHEBYSHEV  z = p(D^-1 A) D^-1 r: `degree` steps (1..8) of Chebyshev
 *                     iteration for A z = r from z = 0 on [lam/ratio, lam]
 *                     (Saad, Iterative Methods, Sect. 12.3), lam = boost x an
 *                     estimate of the largest eigenvalue of D^-1 A: power_iters
 *                     steps v <- D^-1 A v / ||D^-1 A v|| from power_start (device,
 *                     commuted layout n*s) and the quotient v.Av / v.Dv; with
 *                     ENS_PC_LANCZOS in flags the Lanczos estimate from
 *                     power_iters (1..32) steps instead (see ens_mg_pcg).
 * FP64 values and arithmetic (the ENS_F64 SpMV).  flags: ENS_CG_GRAPH,
 * ENS_CG_X0_ZERO, ENS_PC_LANCZOS.  lam_host[s] (may be NULL) receives the estimates (0 for
 * Jacobi).  Other arguments and outputs as ens_cg; work:
 * ens_pcg_workspace_size bytes.  Synchronises `stream`. */
enum { ENS_PC_JACOBI = 1, ENS_PC_CHEBYSHEV = 2 };
/* flag of ens_pcg and ens_mg_pcg: the smoothers' eigenvalue bound by Lanczos
 * (not in the paper: its smoothers take MueLu's power iteration) */
#define ENS_PC_LANCZOS (1 << 24)
int ens_pcg_workspace_size(int32_t num_rows, int s, size_t *bytes);
int ens_pcg(const ens_graph *graph, int s, const double *values, const double *b, double *x, double tol,
            int max_iter, int precond, int degree, double ratio, double boost, int power_iters,
            const double *power_start, int flags, int check_every, void *work, size_t work_bytes,
            int32_t *iters_host, double *relres_host, int32_t *status_host, double *lam_host,
            ens_cg_stats *stats_host, void *stream);

/* ------------------------------- multigrid-preconditioned ensemble CG */
/* The paper's solver (Sect. 3.5, Algorithm 1), geometric form: CG with
 * z = V_0(r), a V-cycle over nested meshes N, N/2, ..., N_L (N_L <= 4).
 * Level l: the ensemble's matrix assembled by the caller on the
 * (N/2^l)^3-cell mesh from the same KL variables (rediscretisation).
 *   P_l  trilinear interpolation from the interior nodes of level l+1 to the
 *        interior nodes of level l (fine 2i <- coarse i, weight 1; 2i+1 <- i,
 *        i+1, weight 1/2 each, per axis; boundary nodes left out), R_l = P_l^T;
 *   S_l  Chebyshev smoother x += p(D^-1 A) D^-1 (b - A x): `degree` steps on
 *        [lam/ratio, lam], lam = boost x the power estimate of ens_pcg
 *        (power_iters steps from the level's power_start), or with
 *        ENS_PC_LANCZOS in flags the Lanczos estimate from power_iters
 *        (1..32) steps from the same start: the largest eigenvalue of the
 *        tridiagonal T_k of Lanczos in the D inner product (Lanczos 1950;
 *        Saad, Iterative Methods, Sect. 6.6), never below the power estimate
 *        from the same start with as many matrix products (5 Lanczos steps
 *        on the 64^3 Q1 levels: about 0.925 of the largest eigenvalue, 10
 *        power steps 0.91); not in the paper, whose smoothers take MueLu's
 *        power iteration;
 *   V_L  x = A_L^-1 b (inverse of the coarsest matrix, Gauss-Jordan once per
 *        call; at most 125 rows);
 *   V_l  x = S(b, 0); r = b - A x; x += P V_{l+1}(R r); x = S(b, x).
 * CG as ens_cg with rho = r.z; FP64 throughout.  flags: ENS_CG_GRAPH,
 * ENS_CG_X0_ZERO, ENS_PC_LANCZOS.  b, x: level-0 vectors (commuted layout).  Returns
 * ENS_ERR_BREAKDOWN if the coarsest matrix is not positive definite.
 * Synchronises `stream`. */
typedef struct ens_mg_level {
    ens_graph graph;            /* the level's mesh graph (ens_graph_build of N) */
    int32_t N;                  /* cells per side: levels[l].N = levels[0].N / 2^l */
    int32_t reserved;
    const double *values;       /* the ensemble's matrix on this level, commuted layout */
    const double *power_start;  /* n*s start vector of the level's eigenvalue estimate */
    const float *values_df;     /* optional: values pre-split into float pairs (ens_assemble_df or
                                   ens_convert_values ENS_F64_DF); the level's SpMVs then run in
                                   double-float (FP64-class, as ens_cg_df); NULL: FP64 SpMVs */
    const float *values_f32;    /* optional, on every level or none: values rounded to FP32
                                   (ens_convert_values ENS_F32); the V-cycle then runs in FP32
                                   (values, vectors, arithmetic) as a mixed-precision
                                   preconditioner of the FP64 CG or (flexible) GMRES; the
                                   set-up stays FP64 */
} ens_mg_level;
int ens_mg_workspace_size(int nlevels, const ens_mg_level *levels, int s, size_t *bytes);
int ens_mg_pcg(int nlevels, const ens_mg_level *levels, int s, const double *b, double *x, double tol,
               int max_iter, int degree, double ratio, double boost, int power_iters, int flags,
               int check_every, void *work, size_t work_bytes, int32_t *iters_host, double *relres_host,
               int32_t *status_host, ens_cg_stats *stats_host, void *stream);

/* ---------------------------------------------------- A8 batched CG */
/* One ensemble of a batch: its graph (by value), size s, values, rhs, x (in:
 * x0, out: solution), optional host outputs iters/relres/status [s], and
 * optional pre-split values (as for ens_cg_df; either every item of a batch
 * gives them, and the batch runs the pre-split double-float SpMV, or none). */
typedef struct ens_batch_item {
    ens_graph graph;
    int32_t s;
    int32_t reserved;
    const double *values;
    const double *b;
    double *x;
    int32_t *iters_host;
    double *relres_host;
    int32_t *status_host;
    const float *values_df;
} ens_batch_item;

/* Solves a batch of ensembles -- any mix of meshes and ensemble sizes -- with
 * one launch per CG phase for the whole batch (a per-CTA work list maps CTAs
 * to (ensemble, row tiles)); each ensemble follows exactly the arithmetic of
 * ens_cg, or of ens_cg_df when the items carry values_df (ENS_ERR_ARG if only
 * some do, or together with ENS_CG_DF64 / ENS_CG_SPLIT64) (same flags:
 * ENS_CG_COUPLED, ENS_CG_DF64, ENS_CG_SPLIT64,
 * ENS_CG_GRAPH replays check_every iterations of the batch as one CUDA
 * graph, ENS_CG_TIME_SPMV).  Not in the paper (Sect. 5 leaves the grouping of
 * samples to future work); it amortises launch latency over small meshes.
 * work: ens_cg_batched_workspace_size bytes.  Synchronises `stream`. */
int ens_cg_batched_workspace_size(int n_items, const ens_batch_item *items, size_t *bytes);
int ens_cg_batched(int n_items, const ens_batch_item *items, double tol, int max_iter, int flags,
                   int check_every, void *work, size_t work_bytes, ens_cg_stats *stats_host,
                   void *stream);

/* ------------------------------------------------- A7 mixed precision */
/* Low-precision copy of ensemble values for the inner solver of ens_cg_mixed.
 *   dtype = ENS_F32 or ENS_BF16; values_lo: float[nnz*s] or bfloat16[nnz*s]
 *   (commuted layout), each value rounded to nearest (BF16 via FP32).
 *   diag_lo (float[num_rows*s], may be NULL): when given, the diagonal entry of
 *   values_lo is stored as 0 and diag_lo[I*s+e] is set so that every row of
 *   the low-precision matrix sums to the FP64 row sum:
 *       diag_lo = fl32( sum_j values[j] - sum_{j != diag} values_lo[j] ).
 *   This keeps the zero row sums of the diffusion stencil, which BF16 rounding
 *   would otherwise break at the size of the smallest eigenvalue. */
int ens_convert_values(const ens_graph *graph, int s, const double *values, int dtype,
                       void *values_lo, float *diag_lo, void *stream);
/* dtype = ENS_F64_DF (for ens_cg_df): values_lo is float2[nnz*s] (commuted
 * layout), each value split by truncation into hi + lo floats (the split of
 * the ENS_F64_DF SpMV, 47 significant bits); a value whose magnitude is
 * outside [2^-103, 2^128) or that is not finite is stored as (NaN, 0).
 * diag_lo must be NULL. */

/* Mixed-precision ensemble CG (iterative refinement; not in the paper, see
 * the A7 row of the design notes): per member,
 *     r = b - A x (FP64 values and arithmetic; the true residual),
 *     stop when ||r|| <= tol*||b|| (status ENS_OK) or after max_outer steps,
 *     solve A_lo d = r/||r|| by FP32 CG (FP32 vectors and accumulation, values
 *     values_lo of dtype_lo with optional diag_lo) to ||r_in|| <= inner_tol
 *     or max_inner iterations,
 *     x += ||r|| d (FP64).
 * Members with b = 0 return x = 0.  outer_iters_host[s] = refinement steps,
 * inner_iters_host[s] = total inner iterations, relres_host[s] = the final
 * true ||b - A x||/||b||.  flags: ENS_CG_TIME_SPMV records CUDA events around
 * the inner SpMV launches (stats_host->spmv_ms / spmv_launches).
 * work: ens_cg_mixed_workspace_size bytes.
 * Synchronises `stream`.  Returns ENS_OK when every member converged. */
int ens_cg_mixed_workspace_size(int32_t num_rows, int s, size_t *bytes);
int ens_cg_mixed(const ens_graph *graph, int s, const double *values, const void *values_lo,
                 int dtype_lo, const float *diag_lo, const double *b, double *x, double tol,
                 int max_outer, double inner_tol, int max_inner, int check_every, int flags, void *work,
                 size_t work_bytes, int32_t *outer_iters_host, int32_t *inner_iters_host,
                 double *relres_host, int32_t *status_host, ens_cg_stats *stats_host,
                 void *stream);

/* ----------------------------------------- A9 learned initial guess */
/* Not in the paper (its CG starts from x = 0, Sect. 4).  A reduced basis of
 * solutions (POD) and a small MLP map the KL variables xi of a sample to a
 * start x0 for ens_cg (with ENS_CG_GUESS_FALLBACK the zero guess stays the
 * fallback, and CG always runs to the same ||r|| <= tol ||b||).
 *
 * Snapshots: X is row-major n x m with leading dimension ldx >= m (column j =
 * solution of sample j).  ens_snapshots_put copies an ensemble solution x
 * (n x s, commuted layout, Eq. 3) into columns col0 .. col0+s-1 of X
 * (device pointers; ENS_ERR_ARG if ldx < col0 + s). */
int ens_snapshots_put(int64_t n, int32_t s, const double *x, double *X, int64_t ldx, int64_t col0,
                      void *stream);

/* POD basis: centres X in place (mean[n] = row means, X -= mean), then the
 * k leading left singular vectors of the centred X by a randomized range
 * finder with power_iters stabilised power iterations (Halko, Martinsson and
 * Tropp, SIAM Review 53 (2011), Algorithms 4.1 and 4.4) and a Rayleigh-Ritz
 * step: Y = X Omega, Q = orth(Y); q times {Z = orth(X^T Q), Q = orth(X Z)};
 * eigen-decomposition of (X^T Q)^T (X^T Q) by cyclic Jacobi; Phi = Q W_k.
 * orth is shifted CholeskyQR3 (Fukaya et al., SIAM J. Sci. Comput. 42 (2020)).
 *   Omega: m x l row-major test matrix (device; drawn by the caller),
 *          1 <= k <= l <= min(80, m - 1), l <= n, 0 <= power_iters <= 8;
 *   Phi: n x k row-major (device), column i scaled to unit 2-norm and signed
 *        so that its largest-magnitude entry (first on ties) is positive;
 *   sigma: k singular-value estimates (device), descending.
 * All arithmetic FP64.  Returns ENS_ERR_BREAKDOWN if a Gram matrix is not
 * positive definite (centred snapshots of numerical rank below l).
 * Synchronises `stream`. */
int ens_pod_workspace_size(int64_t n, int32_t m, int32_t l, size_t *bytes);
int ens_pod(int64_t n, int32_t m, double *X, int64_t ldx, int32_t k, int32_t l, const double *Omega,
            int32_t power_iters, double *mean, double *Phi, double *sigma, void *work, size_t work_bytes,
            void *stream);

/* Training targets: coefficients C = X^T Phi (m x k) of the centred
 * snapshots, coef_mean[k] and coef_scale[k] = per-column mean and population
 * standard deviation (1 where it is 0), T = (C - coef_mean) / coef_scale as
 * float[m x k] row-major.  FP64 except the final rounding of T. */
int ens_pod_targets_workspace_size(int64_t n, int32_t m, int32_t k, size_t *bytes);
int ens_pod_targets(int64_t n, int32_t m, const double *X, int64_t ldx, int32_t k, const double *Phi,
                    double *coef_mean, double *coef_scale, float *T, void *work, size_t work_bytes,
                    void *stream);

/* dst[i] = (float)src[i] (round to nearest), e.g. the FP32 copy of Phi. */
int ens_to_f32(int64_t count, const double *src, float *dst, void *stream);

/* MLP d0 -> d1 -> d2 -> d3 (dims[4], host array, each 1..4096): three affine
 * layers, the exact GELU g(z) = z (1 + erf(z / sqrt 2)) / 2 after the first
 * two, FP32.  Parameters: one float vector in the order W1 [d1 x d0], b1
 * [d1], W2 [d2 x d1], b2 [d2], W3 [d3 x d2], b3 [d3] (row-major, W_l maps
 * layer l-1 to layer l: z = W a + b).  Inputs xin [batch x d0], outputs and
 * targets [batch x d3], row-major float (device).
 * ens_mlp_init: He-uniform start from uniform draws u[count] in [-1, 1]:
 * W_l = u sqrt(6 / fan_in), b_l = 0. */
int ens_mlp_param_count(const int32_t *dims, int64_t *count);
int ens_mlp_init(const int32_t *dims, const float *u, float *params, void *stream);
int ens_mlp_workspace_size(const int32_t *dims, int32_t batch, size_t *bytes);
int ens_mlp_forward(const int32_t *dims, const float *params, int32_t batch, const float *xin, float *y,
                    void *work, size_t work_bytes, void *stream);
/* Gradient of the mean squared error L = sum (y - target)^2 / (batch d3)
 * with respect to the parameters (grad: float[count], device; loss: device
 * float or NULL).  FP32 with sums in a fixed order (deterministic). */
int ens_mlp_grad(const int32_t *dims, const float *params, int32_t batch, const float *xin, const float *target,
                 float *grad, float *loss, void *work, size_t work_bytes, void *stream);
/* One Adam step (Kingma and Ba, ICLR 2015) on P parameters: with t = step[0],
 * m = b1 m + (1 - b1) g, v = b2 v + (1 - b2) g^2,
 * w -= lr_t (m / (1 - b1^(t+1))) / (sqrt(v / (1 - b2^(t+1))) + eps),
 * lr_t = lr0 (1 + cos(pi t / total_steps)) / 2; then step[0] = t + 1.
 * step: device int64[2]; step[1] is scratch that must be 0 before the first
 * call (every call leaves it 0). */
int ens_mlp_adam(int64_t P, float *params, const float *grad, float *m, float *v, int64_t *step,
                 int64_t total_steps, float lr0, float beta1, float beta2, float eps, void *stream);
/* `epochs` passes over n_samples (a positive multiple of batch) in fixed
 * consecutive mini-batches, each an ens_mlp_grad + ens_mlp_adam step on
 * params, m, v, step (as above; step[0] must be a multiple of
 * n_samples / batch).  epoch_loss (device float[epochs] or NULL) receives
 * each epoch's mean batch loss.  use_graph != 0 captures one epoch as a CUDA
 * graph and replays it.  work: ens_mlp_workspace_size(dims, batch). */
int ens_mlp_train(const int32_t *dims, float *params, float *m, float *v, int64_t *step, int64_t n_samples,
                  const float *xin, const float *target, int32_t batch, int32_t epochs, int64_t total_steps,
                  float lr0, float beta1, float beta2, float eps, float *epoch_loss, int32_t use_graph,
                  void *work, size_t work_bytes, void *stream);

/* Learned start of one ensemble: for each member e (s <= 32),
 *   chat_e = MLP(xi_e) with xi_e[k] = xi[k*s + e] (the ens_assemble input,
 *            k < dims[0], rounded to float),
 *   x0[i*s + e] = mean[i] + sum_k Phi32[i][k] (coef_mean[k] + coef_scale[k] chat_e[k]),
 * the sum over k = dims[3] <= 256 in FP32, mean added in FP64.  Phi32: float
 * n x dims[3] row-major.  Synchronises nothing. */
int ens_guess_workspace_size(const int32_t *dims, int32_t s, size_t *bytes);
int ens_guess(const int32_t *dims, const float *params, int64_t n, int32_t s, const double *xi,
              const double *mean, const float *Phi32, const double *coef_mean, const double *coef_scale,
              double *x0, void *work, size_t work_bytes, void *stream);

/* ---------------------------------- NEXT-4 nonlinear advection-diffusion
 * The model problem of Sect. 4 (Eq. 7) with alpha, beta != 0, discretised on
 * the Q1 hex mesh of the linear problem (source 1, u = 0 on the boundary):
 *   F_i(u) = (A u)_i + alpha int phi_i v.grad(u_h) + beta int phi_i u_h^2 - b_i
 *   J(u)   = dF/du = A + alpha C + 2 beta M(u),
 *            C_ij = int phi_i v.grad(phi_j),  M(u)_ij = int phi_i phi_j u_h,
 * with A, b the ensemble's diffusion matrix and load (ens_assemble); boundary
 * rows of F and J are those of A (identity), boundary columns of J are 0.
 * v is a constant velocity; all integrals are exact (2x2x2 Gauss would be).
 * Newton's method (Eq. 10) solves J(u_k) du = -F(u_k), u_{k+1} = u_k + du,
 * per member, with restarted GMRES (one of the Belos solvers of Sect. 3.4;
 * flexible right-preconditioned form, classical Gram-Schmidt applied twice,
 * Givens rotations) for the non-symmetric J.
 * The paper's experiments take alpha = beta = 0; the velocity, the source and
 * the GMRES preconditioner (the V-cycle of the diffusion operator A, fixed for
 * all Newton steps) are this library's readings. */
enum {
    ENS_NL_PRECOND_NONE = 0,  /* plain GMRES */
    ENS_NL_PRECOND_MG = 1     /* right preconditioner: the V-cycle of ens_mg_pcg on levels[] */
};

/* C on the graph of the N^3-cell mesh for the velocity v (host double[3]):
 * C[nnz] FP64, one matrix for every member; boundary rows and columns 0.
 * Asynchronous. */
int ens_nl_advection(const ens_graph *g, int32_t N, const double *v, double *C, void *stream);

/* J[nnz*s] = J(u) and F[n*s] = F(u) in one pass, commuted layout.  A: the
 * ensemble's diffusion values; C: ens_nl_advection; u must vanish on the
 * boundary.  work: ens_nl_jacobian_workspace_size bytes of device memory.
 * ENS_ERR_ARG if an interior row of g is not its 27-node window (sorted).
 * Synchronises `stream`. */
int ens_nl_jacobian_workspace_size(size_t *bytes);
int ens_nl_jacobian(const ens_graph *g, int32_t N, int s, const double *A, const double *C, double alpha, double beta,
                    const double *b, const double *u, double *J, double *F, void *work, void *stream);

/* GMRES(restart) for values * x = b from x = 0, per member, to
 * ||b - values x|| <= tol ||b|| (the Givens residual estimate; relres_host
 * gets the true relative residual).  values: ensemble matrix on the graph of
 * levels[0]; precond ENS_NL_PRECOND_MG takes the V-cycle of ens_mg_pcg with
 * levels[] (the diffusion hierarchy), degree, ratio, boost and power_iters;
 * ENS_NL_PRECOND_NONE needs levels[0] only (its graph and N).
 * 1 <= restart <= 64.  The host polls every check_every steps.
 * work: ens_gmres_workspace_size bytes.  Synchronises `stream`. */
int ens_gmres_workspace_size(int nlevels, const ens_mg_level *levels, int s, int restart, int precond,
                             size_t *bytes);
int ens_gmres(int nlevels, const ens_mg_level *levels, int s, const double *values, const double *b, double *x,
              double tol, int restart, int max_iter, int precond, int degree, double ratio, double boost,
              int power_iters, int check_every, void *work, size_t work_bytes, int32_t *iters_host,
              double *relres_host, int32_t *status_host, ens_cg_stats *stats_host, void *stream);

typedef struct ens_newton_params {
    double alpha, beta;     /* advection and reaction coefficients (Eq. 7) */
    double tol;             /* Newton: stop when ||F(u)|| <= tol ||F(u_0)|| */
    double lin_tol;         /* GMRES: ||J du + F|| <= lin_tol ||F(u_k)|| */
    int32_t max_newton;     /* Newton steps at most */
    int32_t restart;        /* GMRES restart length, 1..64 */
    int32_t max_lin;        /* GMRES steps per Newton step at most */
    int32_t precond;        /* ENS_NL_PRECOND_NONE / _MG */
    int32_t degree;         /* V-cycle: Chebyshev smoother degree */
    int32_t power_iters;    /* V-cycle: power steps of the eigenvalue estimate (Lanczos steps with
                               ENS_PC_LANCZOS) */
    int32_t check_every;    /* GMRES steps between host polls */
    int32_t flags;          /* 0, or ENS_PC_LANCZOS: the V-cycle's eigenvalue bounds by Lanczos */
    double ratio, boost;    /* V-cycle: smoother interval [lam/ratio, lam], lam = boost x estimate */
} ens_newton_params;

/* Newton's method for F(u) = 0 per member from the caller's u (in: u_0, 0 on
 * the boundary; out: the solution).  levels[0].values = A (the diffusion
 * values, also the finest level of the preconditioner's hierarchy); C from
 * ens_nl_advection; b the load.  Per member: newton_iters (steps taken),
 * lin_iters (GMRES steps summed), relres = ||F(u)|| / ||F(u_0)||, status
 * (ENS_ERR_NOT_CONVERGED after max_newton steps).  With ENS_NL_PRECOND_MG
 * and levels[0].values_df the V-cycle's finest level and the GMRES SpMV run
 * in the pre-split double-float form (the Jacobian is then also written as
 * float pairs).  work: ens_newton_workspace_size bytes.  Synchronises
 * `stream`. */
int ens_newton_workspace_size(int nlevels, const ens_mg_level *levels, int s, const ens_newton_params *p,
                              size_t *bytes);
int ens_newton(int nlevels, const ens_mg_level *levels, int s, const double *C, const double *b, double *u,
               const ens_newton_params *p, void *work, size_t work_bytes, int32_t *newton_iters_host,
               int32_t *lin_iters_host, double *relres_host, int32_t *status_host, ens_cg_stats *stats_host,
               void *stream);

#ifdef __cplusplus
}
#endif
#endif /* ENS_H */
