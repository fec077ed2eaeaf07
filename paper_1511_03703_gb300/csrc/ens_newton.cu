// ens_newton.cu -- the nonlinear advection-diffusion problem of the paper's
// model (Sect. 4, Eq. 7 with alpha, beta != 0) solved by Newton's method
// (Eq. 10) with restarted GMRES for the non-symmetric Jacobian, right-
// preconditioned by the multigrid V-cycle of the diffusion operator
// (ens_mg_solver.cuh) or by nothing.
//
// On the Q1 hex mesh of the linear problem (u = 0 on the boundary):
//   F_i(u) = (A u)_i + alpha int phi_i v.grad(u_h) + beta int phi_i u_h^2 - b_i
//   J(u)   = A + alpha C + 2 beta M(u),  C_ij = int phi_i v.grad(phi_j),
//            M(u)_ij = int phi_i phi_j u_h
// boundary rows of J and F those of A (identity), boundary columns of J 0.
// v is a constant velocity, so C is one matrix per mesh.  For a constant v
// and the uniform mesh, both C and M(u) are sums of tensor products of 1-D
// integrals of hat functions (all exact: the integrands are of degree <= 3 per
// coordinate):
//   C_ij  = h^2 sum_d v_d g(a_d) prod_{d' != d} m(a_d'),   a = offset of j from i
//   M_ij  = h^3 sum_c prod_d w(a_d, c_d) u_{i+c},          c in {-1,0,1}^3
// with m(0) = 2/3, m(+-1) = 1/6; g(0) = 0, g(+-1) = +-1/2; and w(a, c) the
// integral of hat_0 hat_a hat_c over the 1-D cells holding all three nodes
// (w(0,0) = 1/2; 1/12 for the pairs (0,+-1), (+-1,0), (+-1,+-1); 0 for (+-1,-+1)).
// M is formed per row by sum factorisation over the 27-node window of the row,
// in float-pair (double-float) arithmetic on the FP32 pipe.
//
// GMRES (Saad, Sect. 6.5 and 9.3.2) per member with classical Gram-Schmidt
// applied twice (CGS2), in the flexible right-preconditioned form (Saad,
// Sect. 9.4.1: the preconditioned vectors z_j are kept, x += Z y, which equals
// x += M^-1 V y for a fixed preconditioner and also admits the FP32 V-cycle):
// every step is four row-parallel kernels after the preconditioner (w = J z
// with the dots v_i.w; two orthogonalisation passes, the second with ||w||
// and the Givens update in its last CTA; the normalisation).  All reductions use the chunk trees of the CG, so every
// member's result is independent of the ensemble size.  Vectors, dots,
// Gram-Schmidt and Givens arithmetic are FP64; the GMRES SpMV is FP64 or, with
// a pre-split level 0, the pre-split double-float form on a split copy of J.
#include "ens_mg_solver.cuh"

namespace ens {

constexpr int kGmMaxRestart = 64;

// ------------------------------------------------------------ device state
struct NlState {            // Newton (and the right-hand-side norm of ens_gmres)
    double f0[32], fn[32];  // ||F(u_0)||, ||F(u_k)||
    double inv_fn[32];      // 1 / ||F(u_k)|| (0 when ||F|| = 0)
    int nact[32];           // member takes a Newton step (or a linear solve) now
    int newton_iters[32], lin_iters[32], status[32];
    int active_count;
    int graph_bad;          // an interior row whose entries are not its 27-node window
};

struct GmState {
    double H[kGmMaxRestart + 1][kGmMaxRestart][32];  // Hessenberg matrix after the rotations
    double hA[kGmMaxRestart + 1][32], hB[kGmMaxRestart + 1][32];  // the two Gram-Schmidt passes
    double cs[kGmMaxRestart][32], sn[kGmMaxRestart][32];
    double g[kGmMaxRestart + 1][32];
    double y[kGmMaxRestart][32];
    double beta0[32], scale[32];
    int active[32], conv[32], k[32], iters[32];
    int active_count;   // members iterating in the current cycle
    int pending_count;  // members not converged and under max_iter (need a restart)
};

// ------------------------------------------------------------ mesh helpers
__device__ __forceinline__ void node_ijk(int64_t I, int n1, int &i, int &j, int &k) {
    i = (int)(I % n1);
    j = (int)((I / n1) % n1);
    k = (int)(I / ((int64_t)n1 * n1));
}
__device__ __forceinline__ bool on_boundary(int i, int j, int k, int N) {
    return i == 0 || j == 0 || k == 0 || i == N || j == N || k == N;
}

// C on the mesh graph (thread per entry), boundary rows and columns 0
__global__ void nl_advection_kernel(int32_t n, int32_t N, const int32_t *__restrict__ row_map,
                                    const int32_t *__restrict__ col, double v0, double v1, double v2,
                                    double *__restrict__ C) {
    const int n1 = N + 1;
    const double h = 1.0 / N;
    for (int64_t I = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; I < n; I += (int64_t)gridDim.x * blockDim.x) {
        int i, j, k;
        node_ijk(I, n1, i, j, k);
        const bool bi = on_boundary(i, j, k, N);
        for (int32_t p = row_map[I]; p < row_map[I + 1]; ++p) {
            int ci, cj, ck;
            node_ijk(col[p], n1, ci, cj, ck);
            double c = 0.0;
            if (!bi && !on_boundary(ci, cj, ck, N)) {
                const int a[3] = {ci - i, cj - j, ck - k};
                double m[3], g[3];
                for (int d = 0; d < 3; ++d) {
                    m[d] = (a[d] == 0) ? 2.0 / 3.0 : 1.0 / 6.0;
                    g[d] = (a[d] == 0) ? 0.0 : 0.5 * a[d];
                }
                c = h * h * (v0 * g[0] * m[1] * m[2] + v1 * m[0] * g[1] * m[2] + v2 * m[0] * m[1] * g[2]);
            }
            C[p] = c;
        }
    }
}

// ---- the sum factorisation of M(u) in double-float arithmetic (float pairs
// on the FP32 pipe: GB300 runs FP64 at 1/64 of its FP32 rate).  M is a small
// part of J (beta h^3 u against the diffusion entries), so its 2^-44-relative
// float-pair rounding stays far below FP64 rounding of J and F.
struct Dfp {
    float h, l;  // unevaluated sum h + l
};
__device__ __forceinline__ Dfp dfp_of(double v) {  // truncating split (|v| < 2^-103 gives 0)
    Dfp r;
    df_split_trunc(v, r.h, r.l);
    return r;
}
__device__ __forceinline__ Dfp dfp_norm(float s, float e) {  // fast two-sum renormalisation
    const float h = __fadd_rn(s, e);
    return Dfp{h, __fsub_rn(e, __fsub_rn(h, s))};
}
__device__ __forceinline__ Dfp dfp_add(Dfp a, Dfp b) {
    float s, e;
    two_sum(a.h, b.h, s, e);
    return dfp_norm(s, __fadd_rn(e, __fadd_rn(a.l, b.l)));
}
// a * (ch + cl)
__device__ __forceinline__ Dfp dfp_mulc(Dfp a, float ch, float cl) {
    const float p = __fmul_rn(a.h, ch);
    float e = __fmaf_rn(a.h, ch, -p);
    e = __fmaf_rn(a.h, cl, e);
    e = __fmaf_rn(a.l, ch, e);
    return dfp_norm(p, e);
}
__device__ __forceinline__ double dfp_to_double(Dfp a) { return f2d_exact(a.h) + f2d_exact(a.l); }

// a value as the pre-split SpMV reads it: the truncating split, or (NaN, 0)
// outside the split range (the SpMV then recomputes that row in FP64)
__device__ __forceinline__ float2 nl_split_value(double v) {
    float hi, lo;
    return df_split_trunc(v, hi, lo) ? make_float2(hi, lo) : make_float2(__int_as_float(0x7fc00000), 0.0f);
}

// 1/12 as a float pair
constexpr float kK12H = (float)(1.0 / 12.0);
constexpr float kK12L = (float)(1.0 / 12.0 - (double)(float)(1.0 / 12.0));

// one 1-D pass over the 27-node window T[x + 3y + 9z] along the axis of the
// given stride: T(a) <- sum_c w(a, c) T(c)
template <int STRIDE>
__device__ __forceinline__ void window_pass(Dfp (&T)[27]) {
#pragma unroll
    for (int b = 0; b < 27; ++b) {
        if ((b / STRIDE) % 3 != 0) continue;  // b: the window index with this axis' coordinate -1
        const Dfp um = T[b], u0 = T[b + STRIDE], up = T[b + 2 * STRIDE];
        const Dfp half0{0.5f * u0.h, 0.5f * u0.l};  // exact
        T[b] = dfp_mulc(dfp_add(um, u0), kK12H, kK12L);
        T[b + STRIDE] = dfp_add(half0, dfp_mulc(dfp_add(um, up), kK12H, kK12L));
        T[b + 2 * STRIDE] = dfp_mulc(dfp_add(u0, up), kK12H, kK12L);
    }
}

// J and F in one pass (thread per row and member):
//   interior row: J_p = A_p + alpha C_p + 2 beta M_p, N_p = A_p + alpha C_p + beta M_p,
//                 F_i = sum_p N_p u_col(p) - b_i  (M_p = 0 for boundary columns)
//   boundary row: J_p = A_p, F_i = sum_p A_p u_col(p) - b_i
// m2h + m2l: 2 beta h^3 as a float pair (M's integrals carry the factor h^3)
template <int S>
__global__ void __launch_bounds__(256) nl_jacobian_kernel(int32_t n, int32_t N, const int32_t *__restrict__ row_map,
                                                          const int32_t *__restrict__ col,
                                                          const double *__restrict__ A, const double *__restrict__ C,
                                                          double alpha, float m2h, float m2l,
                                                          const double *__restrict__ b,
                                                          const double *__restrict__ u, double *__restrict__ J,
                                                          float2 *__restrict__ Js, double *__restrict__ F,
                                                          NlState *ns) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= (int64_t)n * S) return;
    const int e = (int)(t % S);
    const int64_t I = t / S;
    const int n1 = N + 1;
    int i, j, k;
    node_ijk(I, n1, i, j, k);
    const int32_t p0 = row_map[I], p1 = row_map[I + 1];
    double f = -b[t];
    if (on_boundary(i, j, k, N)) {
        for (int32_t p = p0; p < p1; ++p) {
            const double a = A[(int64_t)p * S + e];
            J[(int64_t)p * S + e] = a;
            if (Js) Js[(int64_t)p * S + e] = nl_split_value(a);
            f = fma(a, u[(int64_t)col[p] * S + e], f);
        }
        F[t] = f;
        return;
    }
    if (p1 - p0 != 27) {
        if (e == 0) atomicExch(&ns->graph_bad, 1);
        return;
    }
    Dfp T[27];
#pragma unroll
    for (int w = 0; w < 27; ++w) {
        const int64_t Jn = I + (w % 3 - 1) + (int64_t)n1 * ((w / 3) % 3 - 1) + (int64_t)n1 * n1 * (w / 9 - 1);
        T[w] = dfp_of(u[Jn * S + e]);
    }
    window_pass<1>(T);
    window_pass<3>(T);
    window_pass<9>(T);
    int bad = 0;
#pragma unroll
    for (int w = 0; w < 27; ++w) {
        const int32_t p = p0 + w;
        const int32_t cj = col[p];
        const int64_t Jn = I + (w % 3 - 1) + (int64_t)n1 * ((w / 3) % 3 - 1) + (int64_t)n1 * n1 * (w / 9 - 1);
        bad |= (cj != Jn);
        // 2 beta M_p (0 for a boundary column)
        const double m2 = on_boundary(i + w % 3 - 1, j + (w / 3) % 3 - 1, k + w / 9 - 1, N)
                              ? 0.0
                              : dfp_to_double(dfp_mulc(T[w], m2h, m2l));
        const double ac = fma(alpha, C[p], A[(int64_t)p * S + e]);
        const double jv = ac + m2;
        J[(int64_t)p * S + e] = jv;
        if (Js) Js[(int64_t)p * S + e] = nl_split_value(jv);
        f = fma(fma(0.5, m2, ac), u[(int64_t)cj * S + e], f);
    }
    if (bad && e == 0) atomicExch(&ns->graph_bad, 1);
    F[t] = f;
}

// ||x||^2 per member (chunk tree); the CTA that completes the tree decides,
// per member, whether a Newton step (mode 0) or a linear solve (mode 1) runs.
//   mode 0 (Newton, step `it`): fn = ||F||; step 0 sets f0 = fn; a member
//     continues while fn > tol f0, up to max_newton steps
//   mode 1 (linear): fn = ||b||; a member with b != 0 is solved
//   mode 2: fn only (the true residual after a linear solve)
template <int S>
__global__ void __launch_bounds__(RowMap<S>::THREADS, 1024 / RowMap<S>::THREADS)
    nl_norm_kernel(int32_t n, const double *__restrict__ x, DotTree tn, NlState *ns, int mode, int it,
                   double tol, int max_newton) {
    constexpr int G = RowMap<S>::G;
    __shared__ double sm[32][S + 1];
    const int r = threadIdx.x / G, g = threadIdx.x % G;
    const int64_t R = (int64_t)blockIdx.x * 32 + r;
    double v0 = 0.0, v1 = 0.0;
    if (R < n) {
        if constexpr (S == 1) {
            if (g == 0) v0 = x[R] * x[R];
        } else {
            const double2 xv = reinterpret_cast<const double2 *>(x)[R * G + g];
            v0 = xv.x * xv.x;
            v1 = xv.y * xv.y;
        }
    }
    chunk_tree<S>(sm, v0, v1, r, g, tn, blockIdx.x, 0);
    if (!dot_tree_propagate(tn, blockIdx.x, 1)) return;
    if (threadIdx.x >= 32) return;
    const int e = threadIdx.x;
    int act = 0;
    if (e < S) {
        const double fn = sqrt(ld_cg(tn.buf[tn.levels] + e));
        ns->fn[e] = fn;
        if (mode != 2) ns->inv_fn[e] = (fn > 0.0) ? 1.0 / fn : 0.0;
        if (mode == 1) {
            ns->f0[e] = fn;
            ns->status[e] = (fn == fn) ? ENS_OK : ENS_ERR_BREAKDOWN;
            act = (fn > 0.0 && fn == fn) ? 1 : 0;
        } else if (mode == 0) {
            if (it == 0) {
                ns->f0[e] = fn;
                ns->status[e] = ENS_OK;
                ns->newton_iters[e] = 0;
                ns->lin_iters[e] = 0;
            }
            const double f0 = ns->f0[e];
            if (!(fn == fn)) {
                ns->status[e] = ENS_ERR_BREAKDOWN;
            } else if (ns->status[e] == ENS_OK && fn > tol * f0) {
                if (ns->newton_iters[e] >= max_newton) ns->status[e] = ENS_ERR_NOT_CONVERGED;
                else act = 1;
            }
        }
        if (mode != 2) ns->nact[e] = act;
    }
    if (mode == 2) return;  // report only (uniform over the warp)
    const unsigned ball = __ballot_sync(0xffffffffu, act);
    if (e == 0) ns->active_count = __popc(ball);
    __threadfence();
}

// u += du for the members that took a Newton step; their counts advance
template <int S>
__global__ void nl_update_kernel(int64_t total, double *__restrict__ u, const double *__restrict__ du,
                                 NlState *ns, const GmState *gs) {
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int e = (int)(t % S);
        if (ns->nact[e]) u[t] += du[t];
    }
    if (blockIdx.x == 0 && threadIdx.x < S) {
        const int e = threadIdx.x;
        if (ns->nact[e]) {
            ns->newton_iters[e] += 1;
            ns->lin_iters[e] += gs->iters[e];
        }
    }
}

// ------------------------------------------------------------ GMRES kernels
struct GmArgs {
    int32_t n;
    const int32_t *row_map, *col;
    const double *vals;  // the operator (J)
    const float2 *vdf;   // its pre-split copy (MODE 3 steps), or NULL
    uint64_t val_bytes;  // bytes of vdf
    const float2 *zs;    // MODE 3: split copy of the preconditioned vector z
    int *split_bad;      // MODE 3: a split copy met a value out of range (FP64 then)
    double *V;           // Krylov basis: restart + 1 blocks of n*S
    int64_t vs;          // n*S
    double *Z;           // flexible form: z_j = M^-1 v_j, restart blocks of n*S (with a preconditioner)
    double *t;           // scratch n*S (the final true residual of ens_gmres)
    double *x;           // the solution
    const double *rhs;   // right-hand side = sign * rhs
    double sign;
    DotTree tm;          // width (restart + 1) * S, used at width (j + 1) * S
    DotTree tn;          // width S
    GmState *gs;
    const NlState *ns;
    double tol;
    int restart, max_iter;
};

template <int S>
__device__ __forceinline__ double2 ld_row2(const double *v, int64_t R, int g) {
    if constexpr (S == 1) return make_double2(v[R], 0.0);
    else return reinterpret_cast<const double2 *>(v)[R * RowMap<S>::G + g];
}
template <int S>
__device__ __forceinline__ void st_row2(double *v, int64_t R, int g, double2 w) {
    if constexpr (S == 1) {
        if (g == 0) v[R] = w.x;
    } else {
        reinterpret_cast<double2 *>(v)[R * RowMap<S>::G + g] = w;
    }
}
// member indices of thread g's two lanes (s = 1: member 0 on thread 0 only)
template <int S>
__device__ __forceinline__ bool row_owner(int g) { return S != 1 || g == 0; }

// start of a solve from x = 0: v_0 = sign * rhs / ||rhs|| for the members
// to solve (0 for the others); the GMRES state of every member
template <int S>
__global__ void gm_start_kernel(GmArgs a) {
    const NlState *ns = a.ns;
    const int64_t total = a.vs;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int e = (int)(t % S);
        a.V[t] = ns->nact[e] ? a.sign * a.rhs[t] * ns->inv_fn[e] : 0.0;
        a.x[t] = 0.0;
    }
    if (blockIdx.x == 0 && threadIdx.x < 32) {
        const int e = threadIdx.x;
        GmState *gs = a.gs;
        int act = 0;
        if (e < S) {
            act = (ns->nact[e] && a.max_iter > 0) ? 1 : 0;
            gs->beta0[e] = ns->fn[e];
            gs->g[0][e] = ns->fn[e];
            gs->active[e] = act;
            gs->conv[e] = ns->nact[e] ? 0 : 1;  // a member to solve with max_iter = 0 stays unconverged
            gs->k[e] = 0;
            gs->iters[e] = 0;
            gs->scale[e] = 0.0;
        }
        const unsigned ball = __ballot_sync(0xffffffffu, act);
        if (e == 0) {
            gs->active_count = __popc(ball);
            gs->pending_count = gs->active_count;
        }
    }
}

// step j, part 1: w = J z (written to V[j+1]) and the first Gram-Schmidt
// dots hA_i = v_i . w, i <= j (tj: the tree tm at width (j + 1) s)
// MODE 3: the SpMV in double-float from the pre-split J and z (as the CG's
// pre-split K1), unless a split copy of z met a value out of range
template <int S, int MODE>
__global__ void __launch_bounds__(RowMap<S>::THREADS, 1024 / RowMap<S>::THREADS)
    gm_spmv_dots_kernel(GmArgs a, int j, const double *__restrict__ zin, DotTree tj) {
    if (ld_cg(&a.gs->active_count) == 0) return;
    constexpr int G = RowMap<S>::G;
    __shared__ ChunkCols cc;
    __shared__ double sm[32][S + 1];
    const int r = threadIdx.x / G, g = threadIdx.x % G;
    const int64_t R = (int64_t)blockIdx.x * 32 + r;
    const bool valid = R < a.n;
    double2 w;
    if constexpr (MODE == 3) {
        const bool staged =
            stage_chunk_pf(cc, a.row_map, a.col, blockIdx.x, a.n, a.vdf, S * 8u, a.val_bytes, 0xffffffffu);
        w = (ld_cg(a.split_bad) == 0) ? chunk_spmv_dfv<S>(cc, staged, a.col, a.vdf, a.vals, a.zs, r, g, valid)
                                      : chunk_spmv<S, double>(cc, staged, a.col, a.vals, zin, r, g, valid);
    } else {
        const bool staged = stage_chunk(cc, a.row_map, a.col, blockIdx.x, a.n);
        w = chunk_spmv<S, double>(cc, staged, a.col, a.vals, zin, r, g, valid);
    }
    if (valid) st_row2<S>(a.V + (int64_t)(j + 1) * a.vs, R, g, w);
    for (int i = 0; i <= j; ++i) {
        double p0 = 0.0, p1 = 0.0;
        if (valid && row_owner<S>(g)) {
            const double2 v = ld_row2<S>(a.V + (int64_t)i * a.vs, R, g);
            p0 = v.x * w.x;
            p1 = v.y * w.y;
        }
        chunk_tree<S>(sm, p0, p1, r, g, tj, blockIdx.x, i * S);
    }
    if (!dot_tree_propagate(tj, blockIdx.x, 1)) return;
    const double *top = tj.buf[tj.levels];
    for (int q = threadIdx.x; q < (j + 1) * S; q += blockDim.x) a.gs->hA[q / S][q % S] = ld_cg(top + q);
    __threadfence();
}

// step j, parts 2 and 3: w -= sum_i h_i v_i with h = hA (pass 0) or hB
// (pass 1).  Pass 0 then forms hB_i = v_i . w; pass 1 forms ||w|| and, in the
// CTA that completes the tree, the new Hessenberg column, the Givens
// rotation, the residual estimate |g_{j+1}| and the member's stop test.
template <int S>
__global__ void __launch_bounds__(RowMap<S>::THREADS, 1024 / RowMap<S>::THREADS)
    gm_orth_kernel(GmArgs a, int j, int pass, DotTree tj) {
    GmState *gs = a.gs;
    if (ld_cg(&gs->active_count) == 0) return;
    constexpr int G = RowMap<S>::G;
    __shared__ double sm[32][S + 1];
    const int r = threadIdx.x / G, g = threadIdx.x % G;
    const int64_t R = (int64_t)blockIdx.x * 32 + r;
    const bool own = R < a.n && row_owner<S>(g);
    const int e0 = (S == 1) ? 0 : 2 * g, e1 = (S == 1) ? 0 : 2 * g + 1;
    double *W = a.V + (int64_t)(j + 1) * a.vs;
    const double(*h)[32] = pass == 0 ? gs->hA : gs->hB;
    double2 w = make_double2(0.0, 0.0);
    if (own) {
        w = ld_row2<S>(W, R, g);
        for (int i = 0; i <= j; ++i) {
            const double2 v = ld_row2<S>(a.V + (int64_t)i * a.vs, R, g);
            w.x = fma(-h[i][e0], v.x, w.x);
            w.y = fma(-h[i][e1], v.y, w.y);
        }
        st_row2<S>(W, R, g, w);
    }
    if (pass == 0) {
        for (int i = 0; i <= j; ++i) {
            double p0 = 0.0, p1 = 0.0;
            if (own) {
                const double2 v = ld_row2<S>(a.V + (int64_t)i * a.vs, R, g);
                p0 = v.x * w.x;
                p1 = v.y * w.y;
            }
            chunk_tree<S>(sm, p0, p1, r, g, tj, blockIdx.x, i * S);
        }
        if (!dot_tree_propagate(tj, blockIdx.x, 1)) return;
        const double *top = tj.buf[tj.levels];
        for (int q = threadIdx.x; q < (j + 1) * S; q += blockDim.x) gs->hB[q / S][q % S] = ld_cg(top + q);
        __threadfence();
        return;
    }
    chunk_tree<S>(sm, w.x * w.x, w.y * w.y, r, g, a.tn, blockIdx.x, 0);
    if (!dot_tree_propagate(a.tn, blockIdx.x, 1)) return;
    if (threadIdx.x >= 32) return;
    const int e = threadIdx.x;
    int act = 0, pend = 0;
    if (e < S) {
        if (gs->active[e]) {
            const double hn = sqrt(ld_cg(a.tn.buf[a.tn.levels] + e));
            for (int i = 0; i <= j; ++i) gs->H[i][j][e] = gs->hA[i][e] + gs->hB[i][e];
            for (int i = 0; i < j; ++i) {  // the earlier rotations
                const double c = gs->cs[i][e], sv = gs->sn[i][e];
                const double a0 = gs->H[i][j][e], a1 = gs->H[i + 1][j][e];
                gs->H[i][j][e] = c * a0 + sv * a1;
                gs->H[i + 1][j][e] = -sv * a0 + c * a1;
            }
            const double hjj = gs->H[j][j][e];
            const double tq = hypot(hjj, hn);
            const double c = (tq == 0.0) ? 1.0 : hjj / tq, sv = (tq == 0.0) ? 0.0 : hn / tq;
            gs->cs[j][e] = c;
            gs->sn[j][e] = sv;
            gs->H[j][j][e] = c * hjj + sv * hn;
            const double gj = gs->g[j][e];
            gs->g[j + 1][e] = -sv * gj;
            gs->g[j][e] = c * gj;
            gs->k[e] = j + 1;
            gs->iters[e] += 1;
            const bool conv = fabs(-sv * gj) <= a.tol * gs->beta0[e] || hn == 0.0;
            gs->scale[e] = (hn > 0.0) ? 1.0 / hn : 0.0;
            if (conv) gs->conv[e] = 1;
            act = (!conv && gs->iters[e] < a.max_iter && j + 1 < a.restart) ? 1 : 0;
            gs->active[e] = act;
        } else {
            gs->scale[e] = 0.0;
        }
        pend = (!gs->conv[e] && gs->iters[e] < a.max_iter) ? 1 : 0;
    }
    const unsigned ball = __ballot_sync(0xffffffffu, act), pball = __ballot_sync(0xffffffffu, pend);
    if (e == 0) {
        gs->active_count = __popc(ball);
        gs->pending_count = __popc(pball);
    }
    __threadfence();
}

// v_{j1} *= 1 / h_{j1, j1-1} (0 for the members that stopped)
template <int S>
__global__ void gm_scale_kernel(GmArgs a, int j1) {
    if (ld_cg(&a.gs->active_count) == 0) return;
    double *v = a.V + (int64_t)j1 * a.vs;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < a.vs;
         t += (int64_t)gridDim.x * blockDim.x)
        v[t] *= a.gs->scale[t % S];
}

// end of a cycle: y = H^-1 g on the member's own k steps (back substitution)
template <int S>
__global__ void gm_solve_kernel(GmArgs a) {
    const int e = threadIdx.x;
    if (e >= S) return;
    GmState *gs = a.gs;
    const int k = gs->k[e];
    for (int i = k - 1; i >= 0; --i) {
        double y = gs->g[i][e];
        for (int l = i + 1; l < k; ++l) y -= gs->H[i][l][e] * gs->y[l][e];
        gs->y[i][e] = y / gs->H[i][i][e];
    }
}

// x += sum_{i < k_e} y_i B_i with B the Krylov basis V (no preconditioner)
// or the preconditioned vectors Z = M^-1 V of the flexible form
template <int S>
__global__ void gm_combine_kernel(GmArgs a, const double *__restrict__ B) {
    const GmState *gs = a.gs;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < a.vs;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int e = (int)(t % S);
        const int k = gs->k[e];
        double acc = 0.0;
        for (int i = 0; i < k; ++i) acc = fma(gs->y[i][e], B[(int64_t)i * a.vs + t], acc);
        a.x[t] += acc;
    }
}

// out = sign * rhs - J x (row per thread pair, as the SpMV)
template <int S>
__global__ void __launch_bounds__(RowMap<S>::THREADS, 1024 / RowMap<S>::THREADS)
    gm_residual_kernel(GmArgs a, double *__restrict__ out) {
    constexpr int G = RowMap<S>::G;
    __shared__ ChunkCols cc;
    const int r = threadIdx.x / G, g = threadIdx.x % G;
    const int64_t R = (int64_t)blockIdx.x * 32 + r;
    const bool valid = R < a.n;
    const bool staged = stage_chunk(cc, a.row_map, a.col, blockIdx.x, a.n);
    const double2 ax = chunk_spmv<S, double>(cc, staged, a.col, a.vals, a.x, r, g, valid);
    if (!valid) return;
    const double2 bv = ld_row2<S>(a.rhs, R, g);
    st_row2<S>(out, R, g, make_double2(a.sign * bv.x - ax.x, a.sign * bv.y - ax.y));
}

// restart: ||r|| of the new residual in V[0]; members still short of the
// tolerance (and under max_iter) start a new cycle with g_0 = ||r||
template <int S>
__global__ void __launch_bounds__(RowMap<S>::THREADS, 1024 / RowMap<S>::THREADS) gm_restart_kernel(GmArgs a) {
    constexpr int G = RowMap<S>::G;
    __shared__ double sm[32][S + 1];
    const int r = threadIdx.x / G, g = threadIdx.x % G;
    const int64_t R = (int64_t)blockIdx.x * 32 + r;
    double2 v = make_double2(0.0, 0.0);
    if (R < a.n && row_owner<S>(g)) v = ld_row2<S>(a.V, R, g);
    chunk_tree<S>(sm, v.x * v.x, v.y * v.y, r, g, a.tn, blockIdx.x, 0);
    if (!dot_tree_propagate(a.tn, blockIdx.x, 1)) return;
    if (threadIdx.x >= 32) return;
    const int e = threadIdx.x;
    GmState *gs = a.gs;
    int act = 0;
    if (e < S) {
        const double rn = sqrt(ld_cg(a.tn.buf[a.tn.levels] + e));
        gs->k[e] = 0;
        if (!gs->conv[e] && gs->iters[e] < a.max_iter) {
            if (rn > 0.0) {
                act = 1;
                gs->g[0][e] = rn;
                gs->scale[e] = 1.0 / rn;
            } else {
                gs->conv[e] = 1;
                gs->scale[e] = 0.0;
            }
        } else {
            gs->scale[e] = 0.0;
        }
        gs->active[e] = act;
    }
    const unsigned ball = __ballot_sync(0xffffffffu, act);
    if (e == 0) {
        gs->active_count = __popc(ball);
        gs->pending_count = gs->active_count;
    }
    __threadfence();
}

// ------------------------------------------------------------ host side
// 2 beta h^3 (h = 1/N) as a float pair for nl_jacobian_kernel
static void nl_m2_split(double beta, int N, float *hi, float *lo) {
    const double c = 2.0 * beta / ((double)N * N * N);
    *hi = (float)c;
    *lo = (float)(c - (double)*hi);
}

struct NlBufs {
    NlState *ns;
    GmState *gs;
    double *V, *Z, *t, *du, *J, *F;
    float2 *Js;  // pre-split J (Newton with a pre-split level 0 of the preconditioner)
    char *tm, *tn;
};

// workspace: states, Krylov basis V, preconditioned basis Z (with a
// preconditioner), t, trees; Newton adds du, J and F (and
// the split J when level 0 of the preconditioner is pre-split); with the
// multigrid preconditioner the hierarchy follows (mg_layout)
static size_t nl_layout(int nlevels, const ens_mg_level *lv, int s, int restart, bool newton, bool precond,
                        char *base, NlBufs *b, std::vector<MgLevel> *mglv, double **inv, int **bad) {
    size_t off = 0;
    auto take = [&](size_t bytes) -> char * {
        char *p = base ? base + off : nullptr;
        off += mg_align(bytes);
        return p;
    };
    const int64_t n = lv[0].graph.num_rows, nnz = lv[0].graph.num_entries;
    const size_t vb = sizeof(double) * (size_t)n * s;
    NlBufs o;
    memset(&o, 0, sizeof(o));
    o.ns = reinterpret_cast<NlState *>(take(sizeof(NlState)));
    o.gs = reinterpret_cast<GmState *>(take(sizeof(GmState)));
    o.V = reinterpret_cast<double *>(take(vb * (size_t)(restart + 1)));
    if (precond) o.Z = reinterpret_cast<double *>(take(vb * (size_t)restart));
    o.t = reinterpret_cast<double *>(take(vb));
    o.tm = take(dot_tree_bytes(n, (restart + 1) * s));
    o.tn = take(dot_tree_bytes(n, s));
    if (newton) {
        o.du = reinterpret_cast<double *>(take(vb));
        o.F = reinterpret_cast<double *>(take(vb));
        o.J = reinterpret_cast<double *>(take(sizeof(double) * (size_t)nnz * s));
        // split J for the pre-split GMRES SpMV (it reads z's split copy, which
        // the FP64-class V-cycle writes; the FP32 V-cycle does not)
        if (precond && lv[0].values_df && !lv[0].values_f32)
            o.Js = reinterpret_cast<float2 *>(take(sizeof(double) * (size_t)nnz * s));
    }
    if (precond) off += mg_layout(nlevels, lv, s, mglv, base ? base + off : nullptr, inv, bad);
    if (base && b) *b = o;
    return off;
}

template <int S>
struct NlSolver {
    GmArgs a;
    MgSolver<S> mg;
    bool precond = false;
    bool pre = false;  // GMRES SpMV in the pre-split form (J and z split; needs a pre-split level 0)
    int check_every = 8;
    int launches = 0, polls = 0;
    unsigned grid = 0, eg = 152 * 4;

    int init(int nlevels, const ens_mg_level *lv, int restart, bool newton, bool pc, int degree, char *work,
             NlBufs *bufs, cudaStream_t st) {
        int *bad = nullptr;
        precond = pc;
        nl_layout(nlevels, lv, S, restart, newton, pc, work, bufs, &mg.lv, &mg.inv, &bad);
        memset(&a, 0, sizeof(a));
        a.n = lv[0].graph.num_rows;
        a.row_map = lv[0].graph.row_map;
        a.col = lv[0].graph.col_entry;
        a.V = bufs->V;
        a.vs = (int64_t)a.n * S;
        a.Z = bufs->Z;
        a.t = bufs->t;
        a.gs = bufs->gs;
        a.ns = bufs->ns;
        a.restart = restart;
        dot_tree_layout(&a.tm, a.n, (restart + 1) * S, bufs->tm);
        dot_tree_layout(&a.tn, a.n, S, bufs->tn);
        grid = MgSolver<S>::chunks(a.n);
        int rc;
        ENS_CUDA_TRY(cudaMemsetAsync(bufs->ns, 0, sizeof(NlState), st));
        ENS_CUDA_TRY(cudaMemsetAsync(bufs->gs, 0, sizeof(GmState), st));
        if ((rc = dot_tree_clear(a.tm, st))) return rc;
        if ((rc = dot_tree_clear(a.tn, st))) return rc;
        if (pc) {
            mg.degree = degree;
            mg.f32 = lv[0].values_f32 != nullptr;  // the FP32 V-cycle (flexible GMRES admits it)
            mg.eg = 152 * 4;
            mg.active = &bufs->gs->active_count;
            mg_bad = bad;
        }
        return ENS_OK;
    }
    int *mg_bad = nullptr;

    int setup_mg(const ens_mg_level *lv, double ratio, double boost, int power_iters, cudaStream_t st,
                 bool lanczos = false) {
        int rc = mg.setup(lv, ratio, boost, power_iters, mg_bad, st, &launches, lanczos);
        if (rc) return rc;
        int hbad = 0;
        ENS_CUDA_TRY(cudaMemcpyAsync(&hbad, mg_bad, sizeof(int), cudaMemcpyDeviceToHost, st));
        ENS_CUDA_TRY(cudaStreamSynchronize(st));
        if (hbad) return fail(ENS_ERR_BREAKDOWN, "ens_newton/ens_gmres: coarsest matrix not positive definite");
        return ENS_OK;
    }

    // one GMRES solve of J x = sign * rhs from x = 0 for the members with
    // ns->nact set (a.vals, a.rhs, a.sign, a.x, a.tol, a.max_iter filled)
    int gmres(cudaStream_t st) {
        constexpr unsigned T = RowMap<S>::THREADS;
        gm_start_kernel<S><<<eg, 256, 0, st>>>(a);
        ++launches;
        int32_t h[2] = {0, 0};
        for (;;) {
            int j = 0;
            while (j < a.restart) {
                for (int q = 0; q < check_every && j < a.restart; ++q, ++j) {
                    const double *zin = a.V + (int64_t)j * a.vs;
                    if (precond) {  // flexible form: z_j = M^-1 v_j kept in Z[j]
                        double *zj = a.Z + (int64_t)j * a.vs;
                        mg.active = &a.gs->active_count;
                        if (mg.f32) mg.vcycle32(0, zin, nullptr, mg.lv[0].x32, zj, st);
                        else mg.vcycle(0, zin, zj, st, pre);  // pre: z's split copy into level 0's xs
                        launches += mg.launches_per_vcycle();
                        zin = zj;
                    }
                    DotTree tj = a.tm;
                    tj.width = (j + 1) * S;
                    if (pre) gm_spmv_dots_kernel<S, 3><<<grid, T, 0, st>>>(a, j, zin, tj);
                    else gm_spmv_dots_kernel<S, 0><<<grid, T, 0, st>>>(a, j, zin, tj);
                    gm_orth_kernel<S><<<grid, T, 0, st>>>(a, j, 0, tj);
                    gm_orth_kernel<S><<<grid, T, 0, st>>>(a, j, 1, tj);
                    gm_scale_kernel<S><<<eg, 256, 0, st>>>(a, j + 1);
                    launches += 4;
                }
                ENS_LAUNCH_CHECK("ens_gmres step");
                ENS_CUDA_TRY(cudaMemcpyAsync(h, &a.gs->active_count, 2 * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
                ENS_CUDA_TRY(cudaStreamSynchronize(st));
                ++polls;
                if (h[0] == 0) break;
            }
            gm_solve_kernel<S><<<1, 32, 0, st>>>(a);
            gm_combine_kernel<S><<<eg, 256, 0, st>>>(a, precond ? a.Z : a.V);
            launches += 2;
            if (h[1] == 0) break;
            gm_residual_kernel<S><<<grid, T, 0, st>>>(a, a.V);
            gm_restart_kernel<S><<<grid, T, 0, st>>>(a);
            gm_scale_kernel<S><<<eg, 256, 0, st>>>(a, 0);
            launches += 3;
        }
        ENS_LAUNCH_CHECK("ens_gmres");
        return ENS_OK;
    }
};

static int nl_check_levels(int nlevels, const ens_mg_level *lv, int s, int precond) {
    if (precond == ENS_NL_PRECOND_MG) return mg_check(nlevels, lv, s);
    if (precond != ENS_NL_PRECOND_NONE) return fail(ENS_ERR_ARG, "precond must be ENS_NL_PRECOND_NONE or _MG");
    if (nlevels < 1 || !lv) return fail(ENS_ERR_ARG, "nlevels >= 1 required");
    if (!supported_s(s)) return fail(ENS_ERR_UNSUPPORTED, "ensemble size s=%d not in {1,4,8,16,32}", s);
    int rc = check_graph(&lv[0].graph);
    if (rc) return rc;
    const int64_t n1 = (int64_t)lv[0].N + 1;
    if (lv[0].N < 1 || lv[0].graph.num_rows != n1 * n1 * n1)
        return fail(ENS_ERR_ARG, "level 0: graph is not that of the %d^3-cell mesh", lv[0].N);
    return ENS_OK;
}

template <int S>
static int gmres_run(int nlevels, const ens_mg_level *lv, const double *vals, const double *b, double *x, double tol,
                     int restart, int max_iter, int precond, int degree, double ratio, double boost, int power_iters,
                     int check_every, void *work, int32_t *iters, double *relres, int32_t *status, ens_cg_stats *stats,
                     cudaStream_t st) {
    NlSolver<S> sv;
    NlBufs bufs;
    int rc = sv.init(nlevels, lv, restart, false, precond == ENS_NL_PRECOND_MG, degree, static_cast<char *>(work),
                     &bufs, st);
    if (rc) return rc;
    sv.check_every = check_every;
    if (sv.precond && (rc = sv.setup_mg(lv, ratio, boost, power_iters, st))) return rc;
    GmArgs &a = sv.a;
    a.vals = vals;
    a.rhs = b;
    a.sign = 1.0;
    a.x = x;
    a.tol = tol;
    a.max_iter = max_iter;
    nl_norm_kernel<S><<<sv.grid, RowMap<S>::THREADS, 0, st>>>(a.n, b, a.tn, bufs.ns, 1, 0, 0.0, 0);
    if ((rc = sv.gmres(st))) return rc;
    // true residual ||b - A x|| (into t)
    gm_residual_kernel<S><<<sv.grid, RowMap<S>::THREADS, 0, st>>>(a, a.t);
    nl_norm_kernel<S><<<sv.grid, RowMap<S>::THREADS, 0, st>>>(a.n, a.t, a.tn, bufs.ns, 2, 0, 0.0, 0);
    sv.launches += 3;
    ENS_LAUNCH_CHECK("ens_gmres final");
    NlState hn;
    GmState *hg = static_cast<GmState *>(malloc(sizeof(GmState)));
    if (!hg) return fail(ENS_ERR_ARG, "ens_gmres: host allocation failed");
    cudaError_t ce = cudaMemcpyAsync(&hn, bufs.ns, sizeof(NlState), cudaMemcpyDeviceToHost, st);
    if (ce == cudaSuccess) ce = cudaMemcpyAsync(hg, bufs.gs, sizeof(GmState), cudaMemcpyDeviceToHost, st);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(st);
    if (ce != cudaSuccess) {
        free(hg);
        return cuda_fail(ce, "ens_gmres results");
    }
    int first_bad = ENS_OK, maxit = 0;
    for (int e = 0; e < S; ++e) {
        const int stv = hn.status[e] != ENS_OK ? hn.status[e] : (hg->conv[e] ? ENS_OK : ENS_ERR_NOT_CONVERGED);
        if (iters) iters[e] = hg->iters[e];
        if (relres) relres[e] = hn.f0[e] > 0.0 ? hn.fn[e] / hn.f0[e] : 0.0;
        if (status) status[e] = stv;
        if (stv != ENS_OK && first_bad == ENS_OK) first_bad = stv;
        maxit = hg->iters[e] > maxit ? hg->iters[e] : maxit;
    }
    free(hg);
    if (stats) {
        memset(stats, 0, sizeof(ens_cg_stats));
        stats->iterations = maxit;
        stats->kernel_launches = sv.launches;
        stats->host_checks = sv.polls;
    }
    if (first_bad != ENS_OK) set_error("ens_gmres: member status %d (%s)", first_bad, ens_status_string(first_bad));
    return first_bad;
}

template <int S>
static int newton_run(int nlevels, const ens_mg_level *lv, const double *C, const double *b, double *u,
                      const ens_newton_params *p, void *work, int32_t *newton_iters, int32_t *lin_iters,
                      double *relres, int32_t *status, ens_cg_stats *stats, cudaStream_t st) {
    NlSolver<S> sv;
    NlBufs bufs;
    int rc = sv.init(nlevels, lv, p->restart, true, p->precond == ENS_NL_PRECOND_MG, p->degree,
                     static_cast<char *>(work), &bufs, st);
    if (rc) return rc;
    sv.check_every = p->check_every;
    if (sv.precond && (rc = sv.setup_mg(lv, p->ratio, p->boost, p->power_iters, st,
                                        (p->flags & ENS_PC_LANCZOS) != 0)))
        return rc;
    GmArgs &a = sv.a;
    a.vals = bufs.J;
    if (bufs.Js) {  // the GMRES SpMV reads J pre-split and z split by the V-cycle
        sv.pre = true;
        a.vdf = bufs.Js;
        a.val_bytes = (uint64_t)lv[0].graph.num_entries * S * 8u;
        a.zs = sv.mg.lv[0].xs;
        a.split_bad = sv.mg.lv[0].split_bad;
    }
    a.rhs = bufs.F;
    a.sign = -1.0;
    a.x = bufs.du;
    a.tol = p->lin_tol;
    a.max_iter = p->max_lin;
    const int32_t n = a.n, N = lv[0].N;
    const unsigned jgrid = (unsigned)(((int64_t)n * S + 255) / 256);
    float m2h, m2l;
    nl_m2_split(p->beta, N, &m2h, &m2l);
    int32_t h[2];
    for (int it = 0; it <= p->max_newton; ++it) {
        nl_jacobian_kernel<S><<<jgrid, 256, 0, st>>>(n, N, a.row_map, a.col, lv[0].values, C, p->alpha, m2h, m2l,
                                                    b, u, bufs.J, bufs.Js, bufs.F, bufs.ns);
        nl_norm_kernel<S><<<sv.grid, RowMap<S>::THREADS, 0, st>>>(n, bufs.F, a.tn, bufs.ns, 0, it, p->tol,
                                                                 p->max_newton);
        sv.launches += 2;
        ENS_LAUNCH_CHECK("ens_newton residual");
        ENS_CUDA_TRY(cudaMemcpyAsync(h, &bufs.ns->active_count, 2 * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
        ENS_CUDA_TRY(cudaStreamSynchronize(st));
        ++sv.polls;
        if (h[1]) return fail(ENS_ERR_ARG, "ens_newton: an interior row of the graph is not its 27-node window");
        if (h[0] == 0) break;
        if ((rc = sv.gmres(st))) return rc;
        nl_update_kernel<S><<<sv.eg, 256, 0, st>>>((int64_t)n * S, u, bufs.du, bufs.ns, bufs.gs);
        ++sv.launches;
    }
    NlState hn;
    ENS_CUDA_TRY(cudaMemcpyAsync(&hn, bufs.ns, sizeof(NlState), cudaMemcpyDeviceToHost, st));
    ENS_CUDA_TRY(cudaStreamSynchronize(st));
    int first_bad = ENS_OK, maxit = 0;
    for (int e = 0; e < S; ++e) {
        if (newton_iters) newton_iters[e] = hn.newton_iters[e];
        if (lin_iters) lin_iters[e] = hn.lin_iters[e];
        if (relres) relres[e] = hn.f0[e] > 0.0 ? hn.fn[e] / hn.f0[e] : 0.0;
        if (status) status[e] = hn.status[e];
        if (hn.status[e] != ENS_OK && first_bad == ENS_OK) first_bad = hn.status[e];
        maxit = hn.newton_iters[e] > maxit ? hn.newton_iters[e] : maxit;
    }
    if (stats) {
        memset(stats, 0, sizeof(ens_cg_stats));
        stats->iterations = maxit;
        stats->kernel_launches = sv.launches;
        stats->host_checks = sv.polls;
    }
    if (first_bad != ENS_OK) set_error("ens_newton: member status %d (%s)", first_bad, ens_status_string(first_bad));
    return first_bad;
}

}  // namespace ens

using namespace ens;

#define NL_DISPATCH(call_template)                 \
    switch (s) {                                   \
        case 1: return call_template(1);           \
        case 4: return call_template(4);           \
        case 8: return call_template(8);           \
        case 16: return call_template(16);         \
        default: return call_template(32);         \
    }

extern "C" int ens_nl_advection(const ens_graph *gp, int32_t N, const double *v, double *C, void *stream) {
    if (!gp) return fail(ENS_ERR_ARG, "NULL graph");
    const ens_graph &g = *gp;
    int rc = check_graph(&g);
    if (rc) return rc;
    const int64_t n1 = (int64_t)N + 1;
    if (N < 1 || g.num_rows != n1 * n1 * n1) return fail(ENS_ERR_ARG, "graph is not that of the %d^3-cell mesh", N);
    if (!v || !C) return fail(ENS_ERR_ARG, "NULL v/C");
    const unsigned grid = (unsigned)((g.num_rows + 255) / 256);
    nl_advection_kernel<<<grid, 256, 0, as_stream(stream)>>>(g.num_rows, N, g.row_map, g.col_entry, v[0], v[1], v[2],
                                                             C);
    ENS_LAUNCH_CHECK("ens_nl_advection");
    return ENS_OK;
}

extern "C" int ens_nl_jacobian(const ens_graph *gp, int32_t N, int s, const double *A, const double *C, double alpha,
                               double beta, const double *b, const double *u, double *J, double *F, void *work,
                               void *stream) {
    if (!gp) return fail(ENS_ERR_ARG, "NULL graph");
    const ens_graph &g = *gp;
    int rc = check_graph(&g);
    if (rc) return rc;
    if (!supported_s(s)) return fail(ENS_ERR_UNSUPPORTED, "ensemble size s=%d not in {1,4,8,16,32}", s);
    const int64_t n1 = (int64_t)N + 1;
    if (N < 1 || g.num_rows != n1 * n1 * n1) return fail(ENS_ERR_ARG, "graph is not that of the %d^3-cell mesh", N);
    if (!A || !C || !b || !u || !J || !F || !work) return fail(ENS_ERR_ARG, "NULL A/C/b/u/J/F/work");
    cudaStream_t st = as_stream(stream);
    NlState *ns = static_cast<NlState *>(work);
    ENS_CUDA_TRY(cudaMemsetAsync(&ns->graph_bad, 0, sizeof(int), st));
    const unsigned grid = (unsigned)(((int64_t)g.num_rows * s + 255) / 256);
    float m2h, m2l;
    nl_m2_split(beta, N, &m2h, &m2l);
#define NL_JAC(SS)                                                                                             \
    nl_jacobian_kernel<SS><<<grid, 256, 0, st>>>(g.num_rows, N, g.row_map, g.col_entry, A, C, alpha, m2h, m2l,  \
                                                 b, u, J, nullptr, F, ns)
    switch (s) {
        case 1: NL_JAC(1); break;
        case 4: NL_JAC(4); break;
        case 8: NL_JAC(8); break;
        case 16: NL_JAC(16); break;
        default: NL_JAC(32); break;
    }
#undef NL_JAC
    ENS_LAUNCH_CHECK("ens_nl_jacobian");
    int bad = 0;
    ENS_CUDA_TRY(cudaMemcpyAsync(&bad, &ns->graph_bad, sizeof(int), cudaMemcpyDeviceToHost, st));
    ENS_CUDA_TRY(cudaStreamSynchronize(st));
    if (bad) return fail(ENS_ERR_ARG, "ens_nl_jacobian: an interior row of the graph is not its 27-node window");
    return ENS_OK;
}

extern "C" int ens_nl_jacobian_workspace_size(size_t *bytes) {
    if (!bytes) return fail(ENS_ERR_ARG, "bytes is NULL");
    *bytes = sizeof(NlState);
    return ENS_OK;
}

static int gmres_args(int nlevels, const ens_mg_level *levels, int s, int restart, int max_iter, int precond,
                      int degree, double ratio, double boost, int power_iters, int check_every, double tol) {
    int rc = nl_check_levels(nlevels, levels, s, precond);
    if (rc) return rc;
    if (restart < 1 || restart > kGmMaxRestart || max_iter < 0 || check_every < 1 || !(tol >= 0.0))
        return fail(ENS_ERR_ARG, "GMRES: 1 <= restart <= %d, max_iter >= 0, check_every >= 1, tol >= 0",
                    kGmMaxRestart);
    if (precond == ENS_NL_PRECOND_MG) {
        if (degree < 1 || degree > kPcMaxDegree || !(ratio > 1.0) || !(boost >= 1.0) || power_iters < 1 ||
            power_iters > 1000)
            return fail(ENS_ERR_ARG, "V-cycle: bad degree/ratio/boost/power_iters");
        for (int l = 0; l < nlevels; ++l)
            if (!levels[l].power_start) return fail(ENS_ERR_ARG, "level %d: NULL power_start", l);
    }
    return ENS_OK;
}

extern "C" int ens_gmres_workspace_size(int nlevels, const ens_mg_level *levels, int s, int restart, int precond,
                                        size_t *bytes) {
    int rc = nl_check_levels(nlevels, levels, s, precond);
    if (rc) return rc;
    if (restart < 1 || restart > kGmMaxRestart) return fail(ENS_ERR_ARG, "1 <= restart <= %d", kGmMaxRestart);
    if (!bytes) return fail(ENS_ERR_ARG, "bytes is NULL");
    *bytes = nl_layout(nlevels, levels, s, restart, false, precond == ENS_NL_PRECOND_MG, nullptr, nullptr, nullptr,
                       nullptr, nullptr);
    return ENS_OK;
}

extern "C" int ens_gmres(int nlevels, const ens_mg_level *levels, int s, const double *values, const double *b,
                         double *x, double tol, int restart, int max_iter, int precond, int degree, double ratio,
                         double boost, int power_iters, int check_every, void *work, size_t work_bytes,
                         int32_t *iters_host, double *relres_host, int32_t *status_host, ens_cg_stats *stats_host,
                         void *stream) {
    int rc = gmres_args(nlevels, levels, s, restart, max_iter, precond, degree, ratio, boost, power_iters,
                        check_every, tol);
    if (rc) return rc;
    if (!values || !b || !x || !work) return fail(ENS_ERR_ARG, "NULL values/b/x/work");
    if (!aligned16(work) || (s > 1 && (!aligned16(b) || !aligned16(x) || !aligned16(values))))
        return fail(ENS_ERR_ALIGN, "values/b/x/work must be 16-byte aligned");
    const size_t need = nl_layout(nlevels, levels, s, restart, false, precond == ENS_NL_PRECOND_MG, nullptr,
                                  nullptr, nullptr, nullptr, nullptr);
    if (work_bytes < need) return fail(ENS_ERR_WORKSPACE, "gmres workspace %zu < %zu bytes", work_bytes, need);
    cudaStream_t st = as_stream(stream);
#define GM_CALL(SS)                                                                                                 \
    gmres_run<SS>(nlevels, levels, values, b, x, tol, restart, max_iter, precond, degree, ratio, boost, power_iters, \
                  check_every, work, iters_host, relres_host, status_host, stats_host, st)
    NL_DISPATCH(GM_CALL)
#undef GM_CALL
}

extern "C" int ens_newton_workspace_size(int nlevels, const ens_mg_level *levels, int s,
                                         const ens_newton_params *p, size_t *bytes) {
    if (!p || !bytes) return fail(ENS_ERR_ARG, "NULL params/bytes");
    int rc = nl_check_levels(nlevels, levels, s, p->precond);
    if (rc) return rc;
    if (p->restart < 1 || p->restart > kGmMaxRestart) return fail(ENS_ERR_ARG, "1 <= restart <= %d", kGmMaxRestart);
    *bytes = nl_layout(nlevels, levels, s, p->restart, true, p->precond == ENS_NL_PRECOND_MG, nullptr, nullptr,
                       nullptr, nullptr, nullptr);
    return ENS_OK;
}

extern "C" int ens_newton(int nlevels, const ens_mg_level *levels, int s, const double *C, const double *b, double *u,
                          const ens_newton_params *p, void *work, size_t work_bytes, int32_t *newton_iters_host,
                          int32_t *lin_iters_host, double *relres_host, int32_t *status_host,
                          ens_cg_stats *stats_host, void *stream) {
    if (!p) return fail(ENS_ERR_ARG, "NULL params");
    int rc = gmres_args(nlevels, levels, s, p->restart, p->max_lin, p->precond, p->degree, p->ratio, p->boost,
                        p->power_iters, p->check_every, p->lin_tol);
    if (rc) return rc;
    if (!(p->tol >= 0.0) || p->max_newton < 0) return fail(ENS_ERR_ARG, "ens_newton: tol >= 0, max_newton >= 0");
    if ((p->flags & ~ENS_PC_LANCZOS) != 0 || ((p->flags & ENS_PC_LANCZOS) && p->power_iters > kLzMaxSteps))
        return fail(ENS_ERR_ARG, "ens_newton: flags 0 or ENS_PC_LANCZOS (with at most %d steps)", kLzMaxSteps);
    if (!levels[0].values || !C || !b || !u || !work) return fail(ENS_ERR_ARG, "NULL values/C/b/u/work");
    if (!aligned16(work) || (s > 1 && (!aligned16(b) || !aligned16(u) || !aligned16(levels[0].values))))
        return fail(ENS_ERR_ALIGN, "values/b/u/work must be 16-byte aligned");
    const size_t need = nl_layout(nlevels, levels, s, p->restart, true, p->precond == ENS_NL_PRECOND_MG, nullptr,
                                  nullptr, nullptr, nullptr, nullptr);
    if (work_bytes < need) return fail(ENS_ERR_WORKSPACE, "newton workspace %zu < %zu bytes", work_bytes, need);
    cudaStream_t st = as_stream(stream);
#define NT_CALL(SS)                                                                                             \
    newton_run<SS>(nlevels, levels, C, b, u, p, work, newton_iters_host, lin_iters_host, relres_host, status_host, \
                   stats_host, st)
    NL_DISPATCH(NT_CALL)
#undef NT_CALL
}
