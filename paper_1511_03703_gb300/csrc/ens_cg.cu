// ens_cg.cu -- ensemble conjugate gradients (Sect. 3.4 solver, Sect. 4 experiments).
//
// Hestenes-Stiefel CG run on every member of the commuted ensemble system at
// once.  By default each member has its own alpha, beta and stopping test
// (dots reduced per member: the vector sum_i u_i^T v_i (x) e_i of Sect. 3.4
// before its members are added), so member e follows the iterates of a
// standalone solve of sample e; members that converge are frozen.  With
// ENS_CG_COUPLED the member dots are summed first, which is the paper's
// coupled ensemble solver of Sect. 3.6.
//
// Launch sequence, no host synchronisation inside an iteration:
//   K0  r = b - A x0, p = r, rho_e = r.r, |b_e|^2   (last CTA: init, stop test)
//   KZ  x_e = 0 for members with b_e = 0 (one-shot)
//   per iteration:
//   K1  q = A p,  pi_e = p.q     (last CTA: alpha_e = rho_e / pi_e, breakdown)
//   K2  r -= alpha q,  r.r       (last CTA: stop test, beta_e, x-update flags)
//   K3  x += alpha p,  p = r + beta p   (x update deferred here so K2 reads 2 vectors)
// Vector traffic per iteration: K1 1 gather + 1 write, K2 2 reads + 1 write,
// K3 3 reads + 2 writes (10 vector passes; +1 write of the split p in df mode).
// The per-member scalar work runs in the CTA that completes each kernel's
// deterministic dot tree.  K2/K3 stream tiles of 4-8 tree chunks per CTA.
// Flag protocol: K2 sets updx_e for members active in its iteration, K3 reads
// them, and the next K1 clears them (also when it exits early).
#include <vector>

#include "ens_spmv.cuh"

namespace ens {

struct CgState {
    double rho[32], alpha[32], beta[32], bnorm[32], relres[32];
    int active[32], updx[32], zerox[32], iters[32], status[32];
    int active_count, updx_any, zero_any, spmv_real;
    int df_bad_any, pad0, pad1, pad2;
    double bnorm_all;
};

struct CgArgs {
    int32_t n;
    const int32_t *row_map;
    const int32_t *col;
    const double *vals;
    const double *b;
    double *x, *r, *p, *q;
    float2 *pdf;  // p split into float pairs (df mode)
    CgState *st;
    DotTree t1;   // width s
    DotTree t2;   // width 2s
    double tol;
    int max_iter;
    int coupled;
};

// mapping of the streaming vector kernels (K2, K3): a CTA owns CPC chunks
template <int S>
struct VecMap {
    static constexpr int VG = (S == 1) ? 1 : S / 2;            // threads per row
    static constexpr int CHUNK_T = 32 * VG;                    // threads per chunk
    static constexpr int THREADS = (S == 32) ? 512 : 256;
    static constexpr int CPP = THREADS / CHUNK_T;              // chunks per pass
    static constexpr int CPC = (S >= 16) ? 4 : 8;              // chunks per CTA
    static constexpr int PASSES = CPC / CPP;
};

__device__ __forceinline__ void store_split(float2 *pdf, int64_t i, double v0, double v1, int *bad) {
    bool ok0, ok1;
    const float2 a = df_split_vec(v0, ok0), b = df_split_vec(v1, ok1);
    reinterpret_cast<float4 *>(pdf)[i >> 1] = make_float4(a.x, a.y, b.x, b.y);
    if (!ok0 || !ok1) *bad = 1;
}
__device__ __forceinline__ void store_split1(float2 *pdf, int64_t i, double v, int *bad) {
    bool ok;
    pdf[i] = df_split_vec(v, ok);
    if (!ok) *bad = 1;
}

// ------------------------------------------------------------------ K0
template <int S, int MODE>
__global__ void __launch_bounds__(RowMap<S>::THREADS, 1024 / RowMap<S>::THREADS) cg_init_kernel(CgArgs a) {
    constexpr int G = RowMap<S>::G;
    __shared__ double sm[32][S + 1];
    const int r = threadIdx.x / G, g = threadIdx.x % G;
    const int64_t R = (int64_t)blockIdx.x * 32 + r;
    __shared__ ChunkCols cc;
    const bool staged = stage_chunk(cc, a.row_map, a.col, blockIdx.x, a.n);
    const double2 axv = chunk_spmv<S, double>(cc, staged, a.col, a.vals, a.x, r, g, R < a.n);
    double rr0 = 0.0, rr1 = 0.0, bb0 = 0.0, bb1 = 0.0;
    if constexpr (S == 1) {
        const double ax = axv.x;
        if (R < a.n) {
            const double bv = a.b[R];
            const double res = bv - ax;
            if (g == 0) {
                a.r[R] = res;
                a.p[R] = res;
                if (MODE != 0) store_split1(a.pdf, R, res, &a.st->df_bad_any);
            }
            rr0 = res * res;
            bb0 = bv * bv;
        }
    } else if (R < a.n) {
        const double2 ax = axv;
        const double2 bv = reinterpret_cast<const double2 *>(a.b)[R * G + g];
        const double2 res = make_double2(bv.x - ax.x, bv.y - ax.y);
        reinterpret_cast<double2 *>(a.r)[R * G + g] = res;
        reinterpret_cast<double2 *>(a.p)[R * G + g] = res;
        if (MODE != 0) store_split(a.pdf, R * S + 2 * g, res.x, res.y, &a.st->df_bad_any);
        rr0 = res.x * res.x; rr1 = res.y * res.y;
        bb0 = bv.x * bv.x; bb1 = bv.y * bv.y;
    }
    chunk_tree<S>(sm, rr0, rr1, r, g, a.t2, blockIdx.x, 0);
    chunk_tree<S>(sm, bb0, bb1, r, g, a.t2, blockIdx.x, S);
    if (!dot_tree_propagate(a.t2, blockIdx.x, 1)) return;
    if (threadIdx.x >= 32) return;
    // epilogue: one lane per member (s <= 32); member sums in member order
    const unsigned FULL = 0xffffffffu;
    const int e = threadIdx.x;
    const double *top = a.t2.buf[a.t2.levels];
    CgState *st = a.st;
    const double rr = (e < S) ? ld_cg(top + e) : 0.0, bb = (e < S) ? ld_cg(top + S + e) : 0.0;
    double rsum = 0.0, bsum = 0.0;
    for (int k = 0; k < S; ++k) {
        rsum += __shfl_sync(FULL, rr, k);
        bsum += __shfl_sync(FULL, bb, k);
    }
    const double bn = sqrt(bb);
    int act = 0, zx = 0;
    if (!a.coupled) {
        if (bb == 0.0) zx = 1;
        else act = (sqrt(rr) <= a.tol * bn) ? 0 : 1;
    } else {
        const bool all_zero = (bsum == 0.0);
        act = (all_zero || sqrt(rsum) <= a.tol * sqrt(bsum)) ? 0 : 1;
        zx = all_zero ? 1 : 0;
    }
    int status = ENS_OK;
    if (a.max_iter == 0 && act) { act = 0; status = ENS_ERR_NOT_CONVERGED; }
    if (e < S) {
        st->rho[e] = rr;
        st->bnorm[e] = bn;
        st->alpha[e] = 0.0; st->beta[e] = 0.0; st->relres[e] = 0.0;
        st->iters[e] = 0; st->updx[e] = 0; st->zerox[e] = zx; st->status[e] = status;
        st->active[e] = act;
    } else {
        act = 0; zx = 0;
    }
    const int ac = __popc(__ballot_sync(FULL, act)), zany = __popc(__ballot_sync(FULL, zx));
    if (e == 0) {
        st->bnorm_all = sqrt(bsum);
        st->active_count = ac;
        st->zero_any = zany;
        st->updx_any = 0;
        st->spmv_real = 0;
    }
    __threadfence();
}

// ------------------------------------------------------------------ KZ
template <int S>
__global__ void cg_zero_kernel(CgArgs a) {
    if (ld_cg(&a.st->zero_any) == 0) return;
    const int64_t total = (int64_t)a.n * S;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x)
        if (a.st->zerox[i % S]) a.x[i] = 0.0;
}

// ------------------------------------------------------------------ K1
template <int S, int MODE>
__global__ void __launch_bounds__(RowMap<S>::THREADS, 1536 / RowMap<S>::THREADS) cg_spmv_kernel(CgArgs a) {
    CgState *st = a.st;
    if (ld_cg(&st->active_count) == 0) {
        if (blockIdx.x == 0 && threadIdx.x == 0 && st->updx_any) {
            for (int e = 0; e < S; ++e) st->updx[e] = 0;
            st->updx_any = 0;
        }
        return;
    }
    constexpr int G = RowMap<S>::G;
    __shared__ double sm[32][S + 1];
    const int r = threadIdx.x / G, g = threadIdx.x % G;
    const int64_t R = (int64_t)blockIdx.x * 32 + r;
    // the split form is used unless a vector element fell outside its range
    const int mode = (MODE != 0 && ld_cg(&st->df_bad_any) != 0) ? 0 : MODE;
    __shared__ ChunkCols cc;
    const bool staged = stage_chunk(cc, a.row_map, a.col, blockIdx.x, a.n);
    double2 apv;
    if (MODE == 1 && mode == 1)
        apv = chunk_spmv_df<S, XPre>(cc, staged, a.col, a.vals, a.pdf, r, g, R < a.n);
    else if (MODE == 2 && mode == 2)
        apv = chunk_spmv_split<S, XPre>(cc, staged, a.col, a.vals, a.p, a.pdf, r, g, R < a.n);
    else
        apv = chunk_spmv<S, double>(cc, staged, a.col, a.vals, a.p, r, g, R < a.n);
    double v0 = 0.0, v1 = 0.0;
    if constexpr (S == 1) {
        const double ap = apv.x;
        if (R < a.n) {
            if (g == 0) a.q[R] = ap;
            v0 = ap * a.p[R];
        }
    } else if (R < a.n) {
        const double2 ap = apv;
        reinterpret_cast<double2 *>(a.q)[R * G + g] = ap;
        const double2 pv = reinterpret_cast<const double2 *>(a.p)[R * G + g];
        v0 = ap.x * pv.x;
        v1 = ap.y * pv.y;
    }
    chunk_tree<S>(sm, v0, v1, r, g, a.t1, blockIdx.x, 0);
    if (!dot_tree_propagate(a.t1, blockIdx.x, 1)) return;
    if (threadIdx.x >= 32) return;
    // epilogue: one lane per member
    const unsigned FULL = 0xffffffffu;
    const int e = threadIdx.x;
    const double *top = a.t1.buf[a.t1.levels];
    const double pi = (e < S) ? ld_cg(top + e) : 0.0;
    const double rho = (e < S) ? st->rho[e] : 0.0;
    int act = (e < S) ? st->active[e] : 0;
    if (a.coupled) {
        double pis = 0.0, rhos = 0.0;
        for (int k = 0; k < S; ++k) {
            pis += __shfl_sync(FULL, pi, k);
            rhos += __shfl_sync(FULL, rho, k);
        }
        const bool bad = !(pis > 0.0) || !isfinite(pis);
        if (act) {
            if (bad) { act = 0; st->status[e] = ENS_ERR_BREAKDOWN; }
            else st->alpha[e] = rhos / pis;
        }
    } else if (act) {
        if (!(pi > 0.0) || !isfinite(pi)) { act = 0; st->status[e] = ENS_ERR_BREAKDOWN; }
        else st->alpha[e] = rho / pi;
    }
    if (e < S) {
        st->active[e] = act;
        st->updx[e] = 0;  // consumed by the previous K3
    }
    const int ac = __popc(__ballot_sync(FULL, act));
    if (e == 0) {
        st->spmv_real += 1;
        st->updx_any = 0;
        st->active_count = ac;
    }
    __threadfence();
}

// ------------------------------------------------------------------ K2
template <int S>
__global__ void __launch_bounds__(VecMap<S>::THREADS) cg_resid_kernel(CgArgs a) {
    using VM = VecMap<S>;
    if (ld_cg(&a.st->active_count) == 0) return;
    constexpr int VG = VM::VG;
    const int cip = threadIdx.x / VM::CHUNK_T, lt = threadIdx.x % VM::CHUNK_T;
    const int r = lt / VG, g = lt % VG;
    const CgState *cs = a.st;
    const int m = (S == 1) ? 0 : 2 * g;
    const bool act0 = cs->active[m];
    const bool act1 = (S == 1) ? false : (bool)cs->active[m + 1];
    const double al0 = cs->alpha[m];
    const double al1 = (S == 1) ? 0.0 : cs->alpha[m + 1];
    __shared__ double sm[VM::CPC][32][S + 1];   // per-row products of every chunk
    const int64_t first_chunk = (int64_t)blockIdx.x * VM::CPC;
#pragma unroll
    for (int pass = 0; pass < VM::PASSES; ++pass) {
        const int c = pass * VM::CPP + cip;
        const int64_t R = (first_chunk + c) * 32 + r;
        double v0 = 0.0, v1 = 0.0;
        if (R < a.n) {
            if constexpr (S == 1) {
                double rv = a.r[R];
                if (act0) { rv = fma(-al0, a.q[R], rv); a.r[R] = rv; }
                v0 = rv * rv;
            } else {
                double2 rv = reinterpret_cast<const double2 *>(a.r)[R * VG + g];
                const double2 qv = reinterpret_cast<const double2 *>(a.q)[R * VG + g];
                if (act0) rv.x = fma(-al0, qv.x, rv.x);
                if (act1) rv.y = fma(-al1, qv.y, rv.y);
                if (act0 || act1) reinterpret_cast<double2 *>(a.r)[R * VG + g] = rv;
                v0 = rv.x * rv.x;
                v1 = rv.y * rv.y;
            }
        }
        sm[c][r][m] = v0;
        if constexpr (S > 1) sm[c][r][m + 1] = v1;
    }
    __syncthreads();
    // halving tree over the 32 rows of every chunk, all members packed
#pragma unroll
    for (int h = 16; h >= 1; h >>= 1) {
        for (int it = threadIdx.x; it < VM::CPC * h * S; it += VM::THREADS) {
            const int c = it / (h * S), rem = it % (h * S), i = rem / S, e = rem % S;
            sm[c][i][e] += sm[c][i + h][e];
        }
        __syncthreads();
    }
    for (int it = threadIdx.x; it < VM::CPC * S; it += VM::THREADS) {
        const int c = it / S, e = it % S;
        const int64_t ch = first_chunk + c;
        if (ch < a.t1.count[1]) a.t1.buf[1][ch * S + e] = sm[c][0][e];
    }
    const int nitems = (int)min((int64_t)VM::CPC, a.t1.count[1] - first_chunk);
    if (!dot_tree_propagate(a.t1, first_chunk, nitems)) return;
    if (threadIdx.x >= 32) return;
    // epilogue: one lane per member
    const unsigned FULL = 0xffffffffu;
    const int e = threadIdx.x;
    const double *top = a.t1.buf[a.t1.levels];
    CgState *st = a.st;
    const double rn = (e < S) ? ld_cg(top + e) : 0.0;
    const double rho = (e < S) ? st->rho[e] : 0.0;
    int act = (e < S) ? st->active[e] : 0, ux = 0;
    int it = (e < S) ? st->iters[e] : 0;
    bool conv_all = false;
    double rns = 0.0, ros = 0.0;
    if (a.coupled) {
        for (int k = 0; k < S; ++k) {
            rns += __shfl_sync(FULL, rn, k);
            ros += __shfl_sync(FULL, rho, k);
        }
        conv_all = sqrt(rns) <= a.tol * st->bnorm_all;
    }
    if (act) {
        it += 1;
        ux = 1;
        const bool conv = a.coupled ? conv_all : (sqrt(rn) <= a.tol * st->bnorm[e]);
        if (conv) { act = 0; st->status[e] = ENS_OK; }
        else if (it >= a.max_iter) { act = 0; st->status[e] = ENS_ERR_NOT_CONVERGED; }
        else st->beta[e] = a.coupled ? rns / ros : rn / rho;
    }
    if (e < S) {
        if (a.coupled || ux) st->rho[e] = rn;
        st->iters[e] = it;
        st->updx[e] = ux;
        st->active[e] = act;
    }
    const int ac = __popc(__ballot_sync(FULL, act)), uany = __popc(__ballot_sync(FULL, ux));
    if (e == 0) {
        st->active_count = ac;
        st->updx_any = uany;
    }
    __threadfence();
}

// ------------------------------------------------------------------ K3
template <int S, int MODE>
__global__ void __launch_bounds__(VecMap<S>::THREADS) cg_update_kernel(CgArgs a) {
    using VM = VecMap<S>;
    CgState *st = a.st;
    if (ld_cg(&st->updx_any) == 0) return;
    constexpr int VG = VM::VG;
    const int cip = threadIdx.x / VM::CHUNK_T, lt = threadIdx.x % VM::CHUNK_T;
    const int r = lt / VG, g = lt % VG;
    const int m = (S == 1) ? 0 : 2 * g;
    const bool ux0 = st->updx[m], ac0 = st->active[m];
    const bool ux1 = (S == 1) ? false : (bool)st->updx[m + 1];
    const bool ac1 = (S == 1) ? false : (bool)st->active[m + 1];
    const double al0 = st->alpha[m], be0 = st->beta[m];
    const double al1 = (S == 1) ? 0.0 : st->alpha[m + 1], be1 = (S == 1) ? 0.0 : st->beta[m + 1];
    const int64_t first_chunk = (int64_t)blockIdx.x * VM::CPC;
#pragma unroll 2
    for (int pass = 0; pass < VM::PASSES; ++pass) {
        const int64_t R = (first_chunk + pass * VM::CPP + cip) * 32 + r;
        if (R >= a.n) continue;
        if constexpr (S == 1) {
            const double pv = a.p[R];
            if (ux0) a.x[R] = fma(al0, pv, a.x[R]);
            if (ac0) {
                const double pn = fma(be0, pv, a.r[R]);
                a.p[R] = pn;
                if (MODE != 0) store_split1(a.pdf, R, pn, &st->df_bad_any);
            }
        } else {
            const double2 pv = reinterpret_cast<const double2 *>(a.p)[R * VG + g];
            if (ux0 || ux1) {
                double2 xv = reinterpret_cast<const double2 *>(a.x)[R * VG + g];
                if (ux0) xv.x = fma(al0, pv.x, xv.x);
                if (ux1) xv.y = fma(al1, pv.y, xv.y);
                reinterpret_cast<double2 *>(a.x)[R * VG + g] = xv;
            }
            if (ac0 || ac1) {
                const double2 rv = reinterpret_cast<const double2 *>(a.r)[R * VG + g];
                double2 pn = pv;
                if (ac0) pn.x = fma(be0, pv.x, rv.x);
                if (ac1) pn.y = fma(be1, pv.y, rv.y);
                reinterpret_cast<double2 *>(a.p)[R * VG + g] = pn;
                if (MODE != 0) store_split(a.pdf, R * S + m, pn.x, pn.y, &st->df_bad_any);
            }
        }
    }
}

// ------------------------------------------------------------------ KF
template <int S>
__global__ void __launch_bounds__(RowMap<S>::THREADS, 1024 / RowMap<S>::THREADS) cg_final_kernel(CgArgs a) {
    constexpr int G = RowMap<S>::G;
    __shared__ double sm[32][S + 1];
    const int r = threadIdx.x / G, g = threadIdx.x % G;
    const int64_t R = (int64_t)blockIdx.x * 32 + r;
    __shared__ ChunkCols cc;
    const bool staged = stage_chunk(cc, a.row_map, a.col, blockIdx.x, a.n);
    const double2 axv = chunk_spmv<S, double>(cc, staged, a.col, a.vals, a.x, r, g, R < a.n);
    double v0 = 0.0, v1 = 0.0;
    if constexpr (S == 1) {
        const double ax = axv.x;
        if (R < a.n) { const double res = a.b[R] - ax; v0 = res * res; }
    } else if (R < a.n) {
        const double2 ax = axv;
        const double2 bv = reinterpret_cast<const double2 *>(a.b)[R * G + g];
        const double rx = bv.x - ax.x, ry = bv.y - ax.y;
        v0 = rx * rx;
        v1 = ry * ry;
    }
    chunk_tree<S>(sm, v0, v1, r, g, a.t1, blockIdx.x, 0);
    if (!dot_tree_propagate(a.t1, blockIdx.x, 1)) return;
    const int e = threadIdx.x;
    if (e >= S) return;
    const double *top = a.t1.buf[a.t1.levels];
    const double bn = a.st->bnorm[e];
    a.st->relres[e] = (bn > 0.0) ? sqrt(ld_cg(top + e)) / bn : 0.0;
    __threadfence();
}

// ------------------------------------------------------------ host side
static size_t align256(size_t x) { return (x + 255) / 256 * 256; }

static size_t cg_bytes(int64_t n, int s) {
    return align256(sizeof(CgState)) + 4 * align256(sizeof(double) * (size_t)n * s) +
           dot_tree_bytes(n, s) + dot_tree_bytes(n, 2 * s);
}

template <int S, int MODE>
struct CgKernels {
    static unsigned vec_grid(const CgArgs &a) {
        return (unsigned)((a.t1.count[1] + VecMap<S>::CPC - 1) / VecMap<S>::CPC);
    }
    static void init(const CgArgs &a, unsigned grid, cudaStream_t st) {
        cg_init_kernel<S, MODE><<<grid, RowMap<S>::THREADS, 0, st>>>(a);
        cg_zero_kernel<S><<<152 * 2, 256, 0, st>>>(a);
    }
    static void spmv(const CgArgs &a, unsigned grid, cudaStream_t st) {
        cg_spmv_kernel<S, MODE><<<grid, RowMap<S>::THREADS, 0, st>>>(a);
    }
    static void resid(const CgArgs &a, unsigned, cudaStream_t st) {
        cg_resid_kernel<S><<<vec_grid(a), VecMap<S>::THREADS, 0, st>>>(a);
    }
    static void update(const CgArgs &a, unsigned, cudaStream_t st) {
        cg_update_kernel<S, MODE><<<vec_grid(a), VecMap<S>::THREADS, 0, st>>>(a);
    }
    static void final_(const CgArgs &a, unsigned grid, cudaStream_t st) {
        cg_final_kernel<S><<<grid, RowMap<S>::THREADS, 0, st>>>(a);
    }
};

struct CgHostOut {
    int32_t *iters;
    double *relres;
    int32_t *status;
    ens_cg_stats *stats;
};

template <int S, int MODE>
static int cg_run(const ens_graph *g, const double *vals, const double *b, double *x, double tol,
                  int max_iter, int flags, int check_every, void *work, CgHostOut out,
                  cudaStream_t st) {
    using K = CgKernels<S, MODE>;
    const int64_t n = g->num_rows;
    char *w = static_cast<char *>(work);
    CgArgs a;
    a.n = g->num_rows;
    a.row_map = g->row_map;
    a.col = g->col_entry;
    a.vals = vals;
    a.b = b;
    a.x = x;
    a.st = reinterpret_cast<CgState *>(w);
    w += align256(sizeof(CgState));
    a.r = reinterpret_cast<double *>(w); w += align256(sizeof(double) * (size_t)n * S);
    a.p = reinterpret_cast<double *>(w); w += align256(sizeof(double) * (size_t)n * S);
    a.q = reinterpret_cast<double *>(w); w += align256(sizeof(double) * (size_t)n * S);
    a.pdf = reinterpret_cast<float2 *>(w); w += align256(sizeof(double) * (size_t)n * S);
    dot_tree_layout(&a.t1, n, S, w);
    w += dot_tree_bytes(n, S);
    dot_tree_layout(&a.t2, n, 2 * S, w);
    a.tol = tol;
    a.max_iter = max_iter;
    a.coupled = (flags & ENS_CG_COUPLED) ? 1 : 0;
    const unsigned grid = (unsigned)a.t1.count[1];
    int rc;
    if ((rc = dot_tree_clear(a.t1, st))) return rc;
    if ((rc = dot_tree_clear(a.t2, st))) return rc;
    ENS_CUDA_TRY(cudaMemsetAsync(a.st, 0, sizeof(CgState), st));

    const bool timing = (flags & ENS_CG_TIME_SPMV) != 0;
    const bool use_graph = (flags & ENS_CG_GRAPH) != 0 && !timing;
    int launches = 0, polls = 0;
    std::vector<cudaEvent_t> ev;
    std::vector<float> spmv_ms;
    if (timing) {
        ev.resize(2 * (size_t)check_every);
        for (auto &e : ev) ENS_CUDA_TRY(cudaEventCreate(&e));
    }
    auto destroy_events = [&]() { for (auto &e : ev) cudaEventDestroy(e); };

    K::init(a, grid, st);
    launches += 2;
    ENS_LAUNCH_CHECK("cg_init_kernel");

    cudaGraphExec_t gexec = nullptr;
    cudaGraph_t graph = nullptr;
    if (use_graph) {
        // capture on a private stream (the legacy default stream cannot be
        // captured); the graph is then launched on the caller's stream
        cudaStream_t cap;
        ENS_CUDA_TRY(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
        cudaError_t ce = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
        if (ce == cudaSuccess) {
            for (int i = 0; i < check_every; ++i) {
                K::spmv(a, grid, cap);
                K::resid(a, grid, cap);
                K::update(a, grid, cap);
            }
            ce = cudaStreamEndCapture(cap, &graph);
        }
        cudaStreamDestroy(cap);
        if (ce != cudaSuccess) return cuda_fail(ce, "cg iteration graph capture");
        ce = cudaGraphInstantiate(&gexec, graph, 0);
        if (ce != cudaSuccess) { cudaGraphDestroy(graph); return cuda_fail(ce, "cudaGraphInstantiate"); }
    }

    int32_t flags_h[2];
    int iter_blocks = 0;
    const int max_blocks = max_iter / check_every + 3;
    rc = ENS_OK;
    while (iter_blocks < max_blocks) {
        if (use_graph) {
            cudaError_t ce = cudaGraphLaunch(gexec, st);
            if (ce != cudaSuccess) { rc = cuda_fail(ce, "cudaGraphLaunch"); break; }
        } else {
            for (int i = 0; i < check_every; ++i) {
                if (timing) cudaEventRecord(ev[2 * i], st);
                K::spmv(a, grid, st);
                if (timing) cudaEventRecord(ev[2 * i + 1], st);
                K::resid(a, grid, st);
                K::update(a, grid, st);
            }
        }
        launches += 3 * check_every;
        ++iter_blocks;
        cudaError_t ce = cudaGetLastError();
        if (ce != cudaSuccess) { rc = cuda_fail(ce, "cg iteration launch"); break; }
        ce = cudaMemcpyAsync(flags_h, &a.st->active_count, 2 * sizeof(int32_t), cudaMemcpyDeviceToHost, st);
        if (ce == cudaSuccess) ce = cudaStreamSynchronize(st);
        if (ce != cudaSuccess) { rc = cuda_fail(ce, "cg convergence poll"); break; }
        ++polls;
        if (timing) {
            for (int i = 0; i < check_every; ++i) {
                float ms = 0.f;
                cudaEventElapsedTime(&ms, ev[2 * i], ev[2 * i + 1]);
                spmv_ms.push_back(ms);
            }
        }
        if (flags_h[0] == 0 && flags_h[1] == 0) break;
    }
    if (gexec) cudaGraphExecDestroy(gexec);
    if (graph) cudaGraphDestroy(graph);
    if (rc != ENS_OK) { destroy_events(); return rc; }

    K::final_(a, grid, st);
    ++launches;
    ENS_LAUNCH_CHECK("cg_final_kernel");
    CgState hs;
    ENS_CUDA_TRY(cudaMemcpyAsync(&hs, a.st, sizeof(CgState), cudaMemcpyDeviceToHost, st));
    ENS_CUDA_TRY(cudaStreamSynchronize(st));
    destroy_events();
    int maxit = 0, first_bad = ENS_OK;
    for (int e = 0; e < S; ++e) {
        if (out.iters) out.iters[e] = hs.iters[e];
        if (out.relres) out.relres[e] = hs.relres[e];
        if (out.status) out.status[e] = hs.status[e];
        maxit = hs.iters[e] > maxit ? hs.iters[e] : maxit;
        if (hs.status[e] != ENS_OK && first_bad == ENS_OK) first_bad = hs.status[e];
    }
    if (out.stats) {
        out.stats->iterations = maxit;
        out.stats->kernel_launches = launches;
        out.stats->host_checks = polls;
        out.stats->spmv_launches = 0;
        out.stats->spmv_ms = 0.0;
        if (timing) {
            const int real = hs.spmv_real < (int)spmv_ms.size() ? hs.spmv_real : (int)spmv_ms.size();
            double tot = 0.0;
            for (int i = 0; i < real; ++i) tot += spmv_ms[i];
            out.stats->spmv_launches = real;
            out.stats->spmv_ms = tot;
        }
    }
    if (first_bad != ENS_OK)
        set_error("ens_cg: member status %d (%s)", first_bad, ens_status_string(first_bad));
    return first_bad;
}

template <int S>
static int cg_dispatch_df(const ens_graph *g, const double *vals, const double *b, double *x,
                          double tol, int max_iter, int flags, int check_every, void *work,
                          CgHostOut out, cudaStream_t st) {
    if (flags & ENS_CG_SPLIT64)
        return cg_run<S, 2>(g, vals, b, x, tol, max_iter, flags, check_every, work, out, st);
    if (flags & ENS_CG_DF64)
        return cg_run<S, 1>(g, vals, b, x, tol, max_iter, flags, check_every, work, out, st);
    return cg_run<S, 0>(g, vals, b, x, tol, max_iter, flags, check_every, work, out, st);
}

}  // namespace ens

using namespace ens;

extern "C" int ens_cg_workspace_size(int32_t num_rows, int s, size_t *bytes) {
    if (num_rows < 0) return fail(ENS_ERR_ARG, "num_rows < 0");
    if (!supported_s(s)) return fail(ENS_ERR_UNSUPPORTED, "ensemble size s=%d not in {1,4,8,16,32}", s);
    if (!bytes) return fail(ENS_ERR_ARG, "bytes is NULL");
    *bytes = cg_bytes(num_rows, s);
    return ENS_OK;
}

extern "C" int ens_cg(const ens_graph *graph, int s, const double *values, const double *b,
                      double *x, double tol, int max_iter, int flags, int check_every, void *work,
                      size_t work_bytes, int32_t *iters_host, double *relres_host,
                      int32_t *status_host, ens_cg_stats *stats_host, void *stream) {
    int rc = check_graph(graph);
    if (rc) return rc;
    if (!supported_s(s)) return fail(ENS_ERR_UNSUPPORTED, "ensemble size s=%d not in {1,4,8,16,32}", s);
    if (graph->num_rows == 0) return fail(ENS_ERR_ARG, "empty graph");
    if (!values || !b || !x || !work) return fail(ENS_ERR_ARG, "NULL values/b/x/work");
    if (!(tol >= 0.0) || max_iter < 0 || check_every < 1)
        return fail(ENS_ERR_ARG, "tol=%g max_iter=%d check_every=%d", tol, max_iter, check_every);
    if (!aligned16(work) || (s > 1 && (!aligned16(values) || !aligned16(b) || !aligned16(x))))
        return fail(ENS_ERR_ALIGN, "values/b/x/work must be 16-byte aligned");
    const size_t need = cg_bytes(graph->num_rows, s);
    if (work_bytes < need) return fail(ENS_ERR_WORKSPACE, "cg workspace %zu < %zu bytes", work_bytes, need);
    CgHostOut out{iters_host, relres_host, status_host, stats_host};
    cudaStream_t st = as_stream(stream);
    switch (s) {
        case 1: return cg_dispatch_df<1>(graph, values, b, x, tol, max_iter, flags, check_every, work, out, st);
        case 4: return cg_dispatch_df<4>(graph, values, b, x, tol, max_iter, flags, check_every, work, out, st);
        case 8: return cg_dispatch_df<8>(graph, values, b, x, tol, max_iter, flags, check_every, work, out, st);
        case 16: return cg_dispatch_df<16>(graph, values, b, x, tol, max_iter, flags, check_every, work, out, st);
        default: return cg_dispatch_df<32>(graph, values, b, x, tol, max_iter, flags, check_every, work, out, st);
    }
}
