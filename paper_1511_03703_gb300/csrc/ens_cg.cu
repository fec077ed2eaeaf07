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
#include <stdlib.h>

#include <vector>

#include "ens_spmv.cuh"

namespace ens {

struct CgState {
    double rho[32], alpha[32], beta[32], bnorm[32], relres[32];
    int active[32], updx[32], zerox[32], iters[32], status[32], fb[32];
    int active_count, updx_any, zero_any, spmv_real;
    int df_bad_any, fb_count, pad1, pad2;
    double bnorm_all;
};

struct CgArgs {
    int32_t n;
    const int32_t *row_map;
    const int32_t *col;
    const double *vals;
    const float2 *vdf;  // values pre-split into float pairs (MODE 3), else NULL
    const double *b;
    double *x, *r, *p, *q;
    float2 *pdf;  // p split into float pairs (df modes)
    CgState *st;
    DotTree t1;   // width s
    DotTree t2;   // width 2s
    double tol;
    int max_iter;
    int coupled;
    int fallback;  // restart from x = 0 members whose ||b - A x0|| >= ||b||
    int x0_zero;   // the caller states x0 = 0: r0 = b without the initial SpMV
    uint32_t pf_cap;       // bytes of each chunk's value block prefetched into L2 by K1
    uint64_t val_bytes;    // size of the value array read by K1 (8 bytes per value in every form)
};

// mapping of the streaming vector kernels (K2, K3): a CTA of TH threads owns
// CPC chunks, CPP of them at a time
template <int S, int TH = (S == 32) ? 512 : 256>
struct VecMap {
    static constexpr int VG = (S == 1) ? 1 : S / 2;            // threads per row
    static constexpr int CHUNK_T = 32 * VG;                    // threads per chunk
    static constexpr int THREADS = TH;
    static constexpr int CPP = THREADS / CHUNK_T;              // chunks per pass
    static constexpr int CPC0 = (S >= 16) ? 4 : 8;
    static constexpr int CPC = (CPC0 > CPP) ? CPC0 : CPP;      // chunks per CTA
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
    double2 axv = make_double2(0.0, 0.0);  // A x0 = 0 when the caller states x0 = 0
    if (!a.x0_zero) {
        const bool staged = stage_chunk(cc, a.row_map, a.col, blockIdx.x, a.n);
        axv = chunk_spmv<S, double>(cc, staged, a.col, a.vals, a.x, r, g, R < a.n);
    }
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
    const double rrx = (e < S) ? ld_cg(top + e) : 0.0, bb = (e < S) ? ld_cg(top + S + e) : 0.0;
    // zero-guess fallback: a start no better than x = 0 (or not finite) is
    // replaced by x = 0, r = p = b, whose r.r is b.b in the same tree order
    const bool fbk = a.fallback && e < S && bb != 0.0 && !(rrx < bb);
    const double rr = fbk ? bb : rrx;
    double rsum = 0.0, bsum = 0.0;
    for (int k = 0; k < S; ++k) {
        rsum += __shfl_sync(FULL, rr, k);
        bsum += __shfl_sync(FULL, bb, k);
    }
    const double bn = sqrt(bb);
    int act = 0, zx = fbk ? 1 : 0;
    if (!a.coupled) {
        if (bb == 0.0) zx = 1;
        else act = (sqrt(rr) <= a.tol * bn) ? 0 : 1;
    } else {
        const bool all_zero = (bsum == 0.0);
        act = (all_zero || sqrt(rsum) <= a.tol * sqrt(bsum)) ? 0 : 1;
        zx = (all_zero || fbk) ? 1 : 0;
    }
    int status = ENS_OK;
    if (a.max_iter == 0 && act) { act = 0; status = ENS_ERR_NOT_CONVERGED; }
    if (e < S) {
        st->rho[e] = rr;
        st->bnorm[e] = bn;
        st->alpha[e] = 0.0; st->beta[e] = 0.0; st->relres[e] = 0.0;
        st->iters[e] = 0; st->updx[e] = 0; st->zerox[e] = zx; st->status[e] = status;
        st->active[e] = act;
        st->fb[e] = fbk ? 1 : 0;
    } else {
        act = 0; zx = 0;
    }
    const int ac = __popc(__ballot_sync(FULL, act)), zany = __popc(__ballot_sync(FULL, zx));
    const int nfb = __popc(__ballot_sync(FULL, fbk));
    if (e == 0) {
        st->bnorm_all = sqrt(bsum);
        st->active_count = ac;
        st->zero_any = zany;
        st->fb_count = nfb;
        st->updx_any = 0;
        st->spmv_real = 0;
    }
    __threadfence();
}

// ------------------------------------------------------------------ KZ
// x = 0 for members with b = 0 or a rejected start; for the latter also
// r = p = b (and the split copy of p)
template <int S, int MODE>
__global__ void cg_zero_kernel(CgArgs a) {
    if (ld_cg(&a.st->zero_any) == 0) return;
    const int64_t total = (int64_t)a.n * S;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int e = (int)(i % S);
        if (!a.st->zerox[e]) continue;
        a.x[i] = 0.0;
        if (a.st->fb[e]) {
            const double bv = a.b[i];
            a.r[i] = bv;
            a.p[i] = bv;
            if (MODE != 0) store_split1(a.pdf, i, bv, &a.st->df_bad_any);
        }
    }
}

// ------------------------------------------------------------------ K1
// Body of the batched kernel: NSUB chunks of one ensemble per CTA, each on
// its own thread group.  Its arithmetic is that of cg_spmv_kernel below (kept
// as a separate copy because the shared form needs more registers there).
template <int S, int NSUB>
struct K1Smem {
    double sm[NSUB][32][S + 1];
    ChunkCols cc[NSUB];
};

template <int S, int MODE, int NSUB>
__device__ __forceinline__ void k1_body(const CgArgs &a, const int cta, K1Smem<S, NSUB> &sh) {
    CgState *st = a.st;
    if (ld_cg(&st->active_count) == 0) {
        if (cta == 0 && threadIdx.x == 0 && st->updx_any) {
            for (int e = 0; e < S; ++e) st->updx[e] = 0;
            st->updx_any = 0;
        }
        return;
    }
    constexpr int G = RowMap<S>::G, T = RowMap<S>::THREADS;
    const int sub = (NSUB == 1) ? 0 : (int)threadIdx.x / T;
    const int ltid = (NSUB == 1) ? (int)threadIdx.x : (int)threadIdx.x % T;
    const int r = ltid / G, g = ltid % G;
#define K1_CHUNK ((int64_t)cta * NSUB + sub)
    const int64_t chunk = K1_CHUNK;
    const bool valid = chunk * 32 + r < a.n;
    // the split / double-float forms are used unless a vector element fell outside their range
    const int mode = (MODE != 0 && ld_cg(&st->df_bad_any) != 0) ? 0 : MODE;
    const bool staged = (NSUB == 1) ? stage_chunk(sh.cc[0], a.row_map, a.col, chunk, a.n)
                                    : stage_chunk_sub(sh.cc[sub], a.row_map, a.col, chunk, a.n, ltid, T);
    double2 apv;
    if (MODE == 1 && mode == 1)
        apv = chunk_spmv_df<S, XPre>(sh.cc[sub], staged, a.col, a.vals, a.pdf, r, g, valid);
    else if (MODE == 2 && mode == 2)
        apv = chunk_spmv_split<S, XPre>(sh.cc[sub], staged, a.col, a.vals, a.p, a.pdf, r, g, valid);
    else
        apv = chunk_spmv<S, double>(sh.cc[sub], staged, a.col, a.vals, a.p, r, g, valid);
    double v0 = 0.0, v1 = 0.0;
    const int64_t R = K1_CHUNK * 32 + r;
    if constexpr (S == 1) {
        if (valid) {
            if (g == 0) a.q[R] = apv.x;
            v0 = apv.x * a.p[R];
        }
    } else if (valid) {
        reinterpret_cast<double2 *>(a.q)[R * G + g] = apv;
        const double2 pv = reinterpret_cast<const double2 *>(a.p)[R * G + g];
        v0 = apv.x * pv.x;
        v1 = apv.y * pv.y;
    }
    if constexpr (NSUB == 1) chunk_tree<S>(sh.sm[0], v0, v1, r, g, a.t1, K1_CHUNK, 0);
    else chunk_tree_sub<S>(sh.sm[sub], v0, v1, r, g, a.t1, K1_CHUNK, 0, ltid, T);
    const int nitems = (NSUB == 1) ? 1 : (int)min((int64_t)NSUB, a.t1.count[1] - (int64_t)cta * NSUB);
    if (!dot_tree_propagate(a.t1, (int64_t)cta * NSUB, nitems)) return;
#undef K1_CHUNK
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

// single-ensemble K1 (one chunk per CTA); same arithmetic as k1_body
#ifndef ENS_K1_DFV_THREADS_PER_SM
#define ENS_K1_DFV_THREADS_PER_SM 1536
#endif
template <int S, int MODE>
struct K1Occ {
    static constexpr int THREADS_PER_SM = (MODE == 3) ? ENS_K1_DFV_THREADS_PER_SM : 1536;
};

template <int S, int MODE>
__global__ void __launch_bounds__(RowMap<S>::THREADS, K1Occ<S, MODE>::THREADS_PER_SM / RowMap<S>::THREADS)
    cg_spmv_kernel(CgArgs a) {
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
    const void *vblock = (MODE == 3) ? static_cast<const void *>(a.vdf) : static_cast<const void *>(a.vals);
    const bool staged = stage_chunk_pf(cc, a.row_map, a.col, blockIdx.x, a.n, vblock, S * 8u, a.val_bytes,
                                       a.pf_cap);
    double2 apv;
    if (MODE == 1 && mode == 1)
        apv = chunk_spmv_df<S, XPre>(cc, staged, a.col, a.vals, a.pdf, r, g, R < a.n);
    else if (MODE == 3 && mode == 3)
        apv = chunk_spmv_dfv<S>(cc, staged, a.col, a.vdf, a.vals, a.pdf, r, g, R < a.n);
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
// v*v of an FP64 value as an unevaluated float pair: v split by truncation
// into hi + lo (47 bits), hi*hi exact by FMA error recovery, 2 hi lo added to
// the error term (lo*lo, below 2^-46 |v*v|, is dropped); values outside the
// split range square in FP64 and round to a pair (out of line, so that the
// FP64 instructions stay off the common path)
__device__ __noinline__ float2 df_square_wide(double v) {
    const double q = v * v;
    const float qh = (float)q;
    return make_float2(qh, (float)(q - (double)qh));
}

__device__ __forceinline__ float2 df_square(double v) {
    float hi, lo;
    if (!df_split_trunc(v, hi, lo)) return df_square_wide(v);
    const float p = __fmul_rn(hi, hi);
    float e = __fmaf_rn(hi, hi, -p);
    e = __fmaf_rn(2.0f * hi, lo, e);
    return make_float2(p, e);
}

// (a.x + a.y) + (b.x + b.y) as a float pair: TwoSum of the leading parts,
// the trailing parts and the rounding error summed
__device__ __forceinline__ float2 df_add(float2 a, float2 b) {
    float s, t;
    two_sum(a.x, b.x, s, t);
    return make_float2(s, __fadd_rn(__fadd_rn(a.y, b.y), t));
}

template <int S, int TH>
__device__ __forceinline__ void k2_body(const CgArgs &a, int cta,
                                        double (*sm)[32][S + 1] /* [CPC][32][S+1] */) {
    using VM = VecMap<S, TH>;
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
    const int64_t first_chunk = (int64_t)cta * VM::CPC;
    // r.r: squares and the chunk's 32-row tree in double-float on the FP32
    // pipe (the FP64 pipe keeps only the r update); the chunk sums enter the
    // FP64 dot tree above the chunk
    float2(*sf)[32][S + 1] = reinterpret_cast<float2(*)[32][S + 1]>(sm);
#pragma unroll
    for (int pass = 0; pass < VM::PASSES; ++pass) {
        const int c = pass * VM::CPP + cip;
        const int64_t R = (first_chunk + c) * 32 + r;
        float2 v0 = make_float2(0.f, 0.f), v1 = make_float2(0.f, 0.f);
        if (R < a.n) {
            if constexpr (S == 1) {
                double rv = a.r[R];
                if (act0) { rv = fma(-al0, a.q[R], rv); a.r[R] = rv; }
                v0 = df_square(rv);
            } else {
                double2 rv = reinterpret_cast<const double2 *>(a.r)[R * VG + g];
                const double2 qv = reinterpret_cast<const double2 *>(a.q)[R * VG + g];
                if (act0) rv.x = fma(-al0, qv.x, rv.x);
                if (act1) rv.y = fma(-al1, qv.y, rv.y);
                if (act0 || act1) reinterpret_cast<double2 *>(a.r)[R * VG + g] = rv;
                v0 = df_square(rv.x);
                v1 = df_square(rv.y);
            }
        }
        sf[c][r][m] = v0;
        if constexpr (S > 1) sf[c][r][m + 1] = v1;
    }
    __syncthreads();
    // halving tree over the 32 rows of every chunk, all members packed
#pragma unroll
    for (int h = 16; h >= 1; h >>= 1) {
        for (int it = threadIdx.x; it < VM::CPC * h * S; it += VM::THREADS) {
            const int c = it / (h * S), rem = it % (h * S), i = rem / S, e = rem % S;
            sf[c][i][e] = df_add(sf[c][i][e], sf[c][i + h][e]);
        }
        __syncthreads();
    }
    for (int it = threadIdx.x; it < VM::CPC * S; it += VM::THREADS) {
        const int c = it / S, e = it % S;
        const int64_t ch = first_chunk + c;
        if (ch < a.t1.count[1]) a.t1.buf[1][ch * S + e] = f2d_exact(sf[c][0][e].x) + f2d_exact(sf[c][0][e].y);
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
template <int S, int MODE, int TH>
__device__ __forceinline__ void k3_body(const CgArgs &a, int cta) {
    using VM = VecMap<S, TH>;
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
    const int64_t first_chunk = (int64_t)cta * VM::CPC;
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

template <int S>
__global__ void __launch_bounds__(VecMap<S>::THREADS) cg_resid_kernel(CgArgs a) {
    __shared__ double sm[VecMap<S>::CPC][32][S + 1];   // per-row products of every chunk
    k2_body<S, VecMap<S>::THREADS>(a, blockIdx.x, sm);
}

template <int S, int MODE>
__global__ void __launch_bounds__(VecMap<S>::THREADS) cg_update_kernel(CgArgs a) {
    k3_body<S, MODE, VecMap<S>::THREADS>(a, blockIdx.x);
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

// Bytes of each chunk's value block that K1 prefetches into L2 at its start:
// the whole block for the pre-split double-float form, whose SpMV is bound by
// memory latency without it (measured on the 64^3 mesh: 0.425 -> 0.372 ms at
// s = 32); none for the FP64-pipe-bound forms.  ENS_L2_PREFETCH (bytes)
// overrides both.
static uint32_t l2_prefetch_cap(int mode) {
    static const long long env = [] {
        const char *e = getenv("ENS_L2_PREFETCH");
        return e ? (long long)strtoull(e, nullptr, 10) : -1LL;
    }();
    if (env >= 0) return (uint32_t)(env > 0xffffffffLL ? 0xffffffffLL : env);
    return mode == 3 ? 0xffffffffu : 0u;
}

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
        cg_zero_kernel<S, MODE><<<152 * 2, 256, 0, st>>>(a);
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
static int cg_run(const ens_graph *g, const double *vals, const float2 *vdf, const double *b, double *x,
                  double tol, int max_iter, int flags, int check_every, void *work, CgHostOut out,
                  cudaStream_t st) {
    using K = CgKernels<S, MODE>;
    const int64_t n = g->num_rows;
    char *w = static_cast<char *>(work);
    CgArgs a;
    a.n = g->num_rows;
    a.row_map = g->row_map;
    a.col = g->col_entry;
    a.vals = vals;
    a.vdf = vdf;
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
    a.fallback = (flags & ENS_CG_GUESS_FALLBACK) ? 1 : 0;
    a.x0_zero = (flags & ENS_CG_X0_ZERO) ? 1 : 0;
    a.pf_cap = l2_prefetch_cap(MODE);
    a.val_bytes = (uint64_t)g->num_entries * S * 8u;
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
        out.stats->guess_fallbacks = hs.fb_count;
        out.stats->reserved = 0;
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
static int cg_dispatch_df(const ens_graph *g, const double *vals, const float2 *vdf, const double *b,
                          double *x, double tol, int max_iter, int flags, int check_every, void *work,
                          CgHostOut out, cudaStream_t st) {
    if (vdf) return cg_run<S, 3>(g, vals, vdf, b, x, tol, max_iter, flags, check_every, work, out, st);
    if (flags & ENS_CG_SPLIT64)
        return cg_run<S, 2>(g, vals, nullptr, b, x, tol, max_iter, flags, check_every, work, out, st);
    if (flags & ENS_CG_DF64)
        return cg_run<S, 1>(g, vals, nullptr, b, x, tol, max_iter, flags, check_every, work, out, st);
    return cg_run<S, 0>(g, vals, nullptr, b, x, tol, max_iter, flags, check_every, work, out, st);
}

// ------------------------------------------------------------ batched
// One launch per CG phase for a whole batch of ensembles (different meshes
// and ensemble sizes): every CTA looks up its ensemble in a per-CTA table and
// runs the same bodies as the single-ensemble kernels, with 512-thread CTAs
// holding 512 / RowMap<s>::THREADS chunks (K1) or VecMap<s, 512>::CPC chunks
// (K2, K3) of that ensemble.  Arithmetic is identical to ens_cg.
constexpr int kBatchThreads = 512;

template <int S>
struct BatchK1 {
    static constexpr int NSUB = kBatchThreads / RowMap<S>::THREADS;
    using Smem = K1Smem<S, NSUB>;
};

constexpr size_t cmax(size_t a, size_t b) { return a > b ? a : b; }
constexpr size_t kBatchK1Smem =
    cmax(cmax(cmax(sizeof(BatchK1<1>::Smem), sizeof(BatchK1<4>::Smem)),
              cmax(sizeof(BatchK1<8>::Smem), sizeof(BatchK1<16>::Smem))),
         sizeof(BatchK1<32>::Smem));
template <int S>
constexpr size_t batch_k2_smem() { return sizeof(double) * VecMap<S, kBatchThreads>::CPC * 32 * (S + 1); }
constexpr size_t kBatchK2Smem = cmax(cmax(cmax(batch_k2_smem<1>(), batch_k2_smem<4>()),
                                          cmax(batch_k2_smem<8>(), batch_k2_smem<16>())),
                                     batch_k2_smem<32>());

struct BItem {
    CgArgs a;
    int S;
    int k1_cta0, v_cta0;
};

struct BatchTables {
    const BItem *items;
    const int *k1_map;  // CTA -> item for K1 launches
    const int *v_map;   // CTA -> item for K2 / K3 launches
};

template <int MODE>
__global__ void __launch_bounds__(kBatchThreads, 2) cg_spmv_batched(BatchTables bt) {
    __shared__ __align__(16) unsigned char raw[kBatchK1Smem];
    const BItem &it = bt.items[__ldg(bt.k1_map + blockIdx.x)];
    const int cta = blockIdx.x - it.k1_cta0;
    switch (it.S) {
        case 1: k1_body<1, MODE, BatchK1<1>::NSUB>(it.a, cta, *reinterpret_cast<BatchK1<1>::Smem *>(raw)); break;
        case 4: k1_body<4, MODE, BatchK1<4>::NSUB>(it.a, cta, *reinterpret_cast<BatchK1<4>::Smem *>(raw)); break;
        case 8: k1_body<8, MODE, BatchK1<8>::NSUB>(it.a, cta, *reinterpret_cast<BatchK1<8>::Smem *>(raw)); break;
        case 16: k1_body<16, MODE, BatchK1<16>::NSUB>(it.a, cta, *reinterpret_cast<BatchK1<16>::Smem *>(raw)); break;
        default: k1_body<32, MODE, BatchK1<32>::NSUB>(it.a, cta, *reinterpret_cast<BatchK1<32>::Smem *>(raw)); break;
    }
}

template <int S>
__device__ __forceinline__ void k2_batched_s(const CgArgs &a, int cta, unsigned char *raw) {
    k2_body<S, kBatchThreads>(a, cta, reinterpret_cast<double(*)[32][S + 1]>(raw));
}

__global__ void __launch_bounds__(kBatchThreads) cg_resid_batched(BatchTables bt) {
    __shared__ __align__(16) unsigned char raw[kBatchK2Smem];
    const BItem &it = bt.items[__ldg(bt.v_map + blockIdx.x)];
    const int cta = blockIdx.x - it.v_cta0;
    switch (it.S) {
        case 1: k2_batched_s<1>(it.a, cta, raw); break;
        case 4: k2_batched_s<4>(it.a, cta, raw); break;
        case 8: k2_batched_s<8>(it.a, cta, raw); break;
        case 16: k2_batched_s<16>(it.a, cta, raw); break;
        default: k2_batched_s<32>(it.a, cta, raw); break;
    }
}

template <int MODE>
__global__ void __launch_bounds__(kBatchThreads) cg_update_batched(BatchTables bt) {
    const BItem &it = bt.items[__ldg(bt.v_map + blockIdx.x)];
    const int cta = blockIdx.x - it.v_cta0;
    switch (it.S) {
        case 1: k3_body<1, MODE, kBatchThreads>(it.a, cta); break;
        case 4: k3_body<4, MODE, kBatchThreads>(it.a, cta); break;
        case 8: k3_body<8, MODE, kBatchThreads>(it.a, cta); break;
        case 16: k3_body<16, MODE, kBatchThreads>(it.a, cta); break;
        default: k3_body<32, MODE, kBatchThreads>(it.a, cta); break;
    }
}

// sums of the convergence words of all ensembles (one thread per ensemble)
__global__ void batch_poll_kernel(const BItem *items, int n_items, int *out) {
    __shared__ int s_act, s_upd;
    if (threadIdx.x == 0) { s_act = 0; s_upd = 0; }
    __syncthreads();
    for (int i = threadIdx.x; i < n_items; i += blockDim.x) {
        const CgState *st = items[i].a.st;
        atomicAdd(&s_act, ld_cg(&st->active_count));
        atomicAdd(&s_upd, ld_cg(&st->updx_any));
    }
    __syncthreads();
    if (threadIdx.x == 0) { out[0] = s_act; out[1] = s_upd; }
}

static void cg_layout_args(CgArgs &a, const ens_graph *g, int S, const double *vals,
                           const double *b, double *x, double tol, int max_iter, int flags,
                           void *work) {
    const int64_t n = g->num_rows;
    char *w = static_cast<char *>(work);
    a.n = g->num_rows;
    a.row_map = g->row_map;
    a.col = g->col_entry;
    a.vals = vals;
    a.vdf = nullptr;
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
    a.fallback = (flags & ENS_CG_GUESS_FALLBACK) ? 1 : 0;
    a.x0_zero = (flags & ENS_CG_X0_ZERO) ? 1 : 0;
    a.pf_cap = 0;
    a.val_bytes = 0;
}

template <int MODE>
static void launch_single(int which, int S, const CgArgs &a, cudaStream_t st) {
    const unsigned grid = (unsigned)a.t1.count[1];
#define ENS_ONE(SS)                                                        \
    if (which == 0) CgKernels<SS, MODE>::init(a, grid, st);                \
    else CgKernels<SS, MODE>::final_(a, grid, st);
    switch (S) {
        case 1: { ENS_ONE(1) break; }
        case 4: { ENS_ONE(4) break; }
        case 8: { ENS_ONE(8) break; }
        case 16: { ENS_ONE(16) break; }
        default: { ENS_ONE(32) break; }
    }
#undef ENS_ONE
}

static int64_t batch_k1_ctas(int S, int64_t chunks) {
    const int nsub = kBatchThreads / (32 * ((S == 1) ? 2 : S / 2));
    return (chunks + nsub - 1) / nsub;
}
static int64_t batch_v_ctas(int S, int64_t chunks) {
    int cpc = 0;
    switch (S) {
        case 1: cpc = VecMap<1, kBatchThreads>::CPC; break;
        case 4: cpc = VecMap<4, kBatchThreads>::CPC; break;
        case 8: cpc = VecMap<8, kBatchThreads>::CPC; break;
        case 16: cpc = VecMap<16, kBatchThreads>::CPC; break;
        default: cpc = VecMap<32, kBatchThreads>::CPC; break;
    }
    return (chunks + cpc - 1) / cpc;
}

struct BatchPlan {
    size_t head;           // items + poll words + CTA maps
    int64_t k1_total, v_total;
    size_t total;
};

static BatchPlan batch_plan(int n_items, const ens_batch_item *items) {
    BatchPlan p{};
    for (int i = 0; i < n_items; ++i) {
        const int64_t chunks = ((int64_t)items[i].graph.num_rows + 31) / 32;
        p.k1_total += batch_k1_ctas(items[i].s, chunks);
        p.v_total += batch_v_ctas(items[i].s, chunks);
    }
    p.head = align256(sizeof(BItem) * n_items) + 256 + align256(sizeof(int) * (size_t)p.k1_total) +
             align256(sizeof(int) * (size_t)p.v_total);
    p.total = p.head;
    for (int i = 0; i < n_items; ++i) p.total += cg_bytes(items[i].graph.num_rows, items[i].s);
    return p;
}

template <int MODE>
static int batched_run(int n_items, const ens_batch_item *items, double tol, int max_iter,
                       int flags, int check_every, void *work, ens_cg_stats *stats,
                       cudaStream_t st) {
    const BatchPlan plan = batch_plan(n_items, items);
    char *w = static_cast<char *>(work);
    BItem *d_items = reinterpret_cast<BItem *>(w);
    int *d_poll = reinterpret_cast<int *>(w + align256(sizeof(BItem) * n_items));
    int *d_k1map = reinterpret_cast<int *>(w + align256(sizeof(BItem) * n_items) + 256);
    int *d_vmap = d_k1map + align256(sizeof(int) * (size_t)plan.k1_total) / sizeof(int);
    char *wi = w + plan.head;
    std::vector<BItem> h(n_items);
    std::vector<int> k1map((size_t)plan.k1_total), vmap((size_t)plan.v_total);
    int64_t k1c = 0, vc = 0;
    int rc;
    for (int i = 0; i < n_items; ++i) {
        const ens_batch_item &it = items[i];
        cg_layout_args(h[i].a, &it.graph, it.s, it.values, it.b, it.x, tol, max_iter,
                       flags, wi);
        wi += cg_bytes(it.graph.num_rows, it.s);
        h[i].S = it.s;
        const int64_t chunks = h[i].a.t1.count[1];
        const int64_t nk = batch_k1_ctas(it.s, chunks), nv = batch_v_ctas(it.s, chunks);
        h[i].k1_cta0 = (int)k1c;
        h[i].v_cta0 = (int)vc;
        for (int64_t c = 0; c < nk; ++c) k1map[k1c++] = i;
        for (int64_t c = 0; c < nv; ++c) vmap[vc++] = i;
        if ((rc = dot_tree_clear(h[i].a.t1, st))) return rc;
        if ((rc = dot_tree_clear(h[i].a.t2, st))) return rc;
        ENS_CUDA_TRY(cudaMemsetAsync(h[i].a.st, 0, sizeof(CgState), st));
    }
    ENS_CUDA_TRY(cudaMemcpyAsync(d_items, h.data(), sizeof(BItem) * n_items, cudaMemcpyHostToDevice, st));
    ENS_CUDA_TRY(cudaMemcpyAsync(d_k1map, k1map.data(), sizeof(int) * k1map.size(), cudaMemcpyHostToDevice, st));
    ENS_CUDA_TRY(cudaMemcpyAsync(d_vmap, vmap.data(), sizeof(int) * vmap.size(), cudaMemcpyHostToDevice, st));
    int launches = 0, polls = 0;
    for (int i = 0; i < n_items; ++i) { launch_single<MODE>(0, h[i].S, h[i].a, st); launches += 2; }
    ENS_LAUNCH_CHECK("batched cg init");
    const BatchTables bt{d_items, d_k1map, d_vmap};
    const unsigned g1 = (unsigned)plan.k1_total, gv = (unsigned)plan.v_total;
    const bool timing = (flags & ENS_CG_TIME_SPMV) != 0;
    const bool use_graph = (flags & ENS_CG_GRAPH) != 0 && !timing;
    std::vector<cudaEvent_t> ev;
    std::vector<float> spmv_ms;
    if (timing) {
        ev.resize(2 * (size_t)check_every);
        for (auto &e : ev) ENS_CUDA_TRY(cudaEventCreate(&e));
    }
    struct EvGuard {
        std::vector<cudaEvent_t> &v;
        ~EvGuard() { for (auto &e : v) cudaEventDestroy(e); }
    } guard{ev};
    auto iteration = [&](cudaStream_t s2, int i) {
        if (timing) cudaEventRecord(ev[2 * i], s2);
        cg_spmv_batched<MODE><<<g1, kBatchThreads, 0, s2>>>(bt);
        if (timing) cudaEventRecord(ev[2 * i + 1], s2);
        cg_resid_batched<<<gv, kBatchThreads, 0, s2>>>(bt);
        cg_update_batched<MODE><<<gv, kBatchThreads, 0, s2>>>(bt);
    };
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t gexec = nullptr;
    if (use_graph) {
        cudaStream_t cap;
        ENS_CUDA_TRY(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
        cudaError_t ce = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
        if (ce == cudaSuccess) {
            for (int i = 0; i < check_every; ++i) iteration(cap, i);
            batch_poll_kernel<<<1, 64, 0, cap>>>(d_items, n_items, d_poll);
            ce = cudaStreamEndCapture(cap, &graph);
        }
        cudaStreamDestroy(cap);
        if (ce != cudaSuccess) return cuda_fail(ce, "batched cg graph capture");
        ce = cudaGraphInstantiate(&gexec, graph, 0);
        if (ce != cudaSuccess) { cudaGraphDestroy(graph); return cuda_fail(ce, "cudaGraphInstantiate"); }
    }
    int32_t hp[2];
    const int max_blocks = max_iter / check_every + 3;
    rc = ENS_OK;
    for (int blk = 0; blk < max_blocks; ++blk) {
        if (use_graph) {
            cudaError_t ce = cudaGraphLaunch(gexec, st);
            if (ce != cudaSuccess) { rc = cuda_fail(ce, "cudaGraphLaunch"); break; }
        } else {
            for (int i = 0; i < check_every; ++i) iteration(st, i);
            batch_poll_kernel<<<1, 64, 0, st>>>(d_items, n_items, d_poll);
        }
        launches += 3 * check_every + 1;
        cudaError_t ce = cudaGetLastError();
        if (ce == cudaSuccess) ce = cudaMemcpyAsync(hp, d_poll, sizeof(hp), cudaMemcpyDeviceToHost, st);
        if (ce == cudaSuccess) ce = cudaStreamSynchronize(st);
        if (ce != cudaSuccess) { rc = cuda_fail(ce, "batched cg iteration"); break; }
        ++polls;
        if (timing)
            for (int i = 0; i < check_every; ++i) {
                float ms = 0.f;
                cudaEventElapsedTime(&ms, ev[2 * i], ev[2 * i + 1]);
                spmv_ms.push_back(ms);
            }
        if (hp[0] == 0 && hp[1] == 0) break;
    }
    if (gexec) cudaGraphExecDestroy(gexec);
    if (graph) cudaGraphDestroy(graph);
    if (rc != ENS_OK) return rc;
    for (int i = 0; i < n_items; ++i) { launch_single<MODE>(1, h[i].S, h[i].a, st); ++launches; }
    ENS_LAUNCH_CHECK("batched cg final");
    std::vector<CgState> hs(n_items);
    for (int i = 0; i < n_items; ++i)
        ENS_CUDA_TRY(cudaMemcpyAsync(&hs[i], h[i].a.st, sizeof(CgState), cudaMemcpyDeviceToHost, st));
    ENS_CUDA_TRY(cudaStreamSynchronize(st));
    int first_bad = ENS_OK, maxit = 0, real = 0, nfb = 0;
    for (int i = 0; i < n_items; ++i) {
        nfb += hs[i].fb_count;
        const ens_batch_item &it = items[i];
        for (int e = 0; e < it.s; ++e) {
            if (it.iters_host) it.iters_host[e] = hs[i].iters[e];
            if (it.relres_host) it.relres_host[e] = hs[i].relres[e];
            if (it.status_host) it.status_host[e] = hs[i].status[e];
            if (hs[i].status[e] != ENS_OK && first_bad == ENS_OK) first_bad = hs[i].status[e];
            maxit = hs[i].iters[e] > maxit ? hs[i].iters[e] : maxit;
        }
        real = hs[i].spmv_real > real ? hs[i].spmv_real : real;
    }
    if (stats) {
        stats->iterations = maxit;
        stats->kernel_launches = launches;
        stats->host_checks = polls;
        stats->guess_fallbacks = nfb;
        stats->reserved = 0;
        stats->spmv_launches = 0;
        stats->spmv_ms = 0.0;
        if (timing) {
            const int nreal = real < (int)spmv_ms.size() ? real : (int)spmv_ms.size();
            double tot = 0.0;
            for (int i = 0; i < nreal; ++i) tot += spmv_ms[i];
            stats->spmv_launches = nreal;
            stats->spmv_ms = tot;
        }
    }
    if (first_bad != ENS_OK)
        set_error("ens_cg_batched: member status %d (%s)", first_bad, ens_status_string(first_bad));
    return first_bad;
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

static int cg_entry(const ens_graph *graph, int s, const double *values, const float2 *vdf, const double *b,
                    double *x, double tol, int max_iter, int flags, int check_every, void *work,
                    size_t work_bytes, int32_t *iters_host, double *relres_host, int32_t *status_host,
                    ens_cg_stats *stats_host, void *stream) {
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
        case 1: return cg_dispatch_df<1>(graph, values, vdf, b, x, tol, max_iter, flags, check_every, work, out, st);
        case 4: return cg_dispatch_df<4>(graph, values, vdf, b, x, tol, max_iter, flags, check_every, work, out, st);
        case 8: return cg_dispatch_df<8>(graph, values, vdf, b, x, tol, max_iter, flags, check_every, work, out, st);
        case 16: return cg_dispatch_df<16>(graph, values, vdf, b, x, tol, max_iter, flags, check_every, work, out, st);
        default: return cg_dispatch_df<32>(graph, values, vdf, b, x, tol, max_iter, flags, check_every, work, out, st);
    }
}

extern "C" int ens_cg(const ens_graph *graph, int s, const double *values, const double *b,
                      double *x, double tol, int max_iter, int flags, int check_every, void *work,
                      size_t work_bytes, int32_t *iters_host, double *relres_host,
                      int32_t *status_host, ens_cg_stats *stats_host, void *stream) {
    return cg_entry(graph, s, values, nullptr, b, x, tol, max_iter, flags, check_every, work, work_bytes,
                    iters_host, relres_host, status_host, stats_host, stream);
}

extern "C" int ens_cg_df(const ens_graph *graph, int s, const double *values, const void *values_df,
                         const double *b, double *x, double tol, int max_iter, int flags, int check_every,
                         void *work, size_t work_bytes, int32_t *iters_host, double *relres_host,
                         int32_t *status_host, ens_cg_stats *stats_host, void *stream) {
    if (!values_df) return fail(ENS_ERR_ARG, "ens_cg_df: values_df is NULL");
    if (s > 1 && !aligned16(values_df)) return fail(ENS_ERR_ALIGN, "ens_cg_df: values_df must be 16-byte aligned");
    return cg_entry(graph, s, values, static_cast<const float2 *>(values_df), b, x, tol, max_iter,
                    flags & ~(ENS_CG_DF64 | ENS_CG_SPLIT64), check_every, work, work_bytes, iters_host,
                    relres_host, status_host, stats_host, stream);
}

static int check_batch(int n_items, const ens_batch_item *items) {
    if (n_items < 1 || n_items > 4096) return fail(ENS_ERR_ARG, "n_items=%d outside [1, 4096]", n_items);
    if (!items) return fail(ENS_ERR_ARG, "items is NULL");
    for (int i = 0; i < n_items; ++i) {
        int rc = check_graph(&items[i].graph);
        if (rc) return rc;
        if (!supported_s(items[i].s))
            return fail(ENS_ERR_UNSUPPORTED, "item %d: ensemble size s=%d not in {1,4,8,16,32}", i, items[i].s);
        if (items[i].graph.num_rows == 0) return fail(ENS_ERR_ARG, "item %d: empty graph", i);
        if (!items[i].values || !items[i].b || !items[i].x)
            return fail(ENS_ERR_ARG, "item %d: NULL values/b/x", i);
        if (items[i].s > 1 && (!aligned16(items[i].values) || !aligned16(items[i].b) || !aligned16(items[i].x)))
            return fail(ENS_ERR_ALIGN, "item %d: values/b/x must be 16-byte aligned", i);
    }
    return ENS_OK;
}

extern "C" int ens_cg_batched_workspace_size(int n_items, const ens_batch_item *items, size_t *bytes) {
    int rc = check_batch(n_items, items);
    if (rc) return rc;
    if (!bytes) return fail(ENS_ERR_ARG, "bytes is NULL");
    *bytes = batch_plan(n_items, items).total;
    return ENS_OK;
}

extern "C" int ens_cg_batched(int n_items, const ens_batch_item *items, double tol, int max_iter,
                              int flags, int check_every, void *work, size_t work_bytes,
                              ens_cg_stats *stats_host, void *stream) {
    int rc = check_batch(n_items, items);
    if (rc) return rc;
    if (!(tol >= 0.0) || max_iter < 0 || check_every < 1)
        return fail(ENS_ERR_ARG, "tol=%g max_iter=%d check_every=%d", tol, max_iter, check_every);
    if (!work || !aligned16(work)) return fail(ENS_ERR_ALIGN, "work must be a 16-byte aligned device pointer");
    const size_t need = batch_plan(n_items, items).total;
    if (work_bytes < need) return fail(ENS_ERR_WORKSPACE, "batched workspace %zu < %zu bytes", work_bytes, need);
    cudaStream_t st = as_stream(stream);
    if (flags & ENS_CG_SPLIT64) return batched_run<2>(n_items, items, tol, max_iter, flags, check_every, work, stats_host, st);
    if (flags & ENS_CG_DF64) return batched_run<1>(n_items, items, tol, max_iter, flags, check_every, work, stats_host, st);
    return batched_run<0>(n_items, items, tol, max_iter, flags, check_every, work, stats_host, st);
}
