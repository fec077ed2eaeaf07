// ens_cg_kernels.cuh -- device side of the ensemble CG: state, arguments and
// the K0/KZ/K1/K2/K3/KF kernels (shared by ens_cg.cu and ens_pcg.cu).
#pragma once
#include "ens_spmv.cuh"

namespace ens {


struct CgState {
    double rho[32], alpha[32], beta[32], bnorm[32], relres[32];
    int active[32], updx[32], zerox[32], iters[32], status[32], fb[32];
    int active_count, updx_any, zero_any, spmv_real;
    int df_bad_any, fb_count, loop_blocks, pad2;   // loop_blocks: blocks run by the device loop
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
    int k2_pf;             // K2 prefetches its CTA's r and q blocks into L2 at its start
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
// q = A p and the per-member p.q for NSUB chunks of one ensemble per CTA,
// each chunk on its own group of 32 * RowMap<S>::G threads (the standalone
// kernel and the batched one share this body).  NSUB changes only the launch
// mapping: every sum is ordered by row index, so results are bitwise the same
// for every NSUB.
template <int S, int NSUB>
struct K1Smem {
    double sm[NSUB][32][S + 1];
    ChunkCols cc[NSUB];
};

template <int S>
__device__ __forceinline__ void k1_epilogue(const CgArgs &a);

// EXIT_FIRST: test for a stopped ensemble before staging anything.  The batched
// kernel sets it: its converged items' CTAs run every remaining iteration, and
// staging (with the L2 prefetch of their values) before the test made them
// read DRAM for nothing (the 2048-sample 16^3-64^3 batch solve took 2319 ms
// against 2190).  The single-ensemble kernels stage first, so the staging
// loads overlap the load of the active count.
template <int S, int MODE, int NSUB, bool EXIT_FIRST = false>
__device__ __forceinline__ void k1_body(const CgArgs &a, const int cta, K1Smem<S, NSUB> &sh) {
    CgState *st = a.st;
    if (EXIT_FIRST && ld_cg(&st->active_count) == 0) {
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
    bool staged;
    if constexpr (NSUB == 1) {
        if (MODE == 3) staged = stage_chunk_pf(sh.cc[0], a.row_map, a.col, chunk, a.n, a.vdf, S * 8u, a.val_bytes,
                                               a.pf_cap);
        else staged = stage_chunk(sh.cc[0], a.row_map, a.col, chunk, a.n);
    } else if (MODE == 3) {
        staged = stage_chunk_sub<stage_unroll(T)>(sh.cc[sub], a.row_map, a.col, chunk, a.n, ltid, T, a.vdf, S * 8u,
                                                  a.val_bytes, a.pf_cap);
    } else {
        staged = stage_chunk_sub<stage_unroll(T)>(sh.cc[sub], a.row_map, a.col, chunk, a.n, ltid, T);
    }
    if (!EXIT_FIRST && ld_cg(&st->active_count) == 0) {   // every member stopped: a launch queued past convergence
        if (cta == 0 && threadIdx.x == 0 && st->updx_any) {
            for (int e = 0; e < S; ++e) st->updx[e] = 0;
            st->updx_any = 0;
        }
        return;
    }
    // the split / double-float forms are used unless a vector element fell outside their range
    const int mode = (MODE != 0 && ld_cg(&st->df_bad_any) != 0) ? 0 : MODE;
    double2 apv;
    if (MODE == 1 && mode == 1)
        apv = chunk_spmv_df<S, XPre>(sh.cc[sub], staged, a.col, a.vals, a.pdf, r, g, valid);
    else if (MODE == 3 && mode == 3)
        apv = chunk_spmv_dfv<S>(sh.cc[sub], staged, a.col, a.vdf, a.vals, a.pdf, r, g, valid);
    else if (MODE == 2 && mode == 2)
        apv = chunk_spmv_split<S, XPre>(sh.cc[sub], staged, a.col, a.vals, a.p, a.pdf, r, g, valid);
    else
        apv = chunk_spmv<S, double>(sh.cc[sub], staged, a.col, a.vals, a.p, r, g, valid);
    double v0 = 0.0, v1 = 0.0;
    const int64_t R = K1_CHUNK * 32 + r;
    const bool pre = (MODE == 1 || MODE == 3) && mode == MODE;  // p.q from the split p, as cg_spmv_kernel
    if constexpr (S == 1) {
        if (valid) {
            if (g == 0) a.q[R] = apv.x;
            double pr;
            if (pre) {
                const float2 h = a.pdf[R];
                pr = f2d_exact(h.x) + f2d_exact(h.y);
            } else {
                pr = a.p[R];
            }
            v0 = apv.x * pr;
        }
    } else if (valid) {
        reinterpret_cast<double2 *>(a.q)[R * G + g] = apv;
        double2 pv;
        if (pre) {
            const float4 h = reinterpret_cast<const float4 *>(a.pdf)[R * G + g];
            pv = make_double2(f2d_exact(h.x) + f2d_exact(h.y), f2d_exact(h.z) + f2d_exact(h.w));
        } else {
            pv = reinterpret_cast<const double2 *>(a.p)[R * G + g];
        }
        v0 = apv.x * pv.x;
        v1 = apv.y * pv.y;
    }
    if constexpr (NSUB == 1) chunk_tree<S>(sh.sm[0], v0, v1, r, g, a.t1, K1_CHUNK, 0);
    else chunk_tree_sub<S>(sh.sm[sub], v0, v1, r, g, a.t1, K1_CHUNK, 0, ltid, T);
    const int nitems = (NSUB == 1) ? 1 : (int)min((int64_t)NSUB, a.t1.count[1] - (int64_t)cta * NSUB);
    if (!dot_tree_propagate(a.t1, (int64_t)cta * NSUB, nitems)) return;
#undef K1_CHUNK
    if (threadIdx.x >= 32) return;
    k1_epilogue<S>(a);
}

// K1's per-member scalar work, run by warp 0 of the CTA that produced the
// top of p.q's tree: alpha = rho / p.q, breakdown, the active count
template <int S>
__device__ __forceinline__ void k1_epilogue(const CgArgs &a) {
    CgState *st = a.st;
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
        st->updx[e] = act;  // this iteration's K3 updates x of every member still active here
    }
    const int ac = __popc(__ballot_sync(FULL, act));
    if (e == 0) {
        st->spmv_real += 1;
        st->updx_any = ac;
        st->active_count = ac;
    }
    __threadfence();
}

// K1 with one chunk per CTA: the arithmetic of k1_body<S, MODE, 1>, written
// out with fewer live indices so that it keeps to 40 registers (3 CTAs of 512
// threads per SM at s = 32) with little spilling.  VEC: column staging with
// 16-byte loads; WARP: chunk tree by warp shuffles (see chunk_tree).
// DEFER: the CTA writes only its chunk's p.q partials (level 1 of the tree);
// cg_spmv_reduce_kernel, launched next, does the upper levels in the same
// order and the epilogue, so no CTA of K1 waits on a fence and an atomic.
template <int S, int MODE, bool VEC, bool WARP, bool DEFER = false>
__device__ __forceinline__ void k1_single(const CgArgs &a) {
    CgState *st = a.st;
    constexpr int G = RowMap<S>::G;
    __shared__ double sm[32][S + 1];
    const int r = threadIdx.x / G, g = threadIdx.x % G;
    const int64_t R = (int64_t)blockIdx.x * 32 + r;
    __shared__ ChunkCols cc;
    const void *vblock = (MODE == 3) ? static_cast<const void *>(a.vdf) : static_cast<const void *>(a.vals);
    const bool staged = stage_chunk_pf<VEC, stage_unroll(RowMap<S>::THREADS)>(cc, a.row_map, a.col, blockIdx.x, a.n,
                                                                            vblock, S * 8u, a.val_bytes,
                                            a.pf_cap);
    if (ld_cg(&st->active_count) == 0) {   // every member stopped: a launch queued past convergence
        if (blockIdx.x == 0 && threadIdx.x == 0 && st->updx_any) {
            for (int e = 0; e < S; ++e) st->updx[e] = 0;
            st->updx_any = 0;
        }
        return;
    }
    // the split / double-float forms are used unless a vector element fell outside their range
    const int mode = (MODE != 0 && ld_cg(&st->df_bad_any) != 0) ? 0 : MODE;
    double2 apv;
    if (MODE == 1 && mode == 1)
        apv = chunk_spmv_df<S, XPre>(cc, staged, a.col, a.vals, a.pdf, r, g, R < a.n);
    else if (MODE == 3 && mode == 3)
        apv = chunk_spmv_dfv<S>(cc, staged, a.col, a.vdf, a.vals, a.pdf, r, g, R < a.n);
    else if (MODE == 2 && mode == 2)
        apv = chunk_spmv_split<S, XPre>(cc, staged, a.col, a.vals, a.p, a.pdf, r, g, R < a.n);
    else
        apv = chunk_spmv<S, double>(cc, staged, a.col, a.vals, a.p, r, g, R < a.n);
    // p.q: the double-float forms take p as the SpMV saw it, hi + lo of the
    // split copy (exact in FP64), which saves reading the FP64 p
    const bool pre = (MODE == 1 || MODE == 3) && mode == MODE;
    double v0 = 0.0, v1 = 0.0;
    if constexpr (S == 1) {
        const double ap = apv.x;
        if (R < a.n) {
            if (g == 0) a.q[R] = ap;
            double pr;
            if (pre) {
                const float2 h = a.pdf[R];
                pr = f2d_exact(h.x) + f2d_exact(h.y);
            } else {
                pr = a.p[R];
            }
            v0 = ap * pr;
        }
    } else if (R < a.n) {
        const double2 ap = apv;
        reinterpret_cast<double2 *>(a.q)[R * G + g] = ap;
        double2 pv;
        if (pre) {
            const float4 h = reinterpret_cast<const float4 *>(a.pdf)[R * G + g];
            pv = make_double2(f2d_exact(h.x) + f2d_exact(h.y), f2d_exact(h.z) + f2d_exact(h.w));
        } else {
            pv = reinterpret_cast<const double2 *>(a.p)[R * G + g];
        }
        v0 = ap.x * pv.x;
        v1 = ap.y * pv.y;
    }
    chunk_tree<S, WARP>(sm, v0, v1, r, g, a.t1, blockIdx.x, 0);
    if (DEFER) return;
    if (!dot_tree_propagate(a.t1, blockIdx.x, 1)) return;
    if (threadIdx.x >= 32) return;
    k1_epilogue<S>(a);
}

// standalone K1: NSUB chunks per CTA (NSUB * 32 * RowMap<S>::G <= 1024
// threads); one chunk at up to 1536 threads per SM (40 registers), several
// at up to 1024 (64 registers)
#ifndef ENS_K1_DFV_THREADS_PER_SM
#define ENS_K1_DFV_THREADS_PER_SM 1536
#endif
// Threads per SM the register budget is sized for: 1536 (40 registers) where
// the SpMV runs fastest with the most CTAs in flight (s = 1, 16, 32), 1024
// (64 registers) at s = 4 and 8, where the spilled row-loop state costs more
// than the lost occupancy (64^3 mesh, pre-split form: s = 4 0.115 -> 0.089
// ms, s = 8 0.139 -> 0.134 ms).
template <int S, int MODE, int NSUB>
struct K1Launch {
    static constexpr int THREADS = NSUB * RowMap<S>::THREADS;
    static constexpr int PER_SM = (NSUB > 1 || S == 4 || S == 8) ? 1024
                                  : (MODE == 3) ? ENS_K1_DFV_THREADS_PER_SM : 1536;
    static constexpr int MIN_BLOCKS = (PER_SM / THREADS) > 0 ? PER_SM / THREADS : 1;
};

template <int S, int MODE, int NSUB>
__global__ void __launch_bounds__(K1Launch<S, MODE, NSUB>::THREADS, K1Launch<S, MODE, NSUB>::MIN_BLOCKS)
    cg_spmv_kernel(CgArgs a) {
    if constexpr (NSUB == 1) {
        k1_single<S, MODE, true, (S == 1)>(a);
    } else {
        __shared__ K1Smem<S, NSUB> sh;
        k1_body<S, MODE, NSUB>(a, blockIdx.x, sh);
    }
}

// K1 with the deferred tree (ENS_CG_K1_DEFER): chunk partials only ...
template <int S, int MODE>
__global__ void __launch_bounds__(RowMap<S>::THREADS, K1Launch<S, MODE, 1>::MIN_BLOCKS)
    cg_spmv_partial_kernel(CgArgs a) {
    k1_single<S, MODE, true, (S == 1), true>(a);
}

// ... then one CTA per level-1 group: the group's reduction, the upper levels
// (last arrivers, as in dot_tree_propagate) and K1's epilogue
template <int S>
__global__ void __launch_bounds__(256) cg_spmv_reduce_kernel(CgArgs a) {
    if (ld_cg(&a.st->active_count) == 0) return;   // K1 already cleared the flags
    if (a.t1.levels == 1) {                         // one chunk: its partials are the top
        if (threadIdx.x < 32) k1_epilogue<S>(a);
        return;
    }
    dot_tree_reduce_group(a.t1, blockIdx.x);
    if (!dot_tree_propagate_from(a.t1, 2, blockIdx.x, 1)) return;
    if (threadIdx.x >= 32) return;
    k1_epilogue<S>(a);
}

// Host: chunks of 32 rows per K1 CTA (1, 2, 4 or 8; at most 1024 threads per
// CTA).  k1_launch launches K1 with that mapping; its instantiations live in
// ens_cg_k1_s*.cu (one translation unit per ensemble size).
template <int S>
constexpr int k1_max_nsub() { return (1024 / RowMap<S>::THREADS) >= 8 ? 8 : 1024 / RowMap<S>::THREADS; }
int k1_max_nsub_rt(int s);
int k1_default_nsub(int s, int mode);
template <int S, int MODE>
void k1_launch(const CgArgs &a, int nsub, cudaStream_t st);


// ------------------------------------------------------------------ K2
// v*v of an FP64 value as an unevaluated float pair: v split by truncation
// into hi + lo (47 bits), hi*hi exact by FMA error recovery, 2 hi lo added to
// the error term (lo*lo, below 2^-46 |v*v|, is dropped).  Exact and free of
// FP32 underflow and overflow only for |v| in [2^-50, 2^60): hi*hi is then at
// least 2^-100 (its error term is a normal float) and a chunk's 32 squares
// stay below 2^125.  Zero squares to (0, 0); any other v outside that range
// returns (NaN, 0), which marks its (chunk, member) column for the FP64 sum
// of k2_chunk_rr_fp64.  Integer and FP32 instructions only.
__device__ __forceinline__ float2 df_square(double v) {
    const uint32_t uh = (uint32_t)__double2hiint(v), ul = (uint32_t)__double2loint(v);
    const uint32_t E = (uh >> 20) & 0x7ffu;
    if (E - 973u > 109u) {  // biased exponent outside [973, 1082]: |v| outside [2^-50, 2^60)
        const bool zero = ((uh << 1) | ul) == 0u;
        return make_float2(zero ? 0.0f : __int_as_float(0x7fc00000), 0.0f);
    }
    float hi, lo;
    df_split_trunc(v, hi, lo);
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

// K2's epilogue, in the CTA that produced the top of r.r's tree: one lane
// per member (warp 0) sets the stopping flags and beta
template <int S>
__device__ __forceinline__ void k2_epilogue(const CgArgs &a) {
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
        st->active[e] = act;
    }
    // the x-update flags of this iteration were set by K1's epilogue (K3 may
    // read them while this kernel is still running)
    const int ac = __popc(__ballot_sync(FULL, act));
    if (e == 0) st->active_count = ac;
    __threadfence();
}


// K2's order for a chunk's r.r (the level-1 items of its dot tree): the 32
// rows in 4 slices of 8 consecutive rows, each slice summed row by row in
// float pairs, then the slices combined as (q0 + q2) + (q1 + q3).  It depends
// only on the row index, so a member's r.r is bitwise the same at every s
// and in every launch shape.  Mapping: a (chunk, slice) unit on S threads,
// one member each (r and q loaded 8 rows at a time, all 16 loads in flight
// before the first store); a CTA of TH threads owns CPC chunks.
constexpr int kK2Slices = 4;
constexpr int kK2SliceRows = 32 / kK2Slices;

template <int S, int TH, int CPC>
struct K2Map {
    static_assert(TH % S == 0, "K2: whole units per CTA");
    static constexpr int UNITS = CPC * kK2Slices;   // (chunk, slice) units of a CTA
    static constexpr int UPP = TH / S;              // units per pass
};

// FP64 r.r of one (chunk, member) column whose float-pair sum was marked (a
// value outside the float-pair range): the same slices and combination
// order in FP64.  Called by one thread after a barrier that orders the CTA's
// r stores before it.
static __device__ __noinline__ double k2_chunk_rr_fp64(const double *r, int64_t n, int64_t chunk, int e, int S) {
    double q[kK2Slices];
    for (int k = 0; k < kK2Slices; ++k) {
        double acc = 0.0;
        for (int i = 0; i < kK2SliceRows; ++i) {
            const int64_t R = chunk * 32 + k * kK2SliceRows + i;
            const double x = (R < n) ? r[R * S + e] : 0.0;
            acc = (i == 0) ? x * x : acc + x * x;
        }
        q[k] = acc;
    }
    return (q[0] + q[2]) + (q[1] + q[3]);
}

// EXIT_FIRST: as for k1_body (the batched kernel tests for a stopped ensemble
// before prefetching its r and q blocks).  LB: rows of r and q loaded before
// the first of them is updated (8: a whole slice).  sl: CPC * 4 * S float
// pairs of shared memory.
template <int S, int TH, int CPC, bool EXIT_FIRST = false, int LB = kK2SliceRows>
__device__ __forceinline__ void k2_body(const CgArgs &a, int cta, float2 (*sl)[kK2Slices][S]) {
    using VM = K2Map<S, TH, CPC>;
    const int64_t first_chunk = (int64_t)cta * CPC;
    if (EXIT_FIRST && ld_cg(&a.st->active_count) == 0) return;
    if (a.k2_pf && threadIdx.x == 0) {   // the loads below then read r and q from L2
        const uint64_t b0 = (uint64_t)first_chunk * 32 * S * 8u;
        const uint64_t b1 = (uint64_t)min((first_chunk + CPC) * 32, (int64_t)a.n) * S * 8u;
        l2_prefetch_span(a.r, b0, b1);
        l2_prefetch_span(a.q, b0, b1);
    }
    if (ld_cg(&a.st->active_count) == 0) return;
    const CgState *cs = a.st;
    const int e = threadIdx.x % S;
    const bool act = cs->active[e];
    const double al = cs->alpha[e];
    double *__restrict__ rp = a.r;
    const double *__restrict__ qp = a.q;
    // r -= alpha q (FP64 FMA, the only FP64-pipe work), then the squares and
    // the slice sums as float pairs on the FP32 pipe
#pragma unroll 1
    for (int u = threadIdx.x / S; u < VM::UNITS; u += VM::UPP) {
        const int c = u / kK2Slices, k = u % kK2Slices;
        const int64_t R0 = (first_chunk + c) * 32 + k * kK2SliceRows;
        float2 acc = make_float2(0.f, 0.f);
#pragma unroll
        for (int i0 = 0; i0 < kK2SliceRows; i0 += LB) {
            double rv[LB], qv[LB];
#pragma unroll
            for (int i = 0; i < LB; ++i) {
                rv[i] = 0.0;
                qv[i] = 0.0;
                if (R0 + i0 + i < a.n) {
                    rv[i] = rp[(R0 + i0 + i) * S + e];
                    qv[i] = qp[(R0 + i0 + i) * S + e];
                }
            }
#pragma unroll
            for (int i = 0; i < LB; ++i) {
                if (act && R0 + i0 + i < a.n) {
                    rv[i] = fma(-al, qv[i], rv[i]);
                    rp[(R0 + i0 + i) * S + e] = rv[i];
                }
                const float2 sq = df_square(rv[i]);
                acc = (i0 + i == 0) ? sq : df_add(acc, sq);
            }
        }
        sl[c][k][e] = acc;
    }
    __syncthreads();
    for (int it = threadIdx.x; it < CPC * S; it += TH) {
        const int c = it / S, m = it % S;
        const int64_t ch = first_chunk + c;
        if (ch < a.t1.count[1]) {
            const float2 t = df_add(df_add(sl[c][0][m], sl[c][2][m]), df_add(sl[c][1][m], sl[c][3][m]));
            a.t1.buf[1][ch * S + m] = (t.x == t.x) ? f2d_exact(t.x) + f2d_exact(t.y)
                                                   : k2_chunk_rr_fp64(a.r, a.n, ch, m, S);
        }
    }
    const int nitems = (int)min((int64_t)CPC, a.t1.count[1] - first_chunk);
    if (!dot_tree_propagate(a.t1, first_chunk, nitems)) return;
    if (threadIdx.x >= 32) return;
    k2_epilogue<S>(a);
}

// ------------------------------------------------------------------ K3
// griddepcontrol: the dependent grid may launch (K2), and wait for the
// prerequisite grid's completion and memory (K3); both are no-ops for a
// launch without a programmatic dependency
__device__ __forceinline__ void pdl_launch_dependents() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// K3: x += alpha p for the members K1 left active (the flags and alpha are
// K1's, so this part may run while K2 still runs, when K3 is launched with a
// programmatic dependency on K2), then, after K2 has completed, p = r + beta p
// for the members K2 left active.
template <int S, int MODE, int TH>
__device__ __forceinline__ void k3_body(const CgArgs &a, int cta) {
    using VM = VecMap<S, TH>;
    CgState *st = a.st;
    if (ld_cg(&st->updx_any) == 0) return;
    constexpr int VG = VM::VG;
    const int cip = threadIdx.x / VM::CHUNK_T, lt = threadIdx.x % VM::CHUNK_T;
    const int r = lt / VG, g = lt % VG;
    const int m = (S == 1) ? 0 : 2 * g;
    const bool ux0 = st->updx[m];
    const bool ux1 = (S == 1) ? false : (bool)st->updx[m + 1];
    const double al0 = st->alpha[m];
    const double al1 = (S == 1) ? 0.0 : st->alpha[m + 1];
    const int64_t first_chunk = (int64_t)cta * VM::CPC;
    if constexpr (S == 1) {
        double pv[VM::PASSES];
#pragma unroll
        for (int pass = 0; pass < VM::PASSES; ++pass) {
            const int64_t R = (first_chunk + pass * VM::CPP + cip) * 32 + r;
            pv[pass] = 0.0;
            if (R < a.n) {
                pv[pass] = a.p[R];
                if (ux0) a.x[R] = fma(al0, pv[pass], a.x[R]);
            }
        }
        pdl_wait();
        const bool ac0 = ld_cg(&st->active[m]) != 0;
        const double be0 = ld_cg(&st->beta[m]);
        if (!ac0) return;
#pragma unroll
        for (int pass = 0; pass < VM::PASSES; ++pass) {
            const int64_t R = (first_chunk + pass * VM::CPP + cip) * 32 + r;
            if (R >= a.n) continue;
            const double pn = fma(be0, pv[pass], a.r[R]);
            a.p[R] = pn;
            if (MODE != 0) store_split1(a.pdf, R, pn, &st->df_bad_any);
        }
    } else {
        double2 pv[VM::PASSES];
#pragma unroll
        for (int pass = 0; pass < VM::PASSES; ++pass) {
            const int64_t R = (first_chunk + pass * VM::CPP + cip) * 32 + r;
            pv[pass] = make_double2(0.0, 0.0);
            if (R < a.n) {
                pv[pass] = reinterpret_cast<const double2 *>(a.p)[R * VG + g];
                if (ux0 || ux1) {
                    double2 xv = reinterpret_cast<const double2 *>(a.x)[R * VG + g];
                    if (ux0) xv.x = fma(al0, pv[pass].x, xv.x);
                    if (ux1) xv.y = fma(al1, pv[pass].y, xv.y);
                    reinterpret_cast<double2 *>(a.x)[R * VG + g] = xv;
                }
            }
        }
        pdl_wait();
        const bool ac0 = ld_cg(&st->active[m]) != 0, ac1 = ld_cg(&st->active[m + 1]) != 0;
        const double be0 = ld_cg(&st->beta[m]), be1 = ld_cg(&st->beta[m + 1]);
        if (!(ac0 || ac1)) return;
#pragma unroll
        for (int pass = 0; pass < VM::PASSES; ++pass) {
            const int64_t R = (first_chunk + pass * VM::CPP + cip) * 32 + r;
            if (R >= a.n) continue;
            const double2 rv = reinterpret_cast<const double2 *>(a.r)[R * VG + g];
            double2 pn = pv[pass];
            if (ac0) pn.x = fma(be0, pv[pass].x, rv.x);
            if (ac1) pn.y = fma(be1, pv[pass].y, rv.y);
            reinterpret_cast<double2 *>(a.p)[R * VG + g] = pn;
            if (MODE != 0) store_split(a.pdf, R * S + m, pn.x, pn.y, &st->df_bad_any);
        }
    }
}

// K2's launch: CTAs of TH threads, a (chunk, slice) unit on S threads, so a
// CTA owns TH / (4 S) chunks (at most 32: one level-2 group of the dot tree);
// 3 CTAs per SM (40 registers), a slice's rows loaded 4 at a time.  At 64^3,
// s = 32 a CG iteration took 0.4739 ms so, 0.4788 ms with 2 CTAs per SM and
// 8 rows at a time (64 registers), 0.4781 ms with CTAs of 256 threads at 4
// per SM, and 0.4836 ms with the earlier K2 (two members per thread and a
// shared-memory halving tree over each chunk's 32 rows).
template <int S>
struct K2Launch {
    static constexpr int TH = (S == 1) ? 128 : 512;
    static constexpr int CPC = TH / (kK2Slices * S);
    static constexpr int MIN_BLOCKS = 3;
    static constexpr int LB = 4;
    static_assert(CPC >= 1 && CPC <= 32 && 32 % CPC == 0, "K2: a CTA's chunks lie in one level-2 group");
};

template <int S>
__global__ void __launch_bounds__(K2Launch<S>::TH, K2Launch<S>::MIN_BLOCKS) cg_resid_kernel(CgArgs a) {
    pdl_launch_dependents();   // K3 may start its x update on the SMs this grid leaves idle
    __shared__ float2 sl[K2Launch<S>::CPC][kK2Slices][S];   // slice sums of every chunk
    k2_body<S, K2Launch<S>::TH, K2Launch<S>::CPC, false, K2Launch<S>::LB>(a, blockIdx.x, sl);
}

template <int S, int MODE>
__global__ void __launch_bounds__(VecMap<S>::THREADS, 1536 / VecMap<S>::THREADS) cg_update_kernel(CgArgs a) {
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

}  // namespace ens
