// ens_mg.cu -- multigrid-preconditioned ensemble CG (the paper's solver,
// Sect. 3.5 and Algorithm 1): CG with z = V_0(r), the V-cycle of
// ens_mg_solver.cuh (rho = r.z), reusing the CG kernels: per iteration
//   K1 (q = A p, alpha), MR (r -= alpha q, r.r), the V-cycle, MZ (r.z: stop
//   test, beta), K3 (x += alpha p, p = z + beta p).
// FP64, with the SpMVs of pre-split levels (and K1 when level 0 is pre-split)
// in double-float.  Every launch of an iteration is asynchronous; with ENS_CG_GRAPH
// check_every iterations are replayed as one CUDA graph.
#include "ens_mg_solver.cuh"

namespace ens {

// ------------------------------------------------------------ CG glue
// MR: r -= alpha q for the active members and r.r (-> ps->rr)
template <int S>
__global__ void __launch_bounds__(RowMap<S>::THREADS, 1024 / RowMap<S>::THREADS) mg_pcg_resid_kernel(PcgArgs a) {
    const CgArgs &c = a.c;
    if (ld_cg(&c.st->active_count) == 0) return;
    constexpr int G = RowMap<S>::G;
    __shared__ double sm[32][S + 1];
    const int r = threadIdx.x / G, g = threadIdx.x % G;
    const int64_t R = (int64_t)blockIdx.x * 32 + r;
    const CgState *cs = c.st;
    double v0 = 0.0, v1 = 0.0;
    if (R < c.n && (S != 1 || g == 0)) {
        const int w = (S == 1) ? 1 : 2;
        const int64_t i0 = (S == 1) ? R : R * S + 2 * g;
        for (int j = 0; j < w; ++j) {
            const int64_t i = i0 + j;
            const int e = (S == 1) ? 0 : 2 * g + j;
            double rv = c.r[i];
            if (cs->active[e]) {
                rv = fma(-cs->alpha[e], c.q[i], rv);
                c.r[i] = rv;
            }
            if (j == 0) v0 = rv * rv;
            else v1 = rv * rv;
        }
    }
    chunk_tree<S>(sm, v0, v1, r, g, c.t1, blockIdx.x, 0);
    if (!dot_tree_propagate(c.t1, blockIdx.x, 1)) return;
    const int e = threadIdx.x;
    if (e < S) a.ps->rr[e] = ld_cg(c.t1.buf[c.t1.levels] + e);
    __threadfence();
}

// MZ: r.z, then the stop test and beta (pc_epilogue)
template <int S>
__global__ void __launch_bounds__(RowMap<S>::THREADS, 1024 / RowMap<S>::THREADS) mg_pcg_rz_kernel(PcgArgs a,
                                                                                                 const double *z,
                                                                                                 int init) {
    const CgArgs &c = a.c;
    if (ld_cg(&c.st->active_count) == 0) return;
    constexpr int G = RowMap<S>::G;
    __shared__ double sm[32][S + 1];
    const int r = threadIdx.x / G, g = threadIdx.x % G;
    const int64_t R = (int64_t)blockIdx.x * 32 + r;
    double v0 = 0.0, v1 = 0.0;
    if (R < c.n) {
        if constexpr (S == 1) {
            if (g == 0) v0 = c.r[R] * z[R];
        } else {
            const double2 rv = reinterpret_cast<const double2 *>(c.r)[R * G + g];
            const double2 zv = reinterpret_cast<const double2 *>(z)[R * G + g];
            v0 = rv.x * zv.x;
            v1 = rv.y * zv.y;
        }
    }
    chunk_tree<S>(sm, v0, v1, r, g, c.t1, blockIdx.x, 0);
    if (!dot_tree_propagate(c.t1, blockIdx.x, 1)) return;
    if (threadIdx.x >= 32) return;
    const int e = threadIdx.x;
    const double rz = (e < S) ? ld_cg(c.t1.buf[c.t1.levels] + e) : 0.0;
    const double rr = (e < S) ? a.ps->rr[e] : 0.0;
    pc_epilogue<S>(a, init ? rz : rr, rz, init != 0);
}

// ------------------------------------------------------------ host side
// workspace of the whole solve: the CG state and vectors (r, p, q, z), then
// the hierarchy (mg_layout)
static size_t mg_pcg_layout(int nl, const ens_mg_level *lv, int s, std::vector<MgLevel> *out, char *base,
                            CgArgs *c0, double **zpcg, double **coarse_inv, int **bad) {
    size_t off = 0;
    auto take = [&](size_t bytes) -> char * {
        char *p = base ? base + off : nullptr;
        off += mg_align(bytes);
        return p;
    };
    const int64_t n0 = lv[0].graph.num_rows;
    const size_t v0 = sizeof(double) * (size_t)n0 * s;
    CgState *st = reinterpret_cast<CgState *>(take(sizeof(CgState)));
    double *pr = reinterpret_cast<double *>(take(v0));
    double *pp = reinterpret_cast<double *>(take(v0));
    double *pq = reinterpret_cast<double *>(take(v0));
    double *pz = reinterpret_cast<double *>(take(v0));
    float2 *pdf = lv[0].values_df ? reinterpret_cast<float2 *>(take(v0)) : nullptr;  // split p for K1
    off += mg_layout(nl, lv, s, out, base ? base + off : nullptr, coarse_inv, bad);
    if (base && c0) {
        *c0 = (*out)[0].pa.c;
        c0->st = st;
        c0->r = pr;
        c0->p = pp;
        c0->q = pq;
        c0->pdf = pdf;
        if (pdf) {
            c0->vdf = reinterpret_cast<const float2 *>(lv[0].values_df);
            c0->pf_cap = 0xffffffffu;
            c0->val_bytes = (uint64_t)lv[0].graph.num_entries * s * 8u;
        }
        *zpcg = pz;
    }
    return off;
}

// MODE 3: level 0 has pre-split values, so K1 runs the pre-split SpMV (K3
// writes the split copy of p) and the V-cycle's level-0 SpMVs run in MODE 3
template <int S, int MODE>
static int mg_run(int nl, const ens_mg_level *levels, const double *b, double *x, double tol, int max_iter,
                  int degree, double ratio, double boost, int power_iters, int flags, int check_every, void *work,
                  int32_t *iters_host, double *relres_host, int32_t *status_host, ens_cg_stats *stats,
                  cudaStream_t st) {
    MgSolver<S> mg;
    CgArgs c;
    memset(&c, 0, sizeof(c));
    double *z = nullptr;
    int *bad = nullptr;
    mg_pcg_layout(nl, levels, S, &mg.lv, static_cast<char *>(work), &c, &z, &mg.inv, &bad);
    mg.degree = degree;
    mg.f32 = levels[0].values_f32 != nullptr;
    mg.active = &c.st->active_count;
    mg.eg = 152 * 4;
    c.b = b;
    c.x = x;
    c.tol = tol;
    c.max_iter = max_iter;
    c.x0_zero = (flags & ENS_CG_X0_ZERO) ? 1 : 0;
    PcgArgs pa0 = mg.lv[0].pa;  // level 0: PCG state (rr) and the CG vectors
    pa0.c = c;
    int launches = 0, rc;
    ENS_CUDA_TRY(cudaMemsetAsync(c.st, 0, sizeof(CgState), st));
    if ((rc = mg.setup(levels, ratio, boost, power_iters, bad, st, &launches, (flags & ENS_PC_LANCZOS) != 0)))
        return rc;
    pa0.ps = mg.lv[0].pa.ps;
    ENS_LAUNCH_CHECK("ens_mg_pcg set-up");
    // the PCG trees of level 0 (the set-up reused them; clear again)
    if ((rc = dot_tree_clear(c.t1, st))) return rc;
    if ((rc = dot_tree_clear(c.t2, st))) return rc;
    const unsigned grid = MgSolver<S>::chunks(c.n);
    const unsigned vgrid = (unsigned)((c.t1.count[1] + VecMap<S>::CPC - 1) / VecMap<S>::CPC);
    CgArgs c3 = c;
    c3.r = z;
    auto stage = [&](int init, cudaStream_t s_) {
        if (!init) mg_pcg_resid_kernel<S><<<grid, RowMap<S>::THREADS, 0, s_>>>(pa0);
        if (mg.f32) mg.vcycle32(0, c.r, nullptr, mg.lv[0].x32, z, s_);
        else mg.vcycle(0, c.r, z, s_);
        mg_pcg_rz_kernel<S><<<grid, RowMap<S>::THREADS, 0, s_>>>(pa0, z, init);
        cg_update_kernel<S, MODE><<<vgrid, VecMap<S>::THREADS, 0, s_>>>(c3);
    };
    const int per_iter = 4 + mg.launches_per_vcycle();
    cg_init_kernel<S, MODE><<<grid, RowMap<S>::THREADS, 0, st>>>(c);
    cg_zero_kernel<S, MODE><<<152 * 2, 256, 0, st>>>(c);
    stage(1, st);
    launches += 2 + per_iter - 2;
    ENS_LAUNCH_CHECK("ens_mg_pcg init");
    int hbad = 0;
    ENS_CUDA_TRY(cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, st));
    ENS_CUDA_TRY(cudaStreamSynchronize(st));
    if (hbad) return fail(ENS_ERR_BREAKDOWN, "ens_mg_pcg: coarsest matrix not positive definite");

    const bool use_graph = (flags & ENS_CG_GRAPH) != 0;
    cudaGraphExec_t gexec = nullptr;
    cudaGraph_t graph = nullptr;
    const int max_blocks = max_iter / check_every + 3;
    // graph replay: the convergence test between blocks on the device (while node)
    bool device_loop = use_graph && use_device_loop();
    if (device_loop) {
        auto body = [&](cudaStream_t cap) {
            for (int i = 0; i < check_every; ++i) {
                k1_launch<S, MODE>(c, k1_default_nsub(S, MODE), cap);
                stage(0, cap);
            }
        };
        device_loop = while_graph_fn(body, &c.st->active_count, &c.st->loop_blocks, max_blocks, &graph, &gexec) ==
                      ENS_OK;
        if (device_loop) {
            if ((rc = launch_while_graph(graph, gexec, st))) return rc;
            graph = nullptr;
            gexec = nullptr;
        }
    }
    if (use_graph && !device_loop) {
        cudaStream_t cap;
        ENS_CUDA_TRY(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
        cudaError_t ce = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
        if (ce == cudaSuccess) {
            for (int i = 0; i < check_every; ++i) {
                k1_launch<S, MODE>(c, k1_default_nsub(S, MODE), cap);
                stage(0, cap);
            }
            ce = cudaStreamEndCapture(cap, &graph);
        }
        cudaStreamDestroy(cap);
        if (ce != cudaSuccess) return cuda_fail(ce, "ens_mg_pcg graph capture");
        ce = cudaGraphInstantiate(&gexec, graph, 0);
        if (ce != cudaSuccess) { cudaGraphDestroy(graph); return cuda_fail(ce, "cudaGraphInstantiate"); }
    }
    int32_t hflag[2];
    int polls = 0;
    rc = ENS_OK;
    for (int blk = 0; !device_loop && blk < max_blocks; ++blk) {
        if (use_graph) {
            cudaError_t ce = cudaGraphLaunch(gexec, st);
            if (ce != cudaSuccess) { rc = cuda_fail(ce, "cudaGraphLaunch"); break; }
        } else {
            for (int i = 0; i < check_every; ++i) {
                k1_launch<S, MODE>(c, k1_default_nsub(S, MODE), st);
                stage(0, st);
            }
        }
        launches += (per_iter + 1) * check_every;
        cudaError_t ce = cudaGetLastError();
        if (ce == cudaSuccess)
            ce = cudaMemcpyAsync(hflag, &c.st->active_count, 2 * sizeof(int32_t), cudaMemcpyDeviceToHost, st);
        if (ce == cudaSuccess) ce = cudaStreamSynchronize(st);
        if (ce != cudaSuccess) { rc = cuda_fail(ce, "ens_mg_pcg iteration"); break; }
        ++polls;
        if (hflag[0] == 0 && hflag[1] == 0) break;
    }
    if (gexec) cudaGraphExecDestroy(gexec);
    if (graph) cudaGraphDestroy(graph);
    if (rc != ENS_OK) return rc;
    cg_final_kernel<S><<<grid, RowMap<S>::THREADS, 0, st>>>(c);
    ++launches;
    ENS_LAUNCH_CHECK("ens_mg_pcg final");
    CgState hs;
    ENS_CUDA_TRY(cudaMemcpyAsync(&hs, c.st, sizeof(CgState), cudaMemcpyDeviceToHost, st));
    ENS_CUDA_TRY(cudaStreamSynchronize(st));
    if (device_loop) launches += ((per_iter + 1) * check_every + 1) * hs.loop_blocks;
    int maxit = 0, first_bad = ENS_OK;
    for (int e = 0; e < S; ++e) {
        if (iters_host) iters_host[e] = hs.iters[e];
        if (relres_host) relres_host[e] = hs.relres[e];
        if (status_host) status_host[e] = hs.status[e];
        maxit = hs.iters[e] > maxit ? hs.iters[e] : maxit;
        if (hs.status[e] != ENS_OK && first_bad == ENS_OK) first_bad = hs.status[e];
    }
    if (stats) {
        memset(stats, 0, sizeof(ens_cg_stats));
        stats->iterations = maxit;
        stats->kernel_launches = launches;
        stats->host_checks = polls;
    }
    if (first_bad != ENS_OK) set_error("ens_mg_pcg: member status %d (%s)", first_bad, ens_status_string(first_bad));
    return first_bad;
}

}  // namespace ens

using namespace ens;

extern "C" int ens_mg_workspace_size(int nlevels, const ens_mg_level *levels, int s, size_t *bytes) {
    int rc = mg_check(nlevels, levels, s);
    if (rc) return rc;
    if (!bytes) return fail(ENS_ERR_ARG, "bytes is NULL");
    *bytes = mg_pcg_layout(nlevels, levels, s, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr);
    return ENS_OK;
}

extern "C" int ens_mg_pcg(int nlevels, const ens_mg_level *levels, int s, const double *b, double *x, double tol,
                          int max_iter, int degree, double ratio, double boost, int power_iters, int flags,
                          int check_every, void *work, size_t work_bytes, int32_t *iters_host, double *relres_host,
                          int32_t *status_host, ens_cg_stats *stats_host, void *stream) {
    int rc = mg_check(nlevels, levels, s);
    if (rc) return rc;
    if (!b || !x || !work) return fail(ENS_ERR_ARG, "NULL b/x/work");
    if (!(tol >= 0.0) || max_iter < 0 || check_every < 1 || degree < 1 || degree > kPcMaxDegree ||
        !(ratio > 1.0) || !(boost >= 1.0) || power_iters < 1 || power_iters > 1000 ||
        ((flags & ENS_PC_LANCZOS) && power_iters > kLzMaxSteps))
        return fail(ENS_ERR_ARG, "ens_mg_pcg: bad tol/max_iter/check_every/degree/ratio/boost/power_iters");
    for (int l = 0; l < nlevels; ++l)
        if (!levels[l].power_start) return fail(ENS_ERR_ARG, "ens_mg_pcg: level %d: NULL power_start", l);
    if (!aligned16(work) || (s > 1 && (!aligned16(b) || !aligned16(x))))
        return fail(ENS_ERR_ALIGN, "b/x/work must be 16-byte aligned");
    const size_t need = mg_pcg_layout(nlevels, levels, s, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr);
    if (work_bytes < need) return fail(ENS_ERR_WORKSPACE, "mg workspace %zu < %zu bytes", work_bytes, need);
    cudaStream_t st = as_stream(stream);
    const bool pre = levels[0].values_df != nullptr;
#define MG_CALL(SS, MM)                                                                                        \
    mg_run<SS, MM>(nlevels, levels, b, x, tol, max_iter, degree, ratio, boost, power_iters, flags, check_every, \
                   work, iters_host, relres_host, status_host, stats_host, st)
    switch (s) {
        case 1: return pre ? MG_CALL(1, 3) : MG_CALL(1, 0);
        case 4: return pre ? MG_CALL(4, 3) : MG_CALL(4, 0);
        case 8: return pre ? MG_CALL(8, 3) : MG_CALL(8, 0);
        case 16: return pre ? MG_CALL(16, 3) : MG_CALL(16, 0);
        default: return pre ? MG_CALL(32, 3) : MG_CALL(32, 0);
    }
#undef MG_CALL
}
