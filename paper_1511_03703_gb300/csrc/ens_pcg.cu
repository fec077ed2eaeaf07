// ens_pcg.cu -- preconditioned ensemble CG with Jacobi or Chebyshev
// preconditioning.  The paper preconditions its CG by multigrid whose
// smoothers are order-2 Chebyshev polynomials (Sect. 3.5); here the two
// SpMV-based preconditioners serve on their own, per member:
//   Jacobi     z = D^-1 r
//   Chebyshev  z = p(D^-1 A) D^-1 r, `degree` steps of Chebyshev iteration for
//              A z = r from z = 0 on [lam/ratio, lam] (Saad, Sect. 12.3), lam =
//              boost x a power-iteration estimate of the largest eigenvalue
//              of D^-1 A (the generalized Rayleigh quotient v.Av / v.Dv after
//              `power_iters` normalised steps from a given start vector).
// The CG part reuses the kernels of ens_cg.cu with rho = r.z:
//   K0  r = b - A x0 (as ens_cg)           KP  z = M^-1 r0, rho = r.z, beta = 0
//   per iteration:
//   K1  q = A p, p.q -> alpha              P2  r -= alpha q, z_1 (Jacobi: z), r.r
//   PC  (Chebyshev, degree - 1 times) w = r - A z_k, d, z_{k+1}; the last one r.z
//   K3  x += alpha p, p = z + beta p
// The stop test ||r|| <= tol ||b|| and beta = (r.z)_new / (r.z)_old run in the
// CTA that completes the last tree of the preconditioner stage.  All
// arithmetic is FP64 (the FP64 SpMV form).
#include <stdlib.h>

#include <vector>

#include "ens_pcg_kernels.cuh"

namespace ens {

// P2: r -= alpha q for active members (not at init); z_1 = D^-1 r (Jacobi) or
// D^-1 r / theta (Chebyshev, also d = z_1); dots r.r and r.z_1.  Final when
// degree <= 1.
template <int S>
__global__ void __launch_bounds__(RowMap<S>::THREADS, 1024 / RowMap<S>::THREADS) pc_resid_kernel(PcgArgs a,
                                                                                                 int init) {
    const CgArgs &c = a.c;
    if (ld_cg(&c.st->active_count) == 0) return;
    constexpr int G = RowMap<S>::G;
    __shared__ double sm[32][S + 1];
    const int r = threadIdx.x / G, g = threadIdx.x % G;
    const int64_t R = (int64_t)blockIdx.x * 32 + r;
    const CgState *cs = c.st;
    double rr0 = 0.0, rr1 = 0.0, rz0 = 0.0, rz1 = 0.0;
    if (R < c.n) {
        const int w = (S == 1) ? 1 : 2;
        const int64_t i0 = (S == 1) ? R : R * S + 2 * g;
        for (int k = 0; k < w; ++k) {
            if (S == 1 && g != 0) break;
            const int64_t i = i0 + k;
            const int e = (S == 1) ? 0 : 2 * g + k;
            double rv = c.r[i];
            if (!init && cs->active[e]) {
                rv = fma(-cs->alpha[e], c.q[i], rv);
                c.r[i] = rv;
            }
            double z = rv * a.dinv[i];
            if (a.degree >= 1) {
                z = z * a.ps->inv_theta[e];
                a.d[i] = z;
            }
            a.zk[0][i] = z;
            if (k == 0) { rr0 = rv * rv; rz0 = rv * z; }
            else { rr1 = rv * rv; rz1 = rv * z; }
        }
    }
    // (s = 1: chunk_tree takes the row's value from lane g = 0)
    chunk_tree<S>(sm, rr0, rr1, r, g, c.t2, blockIdx.x, 0);
    chunk_tree<S>(sm, rz0, rz1, r, g, c.t2, blockIdx.x, S);
    if (!dot_tree_propagate(c.t2, blockIdx.x, 1)) return;
    if (threadIdx.x >= 32) return;
    const int e = threadIdx.x;
    const double *top = c.t2.buf[c.t2.levels];
    const double rr = (e < S) ? ld_cg(top + e) : 0.0, rz = (e < S) ? ld_cg(top + S + e) : 0.0;
    if (a.degree <= 1) {
        pc_epilogue<S>(a, rr, rz, init != 0);
    } else {
        if (e < S) a.ps->rr[e] = rr;
        __threadfence();
    }
}

// PC step k (1 <= k < degree): w = r - A z_k, d = rho_k rho_{k-1} d + (2 rho_k / delta) D^-1 w,
// z_{k+1} = z_k + d; the last step also forms r.z and runs the epilogue
template <int S>
__global__ void __launch_bounds__(RowMap<S>::THREADS, 1024 / RowMap<S>::THREADS) pc_cheb_kernel(PcgArgs a, int k,
                                                                                                int init) {
    const CgArgs &c = a.c;
    if (ld_cg(&c.st->active_count) == 0) return;
    constexpr int G = RowMap<S>::G;
    __shared__ double sm[32][S + 1];
    __shared__ ChunkCols cc;
    const int r = threadIdx.x / G, g = threadIdx.x % G;
    const int64_t R = (int64_t)blockIdx.x * 32 + r;
    const double *zin = a.zk[(k - 1) & 1];
    double *zout = a.zk[k & 1];
    const bool last = (k == a.degree - 1);
    const bool staged = stage_chunk(cc, c.row_map, c.col, blockIdx.x, c.n);
    const double2 az = chunk_spmv<S, double>(cc, staged, c.col, c.vals, zin, r, g, R < c.n);
    const PcgState *ps = a.ps;
    double rz0 = 0.0, rz1 = 0.0;
    if (R < c.n && (S != 1 || g == 0)) {
        const int w = (S == 1) ? 1 : 2;
        const int64_t i0 = (S == 1) ? R : R * S + 2 * g;
        for (int j = 0; j < w; ++j) {
            const int64_t i = i0 + j;
            const int e = (S == 1) ? 0 : 2 * g + j;
            const double axv = (j == 0) ? az.x : az.y;
            const double rk = ps->rhoc[k][e], rk1 = ps->rhoc[k - 1][e];
            const double rv = c.r[i];
            const double dv = rk * rk1 * a.d[i] + ps->c2[k][e] * (a.dinv[i] * (rv - axv));
            const double zv = zin[i] + dv;
            a.d[i] = dv;
            zout[i] = zv;
            if (j == 0) rz0 = rv * zv;
            else rz1 = rv * zv;
        }
    }
    if (!last) return;
    chunk_tree<S>(sm, rz0, rz1, r, g, c.t1, blockIdx.x, 0);
    if (!dot_tree_propagate(c.t1, blockIdx.x, 1)) return;
    if (threadIdx.x >= 32) return;
    const int e = threadIdx.x;
    const double rz = (e < S) ? ld_cg(c.t1.buf[c.t1.levels] + e) : 0.0;
    const double rr = (e < S) ? a.ps->rr[e] : 0.0;
    pc_epilogue<S>(a, rr, rz, init != 0);
}


// ------------------------------------------------------------ host side
static size_t pc_align(size_t x) { return (x + 255) / 256 * 256; }

static size_t pcg_bytes(int64_t n, int s) {
    const size_t vec = pc_align(sizeof(double) * (size_t)n * s);
    return pc_align(sizeof(CgState)) + pc_align(sizeof(PcgState)) + 11 * vec + dot_tree_bytes(n, s) +
           dot_tree_bytes(n, 2 * s);
}

struct PcgOut {
    int32_t *iters;
    double *relres;
    int32_t *status;
    double *lam;
    ens_cg_stats *stats;
};

template <int S>
static int pcg_run(const ens_graph *g, const double *vals, const double *b, double *x, double tol, int max_iter,
                   int degree, double ratio, double boost, int power_iters, const double *v0, int flags,
                   int check_every, void *work, PcgOut out, cudaStream_t st) {
    const int64_t n = g->num_rows;
    const size_t vec = pc_align(sizeof(double) * (size_t)n * S);
    char *w = static_cast<char *>(work);
    PcgArgs a;
    CgArgs &c = a.c;
    memset(&a, 0, sizeof(a));
    c.n = g->num_rows;
    c.row_map = g->row_map;
    c.col = g->col_entry;
    c.vals = vals;
    c.vdf = nullptr;
    c.b = b;
    c.x = x;
    c.st = reinterpret_cast<CgState *>(w); w += pc_align(sizeof(CgState));
    a.ps = reinterpret_cast<PcgState *>(w); w += pc_align(sizeof(PcgState));
    c.r = reinterpret_cast<double *>(w); w += vec;
    c.p = reinterpret_cast<double *>(w); w += vec;
    c.q = reinterpret_cast<double *>(w); w += vec;
    c.pdf = reinterpret_cast<float2 *>(w); w += vec;
    a.zk[0] = reinterpret_cast<double *>(w); w += vec;
    a.zk[1] = reinterpret_cast<double *>(w); w += vec;
    a.d = reinterpret_cast<double *>(w); w += vec;
    double *dg = reinterpret_cast<double *>(w); w += vec;
    double *dinv = reinterpret_cast<double *>(w); w += vec;
    a.dg = dg;
    a.dinv = dinv;
    a.v = reinterpret_cast<double *>(w); w += vec;
    a.y = reinterpret_cast<double *>(w); w += vec;
    dot_tree_layout(&c.t1, n, S, w);
    w += dot_tree_bytes(n, S);
    dot_tree_layout(&c.t2, n, 2 * S, w);
    c.tol = tol;
    c.max_iter = max_iter;
    c.coupled = 0;
    c.fallback = 0;
    c.x0_zero = (flags & ENS_CG_X0_ZERO) ? 1 : 0;
    c.pf_cap = 0;
    c.val_bytes = 0;
    a.degree = degree;
    a.boost = boost;
    a.ratio = ratio;
    const unsigned grid = (unsigned)c.t1.count[1];
    const unsigned vgrid = (unsigned)((c.t1.count[1] + VecMap<S>::CPC - 1) / VecMap<S>::CPC);
    int rc;
    if ((rc = dot_tree_clear(c.t1, st))) return rc;
    if ((rc = dot_tree_clear(c.t2, st))) return rc;
    ENS_CUDA_TRY(cudaMemsetAsync(c.st, 0, sizeof(CgState), st));
    ENS_CUDA_TRY(cudaMemsetAsync(a.ps, 0, sizeof(PcgState), st));
    int launches = 0;
    const int64_t nt = n * S;
    pc_diag_kernel<S><<<(unsigned)((nt + 255) / 256), 256, 0, st>>>(c.n, c.row_map, c.col, vals, dg, dinv);
    ++launches;
    if (degree >= 1) {  // largest eigenvalue of D^-1 A, then the Chebyshev parameters
        ENS_CUDA_TRY(cudaMemcpyAsync(a.v, v0, sizeof(double) * (size_t)nt, cudaMemcpyDeviceToDevice, st));
        if (flags & ENS_PC_LANCZOS) {   // c.q holds q_{j-1} (the CG has not started)
            launches += lanczos_bound<S, 0>(a, c.q, grid, power_iters, st);
        } else {
            for (int k = 0; k < power_iters; ++k) {
                pc_power_kernel<S><<<grid, RowMap<S>::THREADS, 0, st>>>(a);
                pc_scale_kernel<S><<<152 * 4, 256, 0, st>>>(a);
                launches += 2;
            }
            pc_rayleigh_kernel<S><<<grid, RowMap<S>::THREADS, 0, st>>>(a);
            ++launches;
        }
    }
    ENS_LAUNCH_CHECK("ens_pcg set-up");
    // final z buffer of the preconditioner stage (K3 reads it as "r")
    CgArgs c3 = c;
    c3.r = a.zk[(degree >= 2) ? ((degree - 1) & 1) : 0];
    auto precond = [&](int init, cudaStream_t s_) {
        pc_resid_kernel<S><<<grid, RowMap<S>::THREADS, 0, s_>>>(a, init);
        for (int k = 1; k < degree; ++k) pc_cheb_kernel<S><<<grid, RowMap<S>::THREADS, 0, s_>>>(a, k, init);
        cg_update_kernel<S, 0><<<vgrid, VecMap<S>::THREADS, 0, s_>>>(c3);
    };
    const int per_iter = 2 + (degree >= 2 ? degree - 1 : 0) + 1;
    cg_init_kernel<S, 0><<<grid, RowMap<S>::THREADS, 0, st>>>(c);
    cg_zero_kernel<S, 0><<<152 * 2, 256, 0, st>>>(c);
    precond(1, st);
    launches += 2 + per_iter - 1;
    ENS_LAUNCH_CHECK("ens_pcg init");

    const bool use_graph = (flags & ENS_CG_GRAPH) != 0;
    cudaGraphExec_t gexec = nullptr;
    cudaGraph_t graph = nullptr;
    const int max_blocks = max_iter / check_every + 3;
    // graph replay: the convergence test between blocks on the device (while node)
    bool device_loop = use_graph && use_device_loop();
    if (device_loop) {
        auto body = [&](cudaStream_t cap) {
            for (int i = 0; i < check_every; ++i) {
                k1_launch<S, 0>(c, k1_default_nsub(S, 0), cap);
                precond(0, cap);
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
                k1_launch<S, 0>(c, k1_default_nsub(S, 0), cap);
                precond(0, cap);
            }
            ce = cudaStreamEndCapture(cap, &graph);
        }
        cudaStreamDestroy(cap);
        if (ce != cudaSuccess) return cuda_fail(ce, "ens_pcg graph capture");
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
                k1_launch<S, 0>(c, k1_default_nsub(S, 0), st);
                precond(0, st);
            }
        }
        launches += per_iter * check_every;
        cudaError_t ce = cudaGetLastError();
        if (ce == cudaSuccess)
            ce = cudaMemcpyAsync(hflag, &c.st->active_count, 2 * sizeof(int32_t), cudaMemcpyDeviceToHost, st);
        if (ce == cudaSuccess) ce = cudaStreamSynchronize(st);
        if (ce != cudaSuccess) { rc = cuda_fail(ce, "ens_pcg iteration"); break; }
        ++polls;
        if (hflag[0] == 0 && hflag[1] == 0) break;
    }
    if (gexec) cudaGraphExecDestroy(gexec);
    if (graph) cudaGraphDestroy(graph);
    if (rc != ENS_OK) return rc;
    cg_final_kernel<S><<<grid, RowMap<S>::THREADS, 0, st>>>(c);
    ++launches;
    ENS_LAUNCH_CHECK("ens_pcg final");
    CgState hs;
    PcgState hp;
    ENS_CUDA_TRY(cudaMemcpyAsync(&hs, c.st, sizeof(CgState), cudaMemcpyDeviceToHost, st));
    ENS_CUDA_TRY(cudaMemcpyAsync(&hp, a.ps, sizeof(PcgState), cudaMemcpyDeviceToHost, st));
    ENS_CUDA_TRY(cudaStreamSynchronize(st));
    if (device_loop) launches += (per_iter * check_every + 1) * hs.loop_blocks;
    int maxit = 0, first_bad = ENS_OK;
    for (int e = 0; e < S; ++e) {
        if (out.iters) out.iters[e] = hs.iters[e];
        if (out.relres) out.relres[e] = hs.relres[e];
        if (out.status) out.status[e] = hs.status[e];
        if (out.lam) out.lam[e] = (degree >= 1) ? hp.lam[e] : 0.0;
        maxit = hs.iters[e] > maxit ? hs.iters[e] : maxit;
        if (hs.status[e] != ENS_OK && first_bad == ENS_OK) first_bad = hs.status[e];
    }
    if (out.stats) {
        memset(out.stats, 0, sizeof(ens_cg_stats));
        out.stats->iterations = maxit;
        out.stats->kernel_launches = launches;
        out.stats->host_checks = polls;
    }
    if (first_bad != ENS_OK)
        set_error("ens_pcg: member status %d (%s)", first_bad, ens_status_string(first_bad));
    return first_bad;
}

}  // namespace ens

using namespace ens;

extern "C" int ens_pcg_workspace_size(int32_t num_rows, int s, size_t *bytes) {
    if (num_rows < 0) return fail(ENS_ERR_ARG, "num_rows < 0");
    if (!supported_s(s)) return fail(ENS_ERR_UNSUPPORTED, "ensemble size s=%d not in {1,4,8,16,32}", s);
    if (!bytes) return fail(ENS_ERR_ARG, "bytes is NULL");
    *bytes = pcg_bytes(num_rows, s);
    return ENS_OK;
}

extern "C" int ens_pcg(const ens_graph *graph, int s, const double *values, const double *b, double *x,
                       double tol, int max_iter, int precond, int degree, double ratio, double boost,
                       int power_iters, const double *power_start, int flags, int check_every, void *work,
                       size_t work_bytes, int32_t *iters_host, double *relres_host, int32_t *status_host,
                       double *lam_host, ens_cg_stats *stats_host, void *stream) {
    int rc = check_graph(graph);
    if (rc) return rc;
    if (!supported_s(s)) return fail(ENS_ERR_UNSUPPORTED, "ensemble size s=%d not in {1,4,8,16,32}", s);
    if (graph->num_rows == 0) return fail(ENS_ERR_ARG, "empty graph");
    if (!values || !b || !x || !work) return fail(ENS_ERR_ARG, "NULL values/b/x/work");
    if (!(tol >= 0.0) || max_iter < 0 || check_every < 1)
        return fail(ENS_ERR_ARG, "tol=%g max_iter=%d check_every=%d", tol, max_iter, check_every);
    int deg = 0;
    if (precond == ENS_PC_CHEBYSHEV) {
        if (degree < 1 || degree > kPcMaxDegree || !(ratio > 1.0) || !(boost >= 1.0) || power_iters < 1 ||
            power_iters > 1000 || ((flags & ENS_PC_LANCZOS) && power_iters > kLzMaxSteps) || !power_start)
            return fail(ENS_ERR_ARG, "chebyshev: 1 <= degree <= %d, ratio > 1, boost >= 1, 1 <= power_iters <= 1000 "
                        "(<= %d Lanczos steps), power_start given", kPcMaxDegree, kLzMaxSteps);
        deg = degree;
    } else if (precond != ENS_PC_JACOBI) {
        return fail(ENS_ERR_UNSUPPORTED, "precond %d (ENS_PC_JACOBI or ENS_PC_CHEBYSHEV)", precond);
    }
    if (!aligned16(work) || (s > 1 && (!aligned16(values) || !aligned16(b) || !aligned16(x))))
        return fail(ENS_ERR_ALIGN, "values/b/x/work must be 16-byte aligned");
    const size_t need = pcg_bytes(graph->num_rows, s);
    if (work_bytes < need) return fail(ENS_ERR_WORKSPACE, "pcg workspace %zu < %zu bytes", work_bytes, need);
    PcgOut out{iters_host, relres_host, status_host, lam_host, stats_host};
    cudaStream_t st = as_stream(stream);
    switch (s) {
        case 1: return pcg_run<1>(graph, values, b, x, tol, max_iter, deg, ratio, boost, power_iters, power_start,
                                  flags, check_every, work, out, st);
        case 4: return pcg_run<4>(graph, values, b, x, tol, max_iter, deg, ratio, boost, power_iters, power_start,
                                  flags, check_every, work, out, st);
        case 8: return pcg_run<8>(graph, values, b, x, tol, max_iter, deg, ratio, boost, power_iters, power_start,
                                  flags, check_every, work, out, st);
        case 16: return pcg_run<16>(graph, values, b, x, tol, max_iter, deg, ratio, boost, power_iters, power_start,
                                    flags, check_every, work, out, st);
        default: return pcg_run<32>(graph, values, b, x, tol, max_iter, deg, ratio, boost, power_iters, power_start,
                                    flags, check_every, work, out, st);
    }
}
