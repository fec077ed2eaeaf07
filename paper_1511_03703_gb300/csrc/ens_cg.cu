// ens_cg.cu -- ensemble conjugate gradients (Sect. 3.4 solver, Sect. 4 experiments).
//
// Hestenes-Stiefel CG run on every member of the commuted ensemble system at
// once.  By default each member has its own alpha, beta and stopping test
// (dots reduced per member: the vector sum_i u_i^T v_i (x) e_i of Sect. 3.4
// before its members are added), so member e follows the iterates of a
// standalone solve of sample e; members that converge are frozen.  With
// ENS_CG_COUPLED the member dots are summed first, which is the paper's
// coupled ensemble solver of Sects. 3.4 and 3.7.
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
// Flag protocol: K1's epilogue sets updx_e for the members still active after
// its breakdown test, K3 reads them (before it waits for K2, when it is
// launched with a programmatic dependency on K2), and a K1 that exits early
// clears them.
#include <stdlib.h>

#include <vector>

#include "ens_cg_kernels.cuh"

namespace ens {

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

// K2 prefetches each CTA's r and q blocks into L2 before its passes; the
// ENS_K2_PREFETCH environment variable (0 or 1) overrides the default
static int k2_prefetch() {
    static const int v = [] {
        const char *e = getenv("ENS_K2_PREFETCH");
        return e ? (atoi(e) != 0) : 1;
    }();
    return v;
}

// K1 rows per CTA: the largest mapping a CTA of 1024 threads holds, and the
// default (measured on the 64^3 mesh; every mapping gives the same bits)
int k1_max_nsub_rt(int s) {
    switch (s) {
        case 1: return k1_max_nsub<1>();
        case 4: return k1_max_nsub<4>();
        case 8: return k1_max_nsub<8>();
        case 16: return k1_max_nsub<16>();
        default: return k1_max_nsub<32>();
    }
}

int k1_default_nsub(int s, int mode) {
    (void)mode;
    (void)s;
    return 1;   // one chunk per CTA measured fastest, or within 1 %, at every s (64^3 mesh)
}

// chunks per K1 CTA from the ENS_CG_K1_CHUNKS field of flags (0: default);
// 0 for the deferred tree (ENS_CG_K1_DEFER); -1 when the field asks for more
// than a 1024-thread CTA holds
static int k1_nsub_from_flags(int flags, int s, int mode) {
    const int f = (flags >> ENS_CG_K1_CHUNKS_SHIFT) & 7;
    if (flags & ENS_CG_K1_DEFER) return (f == 0 || f == 1) ? 0 : -1;
    if (f == 0) return k1_default_nsub(s, mode);
    const int nsub = 1 << (f - 1);
    return (f <= 4 && nsub <= k1_max_nsub_rt(s)) ? nsub : -1;
}

// ------------------------------------------------------ device-side loop
__global__ void loop_ctl_kernel(const int32_t *flags, int32_t *blocks, int max_blocks,
                                cudaGraphConditionalHandle h) {
    const int b = *blocks + 1;
    *blocks = b;
    const bool more = (flags[0] != 0 || flags[1] != 0) && b < max_blocks;
    cudaGraphSetConditional(h, more ? 1u : 0u);
}

static bool use_cg_pdl() {
    static const bool v = [] {
        const char *e = getenv("ENS_CG_PDL");
        return e ? (atoi(e) != 0) : true;
    }();
    return v;
}

bool use_device_loop() {
    static const bool v = [] {
        const char *e = getenv("ENS_DEVICE_LOOP");
        return e ? (atoi(e) != 0) : true;
    }();
    return v;
}

int while_graph(LoopBodyFn body, void *ctx, const int32_t *flags, int32_t *blocks, int max_blocks,
                cudaGraph_t *graph_out, cudaGraphExec_t *exec_out) {
    *graph_out = nullptr;
    *exec_out = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaStream_t cap = nullptr;
    cudaError_t ce = cudaGraphCreate(&graph, 0);
    cudaGraphConditionalHandle h = 0;
    if (ce == cudaSuccess) ce = cudaGraphConditionalHandleCreate(&h, graph, 1u, cudaGraphCondAssignDefault);
    cudaGraph_t bodyg = nullptr;
    if (ce == cudaSuccess) {
        cudaGraphNodeParams np = {};
        np.type = cudaGraphNodeTypeConditional;
        np.conditional.handle = h;
        np.conditional.type = cudaGraphCondTypeWhile;
        np.conditional.size = 1;
        cudaGraphNode_t node;
        ce = cudaGraphAddNode(&node, graph, nullptr, nullptr, 0, &np);
        if (ce == cudaSuccess) bodyg = np.conditional.phGraph_out[0];
    }
    if (ce == cudaSuccess) ce = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
    int rc = ENS_OK;
    if (ce == cudaSuccess) {
        ce = cudaStreamBeginCaptureToGraph(cap, bodyg, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
        if (ce == cudaSuccess) {
            rc = body(ctx, cap);
            loop_ctl_kernel<<<1, 1, 0, cap>>>(flags, blocks, max_blocks, h);
            cudaGraph_t got = nullptr;
            const cudaError_t ce2 = cudaStreamEndCapture(cap, &got);
            if (ce == cudaSuccess) ce = cudaGetLastError();
            if (ce == cudaSuccess) ce = ce2;
        }
    }
    if (cap) cudaStreamDestroy(cap);
    if (ce == cudaSuccess && rc == ENS_OK) ce = cudaGraphInstantiate(&exec, graph, 0);
    if (ce != cudaSuccess || rc != ENS_OK) {
        if (graph) cudaGraphDestroy(graph);
        cudaGetLastError();   // graph API errors are not sticky: clear for the caller's fallback
        return rc != ENS_OK ? rc : fail(ENS_ERR_CUDA, "device loop graph: %s", cudaGetErrorString(ce));
    }
    *graph_out = graph;
    *exec_out = exec;
    return ENS_OK;
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
    static void spmv(const CgArgs &a, int nsub, cudaStream_t st) { k1_launch<S, MODE>(a, nsub, st); }
    static void resid(const CgArgs &a, cudaStream_t st) {
        using L = K2Launch<S>;
        const unsigned grid = (unsigned)((a.t1.count[1] + L::CPC - 1) / L::CPC);
        cg_resid_kernel<S><<<grid, L::TH, 0, st>>>(a);
    }
    // K3 with a programmatic dependency on K2 (ENS_CG_PDL, default on): its
    // first CTAs start their x update as K2's last wave leaves SMs idle
    static void update(const CgArgs &a, cudaStream_t st) {
        if (use_cg_pdl()) {
            cudaLaunchConfig_t cfg = {};
            cfg.gridDim = dim3(vec_grid(a));
            cfg.blockDim = dim3(VecMap<S>::THREADS);
            cfg.dynamicSmemBytes = 0;
            cfg.stream = st;
            cudaLaunchAttribute at[1];
            at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
            at[0].val.programmaticStreamSerializationAllowed = 1;
            cfg.attrs = at;
            cfg.numAttrs = 1;
            cudaLaunchKernelEx(&cfg, cg_update_kernel<S, MODE>, a);
        } else {
            cg_update_kernel<S, MODE><<<vec_grid(a), VecMap<S>::THREADS, 0, st>>>(a);
        }
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
    a.k2_pf = k2_prefetch();
    const unsigned grid = (unsigned)a.t1.count[1];
    const int nsub = k1_nsub_from_flags(flags, S, MODE);
    int rc;
    if ((rc = dot_tree_clear(a.t1, st))) return rc;
    if ((rc = dot_tree_clear(a.t2, st))) return rc;
    ENS_CUDA_TRY(cudaMemsetAsync(a.st, 0, sizeof(CgState), st));

    const bool timing = (flags & ENS_CG_TIME_SPMV) != 0;
    const bool use_graph = (flags & ENS_CG_GRAPH) != 0;
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
    const int max_blocks = max_iter / check_every + 3;
    // ENS_CG_GRAPH without per-launch timing: the convergence test between
    // blocks runs on the device (while node); the host waits once
    bool device_loop = use_graph && !timing && use_device_loop();
    if (device_loop) {
        struct Ctx { const CgArgs *a; int nsub, check_every; } ctx{&a, nsub, check_every};
        LoopBodyFn body = [](void *c, cudaStream_t cap) -> int {
            const Ctx &x = *static_cast<const Ctx *>(c);
            for (int i = 0; i < x.check_every; ++i) {
                K::spmv(*x.a, x.nsub, cap);
                K::resid(*x.a, cap);
                K::update(*x.a, cap);
            }
            return ENS_OK;
        };
        device_loop = while_graph(body, &ctx, &a.st->active_count, &a.st->loop_blocks, max_blocks, &graph,
                                  &gexec) == ENS_OK;
        if (device_loop) {
            const cudaError_t ce = cudaGraphLaunch(gexec, st);
            cudaGraphExecDestroy(gexec);
            cudaGraphDestroy(graph);
            gexec = nullptr;
            graph = nullptr;
            if (ce != cudaSuccess) { destroy_events(); return cuda_fail(ce, "device loop graph launch"); }
        }
    }
    if (use_graph && !device_loop) {
        // capture on a private stream (the legacy default stream cannot be
        // captured); the graph is then launched on the caller's stream.  With
        // ENS_CG_TIME_SPMV the events around each SpMV become event-record
        // nodes of the graph and are read after every replay.
        cudaStream_t cap;
        ENS_CUDA_TRY(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
        cudaError_t ce = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
        if (ce == cudaSuccess) {
            for (int i = 0; i < check_every; ++i) {
                if (timing && ce == cudaSuccess) ce = cudaEventRecordWithFlags(ev[2 * i], cap, cudaEventRecordExternal);
                K::spmv(a, nsub, cap);
                if (timing && ce == cudaSuccess)
                    ce = cudaEventRecordWithFlags(ev[2 * i + 1], cap, cudaEventRecordExternal);
                K::resid(a, cap);
                K::update(a, cap);
            }
            const cudaError_t ce2 = cudaStreamEndCapture(cap, &graph);
            if (ce == cudaSuccess) ce = ce2;
        }
        cudaStreamDestroy(cap);
        if (ce != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            destroy_events();
            return cuda_fail(ce, "cg iteration graph capture");
        }
        ce = cudaGraphInstantiate(&gexec, graph, 0);
        if (ce != cudaSuccess) {
            cudaGraphDestroy(graph);
            destroy_events();
            return cuda_fail(ce, "cudaGraphInstantiate");
        }
    }

    int32_t flags_h[2];
    int iter_blocks = 0;
    rc = ENS_OK;
    while (!device_loop && iter_blocks < max_blocks) {
        if (use_graph) {
            cudaError_t ce = cudaGraphLaunch(gexec, st);
            if (ce != cudaSuccess) { rc = cuda_fail(ce, "cudaGraphLaunch"); break; }
        } else {
            for (int i = 0; i < check_every; ++i) {
                if (timing) cudaEventRecord(ev[2 * i], st);
                K::spmv(a, nsub, st);
                if (timing) cudaEventRecord(ev[2 * i + 1], st);
                K::resid(a, st);
                K::update(a, st);
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
    if (device_loop) launches += (3 * check_every + 1) * hs.loop_blocks;
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

// batched K1 CTA: TH threads (512, or 1024 with ENS_CG_BATCH_K1_WIDE), i.e.
// TH / (32 * RowMap<S>::G) chunks of an ensemble of size S per CTA
template <int S, int TH>
struct BatchK1 {
    static constexpr int NSUB = TH / RowMap<S>::THREADS;
    using Smem = K1Smem<S, NSUB>;
};

constexpr size_t cmax(size_t a, size_t b) { return a > b ? a : b; }
template <int TH>
constexpr size_t batch_k1_smem() {
    return cmax(cmax(cmax(sizeof(typename BatchK1<1, TH>::Smem), sizeof(typename BatchK1<4, TH>::Smem)),
                     cmax(sizeof(typename BatchK1<8, TH>::Smem), sizeof(typename BatchK1<16, TH>::Smem))),
                sizeof(typename BatchK1<32, TH>::Smem));
}
template <int S>
struct BatchK2 {   // the batched K2's chunks per CTA: a (chunk, slice) unit per S threads, one level-2 group at most
    static constexpr int CPC = (kBatchThreads / (kK2Slices * S) < 32) ? kBatchThreads / (kK2Slices * S) : 32;
};
template <int S>
constexpr size_t batch_k2_smem() { return sizeof(float2) * BatchK2<S>::CPC * kK2Slices * S; }
constexpr size_t kBatchK2Smem = cmax(cmax(cmax(batch_k2_smem<1>(), batch_k2_smem<4>()),
                                          cmax(batch_k2_smem<8>(), batch_k2_smem<16>())),
                                     batch_k2_smem<32>());

struct BItem {
    CgArgs a;
    int S;
    int k1_cta0, v_cta0, r_cta0;
};

struct BatchTables {
    const BItem *items;
    const int *k1_map;  // CTA -> item for K1 launches
    const int *v_map;   // CTA -> item for K3 launches
    const int *r_map;   // CTA -> item for K2 launches
};

template <int MODE, int TH>
__global__ void __launch_bounds__(TH, 1024 / TH) cg_spmv_batched(BatchTables bt) {
    extern __shared__ __align__(16) unsigned char raw[];   // batch_k1_smem<TH>() bytes
    const BItem &it = bt.items[__ldg(bt.k1_map + blockIdx.x)];
    const int cta = blockIdx.x - it.k1_cta0;
#define ENS_BK1(SS) \
    k1_body<SS, MODE, BatchK1<SS, TH>::NSUB, true>(it.a, cta, *reinterpret_cast<typename BatchK1<SS, TH>::Smem *>(raw))
    switch (it.S) {
        case 1: ENS_BK1(1); break;
        case 4: ENS_BK1(4); break;
        case 8: ENS_BK1(8); break;
        case 16: ENS_BK1(16); break;
        default: ENS_BK1(32); break;
    }
#undef ENS_BK1
}

template <int S>
__device__ __forceinline__ void k2_batched_s(const CgArgs &a, int cta, unsigned char *raw) {
    k2_body<S, kBatchThreads, BatchK2<S>::CPC, true>(a, cta, reinterpret_cast<float2(*)[kK2Slices][S]>(raw));
}

// 64 registers (a slice's 16 loads in flight per thread), 2 CTAs per SM, as
// the single-ensemble K2
__global__ void __launch_bounds__(kBatchThreads, 2) cg_resid_batched(BatchTables bt) {
    __shared__ __align__(16) unsigned char raw[kBatchK2Smem];
    const BItem &it = bt.items[__ldg(bt.r_map + blockIdx.x)];
    const int cta = blockIdx.x - it.r_cta0;
    switch (it.S) {
        case 1: k2_batched_s<1>(it.a, cta, raw); break;
        case 4: k2_batched_s<4>(it.a, cta, raw); break;
        case 8: k2_batched_s<8>(it.a, cta, raw); break;
        case 16: k2_batched_s<16>(it.a, cta, raw); break;
        default: k2_batched_s<32>(it.a, cta, raw); break;
    }
}

template <int MODE>
__global__ void __launch_bounds__(kBatchThreads, 3) cg_update_batched(BatchTables bt) {
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
    a.k2_pf = k2_prefetch();
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

static int64_t batch_k1_ctas(int S, int64_t chunks, int th = kBatchThreads) {
    const int nsub = th / (32 * ((S == 1) ? 2 : S / 2));
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

static int64_t batch_r_ctas(int S, int64_t chunks) {
    int cpc = 0;
    switch (S) {
        case 1: cpc = BatchK2<1>::CPC; break;
        case 4: cpc = BatchK2<4>::CPC; break;
        case 8: cpc = BatchK2<8>::CPC; break;
        case 16: cpc = BatchK2<16>::CPC; break;
        default: cpc = BatchK2<32>::CPC; break;
    }
    return (chunks + cpc - 1) / cpc;
}

struct BatchPlan {
    size_t head;           // items + poll words + CTA maps
    int64_t k1_total, v_total, r_total;
    size_t total;
};

static BatchPlan batch_plan(int n_items, const ens_batch_item *items) {
    BatchPlan p{};
    for (int i = 0; i < n_items; ++i) {
        const int64_t chunks = ((int64_t)items[i].graph.num_rows + 31) / 32;
        p.k1_total += batch_k1_ctas(items[i].s, chunks);
        p.v_total += batch_v_ctas(items[i].s, chunks);
        p.r_total += batch_r_ctas(items[i].s, chunks);
    }
    p.head = align256(sizeof(BItem) * n_items) + 256 + align256(sizeof(int) * (size_t)p.k1_total) +
             align256(sizeof(int) * (size_t)p.v_total) + align256(sizeof(int) * (size_t)p.r_total);
    p.total = p.head;
    for (int i = 0; i < n_items; ++i) p.total += cg_bytes(items[i].graph.num_rows, items[i].s);
    return p;
}

template <int MODE, int TH>
static void launch_k1_batched(unsigned grid, const BatchTables &bt, cudaStream_t st) {
    cg_spmv_batched<MODE, TH><<<grid, TH, batch_k1_smem<TH>(), st>>>(bt);
}

template <int MODE>
static int batched_run(int n_items, const ens_batch_item *items, double tol, int max_iter,
                       int flags, int check_every, void *work, ens_cg_stats *stats,
                       cudaStream_t st) {
    const BatchPlan plan = batch_plan(n_items, items);
    // K1 CTA size: the plan's CTA maps are sized for 512 threads, the most CTAs
    const int th = (flags & ENS_CG_BATCH_K1_WIDE) ? 1024 : kBatchThreads;
    ENS_CUDA_TRY(cudaFuncSetAttribute(cg_spmv_batched<MODE, 512>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)batch_k1_smem<512>()));
    ENS_CUDA_TRY(cudaFuncSetAttribute(cg_spmv_batched<MODE, 1024>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)batch_k1_smem<1024>()));
    char *w = static_cast<char *>(work);
    BItem *d_items = reinterpret_cast<BItem *>(w);
    int *d_poll = reinterpret_cast<int *>(w + align256(sizeof(BItem) * n_items));
    int *d_k1map = reinterpret_cast<int *>(w + align256(sizeof(BItem) * n_items) + 256);
    int *d_vmap = d_k1map + align256(sizeof(int) * (size_t)plan.k1_total) / sizeof(int);
    int *d_rmap = d_vmap + align256(sizeof(int) * (size_t)plan.v_total) / sizeof(int);
    char *wi = w + plan.head;
    std::vector<BItem> h(n_items);
    std::vector<int> k1map((size_t)plan.k1_total), vmap((size_t)plan.v_total), rmap((size_t)plan.r_total);
    int64_t k1c = 0, vc = 0, rcn = 0;
    int rc;
    for (int i = 0; i < n_items; ++i) {
        const ens_batch_item &it = items[i];
        cg_layout_args(h[i].a, &it.graph, it.s, it.values, it.b, it.x, tol, max_iter,
                       flags, wi);
        if (MODE == 3) {  // pre-split values; a whole-chunk CTA prefetches its value block into L2
            h[i].a.vdf = reinterpret_cast<const float2 *>(it.values_df);
            h[i].a.val_bytes = (uint64_t)it.graph.num_entries * it.s * 8u;
            h[i].a.pf_cap = l2_prefetch_cap(3);
        }
        wi += cg_bytes(it.graph.num_rows, it.s);
        h[i].S = it.s;
        const int64_t chunks = h[i].a.t1.count[1];
        const int64_t nk = batch_k1_ctas(it.s, chunks, th), nv = batch_v_ctas(it.s, chunks),
                      nr = batch_r_ctas(it.s, chunks);
        h[i].k1_cta0 = (int)k1c;
        h[i].v_cta0 = (int)vc;
        h[i].r_cta0 = (int)rcn;
        for (int64_t c = 0; c < nk; ++c) k1map[k1c++] = i;
        for (int64_t c = 0; c < nv; ++c) vmap[vc++] = i;
        for (int64_t c = 0; c < nr; ++c) rmap[rcn++] = i;
        if ((rc = dot_tree_clear(h[i].a.t1, st))) return rc;
        if ((rc = dot_tree_clear(h[i].a.t2, st))) return rc;
        ENS_CUDA_TRY(cudaMemsetAsync(h[i].a.st, 0, sizeof(CgState), st));
    }
    ENS_CUDA_TRY(cudaMemcpyAsync(d_items, h.data(), sizeof(BItem) * n_items, cudaMemcpyHostToDevice, st));
    ENS_CUDA_TRY(cudaMemcpyAsync(d_k1map, k1map.data(), sizeof(int) * k1map.size(), cudaMemcpyHostToDevice, st));
    ENS_CUDA_TRY(cudaMemcpyAsync(d_vmap, vmap.data(), sizeof(int) * vmap.size(), cudaMemcpyHostToDevice, st));
    ENS_CUDA_TRY(cudaMemcpyAsync(d_rmap, rmap.data(), sizeof(int) * rmap.size(), cudaMemcpyHostToDevice, st));
    int launches = 0, polls = 0;
    for (int i = 0; i < n_items; ++i) { launch_single<MODE>(0, h[i].S, h[i].a, st); launches += 2; }
    ENS_LAUNCH_CHECK("batched cg init");
    const BatchTables bt{d_items, d_k1map, d_vmap, d_rmap};
    const unsigned g1 = (unsigned)k1c, gv = (unsigned)plan.v_total, gr = (unsigned)plan.r_total;
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
        if (th == 1024) launch_k1_batched<MODE, 1024>(g1, bt, s2);
        else launch_k1_batched<MODE, 512>(g1, bt, s2);
        if (timing) cudaEventRecord(ev[2 * i + 1], s2);
        cg_resid_batched<<<gr, kBatchThreads, 0, s2>>>(bt);
        cg_update_batched<MODE><<<gv, kBatchThreads, 0, s2>>>(bt);
    };
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t gexec = nullptr;
    const int max_blocks = max_iter / check_every + 3;
    // graph replay without timing: the convergence test between blocks on the
    // device (while node; d_poll[2] counts the blocks)
    bool device_loop = use_graph && !timing && use_device_loop();
    if (device_loop) {
        ENS_CUDA_TRY(cudaMemsetAsync(d_poll + 2, 0, sizeof(int), st));
        auto body = [&](cudaStream_t cap) {
            for (int i = 0; i < check_every; ++i) iteration(cap, i);
            batch_poll_kernel<<<1, 64, 0, cap>>>(d_items, n_items, d_poll);
        };
        device_loop = while_graph_fn(body, d_poll, d_poll + 2, max_blocks, &graph, &gexec) == ENS_OK;
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
    rc = ENS_OK;
    for (int blk = 0; !device_loop && blk < max_blocks; ++blk) {
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
    int32_t loop_blocks = 0;
    if (device_loop) ENS_CUDA_TRY(cudaMemcpyAsync(&loop_blocks, d_poll + 2, sizeof(int), cudaMemcpyDeviceToHost, st));
    ENS_CUDA_TRY(cudaStreamSynchronize(st));
    if (device_loop) launches += (3 * check_every + 2) * loop_blocks;
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
    if (k1_nsub_from_flags(flags, s, 0) < 0)
        return fail(ENS_ERR_ARG, "ENS_CG_K1_CHUNKS field %d: at most %d chunks of 32 rows per K1 CTA at s=%d "
                    "(one with ENS_CG_K1_DEFER)", (flags >> ENS_CG_K1_CHUNKS_SHIFT) & 7, k1_max_nsub_rt(s), s);
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
        if ((items[i].values_df != nullptr) != (items[0].values_df != nullptr))
            return fail(ENS_ERR_ARG, "item %d: either every item gives values_df or none", i);
        if (items[i].values_df && !aligned16(items[i].values_df))
            return fail(ENS_ERR_ALIGN, "item %d: values_df must be 16-byte aligned", i);
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
    if (items[0].values_df) {
        if (flags & (ENS_CG_DF64 | ENS_CG_SPLIT64))
            return fail(ENS_ERR_ARG, "ens_cg_batched: values_df excludes ENS_CG_DF64 / ENS_CG_SPLIT64");
        return batched_run<3>(n_items, items, tol, max_iter, flags, check_every, work, stats_host, st);
    }
    if (flags & ENS_CG_SPLIT64) return batched_run<2>(n_items, items, tol, max_iter, flags, check_every, work, stats_host, st);
    if (flags & ENS_CG_DF64) return batched_run<1>(n_items, items, tol, max_iter, flags, check_every, work, stats_host, st);
    return batched_run<0>(n_items, items, tol, max_iter, flags, check_every, work, stats_host, st);
}
