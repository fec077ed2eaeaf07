// ens_dot_static.cu -- ens_dot for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc at the point where they need a dot
// product: code running while a memory pool is locked or being captured,
// hosts whose allocator is owned by another runtime, or plug-ins that must
// not touch the process's allocation state.  ens_dot_static computes exactly
// what ens_dot computes (same kernel, same reduction tree, bitwise the same
// result) but takes its reduction scratch from a file-scope device array of
// ENS_DOT_STATIC_MAX_BYTES bytes instead of a caller workspace.  Every GPU
// that loads this library holds that array until the process exits.
//
// The device address of the array is looked up once per device and context,
// on the first call made with that device current (cudaGetSymbolAddress), so
// that first call should come before any stream capture.  The cached address
// is keyed on the current context's unique ID as well (cuCtxGetId, reached
// through cudaGetDriverEntryPointByVersion, so the library needs no link
// against the driver): after a device reset, or any other change of the
// primary context, the next call looks the address up again instead of using
// an address of the destroyed context.  All calls share the one array and it
// keeps the previous call's contents; the call clears the arrival counters it
// needs before launching, and calls that overlap on the GPU (different
// streams, or different host threads, at the same time) race on it.
#include <mutex>

#include "ens_internal.cuh"

namespace ens {

int dot_launch(int64_t n, int s, const double *u, const double *v, double *out,
               const DotTree &t, cudaStream_t st);

static __device__ __align__(256) unsigned char g_dot_static_scratch[ENS_DOT_STATIC_MAX_BYTES];

constexpr int kMaxDevices = 64;
static std::mutex g_static_mu;
static void *g_static_ptr[kMaxDevices] = {};
static unsigned long long g_static_ctx[kMaxDevices] = {};

// unique ID of the calling thread's current context (0 if the driver entry
// points are not available; the cache is then per device only)
typedef int (*CtxGetCurrentFn)(void **ctx);
typedef int (*CtxGetIdFn)(void *ctx, unsigned long long *id);
static unsigned long long current_context_id() {
    static CtxGetCurrentFn get_current = nullptr;
    static CtxGetIdFn get_id = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_current = reinterpret_cast<CtxGetCurrentFn>(f);
        f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_id = reinterpret_cast<CtxGetIdFn>(f);
    });
    if (!get_current || !get_id) return 0ull;
    void *ctx = nullptr;
    unsigned long long id = 0ull;
    if (get_current(&ctx) != 0 || !ctx || get_id(ctx, &id) != 0) return 0ull;
    return id;
}

// device address of the scratch array on the current device and context
// (looked up on the first call, and again when the context has changed)
static int static_scratch(void **out) {
    int dev = -1;
    ENS_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return fail(ENS_ERR_UNSUPPORTED, "device ordinal %d", dev);
    const unsigned long long ctx = current_context_id();
    std::lock_guard<std::mutex> lock(g_static_mu);
    if (!g_static_ptr[dev] || ctx == 0ull || g_static_ctx[dev] != ctx) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_dot_static_scratch);   // also makes the primary context current
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(ens_dot_static scratch)");
        g_static_ptr[dev] = p;
        g_static_ctx[dev] = ctx ? ctx : current_context_id();
    }
    *out = g_static_ptr[dev];
    return ENS_OK;
}

}  // namespace ens

using namespace ens;

extern "C" int ens_dot_static(int64_t n, int s, const double *u, const double *v, double *out,
                              void *stream) {
    size_t need;
    int rc = ens_dot_workspace_size(n, s, &need);
    if (rc) return rc;
    if (need > (size_t)ENS_DOT_STATIC_MAX_BYTES)
        return fail(ENS_ERR_UNSUPPORTED,
                    "ens_dot_static: n=%lld, s=%d needs %zu bytes of scratch, above the static "
                    "limit of %u bytes; use ens_dot with a caller workspace",
                    (long long)n, s, need, (unsigned)ENS_DOT_STATIC_MAX_BYTES);
    if (!out || (n > 0 && (!u || !v))) return fail(ENS_ERR_ARG, "NULL u/v/out");
    if (s > 1 && (!aligned16(u) || !aligned16(v))) return fail(ENS_ERR_ALIGN, "u/v must be 16-byte aligned");
    void *base = nullptr;
    if ((rc = static_scratch(&base))) return rc;
    cudaStream_t st = as_stream(stream);
    DotTree t;
    dot_tree_layout(&t, n, s, base);
    if ((rc = dot_tree_clear(t, st))) return rc;
    return dot_launch(n, s, u, v, out, t, st);
}
