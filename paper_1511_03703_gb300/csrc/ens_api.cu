// ens_api.cu -- error reporting, argument checks and dot-tree scratch layout.
#include <stdarg.h>
#include <string.h>

#include "ens_internal.cuh"

namespace ens {

static thread_local char g_err[512] = "";

void set_error(const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}

int fail(int status, const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return status;
}

int cuda_fail(cudaError_t err, const char *what) {
    set_error("%s: %s (%s)", what, cudaGetErrorName(err), cudaGetErrorString(err));
    (void)cudaGetLastError();  // a non-sticky error must not leak into the next call's launch check
    return ENS_ERR_CUDA;
}

int check_graph(const ens_graph *g) {
    if (!g) return fail(ENS_ERR_ARG, "graph is NULL");
    if (g->num_rows < 0 || g->num_entries < 0)
        return fail(ENS_ERR_ARG, "negative graph size (rows %d, entries %lld)", g->num_rows,
                    (long long)g->num_entries);
    if (g->num_entries > INT32_MAX)
        return fail(ENS_ERR_UNSUPPORTED, "num_entries %lld exceeds int32 indexing",
                    (long long)g->num_entries);
    if (g->num_rows > 0 && (!g->row_map || (g->num_entries > 0 && !g->col_entry)))
        return fail(ENS_ERR_ARG, "graph arrays are NULL");
    return ENS_OK;
}

static size_t round_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

static int tree_levels(int64_t n_rows, int64_t *count) {
    int64_t c = (n_rows + 31) / 32;
    if (c < 1) c = 1;
    int L = 1;
    count[1] = c;
    while (c > 1) {
        c = (c + 31) / 32;
        ++L;
        count[L] = c;
    }
    return L;
}

size_t dot_tree_bytes(int64_t n_rows, int width, size_t elem) {
    int64_t count[kTreeMaxLevels + 2] = {0};
    int L = tree_levels(n_rows, count);
    size_t bytes = 0;
    for (int l = 1; l <= L; ++l) bytes += round_up(elem * (size_t)count[l] * width, 256);
    for (int l = 1; l < L; ++l) bytes += round_up(sizeof(int) * (size_t)count[l + 1], 256);
    return bytes;
}

void dot_tree_layout_raw(int *levels, int64_t *count_out, void **buf, int **counter, int64_t n_rows,
                         int width, size_t elem, void *base) {
    int64_t count[kTreeMaxLevels + 2] = {0};
    int L = tree_levels(n_rows, count);
    *levels = L;
    char *p = static_cast<char *>(base);
    for (int l = 1; l <= L; ++l) {
        count_out[l] = count[l];
        buf[l] = p;
        p += round_up(elem * (size_t)count[l] * width, 256);
    }
    for (int l = 1; l < L; ++l) {
        counter[l] = reinterpret_cast<int *>(p);
        p += round_up(sizeof(int) * (size_t)count[l + 1], 256);
    }
}

int dot_tree_clear_raw(int levels, const int64_t *count, int *const *counter, cudaStream_t st) {
    for (int l = 1; l < levels; ++l)
        ENS_CUDA_TRY(cudaMemsetAsync(counter[l], 0, sizeof(int) * (size_t)count[l + 1], st));
    return ENS_OK;
}

}  // namespace ens

extern "C" const char *ens_last_error(void) { return ens::g_err; }

extern "C" const char *ens_status_string(int status) {
    switch (status) {
        case ENS_OK: return "ok";
        case ENS_ERR_ARG: return "invalid argument";
        case ENS_ERR_UNSUPPORTED: return "unsupported";
        case ENS_ERR_ALIGN: return "misaligned pointer";
        case ENS_ERR_CUDA: return "CUDA error";
        case ENS_ERR_NOT_CONVERGED: return "not converged";
        case ENS_ERR_BREAKDOWN: return "CG breakdown";
        case ENS_ERR_NONPOS_COEFF: return "non-positive coefficient";
        case ENS_ERR_TIMEOUT: return "device wait timed out";
        case ENS_ERR_WORKSPACE: return "workspace too small";
        default: return "unknown status";
    }
}

extern "C" int ens_version(void) { return 100; }
