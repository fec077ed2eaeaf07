// ens_spmv.cu -- ens_spmv (commuted-layout SpMV, Fig. 5) and ens_dot (Sect. 3.4).
#include "ens_spmv.cuh"

namespace ens {

template <int S, typename V>
__global__ void __launch_bounds__(RowMap<S>::THREADS, 1536 / RowMap<S>::THREADS) spmv_kernel(
    int32_t n, const int32_t *__restrict__ row_map, const int32_t *__restrict__ col,
    const V *__restrict__ vals, const double *__restrict__ x, double *__restrict__ y) {
    constexpr int G = RowMap<S>::G;
    __shared__ ChunkCols cc;
    const int r = threadIdx.x / G, g = threadIdx.x % G;
    const int64_t R = (int64_t)blockIdx.x * 32 + r;
    const bool staged = stage_chunk(cc, row_map, col, blockIdx.x, n);
    const double2 v = chunk_spmv<S, V>(cc, staged, col, vals, x, r, g, R < n);
    if (R >= n) return;
    if constexpr (S == 1) {
        if (g == 0) y[R] = v.x;
    } else {
        reinterpret_cast<double2 *>(y)[R * G + g] = v;
    }
}

// double-float arithmetic, FP64 values and x (x split on the fly)
template <int S>
__global__ void __launch_bounds__(RowMap<S>::THREADS, 512 / RowMap<S>::THREADS) spmv_df_kernel(
    int32_t n, const int32_t *__restrict__ row_map, const int32_t *__restrict__ col,
    const double *__restrict__ vals, const double *__restrict__ x, double *__restrict__ y) {
    constexpr int G = RowMap<S>::G;
    __shared__ ChunkCols cc;
    const int r = threadIdx.x / G, g = threadIdx.x % G;
    const int64_t R = (int64_t)blockIdx.x * 32 + r;
    const bool staged = stage_chunk(cc, row_map, col, blockIdx.x, n);
    const double2 v = chunk_spmv_df<S, XSplit>(cc, staged, col, vals, x, r, g, R < n);
    if (R >= n) return;
    if constexpr (S == 1) {
        if (g == 0) y[R] = v.x;
    } else {
        reinterpret_cast<double2 *>(y)[R * G + g] = v;
    }
}

// split FP64 / double-float arithmetic (x split on the fly for odd positions)
template <int S>
__global__ void __launch_bounds__(RowMap<S>::THREADS, 1024 / RowMap<S>::THREADS) spmv_split_kernel(
    int32_t n, const int32_t *__restrict__ row_map, const int32_t *__restrict__ col,
    const double *__restrict__ vals, const double *__restrict__ x, double *__restrict__ y) {
    constexpr int G = RowMap<S>::G;
    __shared__ ChunkCols cc;
    const int r = threadIdx.x / G, g = threadIdx.x % G;
    const int64_t R = (int64_t)blockIdx.x * 32 + r;
    const bool staged = stage_chunk(cc, row_map, col, blockIdx.x, n);
    const double2 v = chunk_spmv_split<S, XSplit>(cc, staged, col, vals, x, x, r, g, R < n);
    if (R >= n) return;
    if constexpr (S == 1) {
        if (g == 0) y[R] = v.x;
    } else {
        reinterpret_cast<double2 *>(y)[R * G + g] = v;
    }
}

// pre-split double-float values (ENS_F64_DF copy) with their FP64 originals;
// x FP64, split on the fly; the value block of each chunk prefetched into L2
// as in the CG's SpMV
template <int S>
__global__ void __launch_bounds__(RowMap<S>::THREADS, 1536 / RowMap<S>::THREADS) spmv_dfv_kernel(
    int32_t n, const int32_t *__restrict__ row_map, const int32_t *__restrict__ col,
    const double *__restrict__ vals, const float2 *__restrict__ vdf, uint64_t vdf_bytes,
    const double *__restrict__ x, double *__restrict__ y) {
    constexpr int G = RowMap<S>::G;
    __shared__ ChunkCols cc;
    const int r = threadIdx.x / G, g = threadIdx.x % G;
    const int64_t R = (int64_t)blockIdx.x * 32 + r;
    const bool staged = stage_chunk_pf(cc, row_map, col, blockIdx.x, n, vdf, S * 8u, vdf_bytes, 0xffffffffu);
    const double2 v = chunk_spmv_dfv<S, XSplit>(cc, staged, col, vdf, vals, x, r, g, R < n);
    if (R >= n) return;
    if constexpr (S == 1) {
        if (g == 0) y[R] = v.x;
    } else {
        reinterpret_cast<double2 *>(y)[R * G + g] = v;
    }
}

template <int S>
static int spmv_dfv_s(const ens_graph *g, const double *vals, const float2 *vdf, const double *x, double *y,
                      cudaStream_t st) {
    const int64_t chunks = ((int64_t)g->num_rows + 31) / 32;
    if (chunks == 0) return ENS_OK;
    spmv_dfv_kernel<S><<<(unsigned)chunks, RowMap<S>::THREADS, 0, st>>>(
        g->num_rows, g->row_map, g->col_entry, vals, vdf, (uint64_t)g->num_entries * S * 8u, x, y);
    ENS_LAUNCH_CHECK("spmv_dfv_kernel");
    return ENS_OK;
}

template <int S>
static int spmv_split_s(const ens_graph *g, const double *vals, const double *x, double *y,
                        cudaStream_t st) {
    const int64_t chunks = ((int64_t)g->num_rows + 31) / 32;
    if (chunks == 0) return ENS_OK;
    spmv_split_kernel<S><<<(unsigned)chunks, RowMap<S>::THREADS, 0, st>>>(g->num_rows, g->row_map,
                                                                         g->col_entry, vals, x, y);
    ENS_LAUNCH_CHECK("spmv_split_kernel");
    return ENS_OK;
}

static int spmv_split_dispatch(const ens_graph *g, int s, const void *vals, const double *x,
                               double *y, cudaStream_t st) {
    const double *v = static_cast<const double *>(vals);
    switch (s) {
        case 1: return spmv_split_s<1>(g, v, x, y, st);
        case 4: return spmv_split_s<4>(g, v, x, y, st);
        case 8: return spmv_split_s<8>(g, v, x, y, st);
        case 16: return spmv_split_s<16>(g, v, x, y, st);
        default: return spmv_split_s<32>(g, v, x, y, st);
    }
}

template <int S>
static int spmv_df_s(const ens_graph *g, const double *vals, const double *x, double *y,
                     cudaStream_t st) {
    const int64_t chunks = ((int64_t)g->num_rows + 31) / 32;
    if (chunks == 0) return ENS_OK;
    spmv_df_kernel<S><<<(unsigned)chunks, RowMap<S>::THREADS, 0, st>>>(g->num_rows, g->row_map,
                                                                      g->col_entry, vals, x, y);
    ENS_LAUNCH_CHECK("spmv_df_kernel");
    return ENS_OK;
}

static int spmv_df_dispatch(const ens_graph *g, int s, const void *vals, const double *x,
                            double *y, cudaStream_t st) {
    const double *v = static_cast<const double *>(vals);
    switch (s) {
        case 1: return spmv_df_s<1>(g, v, x, y, st);
        case 4: return spmv_df_s<4>(g, v, x, y, st);
        case 8: return spmv_df_s<8>(g, v, x, y, st);
        case 16: return spmv_df_s<16>(g, v, x, y, st);
        default: return spmv_df_s<32>(g, v, x, y, st);
    }
}

template <int S, typename V>
static int spmv_s(const ens_graph *g, const V *vals, const double *x, double *y, cudaStream_t st) {
    const int64_t chunks = ((int64_t)g->num_rows + 31) / 32;
    if (chunks == 0) return ENS_OK;
    spmv_kernel<S, V><<<(unsigned)chunks, RowMap<S>::THREADS, 0, st>>>(g->num_rows, g->row_map,
                                                                       g->col_entry, vals, x, y);
    ENS_LAUNCH_CHECK("spmv_kernel");
    return ENS_OK;
}

template <typename V>
static int spmv_dispatch(const ens_graph *g, int s, const void *vals, const double *x, double *y,
                         cudaStream_t st) {
    const V *v = static_cast<const V *>(vals);
    switch (s) {
        case 1: return spmv_s<1, V>(g, v, x, y, st);
        case 4: return spmv_s<4, V>(g, v, x, y, st);
        case 8: return spmv_s<8, V>(g, v, x, y, st);
        case 16: return spmv_s<16, V>(g, v, x, y, st);
        default: return spmv_s<32, V>(g, v, x, y, st);
    }
}

// ------------------------------------------------------------------ dot
// one 32-row chunk per CTA, G = max(s/2, 1) threads per row
template <int S>
__global__ void __launch_bounds__(32 * (S == 1 ? 1 : S / 2)) dot_kernel(
    int64_t n, const double *__restrict__ u, const double *__restrict__ v, DotTree t,
    double *__restrict__ out) {
    constexpr int G = (S == 1) ? 1 : S / 2;
    __shared__ double sm[32][S + 1];
    const int r = threadIdx.x / G, g = threadIdx.x % G;
    const int64_t R = (int64_t)blockIdx.x * 32 + r;
    double p0 = 0.0, p1 = 0.0;
    if (R < n) {
        if constexpr (S == 1) {
            p0 = u[R] * v[R];
        } else {
            const double2 a = reinterpret_cast<const double2 *>(u)[R * G + g];
            const double2 b = reinterpret_cast<const double2 *>(v)[R * G + g];
            p0 = a.x * b.x;
            p1 = a.y * b.y;
        }
    }
    if constexpr (S == 1) {
        sm[r][0] = p0;
    } else {
        sm[r][2 * g] = p0;
        sm[r][2 * g + 1] = p1;
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int e = warp; e < S; e += nw) {
        const double w = warp_tree32(sm[lane][e]);
        if (lane == 0) t.buf[1][blockIdx.x * (int64_t)S + e] = w;
    }
    if (dot_tree_propagate(t, blockIdx.x, 1)) {
        for (int e = threadIdx.x; e < S; e += blockDim.x) out[e] = ld_cg(t.buf[t.levels] + e);
    }
}

template <int S>
static int dot_s(int64_t n, const double *u, const double *v, double *out, const DotTree &t,
                 cudaStream_t st) {
    const int64_t chunks = t.count[1];
    dot_kernel<S><<<(unsigned)chunks, 32 * (S == 1 ? 1 : S / 2), 0, st>>>(n, u, v, t, out);
    ENS_LAUNCH_CHECK("dot_kernel");
    return ENS_OK;
}

int dot_launch(int64_t n, int s, const double *u, const double *v, double *out, const DotTree &t,
               cudaStream_t st) {
    switch (s) {
        case 1: return dot_s<1>(n, u, v, out, t, st);
        case 4: return dot_s<4>(n, u, v, out, t, st);
        case 8: return dot_s<8>(n, u, v, out, t, st);
        case 16: return dot_s<16>(n, u, v, out, t, st);
        default: return dot_s<32>(n, u, v, out, t, st);
    }
}

}  // namespace ens

using namespace ens;

extern "C" int ens_spmv(const ens_graph *graph, int s, int dtype, const void *values,
                        const double *x, double *y, void *stream) {
    int rc = check_graph(graph);
    if (rc) return rc;
    if (!supported_s(s)) return fail(ENS_ERR_UNSUPPORTED, "ensemble size s=%d not in {1,4,8,16,32}", s);
    if (graph->num_rows > 0 && (!values || !x || !y)) return fail(ENS_ERR_ARG, "NULL values/x/y");
    if (s > 1 && (!aligned16(values) || !aligned16(x) || !aligned16(y)))
        return fail(ENS_ERR_ALIGN, "values/x/y must be 16-byte aligned for s > 1");
    cudaStream_t st = as_stream(stream);
    switch (dtype) {
        case ENS_F64: return spmv_dispatch<double>(graph, s, values, x, y, st);
        case ENS_F32: return spmv_dispatch<float>(graph, s, values, x, y, st);
        case ENS_BF16: return spmv_dispatch<__nv_bfloat16>(graph, s, values, x, y, st);
        case ENS_F64_DF: return spmv_df_dispatch(graph, s, values, x, y, st);
        case ENS_F64_SPLIT: return spmv_split_dispatch(graph, s, values, x, y, st);
        default: return fail(ENS_ERR_UNSUPPORTED, "dtype %d", dtype);
    }
}

extern "C" int ens_spmv_df(const ens_graph *graph, int s, const double *values, const void *values_df,
                           const double *x, double *y, void *stream) {
    int rc = check_graph(graph);
    if (rc) return rc;
    if (!supported_s(s)) return fail(ENS_ERR_UNSUPPORTED, "ensemble size s=%d not in {1,4,8,16,32}", s);
    if (graph->num_rows > 0 && (!values || !values_df || !x || !y))
        return fail(ENS_ERR_ARG, "NULL values/values_df/x/y");
    if (!aligned16(values_df) || (s > 1 && (!aligned16(values) || !aligned16(x) || !aligned16(y))))
        return fail(ENS_ERR_ALIGN, "values_df (and values/x/y for s > 1) must be 16-byte aligned");
    const float2 *vdf = static_cast<const float2 *>(values_df);
    cudaStream_t st = as_stream(stream);
    switch (s) {
        case 1: return spmv_dfv_s<1>(graph, values, vdf, x, y, st);
        case 4: return spmv_dfv_s<4>(graph, values, vdf, x, y, st);
        case 8: return spmv_dfv_s<8>(graph, values, vdf, x, y, st);
        case 16: return spmv_dfv_s<16>(graph, values, vdf, x, y, st);
        default: return spmv_dfv_s<32>(graph, values, vdf, x, y, st);
    }
}

extern "C" int ens_dot_workspace_size(int64_t n, int s, size_t *bytes) {
    if (n < 0) return fail(ENS_ERR_ARG, "n=%lld < 0", (long long)n);
    if (!supported_s(s)) return fail(ENS_ERR_UNSUPPORTED, "ensemble size s=%d not in {1,4,8,16,32}", s);
    if (!bytes) return fail(ENS_ERR_ARG, "bytes is NULL");
    *bytes = dot_tree_bytes(n, s);
    return ENS_OK;
}

extern "C" int ens_dot(int64_t n, int s, const double *u, const double *v, double *out,
                       void *work, size_t work_bytes, void *stream) {
    size_t need;
    int rc = ens_dot_workspace_size(n, s, &need);
    if (rc) return rc;
    if (!out || (n > 0 && (!u || !v))) return fail(ENS_ERR_ARG, "NULL u/v/out");
    if (!work || work_bytes < need) return fail(ENS_ERR_WORKSPACE, "dot workspace %zu < %zu bytes", work_bytes, need);
    if (!aligned16(work) || (s > 1 && (!aligned16(u) || !aligned16(v))))
        return fail(ENS_ERR_ALIGN, "u/v/work must be 16-byte aligned");
    cudaStream_t st = as_stream(stream);
    DotTree t;
    dot_tree_layout(&t, n, s, work);
    if ((rc = dot_tree_clear(t, st))) return rc;
    return dot_launch(n, s, u, v, out, t, st);
}
