// ens_graph.cu -- CRS graph, ElemGraph and boundary mask of the structured Q1 hex
// mesh (Fig. 2 data structure; NodeIndex / ElemGraph maps of Algorithm 2).
//
// Row I = node (i,j,k) couples to every node that shares a cell with it, i.e.
// (i+di, j+dj, k+dk) with d in {-1,0,1}^3 inside the mesh; columns ascending
// means (dk, dj, di) in lexicographic order.  Per axis a node has f(t) = 2
// neighbour positions on the boundary (t = 0 or N) and 3 inside, so the row
// length is f(i) f(j) f(k) and every offset below is a closed form: the graph
// is integer work and bit-exact without any sort or scan.
#include "ens_internal.cuh"

namespace ens {

__device__ __forceinline__ int axis_f(int t, int N) { return (t == 0 || t == N) ? 2 : 3; }
// sum_{t' < t} f(t')
__device__ __forceinline__ int64_t axis_prefix(int t, int N) {
    if (t <= 0) return 0;
    if (t > N) return 3LL * N + 1;
    return 2 + 3LL * (t - 1);
}

__global__ void graph_row_map_kernel(int N, int32_t *row_map, uint8_t *bmask) {
    const int64_t n = (int64_t)(N + 1) * (N + 1) * (N + 1);
    const int64_t I = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (I > n) return;
    const int64_t F = 3LL * N + 1;
    if (I == n) {
        row_map[n] = (int32_t)(F * F * F);
        return;
    }
    const int i = (int)(I % (N + 1)), j = (int)((I / (N + 1)) % (N + 1)),
              k = (int)(I / ((int64_t)(N + 1) * (N + 1)));
    int64_t off = axis_prefix(k, N) * F * F +
                  axis_f(k, N) * (axis_prefix(j, N) * F + axis_f(j, N) * axis_prefix(i, N));
    row_map[I] = (int32_t)off;
    if (bmask) bmask[I] = (i == 0 || j == 0 || k == 0 || i == N || j == N || k == N) ? 1 : 0;
}

// one warp per row, lane t writes the row's t-th column
__global__ void graph_cols_kernel(int N, const int32_t *__restrict__ row_map,
                                  int32_t *__restrict__ col_entry) {
    const int64_t n = (int64_t)(N + 1) * (N + 1) * (N + 1);
    const int64_t I = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int t = threadIdx.x & 31;
    if (I >= n) return;
    const int i = (int)(I % (N + 1)), j = (int)((I / (N + 1)) % (N + 1)),
              k = (int)(I / ((int64_t)(N + 1) * (N + 1)));
    const int ni = axis_f(i, N), nj = axis_f(j, N), nk = axis_f(k, N);
    if (t >= ni * nj * nk) return;
    const int di = t % ni + (i == 0 ? 0 : -1);
    const int dj = (t / ni) % nj + (j == 0 ? 0 : -1);
    const int dk = t / (ni * nj) + (k == 0 ? 0 : -1);
    const int64_t J = (i + di) + (int64_t)(N + 1) * ((j + dj) + (int64_t)(N + 1) * (k + dk));
    col_entry[row_map[I] + t] = (int32_t)J;
}

// thread per (cell, a, b): entry of (NodeIndex(c,a), NodeIndex(c,b)) in row NodeIndex(c,a)
__global__ void elem_graph_kernel(int N, const int32_t *__restrict__ row_map,
                                  int32_t *__restrict__ elem_graph) {
    const int64_t total = (int64_t)N * N * N * 64;
    const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (idx >= total) return;
    const int64_t c = idx >> 6;
    const int a = (int)(idx >> 3) & 7, b = (int)idx & 7;
    const int ci = (int)(c % N), cj = (int)((c / N) % N), ck = (int)(c / ((int64_t)N * N));
    const int i = ci + (a & 1), j = cj + ((a >> 1) & 1), k = ck + ((a >> 2) & 1);
    const int di = (b & 1) - (a & 1), dj = ((b >> 1) & 1) - ((a >> 1) & 1),
              dk = ((b >> 2) & 1) - ((a >> 2) & 1);
    const int ni = axis_f(i, N), nj = axis_f(j, N);
    const int pi = di - (i == 0 ? 0 : -1), pj = dj - (j == 0 ? 0 : -1),
              pk = dk - (k == 0 ? 0 : -1);
    const int64_t I = i + (int64_t)(N + 1) * (j + (int64_t)(N + 1) * k);
    elem_graph[idx] = row_map[I] + (pk * nj + pj) * ni + pi;
}

}  // namespace ens

using namespace ens;

extern "C" int ens_mesh_sizes(int N, int32_t *num_rows, int64_t *num_entries, int64_t *num_cells) {
    if (N < 1 || N > 400) return fail(ENS_ERR_UNSUPPORTED, "N=%d outside [1, 400]", N);
    const int64_t F = 3LL * N + 1;
    if (num_rows) *num_rows = (int32_t)((int64_t)(N + 1) * (N + 1) * (N + 1));
    if (num_entries) *num_entries = F * F * F;
    if (num_cells) *num_cells = (int64_t)N * N * N;
    return ENS_OK;
}

extern "C" int ens_graph_build(int N, int32_t *row_map, int32_t *col_entry, int32_t *elem_graph,
                               uint8_t *bmask, void *stream) {
    int32_t n;
    int64_t nnz, nc;
    int rc = ens_mesh_sizes(N, &n, &nnz, &nc);
    if (rc) return rc;
    if (!row_map || !col_entry) return fail(ENS_ERR_ARG, "row_map/col_entry NULL");
    cudaStream_t st = as_stream(stream);
    const int bs = 256;
    graph_row_map_kernel<<<(unsigned)((n + 1 + bs - 1) / bs), bs, 0, st>>>(N, row_map, bmask);
    ENS_LAUNCH_CHECK("graph_row_map_kernel");
    graph_cols_kernel<<<(unsigned)(((int64_t)n * 32 + bs - 1) / bs), bs, 0, st>>>(N, row_map,
                                                                                   col_entry);
    ENS_LAUNCH_CHECK("graph_cols_kernel");
    if (elem_graph) {
        elem_graph_kernel<<<(unsigned)((nc * 64 + bs - 1) / bs), bs, 0, st>>>(N, row_map,
                                                                              elem_graph);
        ENS_LAUNCH_CHECK("elem_graph_kernel");
    }
    return ENS_OK;
}
