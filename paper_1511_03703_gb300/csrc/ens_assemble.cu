// ens_assemble.cu -- ensemble finite-element assembly (Algorithm 2, Sect. 4).
//
// The coefficient is affine in the KL variables, so the element integrals of
// Algorithm 2 split by linearity: member e's matrix is
//     A_e = kappa0 * A^0 + sum_k (sigma * xi_k^e) * A^k,
// where A^k (ens_mode_matrices) integrates kappa_k over each cell with the
// same 2x2x2 Gauss rule.  All sample-independent work (NodeIndex/ElemGraph,
// basis gradients, kappa_k at the Gauss points) is done once per mesh; what
// remains per ensemble is M+1 fused multiply-adds per value, with the
// ensemble dimension contiguous so each mode value is read once per entry and
// used by all s members, and the output written as packed 16-byte stores.
#include "ens_internal.cuh"

namespace ens {

constexpr int kAsmMaxCoef = 65 * 32;

// thread per (entry, member pair); S = 1: thread per entry
template <int S>
__global__ void __launch_bounds__(256) assemble_values_kernel(
    int64_t nnz, int M, const double *__restrict__ modes, const double *__restrict__ xi,
    double sigma, double kappa0, double *__restrict__ values) {
    __shared__ double coef[kAsmMaxCoef];  // coef[k*S + e]
    for (int i = threadIdx.x; i < (M + 1) * S; i += blockDim.x)
        coef[i] = (i < S) ? kappa0 : sigma * xi[i - S];
    __syncthreads();
    constexpr int G = (S == 1) ? 1 : S / 2;
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t e = t / G;
    const int g = (int)(t % G);
    if (e >= nnz) return;
    if constexpr (S == 1) {
        double v = coef[0] * __ldg(modes + e);
        for (int k = 1; k <= M; ++k) v = fma(coef[k], __ldg(modes + (int64_t)k * nnz + e), v);
        values[e] = v;
    } else {
        const int m0 = 2 * g;
        const double mk0 = __ldg(modes + e);
        double v0 = coef[m0] * mk0, v1 = coef[m0 + 1] * mk0;
        for (int k = 1; k <= M; ++k) {
            const double mk = __ldg(modes + (int64_t)k * nnz + e);
            v0 = fma(coef[k * S + m0], mk, v0);
            v1 = fma(coef[k * S + m0 + 1], mk, v1);
        }
        reinterpret_cast<double2 *>(values)[e * G + g] = make_double2(v0, v1);
    }
}

// thread per (row, member): right-hand side and the Dirichlet identity rows
template <int S>
__global__ void assemble_rows_kernel(int32_t n, const int32_t *__restrict__ row_map,
                                     const int32_t *__restrict__ col_entry,
                                     const uint8_t *__restrict__ bmask,
                                     const double *__restrict__ load, double *__restrict__ values,
                                     double *__restrict__ b) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t I = t / S;
    const int e = (int)(t % S);
    if (I >= n) return;
    b[t] = load[I];
    if (bmask[I]) {
        for (int32_t p = row_map[I]; p < row_map[I + 1]; ++p)
            if (col_entry[p] == I) values[(int64_t)p * S + e] = 1.0;
    }
}

template <int S>
static int assemble_s(const ens_graph *g, const uint8_t *bmask, int M, const double *modes,
                      const double *load, const double *xi, double sigma, double kappa0,
                      double *values, double *b, cudaStream_t st) {
    constexpr int G = (S == 1) ? 1 : S / 2;
    const int bs = 256;
    const int64_t nthr = g->num_entries * G;
    if (nthr > 0) {
        assemble_values_kernel<S><<<(unsigned)((nthr + bs - 1) / bs), bs, 0, st>>>(
            g->num_entries, M, modes, xi, sigma, kappa0, values);
        ENS_LAUNCH_CHECK("assemble_values_kernel");
    }
    const int64_t nr = (int64_t)g->num_rows * S;
    if (nr > 0) {
        assemble_rows_kernel<S><<<(unsigned)((nr + bs - 1) / bs), bs, 0, st>>>(
            g->num_rows, g->row_map, g->col_entry, bmask, load, values, b);
        ENS_LAUNCH_CHECK("assemble_rows_kernel");
    }
    return ENS_OK;
}

}  // namespace ens

using namespace ens;

extern "C" int ens_assemble(const ens_graph *graph, const uint8_t *bmask, int s, int M,
                            const double *modes, const double *load, const double *xi,
                            double sigma, double kappa0, double *values, double *b,
                            void *stream) {
    int rc = check_graph(graph);
    if (rc) return rc;
    if (!supported_s(s)) return fail(ENS_ERR_UNSUPPORTED, "ensemble size s=%d not in {1,4,8,16,32}", s);
    if (M < 0 || M > 64) return fail(ENS_ERR_UNSUPPORTED, "M=%d outside [0, 64]", M);
    if (!bmask || !modes || !load || !values || !b || (M > 0 && !xi))
        return fail(ENS_ERR_ARG, "NULL pointer argument");
    if (s > 1 && (!aligned16(values) || !aligned16(b)))
        return fail(ENS_ERR_ALIGN, "values/b must be 16-byte aligned");
    cudaStream_t st = as_stream(stream);
    switch (s) {
        case 1: return assemble_s<1>(graph, bmask, M, modes, load, xi, sigma, kappa0, values, b, st);
        case 4: return assemble_s<4>(graph, bmask, M, modes, load, xi, sigma, kappa0, values, b, st);
        case 8: return assemble_s<8>(graph, bmask, M, modes, load, xi, sigma, kappa0, values, b, st);
        case 16: return assemble_s<16>(graph, bmask, M, modes, load, xi, sigma, kappa0, values, b, st);
        default: return assemble_s<32>(graph, bmask, M, modes, load, xi, sigma, kappa0, values, b, st);
    }
}
