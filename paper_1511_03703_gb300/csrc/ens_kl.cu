// ens_kl.cu -- Karhunen-Loeve setup and the sample-independent mode matrices.
//
// Sect. 4, Eq. 9-10: a(x, y) = kappa0 + sigma * sum_k kappa_k(x) y_k, with
// kappa_k the eigenfunctions of exp(-|x-x'|_1 / L) on [0,1]^3 scaled by
// sqrt(lambda_k).  Because the L1 kernel is a product of 1D kernels, every 3D
// eigenpair is a product of three 1D eigenpairs.  In 1D on [0,1] (centre 1/2,
// half-width a = 1/2, c = 1/L) the eigenfunctions are cos(w (x-1/2)) with
// c cos(w a) = w sin(w a) (even) and sin(w (x-1/2)) with w cos(w a) = -c sin(w a)
// (odd), eigenvalue 2c / (w^2 + c^2).  1D mode p is the (p/2)-th root of the
// even equation in (n pi/a, (n+1/2) pi/a) for even p and of the odd equation
// in ((n+1/2) pi/a, (n+1) pi/a) for odd p; each bracket holds exactly one root.
//
// The 3D modes are ranked by eigenvalue (the product of the three 1D values
// taken in ascending index order, so permuted triples tie exactly), ties by
// (p,q,r) ascending with p the x index.  A triple can only be among the top M
// if (p+1)(q+1)(r+1) <= M, because every componentwise-smaller triple has a
// strictly larger eigenvalue; that bounds the candidate set.
#include "ens_internal.cuh"

namespace ens {

constexpr int kMaxM = 64;
constexpr int kMaxCand = 2048;

__device__ double kl_even(double w, double c) { return c * cos(0.5 * w) - w * sin(0.5 * w); }
__device__ double kl_odd(double w, double c) { return w * cos(0.5 * w) + c * sin(0.5 * w); }

// one block of >= 64 threads
__global__ void kl_modes_kernel(int M, double L, double *hdr) {
    __shared__ double om[kMaxM], la[kMaxM];
    __shared__ int cand[kMaxCand];
    __shared__ double cl[kMaxCand];
    __shared__ int ncand;
    const double c = 1.0 / L;
    const int tid = threadIdx.x;
    if (tid < M) {
        const int p = tid, n = p / 2, odd = p & 1;
        // brackets in units of pi / a with a = 1/2
        double lo = odd ? (2.0 * n + 1.0) * M_PI : 2.0 * n * M_PI;
        double hi = odd ? (2.0 * n + 2.0) * M_PI : (2.0 * n + 1.0) * M_PI;
        double flo = odd ? kl_odd(lo, c) : kl_even(lo, c);
        for (int it = 0; it < 2000; ++it) {
            double mid = 0.5 * (lo + hi);
            if (!(mid > lo && mid < hi)) break;
            double fm = odd ? kl_odd(mid, c) : kl_even(mid, c);
            if (fm == 0.0) { lo = hi = mid; break; }
            if ((fm > 0.0) == (flo > 0.0)) { lo = mid; flo = fm; } else { hi = mid; }
        }
        const double w = 0.5 * (lo + hi);
        om[p] = w;
        la[p] = 2.0 * c / (w * w + c * c);
    }
    if (tid == 0) {
        int nc = 0;
        for (int p = 0; p < M; ++p)
            for (int q = 0; q < M; ++q)
                for (int r = 0; r < M; ++r)
                    if ((p + 1) * (q + 1) * (r + 1) <= M && nc < kMaxCand)
                        cand[nc++] = p | (q << 8) | (r << 16);
        ncand = nc;
    }
    __syncthreads();
    for (int i = tid; i < ncand; i += blockDim.x) {
        int p = cand[i] & 255, q = (cand[i] >> 8) & 255, r = (cand[i] >> 16) & 255;
        int a = min(p, min(q, r)), b2 = max(p, max(q, r)), m = p + q + r - a - b2;
        cl[i] = (la[a] * la[m]) * la[b2];
    }
    __syncthreads();
    // rank = number of candidates ahead in (lambda desc, pqr asc); pqr packed so that
    // lexicographic (p,q,r) order equals integer order of p<<16 | q<<8 | r
    for (int i = tid; i < ncand; i += blockDim.x) {
        int key_i = ((cand[i] & 255) << 16) | (cand[i] & 0xff00) | ((cand[i] >> 16) & 255);
        int rank = 0;
        for (int j = 0; j < ncand; ++j) {
            int key_j = ((cand[j] & 255) << 16) | (cand[j] & 0xff00) | ((cand[j] >> 16) & 255);
            rank += (cl[j] > cl[i]) || (cl[j] == cl[i] && key_j < key_i);
        }
        if (rank < M) {
            hdr[rank] = cl[i];                               // lambda3
            hdr[M + 3 * rank + 0] = (double)(cand[i] & 255);  // p
            hdr[M + 3 * rank + 1] = (double)((cand[i] >> 8) & 255);
            hdr[M + 3 * rank + 2] = (double)((cand[i] >> 16) & 255);
        }
    }
    if (tid < M) {
        hdr[4 * M + tid] = om[tid];
        hdr[5 * M + tid] = la[tid];
    }
}

// T[(d*M + k)*2N + t] = phi_{idx_d(k)}(x_t), x_t = (t/2 + g_{t&1}) / N, sqrt(lambda3_k) in d = 0
__global__ void kl_table_kernel(int N, int M, double *table, const double *hdr) {
    const int64_t total = 3LL * M * 2 * N;
    const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (idx >= total) return;
    const int t = (int)(idx % (2 * N));
    const int k = (int)((idx / (2 * N)) % M);
    const int d = (int)(idx / (2LL * N * M));
    const int p = (int)hdr[M + 3 * k + d];
    const double w = hdr[4 * M + p];
    const double g = (t & 1) ? 0.5 + 0.5 / sqrt(3.0) : 0.5 - 0.5 / sqrt(3.0);
    const double x = ((t >> 1) + g) / (double)N;
    const double s2 = sin(w) / (2.0 * w);  // sin(2 w a) / (2 w) with a = 1/2
    double phi = (p & 1) ? sin(w * (x - 0.5)) / sqrt(0.5 - s2) : cos(w * (x - 0.5)) / sqrt(0.5 + s2);
    if (d == 0) phi *= sqrt(hdr[k]);
    table[idx] = phi;
}

// reference-cell gradient products at the Gauss points times w_q h:
// G[q][a][b] = (h/8) sum_d dphi_a/dxi_d (q) * dphi_b/dxi_d (q)
__device__ double q1_gradprod(int q, int a, int b, double h) {
    const double gp[2] = {0.5 - 0.5 / sqrt(3.0), 0.5 + 0.5 / sqrt(3.0)};
    double xi[3] = {gp[q & 1], gp[(q >> 1) & 1], gp[(q >> 2) & 1]};
    double s = 0.0;
    for (int d = 0; d < 3; ++d) {
        double fa = 1.0, fb = 1.0;
        for (int e = 0; e < 3; ++e) {
            int oa = (a >> e) & 1, ob = (b >> e) & 1;
            if (e == d) {
                fa *= oa ? 1.0 : -1.0;
                fb *= ob ? 1.0 : -1.0;
            } else {
                fa *= oa ? xi[e] : 1.0 - xi[e];
                fb *= ob ? xi[e] : 1.0 - xi[e];
            }
        }
        s += fa * fb;
    }
    return s * (h * 0.125);
}

__device__ double q1_phi(int q, int a) {
    const double gp[2] = {0.5 - 0.5 / sqrt(3.0), 0.5 + 0.5 / sqrt(3.0)};
    double v = 1.0;
    for (int e = 0; e < 3; ++e) {
        double x = gp[(q >> e) & 1];
        v *= ((a >> e) & 1) ? x : 1.0 - x;
    }
    return v;
}

__device__ __forceinline__ int axis_n(int t, int N) { return (t == 0 || t == N) ? 2 : 3; }

// Thread per (row, entry position p of the row): a warp takes position p of
// 32 consecutive rows, so the lanes of an interior warp share the same number
// of cells with their rows and run the same FP64 loops (a warp of the 27
// entries of one row would run the diagonal entry's 8 cells on every lane:
// a divergent FP64 instruction still takes the FP64 pipe for the whole warp).
// Positions p, p + gridDim.y, ... for rows longer than gridDim.y.
__global__ void __launch_bounds__(256) mode_matrices_kernel(
    int N, int M, const int32_t *__restrict__ row_map, const int32_t *__restrict__ col_entry,
    int64_t nnz, const double *__restrict__ table, double *__restrict__ modes,
    double *__restrict__ load) {
    __shared__ double Gs[512];
    __shared__ double Ps[64];
    const double h = 1.0 / N;
    for (int i = threadIdx.x; i < 512; i += blockDim.x) Gs[i] = q1_gradprod(i >> 6, (i >> 3) & 7, i & 7, h);
    for (int i = threadIdx.x; i < 64; i += blockDim.x) Ps[i] = q1_phi(i >> 3, i & 7) * (h * h * h * 0.125);
    __syncthreads();
    const int64_t n = (int64_t)(N + 1) * (N + 1) * (N + 1);
    const int64_t I = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (I >= n) return;
    const int n1 = N + 1;
    const int i = (int)(I % n1), j = (int)((I / n1) % n1), k = (int)(I / ((int64_t)n1 * n1));
    const bool brow = (i == 0 || j == 0 || k == 0 || i == N || j == N || k == N);
    const int rs = row_map[I], len = row_map[I + 1] - rs;
    const int twoN = 2 * N;
    const double *T0 = table, *T1 = table + (int64_t)M * twoN, *T2 = table + 2LL * M * twoN;
    for (int pos = blockIdx.y; pos < len; pos += gridDim.y) {
        const int64_t e = rs + pos;
        const int32_t J = col_entry[e];
        const int ji = (int)(J % n1), jj = (int)((J / n1) % n1), jk = (int)(J / ((int64_t)n1 * n1));
        const bool bcol = (ji == 0 || jj == 0 || jk == 0 || ji == N || jj == N || jk == N);
        // cells shared by I and J: per axis, both coordinates in {c, c+1}
        const int ci0 = max(max(i, ji) - 1, 0), ci1 = min(min(i, ji), N - 1);
        const int cj0 = max(max(j, jj) - 1, 0), cj1 = min(min(j, jj), N - 1);
        const int ck0 = max(max(k, jk) - 1, 0), ck1 = min(min(k, jk), N - 1);
        for (int m = 0; m <= M; ++m) {
            double acc = 0.0;
            if (!brow && !bcol) {
                for (int ck = ck0; ck <= ck1; ++ck)
                    for (int cj = cj0; cj <= cj1; ++cj)
                        for (int ci = ci0; ci <= ci1; ++ci) {
                            const int a = (i - ci) | ((j - cj) << 1) | ((k - ck) << 2);
                            const int b = (ji - ci) | ((jj - cj) << 1) | ((jk - ck) << 2);
                            for (int q = 0; q < 8; ++q) {
                                const double g = Gs[(q << 6) | (a << 3) | b];
                                if (m == 0) {
                                    acc += g;
                                } else {
                                    const int tx = 2 * ci + (q & 1), ty = 2 * cj + ((q >> 1) & 1),
                                              tz = 2 * ck + ((q >> 2) & 1);
                                    const int kk = m - 1;
                                    const double kap = __ldg(T0 + (int64_t)kk * twoN + tx) *
                                                       __ldg(T1 + (int64_t)kk * twoN + ty) *
                                                       __ldg(T2 + (int64_t)kk * twoN + tz);
                                    acc = fma(kap, g, acc);
                                }
                            }
                        }
            }
            modes[(int64_t)m * nnz + e] = acc;
        }
    }
    if (blockIdx.y == 0) {
        double f = 0.0;
        if (!brow) {
            for (int ck = max(k - 1, 0); ck <= min(k, N - 1); ++ck)
                for (int cj = max(j - 1, 0); cj <= min(j, N - 1); ++cj)
                    for (int ci = max(i - 1, 0); ci <= min(i, N - 1); ++ci) {
                        const int a = (i - ci) | ((j - cj) << 1) | ((k - ck) << 2);
                        for (int q = 0; q < 8; ++q) f += Ps[(q << 3) | a];
                    }
        }
        load[I] = f;
    }
}

}  // namespace ens

using namespace ens;

extern "C" int ens_kl_table_size(int N, int M, int64_t *num_doubles) {
    if (N < 1 || N > 400) return fail(ENS_ERR_UNSUPPORTED, "N=%d outside [1, 400]", N);
    if (M < 1 || M > kMaxM) return fail(ENS_ERR_UNSUPPORTED, "M=%d outside [1, %d]", M, kMaxM);
    if (num_doubles) *num_doubles = 3LL * M * 2 * N + 6LL * M;
    return ENS_OK;
}

extern "C" int ens_kl_setup(int N, int M, double L, double *kl_table, double *lambda_host,
                            int32_t *pqr_host, void *stream) {
    int64_t sz;
    int rc = ens_kl_table_size(N, M, &sz);
    if (rc) return rc;
    if (!(L > 0.0)) return fail(ENS_ERR_ARG, "correlation length L=%g must be > 0", L);
    if (!kl_table) return fail(ENS_ERR_ARG, "kl_table is NULL");
    cudaStream_t st = as_stream(stream);
    double *hdr = kl_table + 3LL * M * 2 * N;
    kl_modes_kernel<<<1, 128, 0, st>>>(M, L, hdr);
    ENS_LAUNCH_CHECK("kl_modes_kernel");
    const int64_t tot = 3LL * M * 2 * N;
    kl_table_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(N, M, kl_table, hdr);
    ENS_LAUNCH_CHECK("kl_table_kernel");
    if (lambda_host || pqr_host) {
        double tmp[4 * kMaxM];
        ENS_CUDA_TRY(cudaMemcpyAsync(tmp, hdr, sizeof(double) * 4 * M, cudaMemcpyDeviceToHost, st));
        ENS_CUDA_TRY(cudaStreamSynchronize(st));
        for (int k = 0; k < M; ++k) {
            if (lambda_host) lambda_host[k] = tmp[k];
            if (pqr_host)
                for (int d = 0; d < 3; ++d) pqr_host[3 * k + d] = (int32_t)tmp[M + 3 * k + d];
        }
    }
    return ENS_OK;
}

extern "C" int ens_mode_matrices(int N, const ens_graph *graph, int M, const double *kl_table,
                                 double *modes, double *load, void *stream) {
    int rc = check_graph(graph);
    if (rc) return rc;
    int32_t n;
    int64_t nnz;
    if ((rc = ens_mesh_sizes(N, &n, &nnz, nullptr))) return rc;
    if (graph->num_rows != n || graph->num_entries != nnz)
        return fail(ENS_ERR_ARG, "graph does not belong to the N=%d mesh", N);
    if ((rc = ens_kl_table_size(N, M, nullptr))) return rc;
    if (!kl_table || !modes || !load) return fail(ENS_ERR_ARG, "NULL table/modes/load");
    cudaStream_t st = as_stream(stream);
    const int bs = 256;
    // 27 = the longest row of the Q1 hex graph (the kernel strides past it)
    mode_matrices_kernel<<<dim3((unsigned)(((int64_t)n + bs - 1) / bs), 27), bs, 0, st>>>(
        N, M, graph->row_map, graph->col_entry, nnz, kl_table, modes, load);
    ENS_LAUNCH_CHECK("mode_matrices_kernel");
    return ENS_OK;
}
