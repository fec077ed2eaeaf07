// ens_learned.cu -- learned initial guess for ensemble CG (not in the paper):
// a reduced basis of the solutions (POD) and a small MLP that maps the KL
// variables xi to the basis coefficients, trained with hand-written kernels.
//
// POD (FP64): snapshots X (n x m, row-major [node][sample], centred in place)
// -> randomized range finder with one power iteration (Halko, Martinsson and
// Tropp, SIAM Review 2011): Y = X Omega, Q = orth(Y) by CholeskyQR2,
// Y = X (X^T Q), Q = orth(Y), B = Q^T X, eigen-decomposition of B B^T by cyclic
// Jacobi, Phi = Q W_k, sigma_i = sqrt(lambda_i); each column signed so that its
// largest-magnitude entry is positive.
// MLP (FP32): three affine layers d0 -> d1 -> d2 -> d3 with the exact GELU
// x * Phi(x) = x (1 + erf(x / sqrt 2)) / 2 after the first two, MSE loss,
// Adam (Kingma and Ba, 2015).
#include <math.h>

#include <vector>

#include "ens_internal.cuh"

namespace ens {

// ---------------------------------------------------- FP64 tall-skinny GEMMs
// Tiles of 64 rows x up to 80 columns, 256 threads, 4 x 5 outputs per thread.
constexpr int kTR = 64, kTC = 80, kTK = 16;

// C[n x c] = A[n x r] * B[r x c] (+ rowadd[i] if not NULL), A and B row-major
// with leading dimensions lda, ldb; C leading dimension ldc.  c <= 80.
__global__ void __launch_bounds__(256) gemm_nn_f64(int64_t n, int r, int c, const double *__restrict__ A,
                                                   int64_t lda, const double *__restrict__ B, int64_t ldb,
                                                   double *__restrict__ C, int64_t ldc,
                                                   const double *__restrict__ rowadd) {
    __shared__ double sA[kTK][kTR + 1];
    __shared__ double sB[kTK][kTC];
    const int tid = threadIdx.x, tr = tid / 16, tc = tid % 16;
    const int64_t row0 = (int64_t)blockIdx.x * kTR;
    double acc[4][5];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 5; ++j) acc[i][j] = 0.0;
    for (int k0 = 0; k0 < r; k0 += kTK) {
        for (int t = tid; t < kTR * kTK; t += 256) {
            const int i = t / kTK, k = t % kTK;
            const int64_t gi = row0 + i;
            sA[k][i] = (gi < n && k0 + k < r) ? A[gi * lda + k0 + k] : 0.0;
        }
        for (int t = tid; t < kTK * kTC; t += 256) {
            const int k = t / kTC, j = t % kTC;
            sB[k][j] = (k0 + k < r && j < c) ? B[(int64_t)(k0 + k) * ldb + j] : 0.0;
        }
        __syncthreads();
#pragma unroll 4
        for (int k = 0; k < kTK; ++k) {
            double a[4], b[5];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = sA[k][tr * 4 + i];
#pragma unroll
            for (int j = 0; j < 5; ++j) b[j] = sB[k][tc * 5 + j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 5; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int64_t gi = row0 + tr * 4 + i;
        if (gi >= n) continue;
        const double add = rowadd ? rowadd[gi] : 0.0;
#pragma unroll
        for (int j = 0; j < 5; ++j) {
            const int gj = tc * 5 + j;
            if (gj < c) C[gi * ldc + gj] = acc[i][j] + add;
        }
    }
}

// Partial products for C[r x c] = A[n x r]^T * B[n x c]: CTA (tile, split)
// sums rows [split*len, (split+1)*len) of A and B into P[split][r][c].
__global__ void __launch_bounds__(256) gemm_tn_f64_partial(int64_t n, int r, int c,
                                                           const double *__restrict__ A, int64_t lda,
                                                           const double *__restrict__ B, int64_t ldb,
                                                           double *__restrict__ P, int64_t len) {
    __shared__ double sA[kTK][kTR + 1];
    __shared__ double sB[kTK][kTC];
    const int tid = threadIdx.x, tr = tid / 16, tc = tid % 16;
    const int i0 = blockIdx.x * kTR;
    const int split = blockIdx.y;
    const int64_t n0 = (int64_t)split * len, n1 = min(n, n0 + len);
    double acc[4][5];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 5; ++j) acc[i][j] = 0.0;
    for (int64_t k0 = n0; k0 < n1; k0 += kTK) {
        for (int t = tid; t < kTR * kTK; t += 256) {
            const int k = t / kTR, i = t % kTR;
            sA[k][i] = (k0 + k < n1 && i0 + i < r) ? A[(k0 + k) * lda + i0 + i] : 0.0;
        }
        for (int t = tid; t < kTK * kTC; t += 256) {
            const int k = t / kTC, j = t % kTC;
            sB[k][j] = (k0 + k < n1 && j < c) ? B[(k0 + k) * ldb + j] : 0.0;
        }
        __syncthreads();
#pragma unroll 4
        for (int k = 0; k < kTK; ++k) {
            double a[4], b[5];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = sA[k][tr * 4 + i];
#pragma unroll
            for (int j = 0; j < 5; ++j) b[j] = sB[k][tc * 5 + j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 5; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
        }
        __syncthreads();
    }
    double *Ps = P + (int64_t)split * r * c;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int gi = i0 + tr * 4 + i;
        if (gi >= r) continue;
#pragma unroll
        for (int j = 0; j < 5; ++j) {
            const int gj = tc * 5 + j;
            if (gj < c) Ps[(int64_t)gi * c + gj] = acc[i][j];
        }
    }
}

// C[i][j] = sum over splits in order of P[split][i][j]   (deterministic)
__global__ void sum_partials_f64(int nsplit, int64_t rc, const double *__restrict__ P,
                                 double *__restrict__ C, int64_t ldc, int c) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= rc) return;
    double s = 0.0;
    for (int k = 0; k < nsplit; ++k) s += P[(int64_t)k * rc + t];
    C[(t / c) * ldc + t % c] = s;
}

// row means of X (n x m) and X -= mean (in place); warp per row
__global__ void center_rows_f64(int64_t n, int m, double *__restrict__ X, double *__restrict__ mean) {
    const int64_t row = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (row >= n) return;
    double *x = X + row * m;
    double s = 0.0;
    for (int j = lane; j < m; j += 32) s += x[j];
    s = warp_tree32<double>(s);
    const double mu = s / m;
    for (int j = lane; j < m; j += 32) x[j] -= mu;
    if (lane == 0) mean[row] = mu;
}

// ------------------------------------------------------- small dense (1 CTA)
// Cholesky G + shift I = L L^T (l x l, l <= 80), shift = shift_rel * trace(G),
// and Rinv = (L^T)^{-1} (upper), so that Y * Rinv has orthonormal columns when
// G = Y^T Y (up to the shift).  status[0] |= 1 if the matrix is not positive
// definite.
__global__ void chol_rinv_kernel(int l, const double *__restrict__ G, double shift_rel,
                                 double *__restrict__ Rinv, int *status) {
    extern __shared__ double sh[];
    double *Lm = sh;            // l x l
    double *Li = sh + l * l;    // l x l, inverse of L
    const int tid = threadIdx.x;
    __shared__ int bad;
    __shared__ double shift;
    if (tid == 0) {
        bad = 0;
        double tr = 0.0;
        for (int i = 0; i < l; ++i) tr += G[i * l + i];
        shift = shift_rel * tr;
    }
    __syncthreads();
    for (int t = tid; t < l * l; t += blockDim.x) {
        Lm[t] = G[t] + ((t / l == t % l) ? shift : 0.0);
        Li[t] = 0.0;
    }
    __syncthreads();
    for (int k = 0; k < l; ++k) {
        if (tid == 0) {
            const double d = Lm[k * l + k];
            if (!(d > 0.0)) bad = 1;
            Lm[k * l + k] = sqrt(d > 0.0 ? d : 1.0);
        }
        __syncthreads();
        const double dk = Lm[k * l + k];
        for (int i = k + 1 + tid; i < l; i += blockDim.x) Lm[i * l + k] /= dk;
        __syncthreads();
        for (int t = tid; t < (l - k - 1) * (l - k - 1); t += blockDim.x) {
            const int i = k + 1 + t / (l - k - 1), j = k + 1 + t % (l - k - 1);
            if (j <= i) Lm[i * l + j] -= Lm[i * l + k] * Lm[j * l + k];
        }
        __syncthreads();
    }
    // L^{-1} by forward substitution, one column per thread
    for (int j = tid; j < l; j += blockDim.x) {
        for (int i = j; i < l; ++i) {
            double s = (i == j) ? 1.0 : 0.0;
            for (int k = j; k < i; ++k) s -= Lm[i * l + k] * Li[k * l + j];
            Li[i * l + j] = s / Lm[i * l + i];
        }
    }
    __syncthreads();
    for (int t = tid; t < l * l; t += blockDim.x) {
        const int i = t / l, j = t % l;
        Rinv[t] = Li[j * l + i];  // (L^{-1})^T
    }
    if (tid == 0) status[0] |= bad;
}

// Cyclic Jacobi eigen-decomposition of a symmetric l x l matrix (l <= 80):
// on exit lam[i] (descending) and W[:, i] (column i = eigenvector i).
__global__ void jacobi_eig_kernel(int l, const double *__restrict__ C, double *__restrict__ lam,
                                  double *__restrict__ W, int sweeps) {
    extern __shared__ double sh[];
    double *A = sh;            // l x l
    double *V = sh + l * l;    // l x l
    __shared__ double cs[2];
    __shared__ int order[80];
    const int tid = threadIdx.x;
    for (int t = tid; t < l * l; t += blockDim.x) {
        A[t] = C[t];
        V[t] = (t / l == t % l) ? 1.0 : 0.0;
    }
    __syncthreads();
    __shared__ int done;
    for (int sw = 0; sw < sweeps; ++sw) {
        if (tid == 0) {  // stop once the off-diagonal part is at rounding level
            double off = 0.0, tot = 0.0;
            for (int i = 0; i < l; ++i)
                for (int j = 0; j < l; ++j) {
                    const double v = A[i * l + j] * A[i * l + j];
                    tot += v;
                    if (i != j) off += v;
                }
            done = (off <= 1e-34 * tot) ? 1 : 0;
        }
        __syncthreads();
        if (done) break;
        for (int p = 0; p < l - 1; ++p)
            for (int q = p + 1; q < l; ++q) {
                if (tid == 0) {
                    const double apq = A[p * l + q];
                    double c = 1.0, s = 0.0;
                    if (fabs(apq) > 1e-300) {
                        const double tau = (A[q * l + q] - A[p * l + p]) / (2.0 * apq);
                        const double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
                        c = 1.0 / sqrt(1.0 + t * t);
                        s = t * c;
                    }
                    cs[0] = c;
                    cs[1] = s;
                }
                __syncthreads();
                const double c = cs[0], s = cs[1];
                if (s != 0.0) {
                    // A <- J^T A J with J the (p,q) rotation; V <- V J
                    for (int k = tid; k < l; k += blockDim.x) {
                        const double akp = A[k * l + p], akq = A[k * l + q];
                        A[k * l + p] = c * akp - s * akq;
                        A[k * l + q] = s * akp + c * akq;
                    }
                    __syncthreads();
                    for (int k = tid; k < l; k += blockDim.x) {
                        const double apk = A[p * l + k], aqk = A[q * l + k];
                        A[p * l + k] = c * apk - s * aqk;
                        A[q * l + k] = s * apk + c * aqk;
                        const double vkp = V[k * l + p], vkq = V[k * l + q];
                        V[k * l + p] = c * vkp - s * vkq;
                        V[k * l + q] = s * vkp + c * vkq;
                    }
                }
                __syncthreads();
            }
    }
    if (tid == 0) {  // order by eigenvalue, descending (selection sort, l <= 80)
        for (int i = 0; i < l; ++i) order[i] = i;
        for (int i = 0; i < l; ++i) {
            int b = i;
            for (int j = i + 1; j < l; ++j)
                if (A[order[j] * l + order[j]] > A[order[b] * l + order[b]]) b = j;
            const int t = order[i]; order[i] = order[b]; order[b] = t;
        }
    }
    __syncthreads();
    for (int t = tid; t < l * l; t += blockDim.x) {
        const int i = t / l, j = t % l;
        W[i * l + j] = V[i * l + order[j]];
    }
    for (int i = tid; i < l; i += blockDim.x) lam[i] = A[order[i] * l + order[i]];
}

// sign of each basis column: largest-magnitude entry positive (CTA per column)
__global__ void sign_fix_kernel(int64_t n, int k, double *__restrict__ Phi) {
    const int j = blockIdx.x;
    double best = 0.0;
    int64_t bi = 0;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
        const double v = fabs(Phi[i * k + j]);
        if (v > best || (v == best && i < bi)) { best = v; bi = i; }
    }
    __shared__ double sv[256];
    __shared__ int64_t si[256];
    sv[threadIdx.x] = best;
    si[threadIdx.x] = bi;
    __syncthreads();
    for (int h = blockDim.x / 2; h > 0; h >>= 1) {
        if ((int)threadIdx.x < h) {
            const double a = sv[threadIdx.x], b = sv[threadIdx.x + h];
            const int64_t ia = si[threadIdx.x], ib = si[threadIdx.x + h];
            if (b > a || (b == a && ib < ia)) { sv[threadIdx.x] = b; si[threadIdx.x] = ib; }
        }
        __syncthreads();
    }
    const bool flip = Phi[si[0] * k + j] < 0.0;
    if (flip)
        for (int64_t i = threadIdx.x; i < n; i += blockDim.x) Phi[i * k + j] = -Phi[i * k + j];
}

// standardised coefficients: for column k of C (m x kk) the mean and the
// population standard deviation over the m rows (CTA per column, fixed
// order), then T[j][k] = (C[j][k] - mean) / scale in FP32
__global__ void coef_stats_kernel(int m, int kk, const double *__restrict__ C, double *__restrict__ mean,
                                  double *__restrict__ scale) {
    __shared__ double sh[256];
    const int k = blockIdx.x, tid = threadIdx.x;
    double s = 0.0;
    for (int j = tid; j < m; j += 256) s += C[(int64_t)j * kk + k];
    sh[tid] = s;
    __syncthreads();
    for (int h = 128; h > 0; h >>= 1) {
        if (tid < h) sh[tid] += sh[tid + h];
        __syncthreads();
    }
    const double mu = sh[0] / m;
    __syncthreads();
    double q = 0.0;
    for (int j = tid; j < m; j += 256) {
        const double d = C[(int64_t)j * kk + k] - mu;
        q += d * d;
    }
    sh[tid] = q;
    __syncthreads();
    for (int h = 128; h > 0; h >>= 1) {
        if (tid < h) sh[tid] += sh[tid + h];
        __syncthreads();
    }
    if (tid == 0) {
        mean[k] = mu;
        const double sd = sqrt(sh[0] / m);
        scale[k] = sd > 0.0 ? sd : 1.0;
    }
}

__global__ void standardise_kernel(int64_t total, int kk, const double *__restrict__ C,
                                   const double *__restrict__ mean, const double *__restrict__ scale,
                                   float *__restrict__ T) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= total) return;
    const int k = (int)(t % kk);
    T[t] = (float)((C[t] - mean[k]) / scale[k]);
}

// -------------------------------------------------------------- MLP (FP32)
struct MlpDims {
    int d0, d1, d2, d3;
    int64_t w1, b1, w2, b2, w3, b3, count;  // offsets in the flat parameter vector
};

static MlpDims mlp_dims(const int32_t *d) {
    MlpDims m;
    m.d0 = d[0]; m.d1 = d[1]; m.d2 = d[2]; m.d3 = d[3];
    m.w1 = 0;
    m.b1 = m.w1 + (int64_t)m.d1 * m.d0;
    m.w2 = m.b1 + m.d1;
    m.b2 = m.w2 + (int64_t)m.d2 * m.d1;
    m.w3 = m.b2 + m.d2;
    m.b3 = m.w3 + (int64_t)m.d3 * m.d2;
    m.count = m.b3 + m.d3;
    return m;
}

__device__ __forceinline__ float gelu_f(float z) { return 0.5f * z * (1.0f + erff(z * 0.70710678118654752f)); }
// derivative of z Phi(z): Phi(z) + z phi(z)
__device__ __forceinline__ float gelu_grad_f(float z) {
    return 0.5f * (1.0f + erff(z * 0.70710678118654752f)) + z * 0.39894228040143268f * expf(-0.5f * z * z);
}

// He-uniform initialisation from uniform draws u in [-1, 1]:
// W_l = u * sqrt(6 / fan_in), biases 0
__global__ void mlp_init_kernel(MlpDims d, const float *__restrict__ u, float *__restrict__ w) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= d.count) return;
    float v;
    if (t < d.b1) v = u[t] * sqrtf(6.0f / d.d0);
    else if (t < d.w2) v = 0.0f;
    else if (t < d.b2) v = u[t] * sqrtf(6.0f / d.d1);
    else if (t < d.w3) v = 0.0f;
    else if (t < d.b3) v = u[t] * sqrtf(6.0f / d.d2);
    else v = 0.0f;
    w[t] = v;
}

// C[i][j] = sum_k A(i,k) B(k,j), A(i,k) = TA ? A[k*lda+i] : A[i*lda+k],
// B(k,j) = TB ? B[j*ldb+k] : B[k*ldb+j]; 32 x 32 tiles, 256 threads, 2 x 2
// outputs each, k ascending in one FMA chain per output.  Epilogues:
//   0: C = acc (+ bias[j]); CTAs of tile column 0 also write colsum[i] =
//      sum_k A(i,k) (the bias gradient when A = dZ^T)
//   1: Z = acc + bias[j] -> C, gelu(Z) -> C2
//   2: C = acc * gelu'(aux[i][j])                  (back through a GELU)
//   3: Y = acc + bias[j]; C = 2 (Y - aux[i][j]) / (M N) (MSE gradient),
//      C2 = (Y - aux)^2
constexpr int kMT = 32, kMK = 32;
template <bool TA, bool TB, int EPI>
__global__ void __launch_bounds__(256) mlp_gemm(int M, int N, int K, const float *__restrict__ A, int lda,
                                                const float *__restrict__ B, int ldb,
                                                const float *__restrict__ bias, float *__restrict__ C,
                                                float *__restrict__ C2, const float *__restrict__ aux,
                                                float *__restrict__ colsum) {
    __shared__ float sA[kMK][kMT + 1];
    __shared__ float sB[kMK][kMT + 1];
    const int tid = threadIdx.x, ty = tid / 16, tx = tid % 16;
    const int i0 = blockIdx.y * kMT, j0 = blockIdx.x * kMT;
    float acc[2][2] = {{0.f, 0.f}, {0.f, 0.f}};
    float csum = 0.f;
    for (int k0 = 0; k0 < K; k0 += kMK) {
        for (int t = tid; t < kMT * kMK; t += 256) {
            int i, k;
            if (TA) { i = t % kMT; k = t / kMT; } else { k = t % kMK; i = t / kMK; }
            const int gi = i0 + i, gk = k0 + k;
            float v = 0.f;
            if (gi < M && gk < K) v = TA ? A[(int64_t)gk * lda + gi] : A[(int64_t)gi * lda + gk];
            sA[k][i] = v;
        }
        for (int t = tid; t < kMT * kMK; t += 256) {
            int j, k;
            if (TB) { k = t % kMK; j = t / kMK; } else { j = t % kMT; k = t / kMT; }
            const int gj = j0 + j, gk = k0 + k;
            float v = 0.f;
            if (gj < N && gk < K) v = TB ? B[(int64_t)gj * ldb + gk] : B[(int64_t)gk * ldb + gj];
            sB[k][j] = v;
        }
        __syncthreads();
#pragma unroll 8
        for (int k = 0; k < kMK; ++k) {
            const float a0 = sA[k][ty * 2], a1 = sA[k][ty * 2 + 1];
            const float b0 = sB[k][tx * 2], b1 = sB[k][tx * 2 + 1];
            acc[0][0] = fmaf(a0, b0, acc[0][0]);
            acc[0][1] = fmaf(a0, b1, acc[0][1]);
            acc[1][0] = fmaf(a1, b0, acc[1][0]);
            acc[1][1] = fmaf(a1, b1, acc[1][1]);
        }
        if (EPI == 0 && colsum != nullptr && blockIdx.x == 0 && tid < kMT)
            for (int k = 0; k < kMK; ++k) csum += sA[k][tid];
        __syncthreads();
    }
    if (EPI == 0 && colsum != nullptr && blockIdx.x == 0 && tid < kMT && i0 + tid < M) colsum[i0 + tid] = csum;
#pragma unroll
    for (int a = 0; a < 2; ++a) {
        const int gi = i0 + ty * 2 + a;
        if (gi >= M) continue;
#pragma unroll
        for (int b = 0; b < 2; ++b) {
            const int gj = j0 + tx * 2 + b;
            if (gj >= N) continue;
            const int64_t o = (int64_t)gi * N + gj;
            float v = acc[a][b];
            if (EPI == 0) {
                C[o] = bias ? v + bias[gj] : v;
            } else if (EPI == 1) {
                v += bias[gj];
                C[o] = v;
                C2[o] = gelu_f(v);
            } else if (EPI == 2) {
                C[o] = v * gelu_grad_f(aux[o]);
            } else {
                v += bias[gj];
                const float d = v - aux[o];
                C[o] = 2.0f * d / ((float)M * (float)N);
                C2[o] = d * d;
            }
        }
    }
}

// mean of count squared errors -> *loss (one CTA, fixed order); with acc, adds
// loss / per_epoch to acc[*step / per_epoch - epoch0] (per-epoch mean of the
// batch losses)
__global__ void mse_reduce_kernel(int64_t count, const float *__restrict__ e2, float *loss,
                                  float *acc, const int64_t *step, int per_epoch, int64_t epoch0) {
    __shared__ float sh[256];
    const int tid = threadIdx.x;
    float s = 0.f;
    for (int64_t t = tid; t < count; t += 256) s += e2[t];
    sh[tid] = s;
    __syncthreads();
    for (int h = 128; h > 0; h >>= 1) {
        if (tid < h) sh[tid] += sh[tid + h];
        __syncthreads();
    }
    if (tid == 0) {
        const float l = sh[0] / (float)count;
        if (loss) *loss = l;
        if (acc) acc[*step / per_epoch - epoch0] += l / (float)per_epoch;
    }
}

// Adam with a cosine-decayed step size: t = *step (0-based),
// lr = lr0 (1 + cos(pi t / total)) / 2, bias corrections with t + 1; the last
// CTA to finish increments *step
__global__ void adam_kernel(int64_t P, float *__restrict__ w, const float *__restrict__ g,
                            float *__restrict__ m, float *__restrict__ v, int64_t *step,
                            unsigned *arrive, int64_t total, float lr0, float beta1, float beta2,
                            float eps) {
    const int64_t t = *step;
    const float lr = 0.5f * lr0 * (1.0f + cosf(3.14159265358979f * (float)((double)t / (double)total)));
    const float c1 = 1.0f - powf(beta1, (float)(t + 1)), c2 = 1.0f - powf(beta2, (float)(t + 1));
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < P) {
        const float gi = g[i];
        const float mi = beta1 * m[i] + (1.0f - beta1) * gi;
        const float vi = beta2 * v[i] + (1.0f - beta2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        w[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        if (atomicAdd(arrive, 1u) == gridDim.x - 1) {
            *arrive = 0u;
            *step = t + 1;
        }
    }
}

// MLP input of an ensemble: xin[e][k] = xi[k*s + e] (k < d0)
__global__ void xi_gather_kernel(int s, int d0, const double *__restrict__ xi, float *__restrict__ xin) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= s * d0) return;
    const int e = t / d0, k = t % d0;
    xin[t] = (float)xi[(int64_t)k * s + e];
}

// x0[i*s+e] = mean[i] + sum_k Phi[i][k] c[e][k], c = coef_mean + coef_scale * chat,
// the sum in FP32 (k ascending), the mean added in FP64
__global__ void guess_apply_kernel(int64_t n, int s, int kk, const double *__restrict__ mean,
                                   const float *__restrict__ Phi, const double *__restrict__ cmean,
                                   const double *__restrict__ cscale, const float *__restrict__ chat,
                                   double *__restrict__ x0) {
    extern __shared__ float cs[];  // s x kk
    for (int t = threadIdx.x; t < s * kk; t += blockDim.x) {
        const int k = t % kk;
        cs[t] = (float)(cmean[k] + cscale[k] * (double)chat[t]);
    }
    __syncthreads();
    const int64_t total = n * s;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = t / s;
        const int e = (int)(t % s);
        const float *ph = Phi + i * kk;
        const float *c = cs + e * kk;
        float acc = 0.f;
        for (int k = 0; k < kk; ++k) acc = fmaf(ph[k], c[k], acc);
        x0[t] = mean[i] + (double)acc;
    }
}

__global__ void sqrt_pos_kernel(int k, const double *__restrict__ lam, double *__restrict__ sigma) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < k) sigma[i] = lam[i] > 0.0 ? sqrt(lam[i]) : 0.0;
}

__global__ void to_f32_kernel(int64_t count, const double *__restrict__ src, float *__restrict__ dst) {
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < count;
         t += (int64_t)gridDim.x * blockDim.x)
        dst[t] = (float)src[t];
}

}  // namespace ens

// ------------------------------------------------------------ host side
namespace ens {
namespace {

size_t al256(size_t x) { return (x + 255) / 256 * 256; }

// row splits of a transposed product over n rows with r output rows: about
// 600 CTAs in all, at least 1024 rows per split
int tn_splits(int64_t n, int r) {
    const int64_t tiles = (r + kTR - 1) / kTR;
    int64_t ns = (600 + tiles - 1) / tiles;
    const int64_t cap = (n + 1023) / 1024;
    if (ns > cap) ns = cap;
    return (int)(ns < 1 ? 1 : ns);
}

void gemm_nn(int64_t n, int r, int c, const double *A, int64_t lda, const double *B, int64_t ldb,
             double *C, int64_t ldc, cudaStream_t st) {
    gemm_nn_f64<<<(unsigned)((n + kTR - 1) / kTR), 256, 0, st>>>(n, r, c, A, lda, B, ldb, C, ldc, nullptr);
}

// C (r x c, ldc) = A^T B over n rows; P holds tn_splits(n, r) * r * c doubles
void gemm_tn(int64_t n, int r, int c, const double *A, int64_t lda, const double *B, int64_t ldb,
             double *C, int64_t ldc, double *P, cudaStream_t st) {
    const int ns = tn_splits(n, r);
    const int64_t len = (n + ns - 1) / ns;
    dim3 grid((unsigned)((r + kTR - 1) / kTR), (unsigned)ns);
    gemm_tn_f64_partial<<<grid, 256, 0, st>>>(n, r, c, A, lda, B, ldb, P, len);
    const int64_t rc = (int64_t)r * c;
    sum_partials_f64<<<(unsigned)((rc + 255) / 256), 256, 0, st>>>(ns, rc, P, C, ldc, c);
}

struct PodWork {
    double *Y, *Q, *Z, *Zq, *P, *G, *Rinv, *W, *lam;
    int *status;
};

size_t pod_bytes(int64_t n, int m, int l, PodWork *w, char *base) {
    const int64_t pmax = std::max<int64_t>((int64_t)tn_splits(n, l) * l * l,
                                           std::max<int64_t>((int64_t)tn_splits(n, m) * m * l,
                                                             (int64_t)tn_splits(m, l) * l * l));
    const size_t sz[9] = {sizeof(double) * (size_t)n * l, sizeof(double) * (size_t)n * l,
                          sizeof(double) * (size_t)m * l, sizeof(double) * (size_t)m * l,
                          sizeof(double) * (size_t)pmax,  sizeof(double) * (size_t)l * l,
                          sizeof(double) * (size_t)l * l, sizeof(double) * (size_t)l * l,
                          sizeof(double) * (size_t)l};
    size_t off = 0;
    double **slots[9] = {w ? &w->Y : nullptr, w ? &w->Q : nullptr, w ? &w->Z : nullptr,
                         w ? &w->Zq : nullptr, w ? &w->P : nullptr, w ? &w->G : nullptr,
                         w ? &w->Rinv : nullptr, w ? &w->W : nullptr, w ? &w->lam : nullptr};
    for (int i = 0; i < 9; ++i) {
        if (w) *slots[i] = reinterpret_cast<double *>(base + off);
        off += al256(sz[i]);
    }
    if (w) w->status = reinterpret_cast<int *>(base + off);
    off += 256;
    return off;
}

// Q (rows x l) = orthonormal basis of the columns of Y (shifted CholeskyQR3,
// Fukaya, Kannan, Nakatsukasa, Yamamoto and Yanagisawa, SIAM J. Sci. Comput.
// 2020: one pass with shift 11 (rows l + l (l + 1)) u ||Y||_F^2, two plain
// passes).  Y is overwritten.
void orth(int64_t rows, int l, double *Y, double *Q, PodWork &w, cudaStream_t st) {
    const double u = 0x1p-53;
    const double shift = 11.0 * ((double)rows * l + (double)l * (l + 1)) * u;
    const size_t shm = 2 * sizeof(double) * (size_t)l * l;
    double *src = Y, *dst = Q;
    for (int pass = 0; pass < 3; ++pass) {
        gemm_tn(rows, l, l, src, l, src, l, w.G, l, w.P, st);
        chol_rinv_kernel<<<1, 256, shm, st>>>(l, w.G, pass == 0 ? shift : 0.0, w.Rinv, w.status);
        gemm_nn(rows, l, l, src, l, w.Rinv, l, dst, l, st);
        std::swap(src, dst);
    }
    // three passes: Y -> Q -> Y -> Q, the result is in Q
}

int check_dims(const int32_t *dims) {
    if (!dims) return fail(ENS_ERR_ARG, "mlp: dims is NULL");
    for (int i = 0; i < 4; ++i)
        if (dims[i] < 1 || dims[i] > 4096) return fail(ENS_ERR_ARG, "mlp: dims[%d] = %d not in 1..4096", i, dims[i]);
    return ENS_OK;
}

struct MlpWork {
    float *Z1, *A1, *Z2, *A2, *Y, *dY, *E2, *dZ2, *dZ1, *grad, *loss;
};

size_t mlp_bytes(const MlpDims &d, int B, MlpWork *w, char *base) {
    const size_t sz[11] = {(size_t)B * d.d1, (size_t)B * d.d1, (size_t)B * d.d2, (size_t)B * d.d2,
                           (size_t)B * d.d3, (size_t)B * d.d3, (size_t)B * d.d3, (size_t)B * d.d2,
                           (size_t)B * d.d1, (size_t)d.count, 1};
    float **slots[11] = {w ? &w->Z1 : nullptr, w ? &w->A1 : nullptr, w ? &w->Z2 : nullptr,
                         w ? &w->A2 : nullptr, w ? &w->Y : nullptr,  w ? &w->dY : nullptr,
                         w ? &w->E2 : nullptr, w ? &w->dZ2 : nullptr, w ? &w->dZ1 : nullptr,
                         w ? &w->grad : nullptr, w ? &w->loss : nullptr};
    size_t off = 0;
    for (int i = 0; i < 11; ++i) {
        if (w) *slots[i] = reinterpret_cast<float *>(base + off);
        off += al256(sizeof(float) * sz[i]);
    }
    return off;
}

dim3 mlp_grid(int M, int N) { return dim3((unsigned)((N + kMT - 1) / kMT), (unsigned)((M + kMT - 1) / kMT)); }

// forward to the last layer's pre-activation: Y = f(xin) (EPI 0 on layer 3),
// or with a target the MSE gradient dY and the squared errors E2 (EPI 3)
void mlp_fwd(const MlpDims &d, const float *W, int B, const float *xin, const float *target, float *y,
             MlpWork &w, cudaStream_t st) {
    mlp_gemm<false, true, 1><<<mlp_grid(B, d.d1), 256, 0, st>>>(B, d.d1, d.d0, xin, d.d0, W + d.w1, d.d0,
                                                                W + d.b1, w.Z1, w.A1, nullptr, nullptr);
    mlp_gemm<false, true, 1><<<mlp_grid(B, d.d2), 256, 0, st>>>(B, d.d2, d.d1, w.A1, d.d1, W + d.w2, d.d1,
                                                                W + d.b2, w.Z2, w.A2, nullptr, nullptr);
    if (target)
        mlp_gemm<false, true, 3><<<mlp_grid(B, d.d3), 256, 0, st>>>(B, d.d3, d.d2, w.A2, d.d2, W + d.w3, d.d2,
                                                                    W + d.b3, w.dY, w.E2, target, nullptr);
    else
        mlp_gemm<false, true, 0><<<mlp_grid(B, d.d3), 256, 0, st>>>(B, d.d3, d.d2, w.A2, d.d2, W + d.w3, d.d2,
                                                                    W + d.b3, y, nullptr, nullptr, nullptr);
}

// back-propagation of dY (after mlp_fwd with a target) into grad
void mlp_bwd(const MlpDims &d, const float *W, int B, const float *xin, float *grad, MlpWork &w,
             cudaStream_t st) {
    mlp_gemm<true, false, 0><<<mlp_grid(d.d3, d.d2), 256, 0, st>>>(d.d3, d.d2, B, w.dY, d.d3, w.A2, d.d2, nullptr,
                                                                   grad + d.w3, nullptr, nullptr, grad + d.b3);
    mlp_gemm<false, false, 2><<<mlp_grid(B, d.d2), 256, 0, st>>>(B, d.d2, d.d3, w.dY, d.d3, W + d.w3, d.d2, nullptr,
                                                                 w.dZ2, nullptr, w.Z2, nullptr);
    mlp_gemm<true, false, 0><<<mlp_grid(d.d2, d.d1), 256, 0, st>>>(d.d2, d.d1, B, w.dZ2, d.d2, w.A1, d.d1, nullptr,
                                                                   grad + d.w2, nullptr, nullptr, grad + d.b2);
    mlp_gemm<false, false, 2><<<mlp_grid(B, d.d1), 256, 0, st>>>(B, d.d1, d.d2, w.dZ2, d.d2, W + d.w2, d.d1, nullptr,
                                                                 w.dZ1, nullptr, w.Z1, nullptr);
    mlp_gemm<true, false, 0><<<mlp_grid(d.d1, d.d0), 256, 0, st>>>(d.d1, d.d0, B, w.dZ1, d.d1, xin, d.d0, nullptr,
                                                                   grad + d.w1, nullptr, nullptr, grad + d.b1);
}

void adam_launch(int64_t P, float *W, const float *g, float *m, float *v, int64_t *step, int64_t total,
                 float lr0, float b1, float b2, float eps, cudaStream_t st) {
    adam_kernel<<<(unsigned)((P + 255) / 256), 256, 0, st>>>(P, W, g, m, v, step,
                                                            reinterpret_cast<unsigned *>(step + 1), total,
                                                            lr0, b1, b2, eps);
}

}  // namespace
}  // namespace ens

// ------------------------------------------------------------ C ABI
using namespace ens;

extern "C" {

int ens_snapshots_put(int64_t n, int32_t s, const double *x, double *X, int64_t ldx, int64_t col0,
                      void *stream) {
    if (n < 1 || s < 1 || !x || !X || col0 < 0 || ldx < col0 + s)
        return fail(ENS_ERR_ARG, "ens_snapshots_put: bad arguments (n=%lld s=%d ldx=%lld col0=%lld)",
                    (long long)n, s, (long long)ldx, (long long)col0);
    ENS_CUDA_TRY(cudaMemcpy2DAsync(X + col0, sizeof(double) * (size_t)ldx, x, sizeof(double) * (size_t)s,
                                   sizeof(double) * (size_t)s, (size_t)n, cudaMemcpyDeviceToDevice,
                                   as_stream(stream)));
    return ENS_OK;
}

int ens_pod_workspace_size(int64_t n, int32_t m, int32_t l, size_t *bytes) {
    if (n < 1 || m < 1 || l < 1 || !bytes) return fail(ENS_ERR_ARG, "ens_pod_workspace_size: bad arguments");
    *bytes = pod_bytes(n, m, l, nullptr, nullptr);
    return ENS_OK;
}

int ens_pod(int64_t n, int32_t m, double *X, int64_t ldx, int32_t k, int32_t l, const double *Omega,
            int32_t power_iters, double *mean, double *Phi, double *sigma, void *work, size_t work_bytes,
            void *stream) {
    if (!X || !Omega || !mean || !Phi || !sigma || !work)
        return fail(ENS_ERR_ARG, "ens_pod: NULL pointer");
    if (m < 2 || ldx < m || l < 1 || l > 80 || k < 1 || k > l || l > m - 1 || n < l || power_iters < 0 ||
        power_iters > 8)
        return fail(ENS_ERR_ARG, "ens_pod: need 1 <= k <= l <= min(80, m - 1), l <= n, 0 <= power_iters <= 8 "
                    "(n=%lld m=%d k=%d l=%d q=%d)", (long long)n, m, k, l, power_iters);
    const size_t need = pod_bytes(n, m, l, nullptr, nullptr);
    if (work_bytes < need) return fail(ENS_ERR_WORKSPACE, "ens_pod: workspace %zu < %zu", work_bytes, need);
    cudaStream_t st = as_stream(stream);
    PodWork w;
    pod_bytes(n, m, l, &w, static_cast<char *>(work));
    const size_t shm = 2 * sizeof(double) * (size_t)l * l;
    ENS_CUDA_TRY(cudaFuncSetAttribute(chol_rinv_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm));
    ENS_CUDA_TRY(cudaFuncSetAttribute(jacobi_eig_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm));
    ENS_CUDA_TRY(cudaMemsetAsync(w.status, 0, sizeof(int), st));
    // centre, range finder with stabilised power iterations
    center_rows_f64<<<(unsigned)((n * 32 + 255) / 256), 256, 0, st>>>(n, m, X, mean);
    gemm_nn(n, m, l, X, ldx, Omega, l, w.Y, l, st);
    orth(n, l, w.Y, w.Q, w, st);
    for (int it = 0; it < power_iters; ++it) {
        gemm_tn(n, m, l, X, ldx, w.Q, l, w.Z, l, w.P, st);   // Z = X^T Q
        orth(m, l, w.Z, w.Zq, w, st);
        gemm_nn(n, m, l, X, ldx, w.Zq, l, w.Y, l, st);      // Y = X Zq
        orth(n, l, w.Y, w.Q, w, st);
    }
    // Rayleigh-Ritz: eigenvectors of (X^T Q)^T (X^T Q) = Q^T X X^T Q
    gemm_tn(n, m, l, X, ldx, w.Q, l, w.Z, l, w.P, st);
    gemm_tn(m, l, l, w.Z, l, w.Z, l, w.G, l, w.P, st);
    jacobi_eig_kernel<<<1, 256, shm, st>>>(l, w.G, w.lam, w.W, 60);
    gemm_nn(n, l, k, w.Q, l, w.W, l, Phi, k, st);
    sign_fix_kernel<<<k, 256, 0, st>>>(n, k, Phi);
    sqrt_pos_kernel<<<1, 128, 0, st>>>(k, w.lam, sigma);
    ENS_LAUNCH_CHECK("ens_pod");
    int bad = 0;
    ENS_CUDA_TRY(cudaMemcpyAsync(&bad, w.status, sizeof(int), cudaMemcpyDeviceToHost, st));
    ENS_CUDA_TRY(cudaStreamSynchronize(st));
    if (bad) return fail(ENS_ERR_BREAKDOWN, "ens_pod: Gram matrix not positive definite (snapshots of numerical "
                         "rank below l = %d)", l);
    return ENS_OK;
}

static size_t targets_bytes(int64_t n, int m, int k) {
    return al256(sizeof(double) * (size_t)m * k) + al256(sizeof(double) * (size_t)tn_splits(n, m) * m * k);
}

int ens_pod_targets_workspace_size(int64_t n, int32_t m, int32_t k, size_t *bytes) {
    if (n < 1 || m < 1 || k < 1 || !bytes) return fail(ENS_ERR_ARG, "ens_pod_targets_workspace_size: bad arguments");
    *bytes = targets_bytes(n, m, k);
    return ENS_OK;
}

int ens_pod_targets(int64_t n, int32_t m, const double *X, int64_t ldx, int32_t k, const double *Phi,
                    double *coef_mean, double *coef_scale, float *T, void *work, size_t work_bytes,
                    void *stream) {
    if (!X || !Phi || !coef_mean || !coef_scale || !T || !work)
        return fail(ENS_ERR_ARG, "ens_pod_targets: NULL pointer");
    if (n < 1 || m < 1 || ldx < m || k < 1 || k > 80)
        return fail(ENS_ERR_ARG, "ens_pod_targets: bad sizes (n=%lld m=%d k=%d)", (long long)n, m, k);
    if (work_bytes < targets_bytes(n, m, k))
        return fail(ENS_ERR_WORKSPACE, "ens_pod_targets: workspace too small");
    cudaStream_t st = as_stream(stream);
    double *C = static_cast<double *>(work);
    double *P = reinterpret_cast<double *>(static_cast<char *>(work) + al256(sizeof(double) * (size_t)m * k));
    gemm_tn(n, m, k, X, ldx, Phi, k, C, k, P, st);  // C = X^T Phi  (m x k)
    coef_stats_kernel<<<k, 256, 0, st>>>(m, k, C, coef_mean, coef_scale);
    const int64_t tot = (int64_t)m * k;
    standardise_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(tot, k, C, coef_mean, coef_scale, T);
    ENS_LAUNCH_CHECK("ens_pod_targets");
    return ENS_OK;
}

int ens_to_f32(int64_t count, const double *src, float *dst, void *stream) {
    if (count < 0 || (count > 0 && (!src || !dst))) return fail(ENS_ERR_ARG, "ens_to_f32: bad arguments");
    if (count == 0) return ENS_OK;
    const int64_t blocks = std::min<int64_t>((count + 255) / 256, 152 * 8);
    to_f32_kernel<<<(unsigned)blocks, 256, 0, as_stream(stream)>>>(count, src, dst);
    ENS_LAUNCH_CHECK("ens_to_f32");
    return ENS_OK;
}

int ens_mlp_param_count(const int32_t *dims, int64_t *count) {
    int rc = check_dims(dims);
    if (rc) return rc;
    if (!count) return fail(ENS_ERR_ARG, "ens_mlp_param_count: count is NULL");
    *count = mlp_dims(dims).count;
    return ENS_OK;
}

int ens_mlp_init(const int32_t *dims, const float *u, float *params, void *stream) {
    int rc = check_dims(dims);
    if (rc) return rc;
    if (!u || !params) return fail(ENS_ERR_ARG, "ens_mlp_init: NULL pointer");
    const MlpDims d = mlp_dims(dims);
    mlp_init_kernel<<<(unsigned)((d.count + 255) / 256), 256, 0, as_stream(stream)>>>(d, u, params);
    ENS_LAUNCH_CHECK("ens_mlp_init");
    return ENS_OK;
}

int ens_mlp_workspace_size(const int32_t *dims, int32_t batch, size_t *bytes) {
    int rc = check_dims(dims);
    if (rc) return rc;
    if (batch < 1 || !bytes) return fail(ENS_ERR_ARG, "ens_mlp_workspace_size: bad arguments");
    *bytes = mlp_bytes(mlp_dims(dims), batch, nullptr, nullptr);
    return ENS_OK;
}

int ens_mlp_forward(const int32_t *dims, const float *params, int32_t batch, const float *xin, float *y,
                    void *work, size_t work_bytes, void *stream) {
    int rc = check_dims(dims);
    if (rc) return rc;
    if (!params || !xin || !y || !work || batch < 1) return fail(ENS_ERR_ARG, "ens_mlp_forward: bad arguments");
    if (work_bytes < mlp_bytes(mlp_dims(dims), batch, nullptr, nullptr))
        return fail(ENS_ERR_WORKSPACE, "ens_mlp_forward: workspace too small");
    const MlpDims d = mlp_dims(dims);
    MlpWork w;
    mlp_bytes(d, batch, &w, static_cast<char *>(work));
    mlp_fwd(d, params, batch, xin, nullptr, y, w, as_stream(stream));
    ENS_LAUNCH_CHECK("ens_mlp_forward");
    return ENS_OK;
}

int ens_mlp_grad(const int32_t *dims, const float *params, int32_t batch, const float *xin, const float *target,
                 float *grad, float *loss, void *work, size_t work_bytes, void *stream) {
    int rc = check_dims(dims);
    if (rc) return rc;
    if (!params || !xin || !target || !grad || !work || batch < 1)
        return fail(ENS_ERR_ARG, "ens_mlp_grad: bad arguments");
    if (work_bytes < mlp_bytes(mlp_dims(dims), batch, nullptr, nullptr))
        return fail(ENS_ERR_WORKSPACE, "ens_mlp_grad: workspace too small");
    cudaStream_t st = as_stream(stream);
    const MlpDims d = mlp_dims(dims);
    MlpWork w;
    mlp_bytes(d, batch, &w, static_cast<char *>(work));
    mlp_fwd(d, params, batch, xin, target, nullptr, w, st);
    mlp_bwd(d, params, batch, xin, grad, w, st);
    if (loss) mse_reduce_kernel<<<1, 256, 0, st>>>((int64_t)batch * d.d3, w.E2, loss, nullptr, nullptr, 1, 0);
    ENS_LAUNCH_CHECK("ens_mlp_grad");
    return ENS_OK;
}

int ens_mlp_adam(int64_t P, float *params, const float *grad, float *m, float *v, int64_t *step,
                 int64_t total_steps, float lr0, float beta1, float beta2, float eps, void *stream) {
    if (P < 1 || !params || !grad || !m || !v || !step || total_steps < 1)
        return fail(ENS_ERR_ARG, "ens_mlp_adam: bad arguments");
    adam_launch(P, params, grad, m, v, step, total_steps, lr0, beta1, beta2, eps, as_stream(stream));
    ENS_LAUNCH_CHECK("ens_mlp_adam");
    return ENS_OK;
}

int ens_mlp_train(const int32_t *dims, float *params, float *m, float *v, int64_t *step, int64_t n_samples,
                  const float *xin, const float *target, int32_t batch, int32_t epochs, int64_t total_steps,
                  float lr0, float beta1, float beta2, float eps, float *epoch_loss, int32_t use_graph,
                  void *work, size_t work_bytes, void *stream) {
    int rc = check_dims(dims);
    if (rc) return rc;
    if (!params || !m || !v || !step || !xin || !target || !work || batch < 1 || epochs < 0 ||
        n_samples < batch || n_samples % batch != 0 || total_steps < 1)
        return fail(ENS_ERR_ARG, "ens_mlp_train: bad arguments (n_samples must be a positive multiple of batch)");
    if (work_bytes < mlp_bytes(mlp_dims(dims), batch, nullptr, nullptr))
        return fail(ENS_ERR_WORKSPACE, "ens_mlp_train: workspace too small");
    if (epochs == 0) return ENS_OK;
    cudaStream_t st = as_stream(stream);
    const MlpDims d = mlp_dims(dims);
    MlpWork w;
    mlp_bytes(d, batch, &w, static_cast<char *>(work));
    const int per_epoch = (int)(n_samples / batch);
    // epoch_loss[e] accumulates from the step count at entry
    int64_t step0 = 0;
    ENS_CUDA_TRY(cudaMemcpyAsync(&step0, step, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    ENS_CUDA_TRY(cudaStreamSynchronize(st));
    if (step0 % per_epoch != 0)
        return fail(ENS_ERR_ARG, "ens_mlp_train: step count %lld is not at an epoch boundary", (long long)step0);
    if (epoch_loss) ENS_CUDA_TRY(cudaMemsetAsync(epoch_loss, 0, sizeof(float) * (size_t)epochs, st));
    const int64_t epoch0 = step0 / per_epoch;
    auto one_epoch = [&](cudaStream_t s) {
        for (int b = 0; b < per_epoch; ++b) {
            const float *xb = xin + (int64_t)b * batch * d.d0;
            const float *tb = target + (int64_t)b * batch * d.d3;
            mlp_fwd(d, params, batch, xb, tb, nullptr, w, s);
            mlp_bwd(d, params, batch, xb, w.grad, w, s);
            if (epoch_loss)
                mse_reduce_kernel<<<1, 256, 0, s>>>((int64_t)batch * d.d3, w.E2, nullptr, epoch_loss, step, per_epoch,
                                                    epoch0);
            adam_launch(d.count, params, w.grad, m, v, step, total_steps, lr0, beta1, beta2, eps, s);
        }
    };
    if (!use_graph) {
        for (int e = 0; e < epochs; ++e) one_epoch(st);
        ENS_LAUNCH_CHECK("ens_mlp_train");
        return ENS_OK;
    }
    cudaStream_t cap;
    ENS_CUDA_TRY(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t gexec = nullptr;
    cudaError_t ce = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
    if (ce == cudaSuccess) {
        one_epoch(cap);
        ce = cudaStreamEndCapture(cap, &graph);
    }
    cudaStreamDestroy(cap);
    if (ce != cudaSuccess) return cuda_fail(ce, "ens_mlp_train: epoch graph capture");
    ce = cudaGraphInstantiate(&gexec, graph, 0);
    if (ce != cudaSuccess) { cudaGraphDestroy(graph); return cuda_fail(ce, "ens_mlp_train: cudaGraphInstantiate"); }
    for (int e = 0; e < epochs && ce == cudaSuccess; ++e) ce = cudaGraphLaunch(gexec, st);
    cudaGraphExecDestroy(gexec);
    cudaGraphDestroy(graph);
    if (ce != cudaSuccess) return cuda_fail(ce, "ens_mlp_train: cudaGraphLaunch");
    ENS_LAUNCH_CHECK("ens_mlp_train");
    return ENS_OK;
}

static size_t guess_bytes(const MlpDims &d, int s) {
    return mlp_bytes(d, s, nullptr, nullptr) + al256(sizeof(float) * (size_t)s * d.d0) +
           al256(sizeof(float) * (size_t)s * d.d3);
}

int ens_guess_workspace_size(const int32_t *dims, int32_t s, size_t *bytes) {
    int rc = check_dims(dims);
    if (rc) return rc;
    if (s < 1 || !bytes) return fail(ENS_ERR_ARG, "ens_guess_workspace_size: bad arguments");
    *bytes = guess_bytes(mlp_dims(dims), s);
    return ENS_OK;
}

int ens_guess(const int32_t *dims, const float *params, int64_t n, int32_t s, const double *xi,
              const double *mean, const float *Phi32, const double *coef_mean, const double *coef_scale,
              double *x0, void *work, size_t work_bytes, void *stream) {
    int rc = check_dims(dims);
    if (rc) return rc;
    if (!params || !xi || !mean || !Phi32 || !coef_mean || !coef_scale || !x0 || !work || n < 1 || s < 1 ||
        s > 32 || dims[3] > 256)
        return fail(ENS_ERR_ARG, "ens_guess: bad arguments (1 <= s <= 32, dims[3] <= 256)");
    if (work_bytes < guess_bytes(mlp_dims(dims), s))
        return fail(ENS_ERR_WORKSPACE, "ens_guess: workspace too small");
    cudaStream_t st = as_stream(stream);
    const MlpDims d = mlp_dims(dims);
    MlpWork w;
    char *base = static_cast<char *>(work);
    const size_t mb = mlp_bytes(d, s, &w, base);
    float *xin = reinterpret_cast<float *>(base + mb);
    float *chat = reinterpret_cast<float *>(base + mb + al256(sizeof(float) * (size_t)s * d.d0));
    xi_gather_kernel<<<(unsigned)((s * d.d0 + 255) / 256), 256, 0, st>>>(s, d.d0, xi, xin);
    mlp_fwd(d, params, s, xin, nullptr, chat, w, st);
    const int64_t blocks = std::min<int64_t>((n * s + 255) / 256, 152 * 8);
    guess_apply_kernel<<<(unsigned)blocks, 256, sizeof(float) * (size_t)s * d.d3, st>>>(
        n, s, d.d3, mean, Phi32, coef_mean, coef_scale, chat, x0);
    ENS_LAUNCH_CHECK("ens_guess");
    return ENS_OK;
}

}  // extern "C"
