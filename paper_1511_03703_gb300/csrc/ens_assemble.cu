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
#include <math.h>
#include <string.h>

#include <algorithm>
#include <mutex>

#include "ens_spmv.cuh"

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

// The same combination with the KL terms in double-float arithmetic on the
// FP32 pipe (GB300 runs FP64 FMAs at 1/64 of the FP32 rate): each
// coefficient sigma*xi_k is split into a rounded float pair, each mode value
// by truncation (47 bits), the terms c_k m_k (k >= 1) are formed as in the
// double-float SpMV and summed as an unevaluated float pair, and the value is
// kappa0 * m_0 + (that sum) by one FP64 FMA.  Two FP64 operations per value
// instead of M + 1; the KL terms carry a relative error of about 2^-46 each.
// A mode value or coefficient outside the split range [2^-103, 2^128) (or
// not finite) makes the thread (the whole CTA, for a coefficient) compute
// its values in FP64 instead.  With vdf the values' truncating split (the
// ENS_F64_DF copy for ens_cg_df) is written as well.
// one member's value by the FP64 combination of assemble_values_kernel (out
// of line: the rare path of the double-float kernel)
static __device__ __noinline__ double asm_value_fp64(const double *coef, int stride, int M,
                                                     const double *__restrict__ modes, int64_t nnz,
                                                     int64_t e) {
    double x = coef[0] * __ldg(modes + e);
    for (int k = 1; k <= M; ++k) x = fma(coef[k * stride], __ldg(modes + (int64_t)k * nnz + e), x);
    return x;
}

// Two members' double-float terms at once with the packed FP32 instructions
// of sm_100+ (add/sub/mul/fma .rn.f32x2: per lane IEEE round-to-nearest, so
// each lane is bitwise the scalar df_term_pre).  The product is kept negated
// (np = -(ah*xh), exact) so that every step is an add, sub, mul or fma:
//   e  = ah*xh - p + ah*xl + al*xh     (fma(ah, xh, np), then two fmas)
//   s  = S + p = S - np;  bb = s - S
//   t  = (S - (s - bb)) + (p - bb) = (S - (s - bb)) - (np + bb)
//   S' = s,  C' = C + (t + e)
__device__ __forceinline__ uint64_t f2_pack(float lo, float hi) {
    uint64_t r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ void f2_unpack(uint64_t v, float &lo, float &hi) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
__device__ __forceinline__ uint64_t f2_add(uint64_t a, uint64_t b) {
    uint64_t r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ uint64_t f2_sub(uint64_t a, uint64_t b) {
    uint64_t r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ uint64_t f2_mul(uint64_t a, uint64_t b) {
    uint64_t r;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ uint64_t f2_fma(uint64_t a, uint64_t b, uint64_t c) {
    uint64_t r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
    return r;
}
// (S, C) += (ah + al) * (xh + xl) for two members; nah = -ah
__device__ __forceinline__ void df_term_pair(uint64_t &S, uint64_t &C, uint64_t ah, uint64_t nah, uint64_t al,
                                             uint64_t xh, uint64_t xl) {
    const uint64_t np = f2_mul(nah, xh);
    uint64_t e = f2_fma(ah, xh, np);
    e = f2_fma(ah, xl, e);
    e = f2_fma(al, xh, e);
    const uint64_t s = f2_sub(S, np);
    const uint64_t bb = f2_sub(s, S);
    const uint64_t t = f2_sub(f2_sub(S, f2_sub(s, bb)), f2_add(np, bb));
    S = s;
    C = f2_add(C, f2_add(t, e));
}

template <int S>
__global__ void __launch_bounds__(256) assemble_values_df_kernel(
    int64_t nnz, int M, const double *__restrict__ modes, const double *__restrict__ xi,
    double sigma, double kappa0, double *__restrict__ values, float2 *__restrict__ vdf) {
    // rounded split of coef[k*S + e], k >= 1: (h, l) per member, or for s >= 2
    // per member pair (h_2j, h_2j+1, l_2j, l_2j+1) at coef4[k*S/2 + j]
    __shared__ __align__(16) float2 coef[kAsmMaxCoef];
    __shared__ double coef64[kAsmMaxCoef];
    __shared__ int coef_bad;
    if (threadIdx.x == 0) coef_bad = 0;
    __syncthreads();
    for (int i = threadIdx.x; i < (M + 1) * S; i += blockDim.x) {
        const double c = (i < S) ? kappa0 : sigma * xi[i - S];
        const float h = (float)c;
        const float l = (float)(c - (double)h);
        const double a = fabs(c);
        if (i >= S && !(c == 0.0 || (a >= 0x1p-103 && a < 0x1p+127))) coef_bad = 1;
        if constexpr (S == 1) {
            coef[i] = make_float2(h, l);
        } else {
            float *q = reinterpret_cast<float *>(coef) + 4 * (i >> 1) + (i & 1);
            q[0] = h;
            q[2] = l;
        }
        coef64[i] = c;
    }
    __syncthreads();
    // W members per thread (up to 8): each mode value is split once for W
    // members, so the split's integer work is spread over more terms
    constexpr int W = (S < 8) ? S : 8;
    constexpr int G = S / W;  // threads per entry
    const int64_t total = nnz * G;
    // grid-stride over (entry, member group): the coefficient split above is
    // done once per CTA
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t e = t / G;
        const int g = (int)(t % G);
        const int m0 = g * W;
        DfAcc A[W];
        bool ok = coef_bad == 0;
        if constexpr (W == 1) {
            A[0] = df_zero();
            for (int k = 1; k <= M; ++k) {
                const double mk = __ldg(modes + (int64_t)k * nnz + e);
                float mh, ml;
                ok &= df_split_trunc(mk, mh, ml);
                const float2 c = coef[k * S + m0];
                df_term_pre(A[0], mh, ml, c.x, c.y);
            }
        } else {
            uint64_t AS[W / 2], AC[W / 2];
#pragma unroll
            for (int j = 0; j < W / 2; ++j) AS[j] = AC[j] = 0ull;  // (+0, +0)
            const float4 *c4 = reinterpret_cast<const float4 *>(coef);
            for (int k = 1; k <= M; ++k) {
                const double mk = __ldg(modes + (int64_t)k * nnz + e);
                float mh, ml;
                ok &= df_split_trunc(mk, mh, ml);
                const uint64_t ah = f2_pack(mh, mh), nah = f2_pack(-mh, -mh), al = f2_pack(ml, ml);
#pragma unroll
                for (int j = 0; j < W / 2; ++j) {
                    const float4 c = c4[(k * S + m0) / 2 + j];
                    df_term_pair(AS[j], AC[j], ah, nah, al, f2_pack(c.x, c.y), f2_pack(c.z, c.w));
                }
            }
#pragma unroll
            for (int j = 0; j < W / 2; ++j) {
                f2_unpack(AS[j], A[2 * j].s, A[2 * j + 1].s);
                f2_unpack(AC[j], A[2 * j].c, A[2 * j + 1].c);
            }
        }
        const double mz = __ldg(modes + e);
        double v[W];
#pragma unroll
        for (int w = 0; w < W; ++w) v[w] = fma(coef64[m0 + w], mz, f2d_exact(A[w].s) + f2d_exact(A[w].c));
        if (!ok) {  // FP64 combination, in the order of assemble_values_kernel
#pragma unroll
            for (int w = 0; w < W; ++w) v[w] = asm_value_fp64(coef64 + m0 + w, S, M, modes, nnz, e);
        }
        double *vo = values + e * S + m0;
        if constexpr (W == 1) {
            vo[0] = v[0];
        } else {
#pragma unroll
            for (int w = 0; w < W; w += 2) reinterpret_cast<double2 *>(vo)[w / 2] = make_double2(v[w], v[w + 1]);
        }
        if (vdf) {
            float2 p[W];
#pragma unroll
            for (int w = 0; w < W; ++w) {
                float h, l;
                p[w] = df_split_trunc(v[w], h, l) ? make_float2(h, l)
                                                  : make_float2(__int_as_float(0x7fc00000), 0.0f);
            }
            float2 *po = vdf + e * S + m0;
            if constexpr (W == 1) {
                po[0] = p[0];
            } else {
#pragma unroll
                for (int w = 0; w < W; w += 2)
                    reinterpret_cast<float4 *>(po)[w / 2] = make_float4(p[w].x, p[w].y, p[w + 1].x, p[w + 1].y);
            }
        }
    }
}

// thread per (row, member): right-hand side and the Dirichlet identity rows
template <int S>
__global__ void assemble_rows_kernel(int32_t n, const int32_t *__restrict__ row_map,
                                     const int32_t *__restrict__ col_entry,
                                     const uint8_t *__restrict__ bmask,
                                     const double *__restrict__ load, double *__restrict__ values,
                                     double *__restrict__ b, float2 *__restrict__ vdf) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t I = t / S;
    const int e = (int)(t % S);
    if (I >= n) return;
    b[t] = load[I];
    if (bmask[I]) {
        for (int32_t p = row_map[I]; p < row_map[I + 1]; ++p)
            if (col_entry[p] == I) {
                values[(int64_t)p * S + e] = 1.0;
                if (vdf) vdf[(int64_t)p * S + e] = make_float2(1.0f, 0.0f);
            }
    }
}

// grid of the grid-stride double-float kernel: one wave of resident CTAs
template <int S>
static unsigned asm_df_grid() {
    static const unsigned g = [] {
        int occ = 0, dev = 0, sms = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, assemble_values_df_kernel<S>, 256, 0);
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        return (unsigned)((occ > 0 ? occ : 1) * (sms > 0 ? sms : 152));
    }();
    return g;
}

// ------------------------------------------------ coefficient positivity
// Member e's coefficient at a Gauss point is
//     a_e(x_q) = kappa0 + sigma * sum_k xi[k*s + e] * kappa_k(x_q),
// kappa_k(x_q) = T[0][k][tx] * T[1][k][ty] * T[2][k][tz] (the separable table
// of ens_kl_setup, T[d][k][t] at kl_table[(d*M + k)*2N + t]).  The stiffness
// matrix is SPD only if a_e > 0 at every Gauss point (Sect. 4's coefficient
// is positive by construction for bounded xi and small sigma).
//   Bound: max_q |kappa_k(x_q)| = prod_d max_t |T[d][k][t]| exactly, so
//     kappa0 - |sigma| * sum_k |xi_k^e| * max_q |kappa_k|  <=  min_q a_e(x_q).
//   Exact: for members whose bound is not positive, the minimum of a_e over all
//     (2N)^3 Gauss coordinates, each evaluated as the sum over k in increasing
//     k of kappa_k * xi_k, then kappa0 + sigma * sum (no fused operations).
// One CTA: the bound of every member into out[e].
__global__ void coeff_bound_kernel(int N, int M, const double *__restrict__ T, int s,
                                   const double *__restrict__ xi, double sigma, double kappa0,
                                   double *__restrict__ out) {
    __shared__ double cmax[64];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int nt = 2 * N;
    for (int k = warp; k < M; k += nw) {
        double prod = 1.0;
        for (int d = 0; d < 3; ++d) {
            double m = 0.0;
            for (int t = lane; t < nt; t += 32) {
                const double v = fabs(T[((int64_t)d * M + k) * nt + t]);
                m = (v > m || v != v) ? v : m;   // a NaN entry propagates
            }
            for (int o = 16; o >= 1; o >>= 1) {
                const double w = __shfl_xor_sync(0xffffffffu, m, o);
                m = (w > m || w != w) ? w : m;
            }
            prod *= m;
        }
        if (lane == 0) cmax[k] = prod;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < s; e += blockDim.x) {
        double sum = 0.0;
        for (int k = 0; k < M; ++k) sum += fabs(xi[(int64_t)k * s + e]) * cmax[k];
        out[e] = kappa0 - fabs(sigma) * sum;
    }
}

// order-preserving key of a double for atomicMin (NaN maps below -inf)
__device__ __forceinline__ unsigned long long order_key(double v) {
    if (v != v) return 0ull;
    const unsigned long long u = (unsigned long long)__double_as_longlong(v);
    return (u >> 63) ? ~u : (u | 0x8000000000000000ull);
}

// Exact minimum of a_e over the Gauss points, members with need[e] != 0:
// thread per Gauss point (grid-stride), warp minimum, then atomicMin on the
// ordered key in key_out[e] (which the host set to all ones).
__global__ void __launch_bounds__(256) coeff_min_kernel(int N, int M, const double *__restrict__ T, int s,
                                                        const double *__restrict__ xi, double sigma,
                                                        double kappa0, const int *__restrict__ need,
                                                        unsigned long long *__restrict__ key_out) {
    const int64_t nt = 2 * N, npts = nt * nt * nt;
    for (int e = 0; e < s; ++e) {
        if (!need[e]) continue;
        unsigned long long best = ~0ull;
        for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < npts;
             q += (int64_t)gridDim.x * blockDim.x) {
            const int64_t tx = q % nt, ty = (q / nt) % nt, tz = q / (nt * nt);
            double sum = 0.0;
            for (int k = 0; k < M; ++k) {
                const double kap = __dmul_rn(__dmul_rn(__ldg(T + (int64_t)k * nt + tx),
                                                       __ldg(T + ((int64_t)M + k) * nt + ty)),
                                             __ldg(T + ((int64_t)2 * M + k) * nt + tz));
                sum = __dadd_rn(sum, __dmul_rn(kap, __ldg(xi + (int64_t)k * s + e)));
            }
            const unsigned long long key = order_key(__dadd_rn(kappa0, __dmul_rn(sigma, sum)));
            best = key < best ? key : best;
        }
        for (int o = 16; o >= 1; o >>= 1) {
            const unsigned long long w = __shfl_xor_sync(0xffffffffu, best, o);
            best = w < best ? w : best;
        }
        if ((threadIdx.x & 31) == 0 && best != ~0ull) atomicMin(key_out + e, best);
    }
}

static double key_to_double(unsigned long long k) {
    if (k == 0ull) return NAN;
    const unsigned long long u = (k >> 63) ? (k & 0x7fffffffffffffffull) : ~k;
    double v;
    memcpy(&v, &u, sizeof v);
    return v;
}

// Pinned, device-mapped host slots for the check's bounds: the bound kernel
// stores its s values straight into host memory, and the host reads them
// after synchronising the stream, with no copy-engine transfer.  A small
// device-to-host copy would queue behind any large copy in flight on another
// stream (a solution read back while the next ensemble assembles) and leave
// the GPU idle for its length.  One block of kSlots slots per device and CUDA
// context, allocated on first use and never freed: a context that is
// destroyed (cudaDeviceReset) releases it, and the next context gets a new
// block.  A slot is held for one check; with none free, or without the
// driver's context id, the check reads its bounds by a copy instead.
constexpr int kSlotDevices = 64, kSlots = 64, kSlotDoubles = 32;
struct SlotBlock {
    double *host;
    double *dev;
    unsigned long long ctx;
    uint64_t used;
};
static std::mutex g_slot_mu;
static SlotBlock g_slot[kSlotDevices];

typedef int (*CtxGetCurrentFn)(void **ctx);
typedef int (*CtxGetIdFn)(void *ctx, unsigned long long *id);
static unsigned long long context_id() {   // 0 when the driver entry points are unavailable
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
    cudaGetLastError();
    if (!get_current || !get_id) return 0ull;
    void *ctx = nullptr;
    unsigned long long id = 0ull;
    if (get_current(&ctx) != 0 || !ctx || get_id(ctx, &id) != 0) return 0ull;
    return id;
}

struct Slot {
    int dev = -1, idx = -1;
    unsigned long long ctx = 0ull;
    double *host = nullptr, *devp = nullptr;
};

static Slot acquire_slot() {
    Slot sl;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kSlotDevices) { cudaGetLastError(); return sl; }
    cudaFree(nullptr);   // the device's primary context current before its id is read
    cudaGetLastError();
    const unsigned long long ctx = context_id();
    if (ctx == 0ull) return sl;
    std::lock_guard<std::mutex> lock(g_slot_mu);
    SlotBlock &b = g_slot[dev];
    if (!b.host || b.ctx != ctx) {   // first use, or the block's context was destroyed
        void *h = nullptr, *d = nullptr;
        if (cudaHostAlloc(&h, sizeof(double) * kSlots * kSlotDoubles, cudaHostAllocMapped) != cudaSuccess ||
            cudaHostGetDevicePointer(&d, h, 0) != cudaSuccess) {
            if (h) cudaFreeHost(h);
            cudaGetLastError();
            return sl;
        }
        b.host = static_cast<double *>(h);
        b.dev = static_cast<double *>(d);
        b.ctx = ctx;
        b.used = 0;
    }
    for (int i = 0; i < kSlots; ++i)
        if (!(b.used & (1ull << i))) {
            b.used |= 1ull << i;
            sl.dev = dev;
            sl.idx = i;
            sl.ctx = ctx;
            sl.host = b.host + (size_t)i * kSlotDoubles;
            sl.devp = b.dev + (size_t)i * kSlotDoubles;
            return sl;
        }
    return sl;
}

static void release_slot(const Slot &sl) {
    if (sl.idx < 0) return;
    std::lock_guard<std::mutex> lock(g_slot_mu);
    SlotBlock &b = g_slot[sl.dev];
    if (b.ctx == sl.ctx) b.used &= ~(1ull << sl.idx);
}

// Host: the positivity check of ens_assemble (synchronises the stream).
// Returns ENS_OK with *bad_member = -1 when every member's coefficient is
// positive at every Gauss point, else the first failing member and its
// minimum.  scratch: device memory of at least 16*s bytes (the call's b).
static int coeff_check(const ens_graph *g, int M, const double *kl_table, int s, const double *xi,
                       double sigma, double kappa0, void *scratch, int *bad_member, double *bad_min,
                       cudaStream_t st) {
    *bad_member = -1;
    *bad_min = 0.0;
    const double cn = cbrt((double)g->num_rows);
    const int N = (int)llround(cn) - 1;
    if (N < 1 || (int64_t)(N + 1) * (N + 1) * (N + 1) != (int64_t)g->num_rows)
        return fail(ENS_ERR_ARG, "kl_table given but num_rows=%d is not (N+1)^3", g->num_rows);
    if (M == 0) {
        if (!(kappa0 > 0.0)) { *bad_member = 0; *bad_min = kappa0; }
        return ENS_OK;
    }
    double hb[32];
    const Slot sl = acquire_slot();
    double *bound = sl.devp ? sl.devp : static_cast<double *>(scratch);
    coeff_bound_kernel<<<1, 256, 0, st>>>(N, M, kl_table, s, xi, sigma, kappa0, bound);
    cudaError_t ce = cudaGetLastError();
    if (ce == cudaSuccess && !sl.devp) ce = cudaMemcpyAsync(hb, bound, sizeof(double) * s, cudaMemcpyDeviceToHost, st);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(st);
    if (ce == cudaSuccess && sl.devp) memcpy(hb, sl.host, sizeof(double) * s);
    release_slot(sl);
    if (ce != cudaSuccess) return cuda_fail(ce, "coefficient bound");
    int need[32], any = 0;
    for (int e = 0; e < s; ++e) { need[e] = !(hb[e] > 0.0); any |= need[e]; }
    if (!any) return ENS_OK;
    // exact minimum for the members the bound does not clear
    unsigned long long *keys = static_cast<unsigned long long *>(scratch);
    int *dneed = reinterpret_cast<int *>(keys + s);
    ENS_CUDA_TRY(cudaMemsetAsync(keys, 0xff, sizeof(unsigned long long) * s, st));
    ENS_CUDA_TRY(cudaMemcpyAsync(dneed, need, sizeof(int) * s, cudaMemcpyHostToDevice, st));
    const int64_t npts = (int64_t)8 * N * N * N;
    const unsigned grid = (unsigned)std::min<int64_t>((npts + 255) / 256, 152 * 8);
    coeff_min_kernel<<<grid, 256, 0, st>>>(N, M, kl_table, s, xi, sigma, kappa0, dneed, keys);
    ENS_LAUNCH_CHECK("coeff_min_kernel");
    unsigned long long hk[32];
    ENS_CUDA_TRY(cudaMemcpyAsync(hk, keys, sizeof(unsigned long long) * s, cudaMemcpyDeviceToHost, st));
    ENS_CUDA_TRY(cudaStreamSynchronize(st));
    for (int e = 0; e < s; ++e) {
        if (!need[e]) continue;
        const double amin = key_to_double(hk[e]);
        if (!(amin > 0.0)) { *bad_member = e; *bad_min = amin; break; }
    }
    return ENS_OK;
}

template <int S>
static int assemble_s(const ens_graph *g, const uint8_t *bmask, int M, const double *modes,
                      const double *load, const double *xi, double sigma, double kappa0,
                      double *values, double *b, bool df, float2 *vdf, cudaStream_t st) {
    constexpr int G = (S == 1) ? 1 : S / 2;
    const int bs = 256;
    const int64_t nthr = g->num_entries * G;
    if (nthr > 0) {
        if (df)
            assemble_values_df_kernel<S><<<(unsigned)std::min<int64_t>((nthr + bs - 1) / bs, asm_df_grid<S>()), bs, 0, st>>>(
                g->num_entries, M, modes, xi, sigma, kappa0, values, vdf);
        else
            assemble_values_kernel<S><<<(unsigned)((nthr + bs - 1) / bs), bs, 0, st>>>(
                g->num_entries, M, modes, xi, sigma, kappa0, values);
        ENS_LAUNCH_CHECK("assemble_values_kernel");
    }
    const int64_t nr = (int64_t)g->num_rows * S;
    if (nr > 0) {
        assemble_rows_kernel<S><<<(unsigned)((nr + bs - 1) / bs), bs, 0, st>>>(
            g->num_rows, g->row_map, g->col_entry, bmask, load, values, b, vdf);
        ENS_LAUNCH_CHECK("assemble_rows_kernel");
    }
    return ENS_OK;
}

static int assemble_entry(const ens_graph *graph, const uint8_t *bmask, int s, int M, const double *kl_table,
                          const double *modes, const double *load, const double *xi, double sigma,
                          double kappa0, double *values, double *b, bool df, float2 *vdf, void *stream) {
    int rc = check_graph(graph);
    if (rc) return rc;
    if (!supported_s(s)) return fail(ENS_ERR_UNSUPPORTED, "ensemble size s=%d not in {1,4,8,16,32}", s);
    if (M < 0 || M > 64) return fail(ENS_ERR_UNSUPPORTED, "M=%d outside [0, 64]", M);
    if (!bmask || !modes || !load || !values || !b || (M > 0 && !xi))
        return fail(ENS_ERR_ARG, "NULL pointer argument");
    if (s > 1 && (!aligned16(values) || !aligned16(b) || (vdf && !aligned16(vdf))))
        return fail(ENS_ERR_ALIGN, "values/b/values_df must be 16-byte aligned");
    cudaStream_t st = as_stream(stream);
    int bad = -1;
    double bad_min = 0.0;
    if (kl_table && graph->num_rows > 0) {   // b (n*s doubles, n >= 8) is the check's scratch
        if (!aligned16(b)) return fail(ENS_ERR_ALIGN, "b must be 16-byte aligned when kl_table is given");
        if ((rc = coeff_check(graph, M, kl_table, s, xi, sigma, kappa0, b, &bad, &bad_min, st))) return rc;
    }
    switch (s) {
        case 1: rc = assemble_s<1>(graph, bmask, M, modes, load, xi, sigma, kappa0, values, b, df, vdf, st); break;
        case 4: rc = assemble_s<4>(graph, bmask, M, modes, load, xi, sigma, kappa0, values, b, df, vdf, st); break;
        case 8: rc = assemble_s<8>(graph, bmask, M, modes, load, xi, sigma, kappa0, values, b, df, vdf, st); break;
        case 16: rc = assemble_s<16>(graph, bmask, M, modes, load, xi, sigma, kappa0, values, b, df, vdf, st); break;
        default: rc = assemble_s<32>(graph, bmask, M, modes, load, xi, sigma, kappa0, values, b, df, vdf, st); break;
    }
    if (rc) return rc;
    if (bad >= 0)
        return fail(ENS_ERR_NONPOS_COEFF, "member %d: coefficient a(x_q) = %.17g <= 0 at a Gauss point "
                    "(values and b written; the matrix is not SPD)", bad, bad_min);
    return ENS_OK;
}

}  // namespace ens

using namespace ens;

extern "C" int ens_assemble(const ens_graph *graph, const uint8_t *bmask, int s, int M, const double *kl_table,
                            const double *modes, const double *load, const double *xi,
                            double sigma, double kappa0, double *values, double *b,
                            void *stream) {
    return assemble_entry(graph, bmask, s, M, kl_table, modes, load, xi, sigma, kappa0, values, b, false, nullptr,
                          stream);
}

extern "C" int ens_assemble_df(const ens_graph *graph, const uint8_t *bmask, int s, int M, const double *kl_table,
                               const double *modes, const double *load, const double *xi,
                               double sigma, double kappa0, double *values, void *values_df, double *b,
                               void *stream) {
    return assemble_entry(graph, bmask, s, M, kl_table, modes, load, xi, sigma, kappa0, values, b, true,
                          static_cast<float2 *>(values_df), stream);
}
