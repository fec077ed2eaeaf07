// ens_cg_k1.cuh -- K1 launches for every rows-per-CTA mapping (included by
// the one-per-ensemble-size translation units ens_cg_k1_s*.cu, so that the
// K1 instantiations compile in parallel).
#pragma once
#include "ens_cg_kernels.cuh"

namespace ens {

template <int S, int MODE, int NSUB>
static void k1_launch_n(const CgArgs &a, cudaStream_t st) {
    const int64_t chunks = a.t1.count[1];
    cg_spmv_kernel<S, MODE, NSUB><<<(unsigned)((chunks + NSUB - 1) / NSUB), NSUB * RowMap<S>::THREADS, 0, st>>>(a);
}

// nsub = 0 selects the deferred tree: one chunk per CTA writing its partials,
// then the reduction kernel over the level-1 groups (ENS_CG_K1_DEFER)
template <int S, int MODE>
void k1_launch(const CgArgs &a, int nsub, cudaStream_t st) {
    constexpr int MAXN = k1_max_nsub<S>();
    if (nsub == 0) {
        const int64_t chunks = a.t1.count[1];
        cg_spmv_partial_kernel<S, MODE><<<(unsigned)chunks, RowMap<S>::THREADS, 0, st>>>(a);
        const unsigned groups = a.t1.levels > 1 ? (unsigned)a.t1.count[2] : 1u;
        cg_spmv_reduce_kernel<S><<<groups, 256, 0, st>>>(a);
        return;
    }
    if (nsub >= 8 && MAXN >= 8) k1_launch_n<S, MODE, (MAXN >= 8 ? 8 : 1)>(a, st);
    else if (nsub >= 4 && MAXN >= 4) k1_launch_n<S, MODE, (MAXN >= 4 ? 4 : 1)>(a, st);
    else if (nsub >= 2 && MAXN >= 2) k1_launch_n<S, MODE, (MAXN >= 2 ? 2 : 1)>(a, st);
    else k1_launch_n<S, MODE, 1>(a, st);
}

}  // namespace ens

#define ENS_K1_INSTANTIATE(S)                                                             \
    template void ens::k1_launch<S, 0>(const ens::CgArgs &, int, cudaStream_t);            \
    template void ens::k1_launch<S, 1>(const ens::CgArgs &, int, cudaStream_t);            \
    template void ens::k1_launch<S, 2>(const ens::CgArgs &, int, cudaStream_t);            \
    template void ens::k1_launch<S, 3>(const ens::CgArgs &, int, cudaStream_t);
