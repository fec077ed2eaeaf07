// ens_cg_k1_s32.cu -- K1 (q = A p, p.q) instantiations for ensemble size 32.
#include "ens_cg_k1.cuh"

ENS_K1_INSTANTIATE(32)
