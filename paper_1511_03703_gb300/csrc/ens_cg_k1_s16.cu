// ens_cg_k1_s16.cu -- K1 (q = A p, p.q) instantiations for ensemble size 16.
#include "ens_cg_k1.cuh"

ENS_K1_INSTANTIATE(16)
