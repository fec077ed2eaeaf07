// ens_cg_k1_s4.cu -- K1 (q = A p, p.q) instantiations for ensemble size 4.
#include "ens_cg_k1.cuh"

ENS_K1_INSTANTIATE(4)
