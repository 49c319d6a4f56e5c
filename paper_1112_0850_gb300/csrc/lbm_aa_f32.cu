// Instantiation of the AA-pattern kernels for population storage format LBM_F32.
#include "lbm_aa.cuh"

template struct lbm::AaOps<LBM_F32>;
