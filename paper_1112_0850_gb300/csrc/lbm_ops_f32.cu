// Instantiation of the kernels for population storage format LBM_F32.
#include "lbm_kernels.cuh"

template struct lbm::Ops<LBM_F32>;
