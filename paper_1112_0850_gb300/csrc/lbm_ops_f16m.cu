// Instantiation of the kernels for population storage format LBM_F16M.
#include "lbm_kernels.cuh"

template struct lbm::Ops<LBM_F16M>;
