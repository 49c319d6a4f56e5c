// Instantiation of the kernels for population storage format LBM_BF16M.
#include "lbm_kernels.cuh"

template struct lbm::Ops<LBM_BF16M>;
