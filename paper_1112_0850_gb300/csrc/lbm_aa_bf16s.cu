// Instantiation of the AA-pattern kernels for population storage format LBM_BF16S.
#include "lbm_aa.cuh"

template struct lbm::AaOps<LBM_BF16S>;
