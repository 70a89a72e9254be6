// Batched runs: FP32 storage, double-float chemical potential.
#define LBVDW_S float
#define LBVDW_R float
#define LBVDW_MU MU_DF
#define LBVDW_NAME df
#include "lb_batch_tu.cuh"
