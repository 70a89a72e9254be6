// Batched runs: FP32 storage, FP64 chemical potential.
#define LBVDW_S float
#define LBVDW_R float
#define LBVDW_MU MU_TBL
#define LBVDW_NAME tbl
#include "lb_batch_tu.cuh"
