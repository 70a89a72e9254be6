// Batched runs: FP64 populations and arithmetic.
#define LBVDW_S double
#define LBVDW_R double
#define LBVDW_MU MU_F64
#define LBVDW_NAME f64
#include "lb_batch_tu.cuh"
