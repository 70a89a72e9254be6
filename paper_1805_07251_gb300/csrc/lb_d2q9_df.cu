// D2Q9 lattice, FP32 deviation storage; double-float arithmetic in mu.
#define LBVDW_LAT 2
#define LBVDW_S float
#define LBVDW_R float
#define LBVDW_MU MU_DF
#define LBVDW_NAME d2q9_df
#define LBVDW_STRIPS 1
#define LBVDW_WS 1
#define LBVDW_CHAIN 1
#include "lb_tu.cuh"
