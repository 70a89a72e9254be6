// D1Q3 lattice, FP32 deviation storage; double-float arithmetic in mu.
#define LBVDW_LAT 1
#define LBVDW_S float
#define LBVDW_R float
#define LBVDW_MU MU_DF
#define LBVDW_NAME d1q3_df
#include "lb_tu.cuh"
