// D2Q9 lattice, FP32 deviation storage; FP64 eta, 1/eta and table-driven logs in mu.
#define LBVDW_LAT 2
#define LBVDW_S float
#define LBVDW_R float
#define LBVDW_MU MU_TBL
#define LBVDW_NAME d2q9_tbl
#define LBVDW_FIELDS d2q9_f32
#define LBVDW_STRIPS 1
#include "lb_tu.cuh"
