// D2Q9 lattice, FP32 deviation storage; FP32 mu (the reference point for the FP64-class mu).
#define LBVDW_LAT 2
#define LBVDW_S float
#define LBVDW_R float
#define LBVDW_MU MU_F32
#define LBVDW_NAME d2q9_f32mu
#define LBVDW_STRIPS 1
#define LBVDW_WS 1
#define LBVDW_CHAIN 1
#include "lb_tu.cuh"
