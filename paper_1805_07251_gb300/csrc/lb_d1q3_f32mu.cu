// D1Q3 lattice, FP32 deviation storage; FP32 mu (the reference point for the FP64-class mu).
#define LBVDW_LAT 1
#define LBVDW_S float
#define LBVDW_R float
#define LBVDW_MU MU_F32
#define LBVDW_NAME d1q3_f32mu
#include "lb_tu.cuh"
