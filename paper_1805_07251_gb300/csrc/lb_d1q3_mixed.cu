// D1Q3 lattice, FP32 deviation storage with FP64 chemical potential.
#define LBVDW_LAT 1
#define LBVDW_S float
#define LBVDW_R float
#define LBVDW_NAME d1q3_mixed
#include "lb_tu.cuh"
