// D2Q9 lattice, FP32 deviation storage with FP64 chemical potential.
#define LBVDW_LAT 2
#define LBVDW_S float
#define LBVDW_R float
#define LBVDW_NAME d2q9_mixed
#include "lb_tu.cuh"
