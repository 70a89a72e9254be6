// D2Q9 lattice, FP64 populations and arithmetic.
#define LBVDW_LAT 2
#define LBVDW_S double
#define LBVDW_R double
#define LBVDW_MU MU_F64
#define LBVDW_NAME d2q9_f64
#define LBVDW_FIELDS d2q9_f64
#include "lb_tu.cuh"
