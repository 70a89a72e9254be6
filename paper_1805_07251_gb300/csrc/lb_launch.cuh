// lb_launch.cuh -- host-side launch wrappers shared by the translation units.
// Each lattice/precision pair lives in its own .cu file so the library builds in
// parallel; lb_api.cu dispatches to them.
#pragma once
#include "lb_kernels.cuh"

namespace lbvdw {

struct StepLaunch {
    const void *fin;
    void *fout;
    DevParams P;
    int ncomp, force, tile_x, tile_y;
    cudaStream_t stream;
};

struct FieldLaunch {
    void *f;               // populations (storage type of the precision)
    const double *rho_in;  // init input
    const double *mom_in;  // init input (may be null)
    double *rho_out;       // moments output
    double *mom_out;       // moments output
    double *partial;       // diagnostics partials [nparts][ncomp + 3]
    int nparts;
    double *diag_out;      // [ncomp + 3]
    DevParams P;
    int ncomp;
    cudaStream_t stream;
};

// supported step tiles (tile_x, tile_y) per lattice; returns false when not compiled
bool step_tile_supported(int lattice, int tile_x, int tile_y);

#define LBVDW_DECLARE(NAME)                                \
    cudaError_t NAME##_step(const StepLaunch &a);          \
    cudaError_t NAME##_init(const FieldLaunch &a);         \
    cudaError_t NAME##_moments(const FieldLaunch &a);      \
    cudaError_t NAME##_diag(const FieldLaunch &a);
LBVDW_DECLARE(d1q3_f64)
LBVDW_DECLARE(d1q3_mixed)
LBVDW_DECLARE(d2q9_f64)
LBVDW_DECLARE(d2q9_mixed)
#undef LBVDW_DECLARE

}  // namespace lbvdw
