// lb_launch.cuh -- host-side launch wrappers shared by the translation units.
// Each lattice/precision pair lives in its own .cu file so the library builds in
// parallel; lb_api.cu dispatches to them.
#pragma once
#include "lb_chain.cuh"
#include "lb_device_guard.cuh"
#include "lb_kernels.cuh"
#include "lbvdw.h"

namespace lbvdw {

struct StepLaunch {
    const void *fin;
    void *fout;
    DevParams P;
    int ncomp, force, tile_x, tile_y;
    int kernel = LB_KERNEL_TILES;  // lb_kernel_kind, resolved (never AUTO here)
    int segs = 0;                  // strips: row segments per strip, 0 = fill the GPU once
    cudaStream_t stream;
};

// Streaming-strip kernel (lb_strip.cuh): strip width and rows per block for N components,
// and whether a lattice can use it.
constexpr int STRIP_TX = 32;
inline int strip_ty(int ncomp) { return ncomp <= 2 ? 8 : 4; }
inline bool strip_shape_ok(int nx, int ny, int ncomp) {
    return nx >= STRIP_TX && nx % STRIP_TX == 0 && ny >= strip_ty(ncomp) && ny % strip_ty(ncomp) == 0;
}

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

// parameter block of a parameter set (lb_api.cu); log tables filled on the host
void make_dev_params(const lb_params &p, DevParams &d, unsigned *err, const LogTables *tbl);

// step launchers: one per lattice and chemical-potential arithmetic
cudaError_t d1q3_f64_step(const StepLaunch &a);
cudaError_t d1q3_tbl_step(const StepLaunch &a);
cudaError_t d1q3_df_step(const StepLaunch &a);
cudaError_t d2q9_f64_step(const StepLaunch &a);
cudaError_t d2q9_tbl_step(const StepLaunch &a);
cudaError_t d2q9_df_step(const StepLaunch &a);
cudaError_t d1q3_f32mu_step(const StepLaunch &a);
cudaError_t d2q9_f32mu_step(const StepLaunch &a);
cudaError_t d2q9_tbl_strip(const StepLaunch &a);
cudaError_t d2q9_df_strip(const StepLaunch &a);
cudaError_t d2q9_f32mu_strip(const StepLaunch &a);
cudaError_t d2q9_df_ws(const StepLaunch &a);
cudaError_t d2q9_f32mu_ws(const StepLaunch &a);
// chained steps (lb_chain.cuh): one step of a chain, launched with programmatic
// serialisation after the previous one when `pdl`; CTAs of the chain kernel resident per SM
cudaError_t d2q9_df_chain(const StepLaunch &a, const ChainArgs &ca, bool pdl);
cudaError_t d2q9_f32mu_chain(const StepLaunch &a, const ChainArgs &ca, bool pdl);
int d2q9_df_chain_ctas_per_sm();
int d2q9_f32mu_chain_ctas_per_sm();

// field launchers: one per lattice and storage type (double / float)
#define LBVDW_DECLARE_FIELDS(NAME)                         \
    cudaError_t NAME##_init(const FieldLaunch &a);         \
    cudaError_t NAME##_moments(const FieldLaunch &a);      \
    cudaError_t NAME##_diag(const FieldLaunch &a);
LBVDW_DECLARE_FIELDS(d1q3_f64)
LBVDW_DECLARE_FIELDS(d1q3_f32)
LBVDW_DECLARE_FIELDS(d2q9_f64)
LBVDW_DECLARE_FIELDS(d2q9_f32)
#undef LBVDW_DECLARE_FIELDS

}  // namespace lbvdw
