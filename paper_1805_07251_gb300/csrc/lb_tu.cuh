// lb_tu.cuh -- body of one lattice/precision translation unit.  Before including,
// define LBVDW_LAT (1 = D1Q3, 2 = D2Q9), LBVDW_S / LBVDW_R (storage and compute
// types), LBVDW_MU (chemical-potential arithmetic, MU_*), LBVDW_NAME (prefix of the
// step launcher) and, in one unit per storage type, LBVDW_FIELDS (prefix of the
// init / moments / diagnostics launchers).
#include "lb_launch.cuh"

namespace lbvdw {

namespace {

constexpr int LATV = LBVDW_LAT;
using SV = LBVDW_S;
using RV = LBVDW_R;
constexpr int MUV = LBVDW_MU;

template <int N, int TX, int TY, int FORCE>
cudaError_t step_one(const StepLaunch &a) {
    dim3 block(TX, TY);
    dim3 grid((a.P.nx + TX - 1) / TX, LATV == 1 ? 1 : (a.P.ny + TY - 1) / TY);
    lb_step_kernel<LATV, N, TX, TY, SV, RV, FORCE, MUV><<<grid, block, 0, a.stream>>>(
        static_cast<const SV *>(a.fin), static_cast<SV *>(a.fout), a.P);
    return cudaGetLastError();
}

template <int TX, int TY, int FORCE>
cudaError_t step_n(const StepLaunch &a) {
    switch (a.ncomp) {
        case 1: return step_one<1, TX, TY, FORCE>(a);
        case 2: return step_one<2, TX, TY, FORCE>(a);
        case 3: return step_one<3, TX, TY, FORCE>(a);
        case 4: return step_one<4, TX, TY, FORCE>(a);
    }
    return cudaErrorInvalidValue;
}

template <int TX, int TY>
cudaError_t step_f(const StepLaunch &a) {
    return a.force == 1 ? step_n<TX, TY, 1>(a) : step_n<TX, TY, 0>(a);
}

unsigned field_grid(const DevParams &P) {
    size_t n = (size_t)P.nx * P.ny;
    size_t g = (n + 255) / 256;
    if (g > 152 * 16) g = 152 * 16;
    return (unsigned)(g ? g : 1);
}

template <int N>
cudaError_t init_one(const FieldLaunch &a) {
    lb_init_kernel<LATV, N, SV><<<field_grid(a.P), 256, 0, a.stream>>>(static_cast<SV *>(a.f), a.rho_in,
                                                                         a.mom_in, a.P);
    return cudaGetLastError();
}

template <int N>
cudaError_t moments_one(const FieldLaunch &a) {
    lb_moments_kernel<LATV, N, SV><<<field_grid(a.P), 256, 0, a.stream>>>(static_cast<const SV *>(a.f),
                                                                            a.rho_out, a.mom_out, a.P);
    return cudaGetLastError();
}

template <int N>
cudaError_t diag_one(const FieldLaunch &a) {
    lb_diag_partial_kernel<LATV, N><<<a.nparts, DIAG_THREADS, 0, a.stream>>>(a.rho_out, a.mom_out,
                                                                               a.partial, a.P);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    lb_diag_final_kernel<N + 3><<<1, DIAG_THREADS, 0, a.stream>>>(a.partial, a.nparts, a.diag_out);
    return cudaGetLastError();
}

}  // namespace

#define LBVDW_CAT2(a, b) a##b
#define LBVDW_CAT(a, b) LBVDW_CAT2(a, b)

cudaError_t LBVDW_CAT(LBVDW_NAME, _step)(const StepLaunch &a) {
#if LBVDW_LAT == 1
    if (a.tile_x == 128) return step_f<128, 1>(a);
    if (a.tile_x == 256) return step_f<256, 1>(a);
    return cudaErrorInvalidConfiguration;
#else
    if (a.tile_x == 32 && a.tile_y == 8) return step_f<32, 8>(a);
    if (a.tile_x == 64 && a.tile_y == 4) return step_f<64, 4>(a);
    if (a.tile_x == 32 && a.tile_y == 16) return step_f<32, 16>(a);
    if (a.tile_x == 64 && a.tile_y == 8) return step_f<64, 8>(a);
    return cudaErrorInvalidConfiguration;
#endif
}

#ifdef LBVDW_FIELDS

cudaError_t LBVDW_CAT(LBVDW_FIELDS, _init)(const FieldLaunch &a) {
    switch (a.ncomp) {
        case 1: return init_one<1>(a);
        case 2: return init_one<2>(a);
        case 3: return init_one<3>(a);
        case 4: return init_one<4>(a);
    }
    return cudaErrorInvalidValue;
}

cudaError_t LBVDW_CAT(LBVDW_FIELDS, _moments)(const FieldLaunch &a) {
    switch (a.ncomp) {
        case 1: return moments_one<1>(a);
        case 2: return moments_one<2>(a);
        case 3: return moments_one<3>(a);
        case 4: return moments_one<4>(a);
    }
    return cudaErrorInvalidValue;
}

cudaError_t LBVDW_CAT(LBVDW_FIELDS, _diag)(const FieldLaunch &a) {
    switch (a.ncomp) {
        case 1: return diag_one<1>(a);
        case 2: return diag_one<2>(a);
        case 3: return diag_one<3>(a);
        case 4: return diag_one<4>(a);
    }
    return cudaErrorInvalidValue;
}
#endif  // LBVDW_FIELDS

}  // namespace lbvdw
