// lb_tu.cuh -- body of one lattice/precision translation unit.  Before including,
// define LBVDW_LAT (1 = D1Q3, 2 = D2Q9), LBVDW_S / LBVDW_R (storage and compute
// types), LBVDW_MU (chemical-potential arithmetic, MU_*), LBVDW_NAME (prefix of the
// step launcher) and, in one unit per storage type, LBVDW_FIELDS (prefix of the
// init / moments / diagnostics launchers).
#include "lb_launch.cuh"
#ifdef LBVDW_STRIPS
#include "lb_strip.cuh"
#endif
#ifdef LBVDW_WS
#include "lb_ws.cuh"
#endif

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

// a.force: bit 0 the "nid" force, bit 1 the moment-space collision (D2Q9, 32 x 8 tiles)
template <int TX, int TY>
cudaError_t step_f(const StepLaunch &a) {
    switch (a.force) {
        case 0: return step_n<TX, TY, 0>(a);
        case 1: return step_n<TX, TY, 1>(a);
        case 2:
        case 3:
            if constexpr (LATV == 2 && TX == 32 && TY == 8)
                return a.force == 2 ? step_n<TX, TY, 2>(a) : step_n<TX, TY, 3>(a);
            break;
    }
    return cudaErrorInvalidConfiguration;
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

#ifdef LBVDW_CHAIN

cudaError_t LBVDW_CAT(LBVDW_NAME, _chain)(const StepLaunch &a, const ChainArgs &ca, bool pdl) {
    if (a.ncomp != 2 || a.tile_x != 32 || a.tile_y != 8) return cudaErrorInvalidConfiguration;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((a.P.nx + 31) / 32, (a.P.ny + 7) / 8);
    cfg.blockDim = dim3(32, 8);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = a.stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = pdl ? 1 : 0;
    const float *fin = static_cast<const float *>(a.fin);
    float *fout = static_cast<float *>(a.fout);
    if (ca.evict_first) {
        switch (a.force) {
            case 0: return cudaLaunchKernelEx(&cfg, lb_chain_kernel<0, MUV, true>, fin, fout, a.P, ca);
            case 1: return cudaLaunchKernelEx(&cfg, lb_chain_kernel<1, MUV, true>, fin, fout, a.P, ca);
            case 2: return cudaLaunchKernelEx(&cfg, lb_chain_kernel<2, MUV, true>, fin, fout, a.P, ca);
            case 3: return cudaLaunchKernelEx(&cfg, lb_chain_kernel<3, MUV, true>, fin, fout, a.P, ca);
        }
        return cudaErrorInvalidConfiguration;
    }
    switch (a.force) {
        case 0: return cudaLaunchKernelEx(&cfg, lb_chain_kernel<0, MUV>, fin, fout, a.P, ca);
        case 1: return cudaLaunchKernelEx(&cfg, lb_chain_kernel<1, MUV>, fin, fout, a.P, ca);
        case 2: return cudaLaunchKernelEx(&cfg, lb_chain_kernel<2, MUV>, fin, fout, a.P, ca);
        case 3: return cudaLaunchKernelEx(&cfg, lb_chain_kernel<3, MUV>, fin, fout, a.P, ca);
    }
    return cudaErrorInvalidConfiguration;
}

int LBVDW_CAT(LBVDW_NAME, _chain_ctas_per_sm)() {
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, lb_chain_kernel<0, MUV>, 256, 0) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return nb;
}

#endif

#ifdef LBVDW_STRIPS

namespace {

// Opt the kernel in to its dynamic shared memory on the current device and return the
// CTAs resident per SM times the SM count; `cache` holds one entry per device and must
// belong to this kernel alone.
template <class K>
int strip_slots(K kern, int threads, size_t smem, int (&cache)[64]) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return -1;
    if (cache[dev] > 0) return cache[dev];
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) return -1;
    int sms = 0, occ = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return -1;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, threads, smem) != cudaSuccess) return -1;
    cache[dev] = sms * (occ > 0 ? occ : 1);
    return cache[dev];
}

template <int N, int TY, int FORCE>
cudaError_t strip_one(const StepLaunch &a) {
    using Lay = StripLayout<N, STRIP_TX, TY, MUV>;
    auto kern = lb_strip_kernel<N, STRIP_TX, TY, RV, FORCE, MUV>;
    static int cache[64];  // one per instantiation, i.e. per kernel
    const int slots = strip_slots(kern, Lay::NT, Lay::bytes, cache);
    if (slots < 0) return cudaErrorInvalidConfiguration;
    const int strips = a.P.nx / STRIP_TX, nblk = a.P.ny / TY;
    int segs = a.segs > 0 ? a.segs : slots / strips;
    if (segs < 1) segs = 1;
    if (segs > nblk) segs = nblk;
    kern<<<strips * segs, Lay::NT, Lay::bytes, a.stream>>>(static_cast<const float *>(a.fin),
                                                            static_cast<float *>(a.fout), a.P, segs);
    return cudaGetLastError();
}

template <int FORCE>
cudaError_t strip_n(const StepLaunch &a) {
    switch (a.ncomp) {
        case 1: return strip_one<1, 8, FORCE>(a);
        case 2: return strip_one<2, 8, FORCE>(a);
        case 3: return strip_one<3, 4, FORCE>(a);
        case 4: return strip_one<4, 4, FORCE>(a);
    }
    return cudaErrorInvalidValue;
}

}  // namespace

cudaError_t LBVDW_CAT(LBVDW_NAME, _strip)(const StepLaunch &a) {
    if (!strip_shape_ok(a.P.nx, a.P.ny, a.ncomp) || a.tile_x != STRIP_TX || a.tile_y != strip_ty(a.ncomp))
        return cudaErrorInvalidConfiguration;
    if (a.force & ~1) return cudaErrorInvalidConfiguration;
    return a.force == 1 ? strip_n<1>(a) : strip_n<0>(a);
}

#ifdef LBVDW_WS
namespace {

// Persistent warp-specialised tiles (lb_ws.cuh): as many CTAs as fit on the GPU at once,
// each walking every gridDim.x-th tile.
template <int FORCE>
cudaError_t ws_one(const StepLaunch &a) {
    using Lay = WsLayout<MUV>;
    auto kern = lb_step_ws_kernel<FORCE, MUV>;
    static int cache[64];  // one per instantiation, i.e. per kernel
    const int slots = strip_slots(kern, WS_THREADS, Lay::bytes, cache);
    if (slots < 0) return cudaErrorInvalidConfiguration;
    const int tiles_x = (a.P.nx + WS_TX - 1) / WS_TX, tiles_y = (a.P.ny + WS_TY - 1) / WS_TY;
    const int ntiles = tiles_x * tiles_y;
    const int grid = slots < ntiles ? slots : ntiles;
    kern<<<grid, WS_THREADS, Lay::bytes, a.stream>>>(static_cast<const float *>(a.fin), static_cast<float *>(a.fout),
                                                      a.P, tiles_x, ntiles);
    return cudaGetLastError();
}

}  // namespace

cudaError_t LBVDW_CAT(LBVDW_NAME, _ws)(const StepLaunch &a) {
    if (a.ncomp != 2 || a.tile_x != WS_TX || a.tile_y != WS_TY) return cudaErrorInvalidConfiguration;
    switch (a.force) {
        case 0: return ws_one<0>(a);
        case 1: return ws_one<1>(a);
        case 2: return ws_one<2>(a);
        case 3: return ws_one<3>(a);
    }
    return cudaErrorInvalidConfiguration;
}
#endif  // LBVDW_WS

#endif  // LBVDW_STRIPS

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
