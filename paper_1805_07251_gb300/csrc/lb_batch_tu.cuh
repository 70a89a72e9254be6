// lb_batch_tu.cuh -- launchers of the batched kernels for one storage/compute type and
// chemical-potential arithmetic.  Define LBVDW_S, LBVDW_R, LBVDW_MU and LBVDW_NAME first.
#include "lb_batch.cuh"
#include "lb_batch_launch.cuh"

namespace lbvdw {
namespace {

using SB = LBVDW_S;
using RB = LBVDW_R;
constexpr int MUB = LBVDW_MU;

template <int N, int TX, int TY, int FORCE>
cudaError_t tiles_one(const BatchLaunch &a) {
    if (a.ntiles == 0) return cudaSuccess;
    lb_batch_tile_kernel<N, TX, TY, SB, RB, FORCE, MUB><<<a.ntiles, dim3(TX, TY), 0, a.stream>>>(
        static_cast<const SB *>(a.pool_in), static_cast<SB *>(a.pool_out), a.runs, a.tiles, a.tbl);
    return cudaGetLastError();
}

template <int TX, int TY, int FORCE>
cudaError_t tiles_n(const BatchLaunch &a) {
    switch (a.ncomp) {
        case 1: return tiles_one<1, TX, TY, FORCE>(a);
        case 2: return tiles_one<2, TX, TY, FORCE>(a);
        case 3: return tiles_one<3, TX, TY, FORCE>(a);
        case 4: return tiles_one<4, TX, TY, FORCE>(a);
    }
    return cudaErrorInvalidValue;
}

template <int TX, int TY>
cudaError_t tiles_f(const BatchLaunch &a) {
    return a.force == 1 ? tiles_n<TX, TY, 1>(a) : tiles_n<TX, TY, 0>(a);
}

template <int N, int FORCE>
cudaError_t resident_one(const BatchLaunch &a) {
    if (a.nd1 == 0 || a.nsteps == 0) return cudaSuccess;
    auto k = lb_d1q3_resident_kernel<N, SB, RB, FORCE, MUB>;
    if (a.nsteps < 0)  // preparation call: raise the dynamic shared-memory limit only
        return cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)a.smem);
    k<<<a.nd1, RESIDENT_THREADS, a.smem, a.stream>>>(static_cast<const SB *>(a.pool_in),
                                                      static_cast<SB *>(a.pool_out), a.runs, a.offsets, a.d1_ids,
                                                      a.nsteps);
    return cudaGetLastError();
}

template <int FORCE>
cudaError_t resident_n(const BatchLaunch &a) {
    switch (a.ncomp) {
        case 1: return resident_one<1, FORCE>(a);
        case 2: return resident_one<2, FORCE>(a);
        case 3: return resident_one<3, FORCE>(a);
        case 4: return resident_one<4, FORCE>(a);
    }
    return cudaErrorInvalidValue;
}

}  // namespace

#define LBVDW_BCAT2(a, b) a##b
#define LBVDW_BCAT(a, b) LBVDW_BCAT2(a, b)

cudaError_t LBVDW_BCAT(LBVDW_NAME, _batch_tiles)(const BatchLaunch &a) {
    if (a.tile_x == 32 && a.tile_y == 8) return tiles_f<32, 8>(a);
    if (a.tile_x == 64 && a.tile_y == 4) return tiles_f<64, 4>(a);
    if (a.tile_x == 32 && a.tile_y == 16) return tiles_f<32, 16>(a);
    if (a.tile_x == 64 && a.tile_y == 8) return tiles_f<64, 8>(a);
    return cudaErrorInvalidConfiguration;
}

cudaError_t LBVDW_BCAT(LBVDW_NAME, _batch_resident)(const BatchLaunch &a) {
    return a.force == 1 ? resident_n<1>(a) : resident_n<0>(a);
}

size_t LBVDW_BCAT(LBVDW_NAME, _resident_smem)(int ncomp, int L) {
    switch (ncomp) {
        case 1: return resident_smem_bytes<1, SB, RB, MUB>(L);
        case 2: return resident_smem_bytes<2, SB, RB, MUB>(L);
        case 3: return resident_smem_bytes<3, SB, RB, MUB>(L);
        case 4: return resident_smem_bytes<4, SB, RB, MUB>(L);
    }
    return 0;
}

}  // namespace lbvdw
