// lb_batch_launch.cuh -- host-side launchers of the batched kernels (lb_batch_tu.cuh).
#pragma once
#include "lb_batch.cuh"

namespace lbvdw {

struct BatchLaunch {
    const void *pool_in;
    void *pool_out;
    const DevParams *runs;     // device array, one parameter block per run
    const size_t *offsets;     // device array, element offset of each run in the pools
    const BatchTile *tiles;    // device array of D2Q9 tiles
    const LogTables *tbl;      // device log tables (shared by every run)
    int ntiles;
    const int *d1_ids;         // device array of D1Q3 run indices
    int nd1;
    int ncomp, force, tile_x, tile_y;
    int nsteps;                // resident kernel: timesteps of this launch (< 0: only raise the
                               // kernel's shared-memory limit, before any graph capture)
    size_t smem;               // resident kernel: dynamic shared memory per CTA
    cudaStream_t stream;
};

#define LBVDW_DECLARE_BATCH(NAME)                                  \
    cudaError_t NAME##_batch_tiles(const BatchLaunch &a);          \
    cudaError_t NAME##_batch_resident(const BatchLaunch &a);       \
    size_t NAME##_resident_smem(int ncomp, int L);
LBVDW_DECLARE_BATCH(f64)
LBVDW_DECLARE_BATCH(tbl)
LBVDW_DECLARE_BATCH(df)
#undef LBVDW_DECLARE_BATCH

}  // namespace lbvdw
