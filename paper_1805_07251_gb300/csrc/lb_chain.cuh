// lb_chain.cuh -- consecutive timesteps of one lb_step call as a chain of overlapping
// grids (programmatic dependent launch) with per-tile completion flags.
//
// Each step is the same fused tile step as lb_step_kernel (two FP32 components in a lane
// pair, 32 x 8 tiles), so the results are bitwise those of one launch per step.  What
// changes is when a tile may start:
//
//   * every CTA lets the next step's grid launch as soon as it runs
//     (griddepcontrol.launch_dependents), so the next grid is scheduled once all CTAs of
//     this one have started, and its CTAs take the SM slots that this grid's last wave
//     frees;
//   * a tile of step s reads the populations that step s - 1 pushed into its 2-node ring
//     and overwrites (by push streaming into a 1-node ring) populations that tiles of step
//     s - 1 read.  Both touch only the 3 x 3 tiles around it when every tile is at least 3
//     nodes wide and high, so it may start once those nine tiles of step s - 1 are done;
//   * the grid's tile rows are rotated by one per step (row r of the lattice is taken by
//     CTA row r - s mod rows), so the first rows that step s schedules need only rows that
//     step s - 1 scheduled first.  The first `release_rows` CTA rows of a step set a flag
//     per tile once its stores are out (release at GPU scope); the first CTA rows of the
//     next step whose three source rows all lie in that set wait on those nine flags
//     (acquire), every other CTA waits for the whole previous grid (griddepcontrol.wait).
//
// The flags hold the step number (mod 2^32, compared with wraparound) of the last step the
// tile finished in a chain, so they never need resetting: a chain's first step is a
// plain stream-ordered launch that waits on nothing.  No wait can form a cycle: a grid
// launches only when every CTA of the previous one is resident or finished, and waits only
// on that grid.  A flag wait is bounded in time; when it runs out the kernel sets ERR_STALL
// and goes on, so the host reports the error instead of the GPU hanging.
#pragma once
#include "lb_kernels.cuh"

namespace lbvdw {

struct ChainArgs {
    unsigned *flag;           // [tiles_y][tiles_x] completion flags of the context
    unsigned step;            // chain step number of this launch (mod 2^32)
    int chained;              // 0: first step of a chain (stream-ordered, waits on nothing)
    int flag_rows;            // CTA rows of the previous step that set flags
    int release_rows;         // CTA rows of this step that set flags (0: no next step)
    int roff;                 // row rotation: CTA row b takes tile row (b + roff) mod rows
    unsigned long long wait_ns;  // bound of one flag wait
    int evict_first;          // population loads marked evict-first in the L2 (lb_chain_kernel<.., true>)
};

__device__ __forceinline__ unsigned ld_acquire_gpu(const unsigned *p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release_gpu(unsigned *p, unsigned v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Wait (acquire) until flag[idx] has reached `step` (mod 2^32), for at most wait_ns;
// false when the bound ran out (ERR_STALL set in *err) or another wait already gave up.
__device__ __forceinline__ bool wait_flag(const unsigned *flag, int idx, unsigned step, unsigned long long wait_ns,
                                          unsigned *err) {
    const unsigned *f = flag + idx;
    if ((int)(ld_acquire_gpu(f) - step) >= 0) return true;
    const unsigned long long t0 = global_ns();
    while ((int)(ld_acquire_gpu(f) - step) < 0) {
        if (global_ns() - t0 > wait_ns || (*(volatile unsigned *)err & ERR_STALL)) {
            atomicOr(err, ERR_STALL);
            return false;
        }
        __nanosleep(32);
    }
    return true;
}

// One chained step: D2Q9, N = 2 FP32 components in one lane pair, 32 x 8 tiles.  EF: the
// population loads carry an evict-first L2 policy (chosen by the host where one population
// buffer fits in the L2 with room to spare, so that the step's output stays resident for the
// next step); the results are the same bits either way.
template <int FORCE, int MU, bool EF = false>
__global__ void __launch_bounds__(256, 5)
    lb_chain_kernel(const float *__restrict__ fin, float *__restrict__ fout, DevParams P, ChainArgs ca) {
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    const int tid = threadIdx.x + 32 * threadIdx.y;
    const int tiles_x = gridDim.x, tiles_y = gridDim.y;
    const int r = (int)((blockIdx.y + (unsigned)ca.roff) % (unsigned)tiles_y);
    if (ca.chained) {
        if ((int)blockIdx.y + 2 < ca.flag_rows) {
            // the 3 x 3 tiles of the previous step around this one, one lane each
            if (tid < 9) {
                const int rr = (r + tid / 3 - 1 + tiles_y) % tiles_y;
                const int xx = ((int)blockIdx.x + tid % 3 - 1 + tiles_x) % tiles_x;
                wait_flag(ca.flag, rr * tiles_x + xx, ca.step, ca.wait_ns, P.err);
            }
            __syncthreads();
        } else {
            asm volatile("griddepcontrol.wait;" ::: "memory");
        }
    }
    // the loads bypass L1: the previous grid may still write this grid's input
    step_tile_pair<2, 1, 32, 8, FORCE, MU, 1, EF>(fin, fout, P, blockIdx.x * 32, r * 8);
    if ((int)blockIdx.y < ca.release_rows) {
        // every thread's stores of the tile come before the flag: the barrier orders them
        // before thread 0's release, whose fence is cumulative over what it orders
        __syncthreads();
        if (tid == 0) st_release_gpu(ca.flag + r * tiles_x + blockIdx.x, ca.step + 1u);
    }
}

}  // namespace lbvdw
