// lb_batch.cuh -- batched independent runs (a phase-diagram sweep) on one GPU.
//
// Runs differ in lattice, size, temperature kT, gamma_mu and mean composition; they
// share the mixture (a, b, kappa, lambda), tau, the number of components and the
// precision.  Two kernels advance them, both built from the single-run device code of
// lb_kernels.cuh (mu_node, collide_node, step_tile), so every run of a batch follows
// exactly the arithmetic of the same run advanced alone:
//
//  * lb_batch_tile_kernel: one CTA per tile of a flat work list covering every D2Q9
//    run; one launch per timestep (a CUDA graph replays them).  Each run has its own
//    parameter block and ping-pong pair of population buffers in two pooled arrays.
//  * lb_d1q3_resident_kernel: one CTA per D1Q3 run; the whole run (populations,
//    densities, chemical potentials) lives in shared memory for all the timesteps of
//    the launch, so those steps touch HBM only at the start and the end.
#pragma once
#include "lb_kernels.cuh"

namespace lbvdw {

// One tile of the flat work list: its run, origin, the run's lattice size, element offset
// in the pools and reference densities (what the tile needs before its parameter block
// arrives).
struct BatchTile {
    int run, x0, y0, nx, ny, pad;
    size_t off;
    float rho_ref[4];
};

// Copy a run's parameter block into shared memory (the single-run kernels get theirs as a
// kernel parameter, whose fields the arithmetic reads for free; read from global memory
// they would be loads on the critical path).  The caller synchronises before use.
__device__ __forceinline__ void stage_params(DevParams &dst, const DevParams *src, int tid, int nthreads) {
    static_assert(sizeof(DevParams) % 8 == 0, "DevParams in 8-byte words");
    const int2 *s = reinterpret_cast<const int2 *>(src);
    int2 *d = reinterpret_cast<int2 *>(&dst);
    for (int k = tid; k < (int)(sizeof(DevParams) / 8); k += nthreads) d[k] = s[k];
}

template <int N, int TX, int TY, class S, class R, int FORCE, int MU>
__global__ void __launch_bounds__(TX *TY, MinBlocks<S, N, TX * TY, PairPath<N, S, R, MU>::value>::value)
    lb_batch_tile_kernel(const S *__restrict__ pool_in, S *__restrict__ pool_out, const DevParams *__restrict__ runs,
                         const BatchTile *__restrict__ tiles, const LogTables *__restrict__ tbl) {
    const BatchTile t = tiles[blockIdx.x];
    const int tid = threadIdx.x + TX * threadIdx.y;
    __shared__ __align__(16) DevParams s_p;
    if constexpr (PairPath<N, S, R, MU>::value) {
        // the parameter block is requested here and stored at the end of the densities
        // phase, which needs only the tile entry: the two global round trips overlap, and
        // the step's first barrier publishes the block
        constexpr int W = (int)(sizeof(DevParams) / 8);
        static_assert(sizeof(DevParams) % 8 == 0 && W <= TX * TY, "one 8-byte word of DevParams per thread");
        int2 w = make_int2(0, 0);
        if (tid < W) w = reinterpret_cast<const int2 *>(runs + t.run)[tid];
        auto hook = [&]() {
            if (tid < W) reinterpret_cast<int2 *>(&s_p)[tid] = w;
        };
        step_tile_pair<2, N / 2, TX, TY, FORCE, MU>(
            pool_in + t.off, pool_out + t.off, s_p, t.x0, t.y0,
            TileGeo{t.nx, t.ny, tbl, {t.rho_ref[0], t.rho_ref[1], t.rho_ref[2], t.rho_ref[3]}}, hook);
    } else {
        stage_params(s_p, runs + t.run, tid, TX * TY);
        __syncthreads();
        step_tile<2, N, TX, TY, S, R, FORCE, MU>(pool_in + t.off, pool_out + t.off, s_p, t.x0, t.y0);
    }
}

// Largest D1Q3 run the resident kernel holds, and its thread count.
constexpr int RESIDENT_THREADS = 1024;
constexpr int RESIDENT_MAX_NODES_PER_THREAD = 4;
constexpr int RESIDENT_MAX_L = RESIDENT_THREADS * RESIDENT_MAX_NODES_PER_THREAD;

// shared memory (bytes) the resident kernel needs for a run of L nodes
template <int N, class S, class R, int MU>
__host__ __device__ constexpr size_t resident_smem_bytes(int L) {
    using MT = typename MuStore<MU>::T;
    return sizeof(S) * (size_t)N * 3 * L + sizeof(R) * (size_t)N * (L + 4) + sizeof(MT) * (size_t)N * (L + 2) +
           sizeof(float) * TblWords<MU>::value + 64;
}

template <int N, class S, class R, int FORCE, int MU>
__global__ void __launch_bounds__(RESIDENT_THREADS)
    lb_d1q3_resident_kernel(const S *__restrict__ pool_in, S *__restrict__ pool_out,
                            const DevParams *__restrict__ runs, const size_t *__restrict__ offsets,
                            const int *__restrict__ run_ids, int nsteps) {
    using MT = typename MuStore<MU>::T;
    constexpr int Q = 3;
    constexpr int NT = RESIDENT_THREADS;
    constexpr int MAXM = RESIDENT_MAX_NODES_PER_THREAD;
    const int run = run_ids[blockIdx.x];
    const int tid = threadIdx.x;
    __shared__ __align__(16) DevParams s_p;
    stage_params(s_p, runs + run, tid, RESIDENT_THREADS);
    __syncthreads();
    const DevParams &P = s_p;
    const int L = P.nx;

    extern __shared__ __align__(16) unsigned char smem[];
    // layout: tables | phi [N][L+2] | rho [N][L+4] | f [N][3][L]
    float *s_tbl = reinterpret_cast<float *>(smem);
    MT *s_phi = reinterpret_cast<MT *>(smem + sizeof(float) * TblWords<MU>::value);
    R *s_rho = reinterpret_cast<R *>(reinterpret_cast<unsigned char *>(s_phi) + sizeof(MT) * (size_t)N * (L + 2));
    S *s_f = reinterpret_cast<S *>(reinterpret_cast<unsigned char *>(s_rho) + sizeof(R) * (size_t)N * (L + 4));
    const int PH = L + 2, RH = L + 4;

    load_tables<MU>(s_tbl, P, tid, NT);
    const S *gin = pool_in + offsets[run];
    for (int k = tid; k < N * Q * L; k += NT) s_f[k] = gin[k];
    __syncthreads();

    unsigned bad = 0;
    for (int step = 0; step < nsteps; ++step) {
        // densities on the run plus a 2-node periodic ring (same sums as step_tile)
        for (int k = tid; k < RH; k += NT) {
            int xx = k - 2;
            xx = xx < 0 ? xx + L : (xx >= L ? xx - L : xx);
#pragma unroll
            for (int c = 0; c < N; ++c) {
                R acc = (R)s_f[(c * Q) * L + xx];
#pragma unroll
                for (int i = 1; i < Q; ++i) acc = v_add(acc, (R)s_f[(c * Q + i) * L + xx]);
                s_rho[c * RH + k] = v_add(pv<R>(P.rho_ref[c], P.rho_ref_f[c]), acc);
            }
        }
        __syncthreads();
        // chemical potentials on the run plus a 1-node ring
        for (int k = tid; k < PH; k += NT) {
            const int ex = k + 1;
            R r[N], lp[N], lin[N];
#pragma unroll
            for (int c = 0; c < N; ++c) {
                r[c] = s_rho[c * RH + ex];
                lp[c] = lap_at<1, R>(s_rho + c * RH, ex, 0, RH);
            }
            lin_node<N, R>(r, lp, P, lin);
            MT phi[N];
            if (!mu_node<N, R, FORCE, MU>(r, lin, P, s_tbl, phi)) bad = 1;
#pragma unroll
            for (int c = 0; c < N; ++c) s_phi[c * PH + k] = phi[c];
        }
        __syncthreads();
        // collision of every node into registers
        R post[MAXM][N][Q];
#pragma unroll
        for (int m = 0; m < MAXM; ++m) {
            const int x = tid + m * NT;
            if (x >= L) continue;
            const int ex = x + 2, mx = x + 1;
            R rho[N], lap[N], gpx[N], gpy[N], grx[N], gry[N], jx[N], jy[N], gr[N][Q];
#pragma unroll
            for (int c = 0; c < N; ++c) {
                rho[c] = s_rho[c * RH + ex];
                lap[c] = lap_at<1, R>(s_rho + c * RH, ex, 0, RH);
                grad_phi<1, R, MT>(s_phi + c * PH, mx, 0, PH, P, gpx[c], gpy[c]);
                if constexpr (!Flags<FORCE>::nid) grad_at<1, R>(s_rho + c * RH, ex, 0, RH, grx[c], gry[c]);
                else grx[c] = gry[c] = (R)0;
                R acc;
#pragma unroll
                for (int i = 0; i < Q; ++i) gr[c][i] = (R)s_f[(c * Q + i) * L + x];
                moments_lane<1>(gr[c], acc, jx[c], jy[c]);
            }
            collide_node<1, N, R, FORCE>(rho, lap, gpx, gpy, grx, gry, jx, jy, P, gr, post[m]);
        }
        __syncthreads();
        // push streaming in place (every read of s_f of this step is done)
#pragma unroll
        for (int m = 0; m < MAXM; ++m) {
            const int x = tid + m * NT;
            if (x >= L) continue;
            const int xe = x + 1 == L ? 0 : x + 1, xw = x == 0 ? L - 1 : x - 1;
#pragma unroll
            for (int c = 0; c < N; ++c) {
                s_f[(c * Q + 0) * L + x] = (S)post[m][c][0];
                s_f[(c * Q + 1) * L + xe] = (S)post[m][c][1];
                s_f[(c * Q + 2) * L + xw] = (S)post[m][c][2];
            }
        }
        __syncthreads();
    }
    if (bad) atomicOr(P.err, ERR_DOMAIN);
    S *gout = pool_out + offsets[run];
    for (int k = tid; k < N * Q * L; k += NT) gout[k] = s_f[k];
}

}  // namespace lbvdw
