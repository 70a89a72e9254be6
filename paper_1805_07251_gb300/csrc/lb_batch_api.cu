// lb_batch_api.cu -- C ABI of batched independent runs (include/lbvdw.h, lb_batch_*).
//
// Layout: two pooled population arrays (ping-pong); run r occupies
// [offset_r, offset_r + N Q nx ny) of each, in the single-run layout [c][i][y][x].
// A timestep of the batch is one lb_batch_tile_kernel launch over the tiles of all D2Q9
// runs; D1Q3 runs are advanced by lb_d1q3_resident_kernel, one launch per chunk of
// timesteps.  lb_batch_step replays CUDA graphs of such chunks.
#include <cmath>
#include <cstring>
#include <map>
#include <new>
#include <string>
#include <utility>
#include <vector>

#include "lb_batch_launch.cuh"
#include "lb_launch.cuh"
#include "lbvdw.h"

using namespace lbvdw;

namespace {
constexpr int GRAPH_CHUNK = 32;  // timesteps per captured graph
}

struct lb_batch {
    lb_params shared;
    int nruns = 0, N = 0;
    std::vector<lb_run_desc> desc;
    std::vector<size_t> offsets;      // element offsets
    std::vector<DevParams> hparams;   // host copies of the run parameter blocks
    std::vector<int> d1, d2;          // run indices by lattice
    size_t pool_elems = 0, elem = 0, max_nodes = 0;
    void *pool[2] = {nullptr, nullptr};
    DevParams *d_params = nullptr;
    size_t *d_offsets = nullptr;
    BatchTile *d_tiles = nullptr;
    int ntiles = 0;
    int *d_d1 = nullptr;
    unsigned *d_err = nullptr;
    LogTables *d_tbl = nullptr;
    double *d_rho = nullptr, *d_mom = nullptr;  // read-back / init scratch (largest run)
    size_t smem = 0;
    int cur = 0;
    int tile_x = 32, tile_y = 8;
    cudaStream_t stream = nullptr;
    std::map<std::pair<int, int>, cudaGraphExec_t> graphs;  // (chunk, parity) -> graph
    int64_t steps = 0, launches = 0;
    bool has_state = false;
    std::string msg;
};

namespace {

lb_status bfail(lb_batch *b, lb_status s, const std::string &m) {
    if (b) b->msg = m;
    return s;
}

#define LB_BCUDA(b, call)                                                                  \
    do {                                                                                   \
        cudaError_t e_ = (call);                                                           \
        if (e_ != cudaSuccess) return bfail((b), LB_E_CUDA, std::string(#call) + ": " +     \
                                                                 cudaGetErrorString(e_));  \
    } while (0)

void clear_graphs(lb_batch *b) {
    for (auto &kv : b->graphs) cudaGraphExecDestroy(kv.second);
    b->graphs.clear();
}

// The tile list of the D2Q9 runs (host copy), with each run's current reference densities.
std::vector<BatchTile> tile_list(const lb_batch *b) {
    std::vector<BatchTile> t;
    for (int r : b->d2) {
        const lb_run_desc &d = b->desc[r];
        const DevParams &P = b->hparams[r];
        for (int y0 = 0; y0 < d.ny; y0 += b->tile_y)
            for (int x0 = 0; x0 < d.nx; x0 += b->tile_x)
                t.push_back({r, x0, y0, d.nx, d.ny, 0, b->offsets[r],
                             {P.rho_ref_f[0], P.rho_ref_f[1], P.rho_ref_f[2], P.rho_ref_f[3]}});
    }
    return t;
}

cudaError_t build_tiles(lb_batch *b) {
    std::vector<BatchTile> t = tile_list(b);
    cudaFree(b->d_tiles);
    b->d_tiles = nullptr;
    b->ntiles = (int)t.size();
    if (t.empty()) return cudaSuccess;
    cudaError_t e = cudaMalloc(&b->d_tiles, sizeof(BatchTile) * t.size());
    if (e != cudaSuccess) return e;
    return cudaMemcpy(b->d_tiles, t.data(), sizeof(BatchTile) * t.size(), cudaMemcpyHostToDevice);
}

// Rewrite the tile list in place (same device array, so captured graphs stay valid) after
// the runs' reference densities changed.
cudaError_t refresh_tiles(lb_batch *b) {
    if (b->ntiles == 0) return cudaSuccess;
    std::vector<BatchTile> t = tile_list(b);
    return cudaMemcpy(b->d_tiles, t.data(), sizeof(BatchTile) * t.size(), cudaMemcpyHostToDevice);
}

BatchLaunch launch_args(lb_batch *b, int parity, int nsteps) {
    BatchLaunch a;
    a.pool_in = b->pool[parity];
    a.pool_out = b->pool[parity ^ 1];
    a.runs = b->d_params;
    a.offsets = b->d_offsets;
    a.tiles = b->d_tiles;
    a.tbl = b->d_tbl;
    a.ntiles = b->ntiles;
    a.d1_ids = b->d_d1;
    a.nd1 = (int)b->d1.size();
    a.ncomp = b->N;
    a.force = b->shared.force_method;
    a.tile_x = b->tile_x;
    a.tile_y = b->tile_y;
    a.nsteps = nsteps;
    a.smem = b->smem;
    a.stream = b->stream;
    return a;
}

cudaError_t launch_tiles(lb_batch *b, const BatchLaunch &a) {
    switch (b->shared.precision) {
        case LB_FP32_MIXED: return tbl_batch_tiles(a);
        case LB_FP32_DFMU: return df_batch_tiles(a);
        default: return f64_batch_tiles(a);
    }
}

cudaError_t launch_resident(lb_batch *b, const BatchLaunch &a) {
    switch (b->shared.precision) {
        case LB_FP32_MIXED: return tbl_batch_resident(a);
        case LB_FP32_DFMU: return df_batch_resident(a);
        default: return f64_batch_resident(a);
    }
}

size_t resident_smem(int precision, int N, int L) {
    switch (precision) {
        case LB_FP32_MIXED: return tbl_resident_smem(N, L);
        case LB_FP32_DFMU: return df_resident_smem(N, L);
        default: return f64_resident_smem(N, L);
    }
}

// Enqueue `len` timesteps starting from pool[parity]: the D1Q3 runs in one resident
// launch (result written to the pool the D2Q9 runs end in) and len tile launches.  When
// `side` is given (both kinds of runs present, under capture), the resident launch goes on
// a branch of its own, forked from and joined back into b->stream by the two events: the
// D1Q3 and D2Q9 runs share no memory (their pool regions and error words are disjoint), so
// the graph lets them run side by side.
cudaError_t enqueue_chunk(lb_batch *b, int parity, int len, cudaStream_t side, cudaEvent_t fork,
                          cudaEvent_t join) {
    if (side) {
        cudaError_t e = cudaEventRecord(fork, b->stream);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(side, fork, 0);
        if (e != cudaSuccess) return e;
    }
    if (!b->d1.empty()) {
        BatchLaunch a = launch_args(b, parity, len);
        a.pool_out = b->pool[parity ^ (len & 1)];
        if (side) a.stream = side;
        cudaError_t e = launch_resident(b, a);
        if (e != cudaSuccess) return e;
    }
    if (b->ntiles > 0) {
        for (int s = 0; s < len; ++s) {
            cudaError_t e = launch_tiles(b, launch_args(b, parity ^ (s & 1), 0));
            if (e != cudaSuccess) return e;
        }
    }
    if (side) {
        cudaError_t e = cudaEventRecord(join, side);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(b->stream, join, 0);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

int64_t chunk_launches(lb_batch *b, int len) {
    return (b->d1.empty() ? 0 : 1) + (b->ntiles > 0 ? len : 0);
}

cudaError_t get_graph(lb_batch *b, int parity, int len, cudaGraphExec_t *out) {
    auto key = std::make_pair(len, parity);
    auto it = b->graphs.find(key);
    if (it != b->graphs.end()) {
        *out = it->second;
        return cudaSuccess;
    }
    cudaStream_t cap = nullptr, side = nullptr;
    cudaEvent_t fork = nullptr, join = nullptr;
    const bool both = !b->d1.empty() && b->ntiles > 0;
    cudaError_t e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
    if (e == cudaSuccess && both) {
        e = cudaStreamCreateWithFlags(&side, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&fork, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&join, cudaEventDisableTiming);
    }
    cudaGraph_t g = nullptr;
    if (e == cudaSuccess) {
        cudaStream_t saved = b->stream;
        b->stream = cap;
        e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            cudaError_t e2 = enqueue_chunk(b, parity, len, side, fork, join);
            e = cudaStreamEndCapture(cap, &g);
            if (e2 != cudaSuccess) e = e2;
        }
        b->stream = saved;
    }
    if (fork) cudaEventDestroy(fork);
    if (join) cudaEventDestroy(join);
    if (side) cudaStreamDestroy(side);
    if (cap) cudaStreamDestroy(cap);
    if (e != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return e;
    }
    cudaGraphExec_t ex = nullptr;
    e = cudaGraphInstantiate(&ex, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return e;
    b->graphs[key] = ex;
    *out = ex;
    return cudaSuccess;
}

}  // namespace

extern "C" {

lb_status lb_batch_create(const lb_params *shared, const lb_run_desc *runs, int32_t nruns, lb_batch **out) {
    if (!shared || !runs || !out || nruns < 1) return LB_E_INVALID;
    *out = nullptr;
    // validate the shared part through the single-run rules on each run's geometry
    const int N = shared->ncomp;
    if (shared->abi != LBVDW_ABI || N < 1 || N > 4) return LB_E_INVALID;
    if (shared->precision != LB_FP64 && shared->precision != LB_FP32_MIXED && shared->precision != LB_FP32_DFMU)
        return LB_E_INVALID;
    if (shared->force_method != LB_FORCE_LOG && shared->force_method != LB_FORCE_NID) return LB_E_INVALID;
    if (!(shared->tau > 0.5)) return LB_E_INVALID;
    // batches run the BGK collision: relaxation times other than tau are single-run only
    if ((shared->tau_shear != 0.0 && shared->tau_shear != shared->tau) ||
        (shared->tau_ghost != 0.0 && shared->tau_ghost != shared->tau))
        return LB_E_INVALID;
    for (int c = 0; c < N; ++c) {
        if (!(shared->b[c] > 0.0)) return LB_E_INVALID;
        for (int cc = 0; cc < N; ++cc)
            if (shared->a[c * 4 + cc] != shared->a[cc * 4 + c] ||
                shared->kappa[c * 4 + cc] != shared->kappa[cc * 4 + c] ||
                shared->lambda[c * 4 + cc] != shared->lambda[cc * 4 + c] ||
                (cc != c && shared->lambda[c * 4 + cc] < 0.0))
                return LB_E_INVALID;
    }
    lb_batch *b = new (std::nothrow) lb_batch;
    if (!b) return LB_E_NOMEM;
    b->shared = *shared;
    b->nruns = nruns;
    b->N = N;
    b->desc.assign(runs, runs + nruns);
    b->elem = shared->precision == LB_FP64 ? sizeof(double) : sizeof(float);
    b->stream = static_cast<cudaStream_t>(shared->stream);
    if (shared->tile_x != 0 || shared->tile_y != 0) {
        b->tile_x = shared->tile_x;
        b->tile_y = shared->tile_y;
    }
    int maxL1 = 0;
    size_t off = 0;
    for (int r = 0; r < nruns; ++r) {
        const lb_run_desc &d = runs[r];
        bool ok = (d.lattice == LB_D1Q3 && d.ny == 1 && d.nx >= 2 && d.nx <= RESIDENT_MAX_L) ||
                  (d.lattice == LB_D2Q9 && d.nx >= 2 && d.ny >= 2 && (int64_t)9 * d.nx * d.ny < ((int64_t)1 << 32));
        ok = ok && d.kT > 0.0 && d.gamma_mu > 0.0 && std::isfinite(d.kT) && std::isfinite(d.gamma_mu) &&
             d.kappa_scale >= 0.0 && std::isfinite(d.kappa_scale);
        if (!ok) {
            delete b;
            return LB_E_INVALID;
        }
        const int Q = d.lattice == LB_D1Q3 ? 3 : 9;
        b->offsets.push_back(off);
        size_t n = (size_t)d.nx * d.ny;
        off += (size_t)N * Q * n;
        off = (off + 63) & ~size_t(63);  // 256-byte aligned run starts (FP32)
        if (n > b->max_nodes) b->max_nodes = n;
        if (d.lattice == LB_D1Q3) {
            b->d1.push_back(r);
            if (d.nx > maxL1) maxL1 = d.nx;
        } else {
            b->d2.push_back(r);
        }
    }
    b->pool_elems = off;
    if (maxL1 > 0) {
        b->smem = resident_smem(shared->precision, N, maxL1);
        // dynamic shared memory plus the kernel's static copy of the run's parameters
        if (b->smem + sizeof(DevParams) > 227 * 1024) {
            delete b;
            return LB_E_INVALID;  // the longest D1Q3 run does not fit one CTA's shared memory
        }
    }
    DeviceGuard dg(shared->device);
    if (!dg.ok()) {
        delete b;
        return LB_E_CUDA;
    }
    bool ok = cudaMalloc(&b->pool[0], b->elem * b->pool_elems) == cudaSuccess &&
              cudaMalloc(&b->pool[1], b->elem * b->pool_elems) == cudaSuccess &&
              cudaMalloc(&b->d_params, sizeof(DevParams) * nruns) == cudaSuccess &&
              cudaMalloc(&b->d_offsets, sizeof(size_t) * nruns) == cudaSuccess &&
              cudaMalloc(&b->d_err, sizeof(unsigned) * nruns) == cudaSuccess &&
              cudaMalloc(&b->d_tbl, sizeof(LogTables)) == cudaSuccess &&
              cudaMalloc(&b->d_rho, sizeof(double) * N * b->max_nodes) == cudaSuccess &&
              cudaMalloc(&b->d_mom, sizeof(double) * N * 2 * b->max_nodes) == cudaSuccess &&
              (b->d1.empty() || cudaMalloc(&b->d_d1, sizeof(int) * b->d1.size()) == cudaSuccess);
    if (!ok) {
        cudaGetLastError();
        lb_batch_destroy(b);
        return LB_E_NOMEM;
    }
    LogTables h;
    fill_log_tables(&h);
    b->hparams.resize(nruns);
    for (int r = 0; r < nruns; ++r) {
        lb_params p = *shared;
        p.lattice = runs[r].lattice;
        p.nx = runs[r].nx;
        p.ny = runs[r].ny;
        p.kT = runs[r].kT;
        p.gamma_mu = runs[r].gamma_mu;
        if (runs[r].kappa_scale > 0.0)
            for (int k = 0; k < 16; ++k) p.kappa[k] = shared->kappa[k] * runs[r].kappa_scale;
        make_dev_params(p, b->hparams[r], b->d_err + r, b->d_tbl);
    }
    if (cudaMemcpy(b->d_tbl, &h, sizeof h, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(b->d_offsets, b->offsets.data(), sizeof(size_t) * nruns, cudaMemcpyHostToDevice) != cudaSuccess ||
        (!b->d1.empty() &&
         cudaMemcpy(b->d_d1, b->d1.data(), sizeof(int) * b->d1.size(), cudaMemcpyHostToDevice) != cudaSuccess) ||
        build_tiles(b) != cudaSuccess) {
        cudaGetLastError();
        lb_batch_destroy(b);
        return LB_E_CUDA;
    }
    if (!b->d1.empty() && launch_resident(b, launch_args(b, 0, -1)) != cudaSuccess) {
        cudaGetLastError();
        lb_batch_destroy(b);
        return LB_E_CUDA;
    }
    *out = b;
    return LB_OK;
}

lb_status lb_batch_init(lb_batch *b, const double *rho_all) {
    if (!b || !rho_all) return LB_E_INVALID;
    const int N = b->N;
    DeviceGuard dg(b->shared.device);
    LB_BCUDA(b, dg.status);
    size_t pos = 0;
    for (int r = 0; r < b->nruns; ++r) {
        const lb_run_desc &d = b->desc[r];
        const size_t n = (size_t)d.nx * d.ny;
        const double *rho = rho_all + pos;
        double mean[4] = {0, 0, 0, 0};
        for (size_t s = 0; s < n; ++s) {
            double eta = 1.0;
            for (int c = 0; c < N; ++c) {
                double v = rho[c * n + s];
                if (!(v > 0.0) || !std::isfinite(v)) {
                    b->has_state = false;
                    return bfail(b, LB_E_DOMAIN, "run " + std::to_string(r) + ": a density is <= 0 or not finite");
                }
                eta -= b->shared.b[c] * v;
                mean[c] += v;
            }
            if (!(eta > 0.0)) {
                b->has_state = false;
                return bfail(b, LB_E_DOMAIN, "run " + std::to_string(r) + ": eta <= 0");
            }
        }
        DevParams &P = b->hparams[r];
        for (int c = 0; c < 4; ++c) {
            double ref = 0.0;
            if (b->shared.precision != LB_FP64 && c < N)
                ref = (double)(float)(b->shared.rho_ref[c] > 0.0 ? b->shared.rho_ref[c] : mean[c] / (double)n);
            P.rho_ref[c] = ref;
            P.rho_ref_f[c] = (float)ref;
        }
        LB_BCUDA(b, cudaMemcpyAsync(b->d_rho, rho, sizeof(double) * N * n, cudaMemcpyHostToDevice, b->stream));
        FieldLaunch a;
        std::memset(&a, 0, sizeof a);
        a.f = static_cast<char *>(b->pool[0]) + b->elem * b->offsets[r];
        a.rho_in = b->d_rho;
        a.mom_in = nullptr;
        a.P = P;
        a.ncomp = N;
        a.stream = b->stream;
        const bool f32 = b->shared.precision != LB_FP64;
        cudaError_t e = d.lattice == LB_D1Q3 ? (f32 ? d1q3_f32_init(a) : d1q3_f64_init(a))
                                             : (f32 ? d2q9_f32_init(a) : d2q9_f64_init(a));
        if (e != cudaSuccess) return bfail(b, LB_E_CUDA, "init kernel");
        LB_BCUDA(b, cudaStreamSynchronize(b->stream));  // d_rho is reused by the next run
        b->launches += 1;
        pos += (size_t)N * n;
    }
    LB_BCUDA(b, cudaMemcpy(b->d_params, b->hparams.data(), sizeof(DevParams) * b->nruns, cudaMemcpyHostToDevice));
    LB_BCUDA(b, refresh_tiles(b));
    LB_BCUDA(b, cudaMemset(b->d_err, 0, sizeof(unsigned) * b->nruns));
    b->cur = 0;
    b->steps = 0;
    b->has_state = true;
    b->msg.clear();
    return LB_OK;
}

lb_status lb_batch_step(lb_batch *b, int64_t nsteps) {
    if (!b) return LB_E_INVALID;
    if (!b->has_state) return bfail(b, LB_E_STATE, "fields not initialised");
    if (nsteps < 0) return bfail(b, LB_E_INVALID, "nsteps < 0");
    DeviceGuard dg(b->shared.device);
    LB_BCUDA(b, dg.status);
    int64_t left = nsteps;
    while (left > 0) {
        int len = left >= GRAPH_CHUNK ? GRAPH_CHUNK : (int)left;
        cudaGraphExec_t g = nullptr;
        cudaError_t e = get_graph(b, b->cur, len, &g);
        if (e != cudaSuccess) return bfail(b, LB_E_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
        LB_BCUDA(b, cudaGraphLaunch(g, b->stream));
        b->cur ^= (len & 1);
        b->steps += len;
        b->launches += chunk_launches(b, len);
        left -= len;
    }
    return LB_OK;
}

lb_status lb_batch_read(lb_batch *b, int32_t run, double *rho, double *mom) {
    if (!b || !rho || run < 0 || run >= b->nruns) return LB_E_INVALID;
    if (!b->has_state) return bfail(b, LB_E_STATE, "fields not initialised");
    DeviceGuard dg(b->shared.device);
    LB_BCUDA(b, dg.status);
    const lb_run_desc &d = b->desc[run];
    const size_t n = (size_t)d.nx * d.ny;
    const int D = d.lattice == LB_D1Q3 ? 1 : 2;
    FieldLaunch a;
    std::memset(&a, 0, sizeof a);
    a.f = static_cast<char *>(b->pool[b->cur]) + b->elem * b->offsets[run];
    a.rho_out = b->d_rho;
    a.mom_out = b->d_mom;
    a.P = b->hparams[run];
    a.ncomp = b->N;
    a.stream = b->stream;
    const bool f32 = b->shared.precision != LB_FP64;
    cudaError_t e = d.lattice == LB_D1Q3 ? (f32 ? d1q3_f32_moments(a) : d1q3_f64_moments(a))
                                         : (f32 ? d2q9_f32_moments(a) : d2q9_f64_moments(a));
    if (e != cudaSuccess) return bfail(b, LB_E_CUDA, "moments kernel");
    b->launches += 1;
    LB_BCUDA(b, cudaMemcpyAsync(rho, b->d_rho, sizeof(double) * b->N * n, cudaMemcpyDeviceToHost, b->stream));
    if (mom)
        LB_BCUDA(b, cudaMemcpyAsync(mom, b->d_mom, sizeof(double) * b->N * D * n, cudaMemcpyDeviceToHost, b->stream));
    LB_BCUDA(b, cudaStreamSynchronize(b->stream));
    return LB_OK;
}

lb_status lb_batch_errors(lb_batch *b, uint32_t *flags) {
    if (!b || !flags) return LB_E_INVALID;
    DeviceGuard dg(b->shared.device);
    LB_BCUDA(b, dg.status);
    LB_BCUDA(b, cudaMemcpyAsync(flags, b->d_err, sizeof(unsigned) * b->nruns, cudaMemcpyDeviceToHost, b->stream));
    LB_BCUDA(b, cudaStreamSynchronize(b->stream));
    return LB_OK;
}

lb_status lb_batch_set_tile(lb_batch *b, int32_t tile_x, int32_t tile_y) {
    if (!b) return LB_E_INVALID;
    bool ok = (tile_x == 32 && tile_y == 8) || (tile_x == 64 && tile_y == 4) || (tile_x == 32 && tile_y == 16) ||
              (tile_x == 64 && tile_y == 8);
    if (!ok) return bfail(b, LB_E_INVALID, "unsupported tile");
    DeviceGuard dg(b->shared.device);
    LB_BCUDA(b, dg.status);
    LB_BCUDA(b, cudaStreamSynchronize(b->stream));
    clear_graphs(b);
    b->tile_x = tile_x;
    b->tile_y = tile_y;
    cudaError_t e = build_tiles(b);
    if (e != cudaSuccess) return bfail(b, LB_E_CUDA, cudaGetErrorString(e));
    return LB_OK;
}

lb_status lb_batch_time_steps(lb_batch *b, int32_t nsteps, double *ms) {
    if (!b || !ms || nsteps < 1) return LB_E_INVALID;
    DeviceGuard dg(b->shared.device);
    LB_BCUDA(b, dg.status);
    cudaEvent_t e0, e1;
    LB_BCUDA(b, cudaEventCreate(&e0));
    LB_BCUDA(b, cudaEventCreate(&e1));
    LB_BCUDA(b, cudaEventRecord(e0, b->stream));
    lb_status s = lb_batch_step(b, nsteps);
    LB_BCUDA(b, cudaEventRecord(e1, b->stream));
    LB_BCUDA(b, cudaEventSynchronize(e1));
    float t = 0.0f;
    LB_BCUDA(b, cudaEventElapsedTime(&t, e0, e1));
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    *ms = t;
    return s;
}

int64_t lb_batch_step_count(const lb_batch *b) { return b ? b->steps : -1; }

int64_t lb_batch_launch_count(const lb_batch *b) { return b ? b->launches : -1; }

const char *lb_batch_last_error(const lb_batch *b) { return b ? b->msg.c_str() : "NULL batch"; }

lb_status lb_batch_destroy(lb_batch *b) {
    if (!b) return LB_OK;
    DeviceGuard dg(b->shared.device);
    if (b->stream) cudaStreamSynchronize(b->stream);
    else cudaDeviceSynchronize();
    clear_graphs(b);
    cudaFree(b->pool[0]);
    cudaFree(b->pool[1]);
    cudaFree(b->d_params);
    cudaFree(b->d_offsets);
    cudaFree(b->d_tiles);
    cudaFree(b->d_d1);
    cudaFree(b->d_err);
    cudaFree(b->d_tbl);
    cudaFree(b->d_rho);
    cudaFree(b->d_mom);
    delete b;
    return LB_OK;
}

}  // extern "C"
