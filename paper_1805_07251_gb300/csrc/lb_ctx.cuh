// lb_ctx.cuh -- the context behind lb_ctx* (private to the library).
#pragma once
#include <string>
#include <vector>

#include "lb_launch.cuh"
#include "lbvdw.h"

struct lb_ctx {
    // checkpointed rollout for the adjoint (lb_rollout_*): copies of the state (in its
    // storage type) every ckpt_every steps, and the number of steps recorded
    std::vector<void *> ckpt;
    int ckpt_every = 0;
    int64_t rollout_steps = -1;
    lb_params p;
    int Q = 0, D = 0;
    size_t n = 0;      // nodes
    size_t elem = 0;   // bytes per stored population
    void *f[2] = {nullptr, nullptr};
    int cur = 0;
    double *rho = nullptr;  // moments scratch [N][n]
    double *mom = nullptr;  // moments scratch [N][D][n]
    double *partial = nullptr;
    int nparts = 0;
    double *diag = nullptr;  // [N + 3]
    unsigned *err = nullptr;
    lbvdw::LogTables *tbl = nullptr;  // device copy of the log tables
    cudaStream_t stream = nullptr;
    lbvdw::DevParams dp{};
    // chained steps (lb_chain.cuh): per-tile completion flags (nullptr: the context's
    // configuration does not chain), the next chain step number, the row rotation of the
    // next step, and the CTA rows of a step that set flags
    unsigned *chain_flag = nullptr;
    unsigned chain_step = 0;
    int chain_roff = 0;
    int chain_rows = 0;
    int chain_evict_first = 0;  // chained steps load their input with an evict-first L2 policy
    int64_t steps = 0, launches = 0;
    bool has_state = false, poisoned = false;
    std::string msg;
};

// One timestep of the context's lattice, precision and kernel organisation (lb_api.cu).
cudaError_t lb_ctx_step(lb_ctx *c, const void *fin, void *fout);

// Whether the context uses the moment-space collision (relaxation times other than tau).
bool lb_ctx_mrt(const lb_ctx *c);
