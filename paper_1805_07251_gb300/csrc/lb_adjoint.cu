// lb_adjoint.cu -- checkpointed rollout and its adjoint (lb_rollout_forward /
// lb_rollout_backward in include/lbvdw.h), for FP64 contexts and for the FP32-storage
// contexts (FP64 or double-float mu in the forward step).
//
// Forward: the context advances nsteps timesteps with its own step kernel and keeps a
// device copy of the state (in its storage type) every ckpt_every steps, and of the
// starting state.  Backward: from the last segment to the first, the segment's states
// are recomputed from its checkpoint into a ring of ckpt_every states by the same step
// kernel (bitwise the forward trajectory), then the adjoint step (lb_adjoint.cuh) runs
// backwards through them: in FP64 for an FP64 context, in FP32 (FP64 mu and FP64
// parameter-gradient sums) for the FP32-storage contexts.  Memory: (nsteps /
// ckpt_every + 1) checkpoints + ckpt_every ring states + a few state-sized adjoint
// arrays, all in the storage type.
#include <cstring>
#include <vector>

#include "lb_adjoint.cuh"
#include "lb_ctx.cuh"

using namespace lbvdw;

namespace {

template <int LAT, int N, class T>
cudaError_t adjoint_step(const T *fbar_next, T *fbar, AdjArrays<T> A, const DevParams &P, int nblocks,
                         double *accum, cudaStream_t st) {
    adj_mu_kernel<LAT, N, T><<<nblocks, ADJ_THREADS, 0, st>>>(A, P);
    adj_local_kernel<LAT, N, T><<<nblocks, ADJ_THREADS, 0, st>>>(fbar_next, fbar, A, P);
    adj_mubar_kernel<LAT, N, T><<<nblocks, ADJ_THREADS, 0, st>>>(A, P);
    // add this step's parameter-gradient partials to the running sums, in block order
    lb_diag_final_kernel<2 * N * N + N><<<1, DIAG_THREADS, 0, st>>>(A.partial, nblocks, A.partial + (size_t)nblocks * (2 * N * N + N));
    adj_accum_kernel<2 * N * N + N><<<1, 32, 0, st>>>(A.partial + (size_t)nblocks * (2 * N * N + N), accum);
    adj_rhobar_kernel<LAT, N, T><<<nblocks, ADJ_THREADS, 0, st>>>(fbar, A, P);
    return cudaGetLastError();
}

template <int LAT, class T>
cudaError_t adjoint_step_n(int N, const T *fbar_next, T *fbar, AdjArrays<T> A, const DevParams &P, int nb,
                           double *accum, cudaStream_t st) {
    switch (N) {
        case 1: return adjoint_step<LAT, 1, T>(fbar_next, fbar, A, P, nb, accum, st);
        case 2: return adjoint_step<LAT, 2, T>(fbar_next, fbar, A, P, nb, accum, st);
        case 3: return adjoint_step<LAT, 3, T>(fbar_next, fbar, A, P, nb, accum, st);
        case 4: return adjoint_step<LAT, 4, T>(fbar_next, fbar, A, P, nb, accum, st);
    }
    return cudaErrorInvalidValue;
}

lb_status rfail(lb_ctx *c, lb_status s, const char *m) {
    c->msg = m;
    return s;
}

struct DevBuf {
    std::vector<void *> ptrs;
    ~DevBuf() {
        for (void *p : ptrs) cudaFree(p);
    }
    template <class T>
    T *get(size_t count) {
        void *p = nullptr;
        if (cudaMalloc(&p, sizeof(T) * count) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        ptrs.push_back(p);
        return static_cast<T *>(p);
    }
    void *bytes(size_t nb) {
        void *p = nullptr;
        if (cudaMalloc(&p, nb) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        ptrs.push_back(p);
        return p;
    }
};

// FP64 moments rho, j of a state in the context's storage type (FP32 storage: deviations
// from w_i rho_ref, the reference density added back in FP64)
cudaError_t moments(lb_ctx *c, const void *f, double *rho, double *mom) {
    FieldLaunch a;
    std::memset(&a, 0, sizeof a);
    a.f = const_cast<void *>(f);
    a.rho_out = rho;
    a.mom_out = mom;
    a.P = c->dp;
    a.ncomp = c->p.ncomp;
    a.stream = c->stream;
    const bool d1 = c->p.lattice == LB_D1Q3;
    if (c->p.precision == LB_FP64) return d1 ? d1q3_f64_moments(a) : d2q9_f64_moments(a);
    return d1 ? d1q3_f32_moments(a) : d2q9_f32_moments(a);
}

// FP32 adjoint: the state's moments in FP32 (and FP64 copies) for the adjoint kernels
template <class T>
cudaError_t moments32(lb_ctx *c, const void *f, AdjArrays<T> A, int nb) {
    if constexpr (sizeof(T) != 4) {
        return cudaErrorInvalidValue;
    } else {
        const float *g = static_cast<const float *>(f);
        const bool d1 = c->p.lattice == LB_D1Q3;
        cudaStream_t st = c->stream;
        switch (c->p.ncomp) {
            case 1: d1 ? adj_moments32_kernel<1, 1><<<nb, ADJ_THREADS, 0, st>>>(g, A, c->dp)
                       : adj_moments32_kernel<2, 1><<<nb, ADJ_THREADS, 0, st>>>(g, A, c->dp); break;
            case 2: d1 ? adj_moments32_kernel<1, 2><<<nb, ADJ_THREADS, 0, st>>>(g, A, c->dp)
                       : adj_moments32_kernel<2, 2><<<nb, ADJ_THREADS, 0, st>>>(g, A, c->dp); break;
            case 3: d1 ? adj_moments32_kernel<1, 3><<<nb, ADJ_THREADS, 0, st>>>(g, A, c->dp)
                       : adj_moments32_kernel<2, 3><<<nb, ADJ_THREADS, 0, st>>>(g, A, c->dp); break;
            case 4: d1 ? adj_moments32_kernel<1, 4><<<nb, ADJ_THREADS, 0, st>>>(g, A, c->dp)
                       : adj_moments32_kernel<2, 4><<<nb, ADJ_THREADS, 0, st>>>(g, A, c->dp); break;
            default: return cudaErrorInvalidValue;
        }
        return cudaGetLastError();
    }
}

template <class T>
lb_status backward(lb_ctx *c, const double *rho_bar_T, double *rho_bar_0, double *grad) {
    const int N = c->p.ncomp, Q = c->Q, D = c->D;
    const size_t n = c->n, state = (size_t)N * Q * n;
    const int k = c->ckpt_every;
    const int64_t T_steps = c->rollout_steps;
    const int nb = (int)((n + ADJ_THREADS - 1) / ADJ_THREADS);
    const int V = 2 * N * N + N;
    DevBuf mem;
    std::vector<void *> ring(k);
    for (int m = 0; m < k; ++m)
        if (!(ring[m] = mem.bytes(c->elem * state))) return rfail(c, LB_E_NOMEM, "ring allocation");
    T *fb[2] = {mem.get<T>(state), mem.get<T>(state)};
    AdjArrays<T> A;
    double *rho = mem.get<double>((size_t)N * n), *jj = mem.get<double>((size_t)N * D * n);
    A.rho = rho;
    A.j = jj;
    A.lap = mem.get<T>((size_t)N * n);
    A.phi = mem.get<double>((size_t)N * n);
    A.rhob = mem.get<T>((size_t)N * n);
    A.jb = mem.get<T>((size_t)N * D * n);
    A.dphib = mem.get<T>((size_t)N * D * n);
    A.drhob = mem.get<T>((size_t)N * D * n);
    A.lapb = mem.get<T>((size_t)N * n);
    A.mub = mem.get<T>((size_t)N * n);
    A.partial = mem.get<double>((size_t)(nb + 1) * V);
    A.rho_t = A.u_t = nullptr;
    if (sizeof(T) == 4) {
        A.rho_t = mem.get<float>((size_t)N * n);
        A.u_t = mem.get<float>((size_t)N * D * n);
        if (!A.rho_t || !A.u_t) return rfail(c, LB_E_NOMEM, "adjoint work allocation");
    }
    double *accum = mem.get<double>(V);
    double *rb0 = mem.get<double>((size_t)N * n);
    if (!fb[0] || !fb[1] || !rho || !jj || !A.lap || !A.phi || !A.rhob || !A.jb || !A.dphib || !A.drhob ||
        !A.lapb || !A.mub || !A.partial || !accum || !rb0)
        return rfail(c, LB_E_NOMEM, "adjoint work allocation");
    cudaStream_t st = c->stream;
    // fbar_T,i = rhobar_T (rho_T = sum_i f_T,i)
    if (cudaMemcpyAsync(rb0, rho_bar_T, sizeof(double) * N * n, cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemsetAsync(accum, 0, sizeof(double) * V, st) != cudaSuccess)
        return rfail(c, LB_E_CUDA, "adjoint set-up");
    const bool d1 = c->p.lattice == LB_D1Q3;
    adj_seed_kernel<T><<<nb, ADJ_THREADS, 0, st>>>(rb0, fb[0], N, Q, n);
    int cur = 0;
    const int64_t nseg = (T_steps + k - 1) / k;
    for (int64_t sgm = nseg - 1; sgm >= 0; --sgm) {
        const int64_t t0 = sgm * k;
        const int len = (int)((t0 + k <= T_steps) ? k : T_steps - t0);
        if (cudaMemcpyAsync(ring[0], c->ckpt[sgm], c->elem * state, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
            return rfail(c, LB_E_CUDA, "ring copy");
        for (int m = 1; m < len; ++m)
            if (lb_ctx_step(c, ring[m - 1], ring[m]) != cudaSuccess) return rfail(c, LB_E_CUDA, "recompute step");
        for (int m = len - 1; m >= 0; --m) {
            const cudaError_t em = sizeof(T) == 4 ? moments32(c, ring[m], A, nb)
                                                   : moments(c, ring[m], rho, jj);
            if (em != cudaSuccess) return rfail(c, LB_E_CUDA, "moments");
            cudaError_t e = d1 ? adjoint_step_n<1, T>(N, fb[cur], fb[cur ^ 1], A, c->dp, nb, accum, st)
                               : adjoint_step_n<2, T>(N, fb[cur], fb[cur ^ 1], A, c->dp, nb, accum, st);
            if (e != cudaSuccess) return rfail(c, LB_E_CUDA, "adjoint step");
            cur ^= 1;
        }
    }
    // f_0 = w_i rho_0 (equilibrium at rest): rhobar_0 = sum_i w_i fbar_0,i
    if (d1) adj_init_transpose_kernel<1, T><<<nb, ADJ_THREADS, 0, st>>>(fb[cur], rb0, N, n);
    else adj_init_transpose_kernel<2, T><<<nb, ADJ_THREADS, 0, st>>>(fb[cur], rb0, N, n);
    if (cudaGetLastError() != cudaSuccess) return rfail(c, LB_E_CUDA, "init transpose");
    if (rho_bar_0 &&
        cudaMemcpyAsync(rho_bar_0, rb0, sizeof(double) * N * n, cudaMemcpyDeviceToHost, st) != cudaSuccess)
        return rfail(c, LB_E_CUDA, "rhobar copy");
    if (grad && cudaMemcpyAsync(grad, accum, sizeof(double) * V, cudaMemcpyDeviceToHost, st) != cudaSuccess)
        return rfail(c, LB_E_CUDA, "gradient copy");
    if (cudaStreamSynchronize(st) != cudaSuccess) return rfail(c, LB_E_CUDA, "synchronise");
    return LB_OK;
}

}  // namespace

extern "C" {

lb_status lb_rollout_forward(lb_ctx *c, int64_t nsteps, int32_t ckpt_every) {
    if (!c || nsteps < 1 || ckpt_every < 1) return LB_E_INVALID;
    if (c->poisoned || !c->has_state) return rfail(c, LB_E_STATE, "fields not initialised or context poisoned");
    if (c->p.force_method != LB_FORCE_LOG || lb_ctx_mrt(c) ||
        (c->p.precision != LB_FP64 && c->p.precision != LB_FP32_MIXED && c->p.precision != LB_FP32_DFMU))
        return rfail(c, LB_E_INVALID,
                     "the adjoint rollout needs the log force, the BGK collision and FP64, FP32_MIXED or "
                     "FP32_DFMU precision");
    DeviceGuard dg(c->p.device);
    if (!dg.ok()) return rfail(c, LB_E_CUDA, "cudaSetDevice");
    for (void *p : c->ckpt) cudaFree(p);
    c->ckpt.clear();
    c->rollout_steps = -1;
    const size_t bytes = c->elem * (size_t)c->p.ncomp * c->Q * c->n;
    const int64_t nck = nsteps / ckpt_every + 1;
    for (int64_t k = 0; k < nck; ++k) {
        void *p = nullptr;
        if (cudaMalloc(&p, bytes) != cudaSuccess) {
            cudaGetLastError();
            for (void *q : c->ckpt) cudaFree(q);
            c->ckpt.clear();
            return rfail(c, LB_E_NOMEM, "checkpoint allocation");
        }
        c->ckpt.push_back(p);
    }
    c->ckpt_every = ckpt_every;
    // one lb_step call per segment between checkpoints (chained where the configuration
    // chains: the same bits as single steps, so the backward recompute repeats them)
    for (int64_t t = 0; t < nsteps;) {
        if (t % ckpt_every == 0) {
            if (cudaMemcpyAsync(c->ckpt[t / ckpt_every], c->f[c->cur], bytes, cudaMemcpyDeviceToDevice, c->stream) !=
                cudaSuccess)
                return rfail(c, LB_E_CUDA, "checkpoint copy");
        }
        int64_t seg = ckpt_every - t % ckpt_every;
        if (seg > nsteps - t) seg = nsteps - t;
        lb_status s = lb_step(c, seg);
        if (s != LB_OK) return s;
        t += seg;
    }
    c->rollout_steps = nsteps;
    return LB_OK;
}

lb_status lb_rollout_backward(lb_ctx *c, const double *rho_bar_T, double *rho_bar_0, double *grad) {
    if (!c || !rho_bar_T) return LB_E_INVALID;
    if (c->rollout_steps < 1) return rfail(c, LB_E_STATE, "no recorded rollout");
    DeviceGuard dg(c->p.device);
    if (!dg.ok()) return rfail(c, LB_E_CUDA, "cudaSetDevice");
    return c->p.precision == LB_FP64 ? backward<double>(c, rho_bar_T, rho_bar_0, grad)
                                     : backward<float>(c, rho_bar_T, rho_bar_0, grad);
}

}  // extern "C"
