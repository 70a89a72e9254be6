// lb_api.cu -- the C ABI declared in include/lbvdw.h: context management,
// argument validation, launches on the context stream and read-back.
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <string>

#include "lbvdw.h"
#include "lb_device_guard.cuh"
#include "lb_launch.cuh"

using namespace lbvdw;

#include "lb_ctx.cuh"

namespace {

const char *k_status[] = {"LB_OK", "LB_E_INVALID", "LB_E_NOMEM", "LB_E_CUDA",
                          "LB_E_DOMAIN", "LB_E_TIMEOUT", "LB_E_STATE"};

lb_status fail(lb_ctx *c, lb_status s, const std::string &m) {
    if (c) {
        c->msg = m;
        if (s == LB_E_DOMAIN || s == LB_E_CUDA || s == LB_E_TIMEOUT) c->poisoned = true;
    }
    return s;
}

lb_status cuda_fail(lb_ctx *c, cudaError_t e, const char *where) {
    return fail(c, LB_E_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define LB_CUDA(ctx, call)                                         \
    do {                                                           \
        cudaError_t e_ = (call);                                   \
        if (e_ != cudaSuccess) return cuda_fail((ctx), e_, #call); \
    } while (0)

bool symmetric(const double *m, int N) {
    for (int i = 0; i < N; ++i)
        for (int j = 0; j < N; ++j)
            if (m[i * 4 + j] != m[j * 4 + i]) return false;
    return true;
}

bool finite_all(const double *m, int cnt) {
    for (int i = 0; i < cnt; ++i)
        if (!std::isfinite(m[i])) return false;
    return true;
}

}  // namespace

// Whether relaxation times other than tau were asked for (the moment-space collision).
bool lb_ctx_mrt(const lb_ctx *c) {
    const double t = c->p.tau, ts = c->p.tau_shear, tg = c->p.tau_ghost;
    return (ts != 0.0 && ts != t) || (tg != 0.0 && tg != t);
}

// One timestep of the context's lattice, precision and kernel organisation from fin to
// fout (the forward step of lb_step; also the recompute step of the adjoint rollout).
cudaError_t lb_ctx_step(lb_ctx *c, const void *fin, void *fout) {
    StepLaunch a;
    a.fin = fin;
    a.fout = fout;
    a.P = c->dp;
    a.ncomp = c->p.ncomp;
    a.force = c->p.force_method | (lb_ctx_mrt(c) ? 2 : 0);
    a.tile_x = c->p.tile_x;
    a.tile_y = c->p.tile_y;
    a.kernel = c->p.kernel;
    a.segs = c->p.segments;
    a.stream = c->stream;
    const bool d1 = c->p.lattice == LB_D1Q3;
    if (a.kernel == LB_KERNEL_WS) return c->p.precision == LB_FP32 ? d2q9_f32mu_ws(a) : d2q9_df_ws(a);
    if (a.kernel == LB_KERNEL_STRIPS)
        return c->p.precision == LB_FP32_MIXED ? d2q9_tbl_strip(a)
                                               : (c->p.precision == LB_FP32 ? d2q9_f32mu_strip(a) : d2q9_df_strip(a));
    switch (c->p.precision) {
        case LB_FP32: return d1 ? d1q3_f32mu_step(a) : d2q9_f32mu_step(a);
        case LB_FP32_MIXED: return d1 ? d1q3_tbl_step(a) : d2q9_tbl_step(a);
        case LB_FP32_DFMU: return d1 ? d1q3_df_step(a) : d2q9_df_step(a);
        default: return d1 ? d1q3_f64_step(a) : d2q9_f64_step(a);
    }
}

namespace {

cudaError_t run_step(lb_ctx *c) { return lb_ctx_step(c, c->f[c->cur], c->f[c->cur ^ 1]); }

// Bound of one wait for a neighbouring tile's flag in a chained step (a tile takes
// microseconds; the bound only turns a fault into an error instead of a hang).
constexpr unsigned long long CHAIN_WAIT_NS = 1000000000ull;

// Whether lb_step chains consecutive steps of this configuration (lb_chain.cuh): the
// two-component FP32 lane-pair step on 32 x 8 tiles, with every ragged tile at least 3
// nodes wide and high so that a tile's step touches only the 3 x 3 tiles around it.
bool chain_eligible(const lb_params &p) {
    const int rx = p.nx % 32, ry = p.ny % 8;
    return p.lattice == LB_D2Q9 && p.ncomp == 2 && (p.precision == LB_FP32_DFMU || p.precision == LB_FP32) &&
           p.kernel == LB_KERNEL_TILES && p.tile_x == 32 && p.tile_y == 8 && (rx == 0 || rx >= 3) &&
           (ry == 0 || ry >= 3);
}

// Step `k` of a chain of `n` (lb_chain.cuh).
cudaError_t run_chain_step(lb_ctx *c, int64_t k, int64_t n) {
    StepLaunch a;
    a.fin = c->f[c->cur];
    a.fout = c->f[c->cur ^ 1];
    a.P = c->dp;
    a.ncomp = c->p.ncomp;
    a.force = c->p.force_method | (lb_ctx_mrt(c) ? 2 : 0);
    a.tile_x = c->p.tile_x;
    a.tile_y = c->p.tile_y;
    a.kernel = c->p.kernel;
    a.stream = c->stream;
    const int rows = (c->p.ny + 7) / 8;
    ChainArgs ca;
    ca.flag = c->chain_flag;
    ca.step = c->chain_step;
    ca.chained = k > 0 ? 1 : 0;
    ca.flag_rows = c->chain_rows;
    ca.release_rows = k + 1 < n ? c->chain_rows : 0;
    ca.roff = c->chain_roff;
    ca.wait_ns = CHAIN_WAIT_NS;
    ca.evict_first = c->chain_evict_first;
    const bool pdl = k > 0;
    cudaError_t e = c->p.precision == LB_FP32 ? d2q9_f32mu_chain(a, ca, pdl) : d2q9_df_chain(a, ca, pdl);
    if (e == cudaSuccess) {
        c->chain_step += 1u;
        c->chain_roff = (c->chain_roff + 1) % rows;
    }
    return e;
}

FieldLaunch field_args(lb_ctx *c) {
    FieldLaunch a;
    a.f = c->f[c->cur];
    a.rho_in = c->rho;
    a.mom_in = nullptr;
    a.rho_out = c->rho;
    a.mom_out = c->mom;
    a.partial = c->partial;
    a.nparts = c->nparts;
    a.diag_out = c->diag;
    a.P = c->dp;
    a.ncomp = c->p.ncomp;
    a.stream = c->stream;
    return a;
}

cudaError_t run_field(lb_ctx *c, int which, const FieldLaunch &a) {
    bool f32 = c->p.precision != LB_FP64;
    bool d1 = c->p.lattice == LB_D1Q3;
    switch (which) {
        case 0: return d1 ? (f32 ? d1q3_f32_init(a) : d1q3_f64_init(a)) : (f32 ? d2q9_f32_init(a) : d2q9_f64_init(a));
        case 1: return d1 ? (f32 ? d1q3_f32_moments(a) : d1q3_f64_moments(a)) : (f32 ? d2q9_f32_moments(a) : d2q9_f64_moments(a));
        default: return d1 ? (f32 ? d1q3_f32_diag(a) : d1q3_f64_diag(a)) : (f32 ? d2q9_f32_diag(a) : d2q9_f64_diag(a));
    }
}

// Synchronise the stream and turn a flagged device error into a status.
lb_status sync_check(lb_ctx *c) {
    unsigned h = 0;
    LB_CUDA(c, cudaMemcpyAsync(&h, c->err, sizeof(unsigned), cudaMemcpyDeviceToHost, c->stream));
    LB_CUDA(c, cudaStreamSynchronize(c->stream));
    if (h & ERR_TIMEOUT) return fail(c, LB_E_TIMEOUT, "a step kernel's wait for its bulk copies ran out");
    if (h & ERR_STALL) return fail(c, LB_E_TIMEOUT, "a chained step's wait for a neighbouring tile ran out");
    if (h & ERR_DOMAIN) return fail(c, LB_E_DOMAIN, "a density or eta <= 0, or a non-finite value, was met");
    return LB_OK;
}

lb_status usable(lb_ctx *c) {
    if (!c) return LB_E_INVALID;
    if (c->poisoned) return fail(c, LB_E_STATE, "context poisoned by an earlier error; set the fields again");
    if (!c->has_state) return fail(c, LB_E_STATE, "fields not initialised");
    return LB_OK;
}

uint64_t params_hash(const lb_params &p) {
    uint64_t h = 1469598103934665603ull;
    auto mix = [&h](const void *d, size_t nb) {
        const unsigned char *b = static_cast<const unsigned char *>(d);
        for (size_t i = 0; i < nb; ++i) { h ^= b[i]; h *= 1099511628211ull; }
    };
    mix(&p.lattice, sizeof p.lattice); mix(&p.nx, sizeof p.nx); mix(&p.ny, sizeof p.ny);
    mix(&p.ncomp, sizeof p.ncomp); mix(&p.precision, sizeof p.precision);
    mix(&p.tau, sizeof p.tau); mix(&p.kT, sizeof p.kT); mix(&p.gamma_mu, sizeof p.gamma_mu);
    mix(p.a, sizeof p.a); mix(p.kappa, sizeof p.kappa); mix(p.lambda, sizeof p.lambda); mix(p.b, sizeof p.b);
    return h;
}

struct StateHeader {
    char magic[8];
    uint32_t abi, lattice;
    int32_t nx, ny, ncomp, precision;
    int64_t steps;
    uint64_t hash;
    double rho_ref_sum;
    char pad[8];
};
static_assert(sizeof(StateHeader) == 64, "state header is 64 bytes");

void split_float(double v, float &hi, float &lo) {
    hi = (float)v;
    lo = (float)(v - (double)hi);
}

}  // namespace

namespace lbvdw {

// Tables of the table-driven logarithms (lb_mu.cuh).  c_j = 1 + j/128; r_j = 1/c_j
// rounded to the working type; T_j = -ln(r_j) in extended precision, split into
// hi + lo.  ln 2 comes from its decimal expansion.
constexpr const char *LN2_DIGITS = "0.69314718055994530941723212145817656807550013436";

void fill_log_tables(LogTables *t) {
    const long double ln2 = strtold(LN2_DIGITS, nullptr);
    for (int j = 0; j < LOG_TBL; ++j) {
        long double cj = 1.0L + (long double)j / LOG_TBL;
        double r64 = (double)(1.0L / cj);
        long double T64 = -logl((long double)r64);
        t->r64[j] = r64;
        t->t64_hi[j] = (double)T64;
        t->t64_lo[j] = (double)(T64 - (long double)t->t64_hi[j]);
        float r32 = (float)(1.0L / cj);
        long double T32 = -logl((long double)r32);
        const float t32_hi = (float)T32;
        t->t32[j] = make_float4(r32, t32_hi, (float)(T32 - (long double)t32_hi), 0.0f);
    }
    // FP64 hi: ln 2 with its low 21 significand bits cleared (e * hi exact for |e| < 2^10)
    double h = (double)ln2;
    uint64_t bits;
    std::memcpy(&bits, &h, sizeof bits);
    bits &= ~((uint64_t(1) << 21) - 1);
    std::memcpy(&h, &bits, sizeof bits);
    t->ln2_hi_d = h;
    t->ln2_lo_d = (double)(ln2 - (long double)h);
    t->ln2_hi_f = (float)ln2;
    t->ln2_lo_f = (float)(ln2 - (long double)t->ln2_hi_f);
}

// Kernel parameter block of a parameter set (FP64 values, their FP32 and double-float
// copies, Psi coefficients); reference densities start at zero (set by the init call).
void make_dev_params(const lb_params &p, DevParams &d, unsigned *err, const LogTables *tbl) {
    d = DevParams{};
    d.nx = p.nx;
    d.ny = p.ny;
    d.omega = 1.0 / p.tau;
    d.psi_g = (p.tau - 0.25) / p.tau;
    d.psi_l = 1.0 / (12.0 * p.tau);
    d.kT = p.kT;
    d.gamma = p.gamma_mu;
    for (int k = 0; k < 16; ++k) {
        d.a[k] = p.a[k];
        d.kappa[k] = p.kappa[k];
        d.lam[k] = p.lambda[k];
        d.a2_f[k] = (float)(2.0 * p.a[k]);
        d.kappa_f[k] = (float)p.kappa[k];
        d.lam_f[k] = (float)p.lambda[k];
    }
    for (int k = 0; k < 4; ++k) {
        d.b[k] = p.b[k];
        d.rho_ref[k] = 0.0;
        d.rho_ref_f[k] = 0.0f;
        split_float(p.b[k], d.b_hi[k], d.b_lo[k]);
    }
    d.err = err;
    d.tbl = tbl;
    d.gkT = p.gamma_mu * p.kT;
    d.ikT_f = (float)(1.0 / p.kT);
    d.gkt3_f = (float)(d.gkT / 3.0);
    d.gkt12_f = (float)(d.gkT / 12.0);
    d.gkt2_f = (float)(d.gkT / 2.0);
    split_float(1.0 / (3.0 * d.gkT), d.cnid_hi, d.cnid_lo);
    d.omega_f = (float)d.omega;
    d.psi_g_f = (float)d.psi_g;
    d.psi_l_f = (float)d.psi_l;
    d.omc = 1.0 - d.omega;
    d.omc_f = (float)d.omc;
    d.lam_fr = p.lambda[1] / (1.0 + 0.5 * p.lambda[1]);
    d.lam_fr_f = (float)d.lam_fr;
    const double ts = p.tau_shear > 0.0 ? p.tau_shear : p.tau, tg = p.tau_ghost > 0.0 ? p.tau_ghost : p.tau;
    d.omega_s = 1.0 / ts;
    d.omega_g = 1.0 / tg;
    d.psi_s = (ts - 0.25) / ts;
    d.omega_s_f = (float)d.omega_s;
    d.omega_g_f = (float)d.omega_g;
    d.psi_s_f = (float)d.psi_s;
    const long double ln2 = strtold(LN2_DIGITS, nullptr);
    d.ln2_hi_f = (float)ln2;
    d.ln2_lo_f = (float)(ln2 - (long double)d.ln2_hi_f);
}

// Per-block sums of the N density fields rho[c][s] (s < n) in a fixed order; the partials
// then go through lb_diag_final_kernel, so the means are deterministic.
template <int N>
__global__ void __launch_bounds__(DIAG_THREADS)
    lb_field_sum_kernel(const double *__restrict__ rho, size_t n, double *__restrict__ partial) {
    double acc[N];
#pragma unroll
    for (int k = 0; k < N; ++k) acc[k] = 0.0;
    for (size_t s = blockIdx.x * (size_t)blockDim.x + threadIdx.x; s < n; s += (size_t)gridDim.x * blockDim.x)
#pragma unroll
        for (int k = 0; k < N; ++k) acc[k] += rho[(size_t)k * n + s];
    block_sum<N>(acc, partial + (size_t)blockIdx.x * N);
}

template <int N>
static cudaError_t field_sums(const double *rho, size_t n, double *partial, int nparts, double *out,
                              cudaStream_t st) {
    lb_field_sum_kernel<N><<<nparts, DIAG_THREADS, 0, st>>>(rho, n, partial);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    lb_diag_final_kernel<N><<<1, DIAG_THREADS, 0, st>>>(partial, nparts, out);
    return cudaGetLastError();
}

}  // namespace lbvdw

extern "C" {

void lb_default_params(lb_params *p) {
    if (!p) return;
    std::memset(p, 0, sizeof *p);
    p->abi = LBVDW_ABI;
    p->lattice = LB_D2Q9;
    p->nx = 64;
    p->ny = 64;
    p->ncomp = 2;
    p->precision = LB_FP64;
    p->force_method = LB_FORCE_LOG;
    p->tau = 1.0;
    p->kT = 1.0 / 3.0;
    p->gamma_mu = 1.0;
}

lb_status lb_create(const lb_params *p, lb_ctx **out) {
    if (!p || !out) return LB_E_INVALID;
    *out = nullptr;
    const int N = p->ncomp;
    if (p->abi != LBVDW_ABI) return LB_E_INVALID;
    if (p->lattice != LB_D1Q3 && p->lattice != LB_D2Q9) return LB_E_INVALID;
    if (N < 1 || N > 4) return LB_E_INVALID;
    if (p->precision != LB_FP64 && p->precision != LB_FP32_MIXED && p->precision != LB_FP32_DFMU &&
        p->precision != LB_FP32)
        return LB_E_INVALID;
    if (p->force_method != LB_FORCE_LOG && p->force_method != LB_FORCE_NID) return LB_E_INVALID;
    if (p->nx < 2) return LB_E_INVALID;
    if (p->lattice == LB_D1Q3 ? p->ny != 1 : p->ny < 2) return LB_E_INVALID;
    if ((int64_t)p->nx * p->ny > (int64_t)1 << 31) return LB_E_INVALID;
    // FP32 storage: the lane-pair kernels address a component's Q planes with 32-bit offsets
    if (p->precision != LB_FP64 && (int64_t)(p->lattice == LB_D1Q3 ? 3 : 9) * p->nx * p->ny >= (int64_t)1 << 32)
        return LB_E_INVALID;
    if (!(p->tau > 0.5) || !(p->kT > 0.0) || !(p->gamma_mu > 0.0) || !std::isfinite(p->tau) ||
        !std::isfinite(p->kT) || !std::isfinite(p->gamma_mu))
        return LB_E_INVALID;
    if (!finite_all(p->a, 16) || !finite_all(p->kappa, 16) || !finite_all(p->lambda, 16) || !finite_all(p->b, 4) ||
        !finite_all(p->rho_ref, 4))
        return LB_E_INVALID;
    if (!symmetric(p->a, N) || !symmetric(p->kappa, N) || !symmetric(p->lambda, N)) return LB_E_INVALID;
    for (int c = 0; c < N; ++c) {
        if (!(p->b[c] > 0.0) || p->rho_ref[c] < 0.0) return LB_E_INVALID;
        for (int cc = 0; cc < N; ++cc)
            if (cc != c && p->lambda[c * 4 + cc] < 0.0) return LB_E_INVALID;
    }
    if (p->check_every < 0) return LB_E_INVALID;
    // moment-space collision: 1/2 < tau_shear <= tau (0 = tau), tau_ghost > 1/2 (0 = tau);
    // D2Q9 tiles of 32 x 8 only
    if (!std::isfinite(p->tau_shear) || !std::isfinite(p->tau_ghost)) return LB_E_INVALID;
    if (p->tau_shear != 0.0 && !(p->tau_shear > 0.5 && p->tau_shear <= p->tau)) return LB_E_INVALID;
    if (p->tau_ghost != 0.0 && !(p->tau_ghost > 0.5)) return LB_E_INVALID;
    const bool mrt = (p->tau_shear != 0.0 && p->tau_shear != p->tau) || (p->tau_ghost != 0.0 && p->tau_ghost != p->tau);
    if (mrt && (p->lattice != LB_D2Q9 || p->kernel == LB_KERNEL_STRIPS ||
                !((p->tile_x == 0 && p->tile_y == 0) || (p->tile_x == 32 && p->tile_y == 8))))
        return LB_E_INVALID;
    if (p->kernel < LB_KERNEL_AUTO || p->kernel > LB_KERNEL_WS || p->segments < 0) return LB_E_INVALID;
    if (p->kernel == LB_KERNEL_WS &&
        (p->lattice != LB_D2Q9 || N != 2 || (p->precision != LB_FP32_DFMU && p->precision != LB_FP32) ||
         !((p->tile_x == 0 && p->tile_y == 0) || (p->tile_x == 32 && p->tile_y == 8))))
        return LB_E_INVALID;

    lb_ctx *c = new (std::nothrow) lb_ctx;
    if (!c) return LB_E_NOMEM;
    c->p = *p;
    // kernel organisation: AUTO takes tiles, the faster organisation on GB300 for every
    // measured workload (strips hold two CTAs per SM, too few warps to hide latency)
    const bool no_tile = p->tile_x == 0 && p->tile_y == 0;
    const bool strips_ok = p->lattice == LB_D2Q9 && p->precision != LB_FP64 && strip_shape_ok(p->nx, p->ny, N);
    int kind = p->kernel;
    if (kind == LB_KERNEL_AUTO) kind = LB_KERNEL_TILES;
    c->p.kernel = kind;
    bool tile_ok;
    if (kind == LB_KERNEL_WS) {
        c->p.tile_x = 32;
        c->p.tile_y = 8;
        tile_ok = true;
    } else if (kind == LB_KERNEL_STRIPS) {
        if (no_tile) {
            c->p.tile_x = STRIP_TX;
            c->p.tile_y = strip_ty(N);
        }
        tile_ok = strips_ok && c->p.tile_x == STRIP_TX && c->p.tile_y == strip_ty(N);
    } else {
        if (no_tile) {
            c->p.tile_x = p->lattice == LB_D1Q3 ? 128 : 32;
            c->p.tile_y = p->lattice == LB_D1Q3 ? 1 : 8;
        }
        tile_ok = p->lattice == LB_D1Q3
                      ? (c->p.tile_y == 1 && (c->p.tile_x == 128 || c->p.tile_x == 256))
                      : ((c->p.tile_x == 32 && c->p.tile_y == 8) || (c->p.tile_x == 64 && c->p.tile_y == 4) ||
                         (c->p.tile_x == 32 && c->p.tile_y == 16) || (c->p.tile_x == 64 && c->p.tile_y == 8));
    }
    if (!tile_ok) { delete c; return LB_E_INVALID; }
    c->Q = p->lattice == LB_D1Q3 ? 3 : 9;
    c->D = p->lattice == LB_D1Q3 ? 1 : 2;
    c->n = (size_t)p->nx * p->ny;
    c->elem = p->precision == LB_FP64 ? sizeof(double) : sizeof(float);
    c->stream = static_cast<cudaStream_t>(p->stream);

    DeviceGuard dg(p->device);
    if (!dg.ok()) { delete c; return LB_E_CUDA; }
    size_t fbytes = c->elem * (size_t)N * c->Q * c->n;
    size_t nparts = (c->n + DIAG_THREADS - 1) / DIAG_THREADS;
    if (nparts > 152 * 8) nparts = 152 * 8;
    c->nparts = (int)nparts;
    bool ok = cudaMalloc(&c->f[0], fbytes) == cudaSuccess && cudaMalloc(&c->f[1], fbytes) == cudaSuccess &&
              cudaMalloc(&c->rho, sizeof(double) * N * c->n) == cudaSuccess &&
              cudaMalloc(&c->mom, sizeof(double) * N * c->D * c->n) == cudaSuccess &&
              cudaMalloc(&c->partial, sizeof(double) * (N + 3) * nparts) == cudaSuccess &&
              cudaMalloc(&c->diag, sizeof(double) * (N + 3)) == cudaSuccess &&
              cudaMalloc(&c->err, sizeof(unsigned)) == cudaSuccess &&
              cudaMalloc(&c->tbl, sizeof(LogTables)) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        lb_destroy(c);
        return LB_E_NOMEM;
    }
    make_dev_params(*p, c->dp, c->err, c->tbl);
    LogTables h;
    fill_log_tables(&h);
    if (cudaMemcpy(c->tbl, &h, sizeof h, cudaMemcpyHostToDevice) != cudaSuccess) {
        cudaGetLastError();
        lb_destroy(c);
        return LB_E_CUDA;
    }
    if (chain_eligible(c->p)) {
        // flags of every tile (zero: no chain step done), and the CTA rows of a step that
        // set them: the rows of one wave of the chain kernel (its resident CTAs) plus the
        // two rows the next step's first CTAs reach beyond them, plus one
        // (a failed occupancy or device query leaves the context unchained: chaining only
        // changes when tiles start, not what they compute)
        const int tx = (p->nx + 31) / 32, ty = (p->ny + 7) / 8;
        int sms = 0, dev = 0;
        const int per_sm = p->precision == LB_FP32 ? d2q9_f32mu_chain_ctas_per_sm() : d2q9_df_chain_ctas_per_sm();
        if (per_sm >= 1 && cudaGetDevice(&dev) == cudaSuccess &&
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && sms >= 1) {
            if (cudaMalloc(&c->chain_flag, sizeof(unsigned) * (size_t)tx * ty) != cudaSuccess) {
                cudaGetLastError();
                c->chain_flag = nullptr;
                lb_destroy(c);
                return LB_E_NOMEM;
            }
            if (cudaMemset(c->chain_flag, 0, sizeof(unsigned) * (size_t)tx * ty) != cudaSuccess) {
                cudaGetLastError();
                lb_destroy(c);
                return LB_E_CUDA;
            }
            const int wave_rows = (per_sm * sms + tx - 1) / tx;
            c->chain_rows = wave_rows + 3 < ty ? wave_rows + 3 : ty;
            c->chain_step = 1u;
            // evict-first input where one population buffer takes at most 60 % of the L2
            // (measured on GB300: 1.7 % faster at 1024^2, 75.5 MB of a 126 MB L2; slower from
            // 1152^2 on, 95.6 MB, where the ring re-reads of a step lose the L2)
            int l2 = 0;
            if (cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, dev) == cudaSuccess && l2 > 0)
                c->chain_evict_first = (double)c->elem * N * c->Q * (double)c->n <= 0.6 * l2 ? 1 : 0;
            else
                cudaGetLastError();
        } else {
            cudaGetLastError();
        }
    }
    *out = c;
    return LB_OK;
}

static lb_status init_common(lb_ctx *c, const double *rho_dev, const double *mom_dev, const double *rho_ref) {
    const int N = c->p.ncomp;
    for (int k = 0; k < 4; ++k) c->dp.rho_ref[k] = 0.0;
    // FP32 storage: the reference density is rounded to a float value, so the float
    // kernels and the FP64 moment sums use the same number
    if (c->p.precision != LB_FP64)
        for (int k = 0; k < N; ++k)
            c->dp.rho_ref[k] = (double)(float)(c->p.rho_ref[k] > 0.0 ? c->p.rho_ref[k] : rho_ref[k]);
    for (int k = 0; k < 4; ++k) c->dp.rho_ref_f[k] = (float)c->dp.rho_ref[k];
    LB_CUDA(c, cudaMemsetAsync(c->err, 0, sizeof(unsigned), c->stream));
    c->cur = 0;
    FieldLaunch a = field_args(c);
    a.rho_in = rho_dev;
    a.mom_in = mom_dev;
    a.P = c->dp;
    cudaError_t e = run_field(c, 0, a);
    if (e != cudaSuccess) return cuda_fail(c, e, "init kernel");
    c->launches += 1;
    c->steps = 0;
    c->has_state = true;
    c->poisoned = false;
    c->rollout_steps = -1;
    c->msg.clear();
    return LB_OK;
}

// Mean density of each component for the FP32 reference densities (when the caller
// gave none), through the deterministic diagnostics reduction on the device; the densities
// are expected in c->rho (copied there from rho_dev when it is another buffer).
static lb_status device_mean(lb_ctx *c, const double *rho_dev, double *mean) {
    const int N = c->p.ncomp;
    bool need_mean = false;
    if (c->p.precision != LB_FP64)
        for (int k = 0; k < N; ++k) need_mean = need_mean || !(c->p.rho_ref[k] > 0.0);
    if (!need_mean) return LB_OK;
    cudaError_t e = cudaErrorInvalidValue;
    switch (N) {
        case 1: e = field_sums<1>(rho_dev, c->n, c->partial, c->nparts, c->diag, c->stream); break;
        case 2: e = field_sums<2>(rho_dev, c->n, c->partial, c->nparts, c->diag, c->stream); break;
        case 3: e = field_sums<3>(rho_dev, c->n, c->partial, c->nparts, c->diag, c->stream); break;
        case 4: e = field_sums<4>(rho_dev, c->n, c->partial, c->nparts, c->diag, c->stream); break;
    }
    if (e != cudaSuccess) return cuda_fail(c, e, "field sum kernel");
    c->launches += 2;
    double h[4];
    LB_CUDA(c, cudaMemcpyAsync(h, c->diag, sizeof(double) * N, cudaMemcpyDeviceToHost, c->stream));
    LB_CUDA(c, cudaStreamSynchronize(c->stream));
    for (int k = 0; k < N; ++k) mean[k] = h[k] / (double)c->n;
    return LB_OK;
}

lb_status lb_init_fields(lb_ctx *c, const double *rho, const double *mom) {
    if (!c || !rho) return LB_E_INVALID;
    const int N = c->p.ncomp;
    DeviceGuard dg(c->p.device);
    LB_CUDA(c, dg.status);
    // the fields go to the device first; the reference densities and the domain check
    // (in the init kernel) are computed there
    LB_CUDA(c, cudaMemcpyAsync(c->rho, rho, sizeof(double) * N * c->n, cudaMemcpyHostToDevice, c->stream));
    double mean[4] = {0, 0, 0, 0};
    lb_status s = device_mean(c, c->rho, mean);
    if (s != LB_OK) return s;
    if (mom)
        LB_CUDA(c, cudaMemcpyAsync(c->mom, mom, sizeof(double) * N * c->D * c->n, cudaMemcpyHostToDevice, c->stream));
    s = init_common(c, c->rho, mom ? c->mom : nullptr, mean);
    if (s != LB_OK) return s;
    unsigned h = 0;
    LB_CUDA(c, cudaMemcpyAsync(&h, c->err, sizeof(unsigned), cudaMemcpyDeviceToHost, c->stream));
    LB_CUDA(c, cudaStreamSynchronize(c->stream));
    if (h & ERR_DOMAIN) {
        c->has_state = false;
        return fail(c, LB_E_DOMAIN, "a density <= 0, eta = 1 - sum b rho <= 0 or a non-finite value in the fields");
    }
    return LB_OK;
}

lb_status lb_init_fields_dev(lb_ctx *c, const double *rho_dev, const double *mom_dev) {
    if (!c || !rho_dev) return LB_E_INVALID;
    DeviceGuard dg(c->p.device);
    LB_CUDA(c, dg.status);
    double mean[4] = {0, 0, 0, 0};
    lb_status s = device_mean(c, rho_dev, mean);
    if (s != LB_OK) return s;
    return init_common(c, rho_dev, mom_dev, mean);
}

lb_status lb_step(lb_ctx *c, int64_t nsteps) {
    lb_status s = usable(c);
    if (s != LB_OK) return s;
    DeviceGuard dg(c->p.device);
    LB_CUDA(c, dg.status);
    if (nsteps < 0) return fail(c, LB_E_INVALID, "nsteps < 0");
    // two or more steps of a chaining configuration: one chain (lb_chain.cuh), cut where
    // the host checks the error word.  Not while the stream is being captured: a replayed
    // graph would repeat the step numbers its launches were captured with, and flags left
    // by an earlier replay would release tiles early.
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    LB_CUDA(c, cudaStreamIsCapturing(c->stream, &cap));
    const bool chain = c->chain_flag != nullptr && nsteps >= 2 && cap == cudaStreamCaptureStatusNone;
    int64_t k = 0;  // step within the current chain
    for (int64_t t = 0; t < nsteps; ++t) {
        cudaError_t e;
        if (chain) {
            int64_t left = nsteps - t;
            if (c->p.check_every > 0) {
                const int64_t to_check = c->p.check_every - c->steps % c->p.check_every;
                if (to_check < left) left = to_check;
            }
            // a chain of one step is the plain step
            e = (k == 0 && left == 1) ? run_step(c) : run_chain_step(c, k, k + left);
            k = left == 1 ? 0 : k + 1;
        } else {
            e = run_step(c);
        }
        if (e != cudaSuccess) return cuda_fail(c, e, "step kernel");
        c->cur ^= 1;
        c->steps += 1;
        c->launches += 1;
        if (c->p.check_every > 0 && c->steps % c->p.check_every == 0) {
            s = sync_check(c);
            if (s != LB_OK) return s;
        }
    }
    return LB_OK;
}

lb_status lb_read_moments_dev(lb_ctx *c, double *rho_dev, double *mom_dev) {
    lb_status s = usable(c);
    if (s != LB_OK) return s;
    DeviceGuard dg(c->p.device);
    LB_CUDA(c, dg.status);
    if (!rho_dev) return fail(c, LB_E_INVALID, "rho output is NULL");
    FieldLaunch a = field_args(c);
    a.rho_out = rho_dev;
    a.mom_out = mom_dev;
    cudaError_t e = run_field(c, 1, a);
    if (e != cudaSuccess) return cuda_fail(c, e, "moments kernel");
    c->launches += 1;
    return LB_OK;
}

lb_status lb_read_moments(lb_ctx *c, double *rho, double *mom) {
    lb_status s = usable(c);
    if (s != LB_OK) return s;
    DeviceGuard dg(c->p.device);
    LB_CUDA(c, dg.status);
    if (!rho) return fail(c, LB_E_INVALID, "rho output is NULL");
    const int N = c->p.ncomp;
    FieldLaunch a = field_args(c);
    cudaError_t e = run_field(c, 1, a);
    if (e != cudaSuccess) return cuda_fail(c, e, "moments kernel");
    c->launches += 1;
    LB_CUDA(c, cudaMemcpyAsync(rho, c->rho, sizeof(double) * N * c->n, cudaMemcpyDeviceToHost, c->stream));
    if (mom)
        LB_CUDA(c, cudaMemcpyAsync(mom, c->mom, sizeof(double) * N * c->D * c->n, cudaMemcpyDeviceToHost, c->stream));
    return sync_check(c);
}

lb_status lb_free_energy(lb_ctx *c, double *F, double *mass, double *mom_total) {
    lb_status s = usable(c);
    if (s != LB_OK) return s;
    DeviceGuard dg(c->p.device);
    LB_CUDA(c, dg.status);
    if (!F) return fail(c, LB_E_INVALID, "F output is NULL");
    const int N = c->p.ncomp;
    FieldLaunch a = field_args(c);
    cudaError_t e = run_field(c, 1, a);
    if (e != cudaSuccess) return cuda_fail(c, e, "moments kernel");
    e = run_field(c, 2, a);
    if (e != cudaSuccess) return cuda_fail(c, e, "diag kernel");
    c->launches += 3;
    double h[7];
    LB_CUDA(c, cudaMemcpyAsync(h, c->diag, sizeof(double) * (N + 3), cudaMemcpyDeviceToHost, c->stream));
    s = sync_check(c);
    if (s != LB_OK) return s;
    *F = h[N];
    if (mass)
        for (int k = 0; k < N; ++k) mass[k] = h[k];
    if (mom_total) {
        mom_total[0] = h[N + 1];
        mom_total[1] = c->D == 2 ? h[N + 2] : 0.0;
    }
    return LB_OK;
}

size_t lb_state_bytes(const lb_ctx *c) {
    if (!c) return 0;
    return sizeof(StateHeader) + c->elem * (size_t)c->p.ncomp * c->Q * c->n;
}

lb_status lb_save_state(lb_ctx *c, void *buf, size_t bytes) {
    lb_status s = usable(c);
    if (s != LB_OK) return s;
    DeviceGuard dg(c->p.device);
    LB_CUDA(c, dg.status);
    if (!buf || bytes < lb_state_bytes(c)) return fail(c, LB_E_INVALID, "state buffer too small");
    StateHeader h;
    std::memset(&h, 0, sizeof h);
    std::memcpy(h.magic, "LBVDWST1", 8);
    h.abi = LBVDW_ABI;
    h.lattice = (uint32_t)c->p.lattice;
    h.nx = c->p.nx; h.ny = c->p.ny; h.ncomp = c->p.ncomp; h.precision = c->p.precision;
    h.steps = c->steps;
    h.hash = params_hash(c->p);
    h.rho_ref_sum = 0.0;
    for (int k = 0; k < 4; ++k) h.rho_ref_sum += c->dp.rho_ref[k] * (k + 1);
    std::memcpy(buf, &h, sizeof h);
    char *dst = static_cast<char *>(buf) + sizeof h;
    LB_CUDA(c, cudaMemcpyAsync(dst, c->f[c->cur], lb_state_bytes(c) - sizeof h, cudaMemcpyDeviceToHost, c->stream));
    return sync_check(c);
}

lb_status lb_load_state(lb_ctx *c, const void *buf, size_t bytes) {
    if (!c || !buf || bytes < lb_state_bytes(c)) return LB_E_INVALID;
    StateHeader h;
    std::memcpy(&h, buf, sizeof h);
    if (std::memcmp(h.magic, "LBVDWST1", 8) != 0 || h.abi != LBVDW_ABI || h.lattice != (uint32_t)c->p.lattice ||
        h.nx != c->p.nx || h.ny != c->p.ny || h.ncomp != c->p.ncomp || h.precision != c->p.precision ||
        h.hash != params_hash(c->p))
        return fail(c, LB_E_INVALID, "saved state does not match this context");
    DeviceGuard dg(c->p.device);
    LB_CUDA(c, dg.status);
    if (c->p.precision != LB_FP64) {
        double sum = 0.0;
        for (int k = 0; k < 4; ++k) sum += c->dp.rho_ref[k] * (k + 1);
        if (!c->has_state || sum != h.rho_ref_sum)
            return fail(c, LB_E_INVALID, "mixed-precision state needs the same reference densities (init first)");
    }
    const char *src = static_cast<const char *>(buf) + sizeof h;
    c->cur = 0;
    LB_CUDA(c, cudaMemcpyAsync(c->f[0], src, lb_state_bytes(c) - sizeof h, cudaMemcpyHostToDevice, c->stream));
    LB_CUDA(c, cudaMemsetAsync(c->err, 0, sizeof(unsigned), c->stream));
    LB_CUDA(c, cudaStreamSynchronize(c->stream));
    c->steps = h.steps;
    c->has_state = true;
    c->poisoned = false;
    c->msg.clear();
    return LB_OK;
}

int64_t lb_step_count(const lb_ctx *c) { return c ? c->steps : -1; }

int64_t lb_launch_count(const lb_ctx *c) { return c ? c->launches : -1; }

int32_t lb_chain_rows(const lb_ctx *c) { return c ? (c->chain_flag ? c->chain_rows : 0) : -1; }

int32_t lb_chain_evict_first(const lb_ctx *c) { return c ? (c->chain_flag ? c->chain_evict_first : 0) : -1; }

lb_status lb_get_params(const lb_ctx *c, lb_params *out) {
    if (!c || !out) return LB_E_INVALID;
    *out = c->p;
    return LB_OK;
}

lb_status lb_destroy(lb_ctx *c) {
    if (!c) return LB_OK;
    DeviceGuard dg(c->p.device);
    if (c->stream) cudaStreamSynchronize(c->stream);
    else cudaDeviceSynchronize();
    cudaFree(c->f[0]);
    cudaFree(c->f[1]);
    cudaFree(c->rho);
    cudaFree(c->mom);
    cudaFree(c->partial);
    cudaFree(c->diag);
    cudaFree(c->err);
    cudaFree(c->tbl);
    cudaFree(c->chain_flag);
    for (void *q : c->ckpt) cudaFree(q);
    delete c;
    return LB_OK;
}

const char *lb_status_str(lb_status s) {
    int k = (int)s;
    return (k >= 0 && k <= 6) ? k_status[k] : "LB_E_UNKNOWN";
}

const char *lb_last_error(const lb_ctx *c) {
    if (!c) return "NULL context";
    return c->msg.c_str();
}

}  // extern "C"
