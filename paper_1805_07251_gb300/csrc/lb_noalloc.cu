// lb_noalloc.cu -- lb_free_energy_noalloc: the diagnostics reduction (moments, then
// per-CTA FP64 partials, then one CTA) with all of its scratch in one file-scope
// device array instead of buffers allocated by a context.
//
// Some callers cannot allocate device memory at the point where they want these
// numbers: code running inside another framework's memory pool or under a fixed
// memory budget, tools that inspect a simulation state handed to them as a bare
// device pointer, and callers that must not trigger an allocation (and the implicit
// synchronisation cudaMalloc/cudaFree can cause) in the middle of their own stream
// work.  This entry point takes the populations and an output pointer from the caller
// and touches no allocator: no cudaMalloc, cudaFree or allocating library routine.
//
// The scratch array (NOALLOC_SCRATCH_DOUBLES doubles, 16 MiB) is a static __device__
// object, so every GPU that loads the library holds it until the process exits.  It is
// shared by every call on a device and keeps the last call's contents; the error word is
// cleared at the start of each call.  Calls that overlap on the GPU (on different
// streams, or from different host threads) race on it: serialise them.  In host code the
// symbol is only a host-side stand-in, so every call looks up the array's device address
// with cudaGetSymbolAddress (the call's device current; the lookup allocates nothing).
// Looking it up on every call, rather than caching it, keeps the address right after a
// device reset or a new primary context.  The first call on a device also loads the
// library's module there, so make it before any stream capture.  The caller's current
// device is restored before the call returns.
#include "lb_device_guard.cuh"
#include "lb_kernels.cuh"
#include "lbvdw.h"

namespace {

using namespace lbvdw;

// moments [N][n] + [N][D][n] doubles, then partials [NOALLOC_MAX_PARTS][N + 3], then the
// error word (one double slot)
constexpr size_t NOALLOC_SCRATCH_DOUBLES = size_t(1) << 21;
constexpr int NOALLOC_MAX_PARTS = 1024;
constexpr size_t NOALLOC_PARTIAL_DOUBLES = size_t(NOALLOC_MAX_PARTS) * 7;
constexpr size_t NOALLOC_FIELD_DOUBLES = NOALLOC_SCRATCH_DOUBLES - NOALLOC_PARTIAL_DOUBLES - 1;

static __device__ __align__(256) double g_noalloc_scratch[NOALLOC_SCRATCH_DOUBLES];

// device address of the scratch array on the current device
cudaError_t scratch_address(double **out) {
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    *out = static_cast<double *>(p);
    return cudaSuccess;
}

__global__ void noalloc_flag_kernel(const unsigned *err, double *out) { *out = (*err != 0u) ? 1.0 : 0.0; }

template <int LAT, int N, class S>
cudaError_t run(const DevParams &P, const S *f, double *scratch, double *out, cudaStream_t st) {
    const size_t n = (size_t)P.nx * P.ny;
    double *rho = scratch;
    double *mom = scratch + (size_t)N * n;
    double *partial = scratch + NOALLOC_FIELD_DOUBLES;
    unsigned *err = reinterpret_cast<unsigned *>(scratch + NOALLOC_FIELD_DOUBLES + NOALLOC_PARTIAL_DOUBLES);
    DevParams Q = P;
    Q.err = err;
    cudaError_t e = cudaMemsetAsync(err, 0, sizeof(unsigned), st);
    if (e != cudaSuccess) return e;
    size_t g = (n + 255) / 256;
    if (g > 152 * 16) g = 152 * 16;
    lb_moments_kernel<LAT, N, S><<<(unsigned)g, 256, 0, st>>>(f, rho, mom, Q);
    int parts = (int)((n + DIAG_THREADS - 1) / DIAG_THREADS);
    if (parts > NOALLOC_MAX_PARTS) parts = NOALLOC_MAX_PARTS;
    lb_diag_partial_kernel<LAT, N><<<parts, DIAG_THREADS, 0, st>>>(rho, mom, partial, Q);
    lb_diag_final_kernel<N + 3><<<1, DIAG_THREADS, 0, st>>>(partial, parts, out);
    noalloc_flag_kernel<<<1, 1, 0, st>>>(err, out + N + 3);
    return cudaGetLastError();
}

template <int LAT, class S>
cudaError_t run_n(int N, const DevParams &P, const S *f, double *scratch, double *out, cudaStream_t st) {
    switch (N) {
        case 1: return run<LAT, 1, S>(P, f, scratch, out, st);
        case 2: return run<LAT, 2, S>(P, f, scratch, out, st);
        case 3: return run<LAT, 3, S>(P, f, scratch, out, st);
        case 4: return run<LAT, 4, S>(P, f, scratch, out, st);
    }
    return cudaErrorInvalidValue;
}

}  // namespace

extern "C" lb_status lb_free_energy_noalloc(const lb_params *p, const void *f_dev, double *out_dev) {
    if (!p || !f_dev || !out_dev) return LB_E_INVALID;
    const int N = p->ncomp;
    if (p->abi != LBVDW_ABI || N < 1 || N > 4) return LB_E_INVALID;
    if (p->lattice != LB_D1Q3 && p->lattice != LB_D2Q9) return LB_E_INVALID;
    if (p->precision != LB_FP64 && p->precision != LB_FP32_MIXED && p->precision != LB_FP32_DFMU &&
        p->precision != LB_FP32)
        return LB_E_INVALID;
    if (p->nx < 2 || (p->lattice == LB_D1Q3 ? p->ny != 1 : p->ny < 2)) return LB_E_INVALID;
    const size_t n = (size_t)p->nx * (size_t)p->ny;
    const size_t D = p->lattice == LB_D1Q3 ? 1 : 2;
    if ((size_t)N * (1 + D) * n > NOALLOC_FIELD_DOUBLES) return LB_E_INVALID;  // beyond the scratch size
    if (!(p->kT > 0.0)) return LB_E_INVALID;
    for (int c = 0; c < N; ++c) {
        if (!(p->b[c] > 0.0)) return LB_E_INVALID;
        if (p->precision != LB_FP64 && !(p->rho_ref[c] > 0.0)) return LB_E_INVALID;
    }
    DeviceGuard dg(p->device);
    if (!dg.ok()) return LB_E_CUDA;
    double *scratch = nullptr;
    if (scratch_address(&scratch) != cudaSuccess) return LB_E_CUDA;

    DevParams P{};
    P.nx = p->nx;
    P.ny = p->ny;
    P.kT = p->kT;
    for (int k = 0; k < 16; ++k) {
        P.a[k] = p->a[k];
        P.kappa[k] = p->kappa[k];
    }
    for (int k = 0; k < 4; ++k) {
        P.b[k] = p->b[k];
        P.rho_ref[k] = p->precision == LB_FP64 ? 0.0 : (double)(float)p->rho_ref[k];
    }
    cudaStream_t st = static_cast<cudaStream_t>(p->stream);
    cudaError_t e;
    if (p->precision == LB_FP64) {
        const double *f = static_cast<const double *>(f_dev);
        e = p->lattice == LB_D1Q3 ? run_n<1>(N, P, f, scratch, out_dev, st) : run_n<2>(N, P, f, scratch, out_dev, st);
    } else {
        const float *f = static_cast<const float *>(f_dev);
        e = p->lattice == LB_D1Q3 ? run_n<1>(N, P, f, scratch, out_dev, st) : run_n<2>(N, P, f, scratch, out_dev, st);
    }
    return e == cudaSuccess ? LB_OK : LB_E_CUDA;
}
