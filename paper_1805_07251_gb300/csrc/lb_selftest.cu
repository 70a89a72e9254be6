// lb_selftest.cu -- device self-test of the chemical-potential logarithms
// (include/lbvdw_selftest.h).
#include <cstring>

#include "lb_chain.cuh"
#include "lb_device_guard.cuh"
#include "lb_kernels.cuh"
#include "lb_strip.cuh"
#include "lbvdw_selftest.h"

namespace lbvdw {
void fill_log_tables(LogTables *t);
}

namespace {

__global__ void selftest_log_kernel(const double *x, long long n, const lbvdw::LogTables *tb, double *o_tbl,
                                    double *o_df, double *o_ref) {
    long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (k >= n) return;
    double v = x[k];
    o_tbl[k] = lbvdw::log64_tbl(v, tb->r64, tb->t64_hi, tb->t64_lo, tb->ln2_hi_d, tb->ln2_lo_d);
    lbvdw::df d = lbvdw::df_log(lbvdw::df_from_double(v), tb->t32, tb->ln2_hi_f, tb->ln2_lo_f);
    o_df[k] = lbvdw::df_to_double(d);
    o_ref[k] = log(v);
}

// 1/x through the double-float reciprocal of the chemical-potential stage (1/eta)
__global__ void selftest_recip_kernel(const double *x, long long n, double *o_df) {
    long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (k >= n) return;
    o_df[k] = lbvdw::df_to_double(lbvdw::df_recip(lbvdw::df_from_double(x[k])));
}

// The bounded mbarrier wait of the streaming-strip kernel on a barrier that completes
// (thread 0 arrives) or never does (nobody arrives): the wait must end either way and
// report the second case in the flag.
__global__ void selftest_wait_kernel(unsigned *flag, unsigned polls, int arrive) {
    __shared__ unsigned long long bar;
    if (threadIdx.x == 0) {
        lbvdw::mbar_init(&bar, 1);
        lbvdw::fence_barrier_init();
    }
    __syncthreads();
    if (arrive && threadIdx.x == 0)
        asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.shared::cta.b64 st, [%0];\n\t}" ::"r"(
                         lbvdw::smem_addr(&bar))
                     : "memory");
    if (!lbvdw::mbar_wait_bounded(&bar, 0, polls)) atomicOr(flag, lbvdw::ERR_TIMEOUT);
}

// The bounded flag wait of the chained steps: one thread waits for flag[0] to reach
// `step`; a wait that runs out sets the stall bit in *err.
__global__ void selftest_flag_wait_kernel(const unsigned *flag, unsigned step, unsigned long long wait_ns,
                                          unsigned *err) {
    if (threadIdx.x == 0) lbvdw::wait_flag(flag, 0, step, wait_ns, err);
}

}  // namespace

extern "C" lb_status lb_selftest_flag_wait(int32_t device, uint64_t wait_ns, int32_t set, uint32_t *flag) {
    if (!flag || wait_ns < 1 || wait_ns > 10000000000ull) return LB_E_INVALID;
    lbvdw::DeviceGuard dg(device);
    if (!dg.ok()) return LB_E_CUDA;
    unsigned *d = nullptr;  // [0] the awaited flag, [1] the error word
    if (cudaMalloc(&d, 2 * sizeof(unsigned)) != cudaSuccess) {
        cudaGetLastError();
        return LB_E_NOMEM;
    }
    const unsigned step = 7u;
    const unsigned h[2] = {set ? step : step - 1u, 0u};
    lb_status st = LB_OK;
    if (cudaMemcpy(d, h, sizeof h, cudaMemcpyHostToDevice) != cudaSuccess) {
        st = LB_E_CUDA;
    } else {
        selftest_flag_wait_kernel<<<1, 32>>>(d, step, (unsigned long long)wait_ns, d + 1);
        if (cudaGetLastError() != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess ||
            cudaMemcpy(flag, d + 1, sizeof(unsigned), cudaMemcpyDeviceToHost) != cudaSuccess)
            st = LB_E_CUDA;
    }
    cudaFree(d);
    return st;
}

extern "C" lb_status lb_selftest_wait(int32_t device, uint32_t polls, int32_t arrive, uint32_t *flag) {
    if (!flag || polls < 1) return LB_E_INVALID;
    lbvdw::DeviceGuard dg(device);
    if (!dg.ok()) return LB_E_CUDA;
    unsigned *d = nullptr;
    if (cudaMalloc(&d, sizeof(unsigned)) != cudaSuccess) {
        cudaGetLastError();
        return LB_E_NOMEM;
    }
    lb_status st = LB_OK;
    if (cudaMemset(d, 0, sizeof(unsigned)) != cudaSuccess) {
        st = LB_E_CUDA;
    } else {
        selftest_wait_kernel<<<1, 64>>>(d, polls, arrive);
        if (cudaGetLastError() != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess ||
            cudaMemcpy(flag, d, sizeof(unsigned), cudaMemcpyDeviceToHost) != cudaSuccess)
            st = LB_E_CUDA;
    }
    cudaFree(d);
    return st;
}

extern "C" lb_status lb_selftest_log(int32_t device, const double *x, int64_t n, double *out_tbl, double *out_df,
                                     double *out_ref) {
    if (!x || !out_tbl || !out_df || !out_ref || n < 1) return LB_E_INVALID;
    lbvdw::DeviceGuard dg(device);
    if (!dg.ok()) return LB_E_CUDA;
    lbvdw::LogTables h;
    lbvdw::fill_log_tables(&h);
    double *d = nullptr;
    lbvdw::LogTables *tb = nullptr;
    size_t bytes = sizeof(double) * (size_t)n;
    if (cudaMalloc(&d, 4 * bytes) != cudaSuccess || cudaMalloc(&tb, sizeof h) != cudaSuccess) {
        cudaFree(d);
        cudaGetLastError();
        return LB_E_NOMEM;
    }
    lb_status st = LB_OK;
    if (cudaMemcpy(d, x, bytes, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(tb, &h, sizeof h, cudaMemcpyHostToDevice) != cudaSuccess) {
        st = LB_E_CUDA;
    } else {
        unsigned grid = (unsigned)((n + 255) / 256);
        selftest_log_kernel<<<grid, 256>>>(d, n, tb, d + n, d + 2 * n, d + 3 * n);
        if (cudaGetLastError() != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess ||
            cudaMemcpy(out_tbl, d + n, bytes, cudaMemcpyDeviceToHost) != cudaSuccess ||
            cudaMemcpy(out_df, d + 2 * n, bytes, cudaMemcpyDeviceToHost) != cudaSuccess ||
            cudaMemcpy(out_ref, d + 3 * n, bytes, cudaMemcpyDeviceToHost) != cudaSuccess)
            st = LB_E_CUDA;
    }
    cudaFree(d);
    cudaFree(tb);
    return st;
}

extern "C" lb_status lb_selftest_recip(int32_t device, const double *x, int64_t n, double *out_df) {
    if (!x || !out_df || n < 1) return LB_E_INVALID;
    lbvdw::DeviceGuard dg(device);
    if (!dg.ok()) return LB_E_CUDA;
    double *d = nullptr;
    size_t bytes = sizeof(double) * (size_t)n;
    if (cudaMalloc(&d, 2 * bytes) != cudaSuccess) {
        cudaGetLastError();
        return LB_E_NOMEM;
    }
    lb_status st = LB_OK;
    if (cudaMemcpy(d, x, bytes, cudaMemcpyHostToDevice) != cudaSuccess) {
        st = LB_E_CUDA;
    } else {
        unsigned grid = (unsigned)((n + 255) / 256);
        selftest_recip_kernel<<<grid, 256>>>(d, n, d + n);
        if (cudaGetLastError() != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess ||
            cudaMemcpy(out_df, d + n, bytes, cudaMemcpyDeviceToHost) != cudaSuccess)
            st = LB_E_CUDA;
    }
    cudaFree(d);
    return st;
}
