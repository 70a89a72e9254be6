// lb_selftest.cu -- device self-test of the chemical-potential logarithms
// (include/lbvdw_selftest.h).
#include <cstring>

#include "lb_kernels.cuh"
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
    lbvdw::df d = lbvdw::df_log(lbvdw::df_from_double(v), tb->r32, tb->t32_hi, tb->t32_lo, tb->ln2_hi_f,
                                tb->ln2_lo_f);
    o_df[k] = lbvdw::df_to_double(d);
    o_ref[k] = log(v);
}

}  // namespace

extern "C" lb_status lb_selftest_log(int32_t device, const double *x, int64_t n, double *out_tbl, double *out_df,
                                     double *out_ref) {
    if (!x || !out_tbl || !out_df || !out_ref || n < 1) return LB_E_INVALID;
    if (cudaSetDevice(device) != cudaSuccess) return LB_E_CUDA;
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
