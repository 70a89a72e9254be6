// lb_device_guard.cuh -- makes a context's device current for the duration of one
// entry point and gives the calling thread its previous current device back on every
// return path, so that a call into the library never changes which device the caller's
// own later CUDA calls go to.
#pragma once
#include <cuda_runtime.h>

namespace lbvdw {

struct DeviceGuard {
    int prev = -1;
    cudaError_t status = cudaSuccess;
    explicit DeviceGuard(int device) {
        if (cudaGetDevice(&prev) != cudaSuccess) {
            prev = -1;
            cudaGetLastError();
        }
        status = cudaSetDevice(device);
    }
    ~DeviceGuard() {
        int now = -1;
        if (prev >= 0 && cudaGetDevice(&now) == cudaSuccess && now != prev) cudaSetDevice(prev);
    }
    bool ok() const { return status == cudaSuccess; }
    DeviceGuard(const DeviceGuard &) = delete;
    DeviceGuard &operator=(const DeviceGuard &) = delete;
};

}  // namespace lbvdw
