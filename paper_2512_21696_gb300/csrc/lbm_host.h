// Host-side helpers of the C-ABI layer shared by its translation units
// (lbm_api.cu, lbm_batch.cu).
#pragma once

#include <cuda_runtime.h>

#include "lbm_context.h"

namespace lbm_host {

// Records the failing call for lbm_last_cuda_error and maps it to a status.
int cuda_fail(cudaError_t e, const char *where);
// LBM_OK or LBM_ERR_ARG for a parameter block (the checks of lbm_create).
int validate_params(const lbm_params *p);
// Fills ctx->dp from ctx->p, the reservoir densities and the constitutive curves.
void fill_device_params(lbm_ctx *ctx);
// Reservoir densities before any lbm_set_pressure: (rho_hi, rho_lo) at both ends.
void default_held(lbm_ctx *ctx);
// Bytes of one population buffer of ctx (2 components, its storage).
size_t pop_bytes(const lbm_ctx *ctx);

#define LBM_CUDA(call)                                   \
    do {                                                 \
        cudaError_t e_ = (call);                         \
        if (e_ != cudaSuccess) return cuda_fail(e_, #call); \
    } while (0)

// Makes the context's device current for the duration of a call.
struct DeviceGuard {
    int prev = -1;
    bool ok = true;
    explicit DeviceGuard(int dev)
    {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) ok = cudaSetDevice(dev) == cudaSuccess;
    }
    ~DeviceGuard()
    {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

}  // namespace lbm_host
