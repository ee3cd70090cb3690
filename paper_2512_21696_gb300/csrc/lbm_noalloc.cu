// Observables reduction that allocates nothing (lbm_observables_noalloc).
//
// Some callers cannot call cudaMalloc at all: code that runs inside a host
// callback or an allocator hook, plug-ins of host applications whose memory
// pool owns the device, and latency-critical loops that must not touch the
// allocator (an allocation can synchronise the device).  This entry point
// serves them: the caller passes the fields and receives lbm_obs, and the
// reduction's per-block partial sums live in a file-scope device array
// instead of context-owned memory.
//
// The array is g_obs_scratch below: (OBS_MAX_BLOCKS + 1) * NOBS doubles =
// 77,952 bytes, which every GPU that loads this library holds until the
// process exits.  Its device address is resolved once per device with
// cudaGetSymbolAddress by the first call on that device (host code must not
// use the symbol itself: on the host it only names a stand-in).  Each call
// overwrites every slot it later reads; the one slot that must start at zero,
// the completion count in the final row, is zero at load and reset by each
// call's last block.  Calls that overlap on the GPU (for example on two
// streams) share the array and race.
#include <atomic>
#include <cmath>
#include <cstring>
#include <mutex>

#include "lbm_obs.cuh"

namespace {

static __device__ __align__(256) double g_obs_scratch[(lbm::OBS_MAX_BLOCKS + 1) * lbm::NOBS];

constexpr int MAX_DEVICES = 64;
std::mutex g_scratch_mutex;
double *g_scratch_ptr[MAX_DEVICES] = {};

// Device address of g_obs_scratch on the current device (resolved once).
cudaError_t scratch_address(int dev, double **out)
{
    std::lock_guard<std::mutex> lock(g_scratch_mutex);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_obs_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_ptr[dev] = static_cast<double *>(p);
    }
    *out = g_scratch_ptr[dev];
    return cudaSuccess;
}

}  // namespace

extern "C" LBM_API int lbm_observables_noalloc(const float *fields, const uint8_t *type, const float *phi, int nx,
                                                int ny, int nz, double G, const double probe[5], void *stream,
                                                lbm_obs *out)
{
    if (!fields || !type || !phi || !probe || !out) return LBM_ERR_ARG;
    if (nx < 1 || ny < 1 || nz < 1) return LBM_ERR_ARG;
    const long long n = (long long)nx * ny * nz;
    if (n > LBM_NOALLOC_MAX_CELLS) return LBM_ERR_ARG;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAX_DEVICES) return LBM_ERR_CUDA;
    double *scratch = nullptr;
    if (scratch_address(dev, &scratch) != cudaSuccess) return LBM_ERR_CUDA;

    lbm::DevParams P;
    std::memset(&P, 0, sizeof(P));
    P.nx = nx;
    P.ny = ny;
    P.nz = nz;
    P.n = (int)n;
    const lbm::ObsArgs O = lbm::obs_args(probe, probe[3], probe[4], G, n);
    const int nb = lbm::obs_blocks((int)n);
    float2 *partial = reinterpret_cast<float2 *>(scratch);  // a float-float pair per double slot
    double *final_row = scratch + (size_t)lbm::OBS_MAX_BLOCKS * lbm::NOBS;
    cudaStream_t s = (cudaStream_t)stream;
    lbm::k_obs_partial<<<nb, lbm::OBS_BLOCK, 0, s>>>(P, O, type, phi, fields, partial, final_row);
    if (cudaGetLastError() != cudaSuccess) return LBM_ERR_CUDA;
    double v[lbm::NOBS];
    if (cudaMemcpyAsync(v, final_row, sizeof(v), cudaMemcpyDeviceToHost, s) != cudaSuccess) return LBM_ERR_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return LBM_ERR_CUDA;
    out->mass[0] = v[0];
    out->mass[1] = v[1];
    out->sat = v[3] > 0 ? v[2] / v[3] : 0.0;
    out->flux_out = v[4] / ((double)ny * nz);
    for (int d = 0; d < 3; ++d) out->flux_vol[d] = v[5 + d] / (double)n;
    out->max_u = v[8];
    out->dp = (v[10] > 0 ? v[9] / v[10] : 0.0) - (v[12] > 0 ? v[11] / v[12] : 0.0);
    out->nan_count = (long long)v[13];
    out->step = 0;
    return out->nan_count > 0 ? LBM_ERR_NUMERIC : LBM_OK;
}
