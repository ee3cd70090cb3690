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
// 58,496 bytes, which every GPU that loads this library holds until the
// process exits.  Host code must not use the symbol itself (on the host it
// only names a stand-in): every call resolves the array's device address in
// the context current to the calling thread with cudaGetSymbolAddress (a
// host-side lookup, small next to the synchronisation the call ends with), so
// the device's primary context, a context the caller made current and a
// primary context re-created after cudaDeviceReset each get the address of
// their own copy of the module.  Each call overwrites every slot it later
// reads; the one slot that must start at zero, the completion count in the
// final row, is zero at load and reset by each call's last block.  Calls that
// overlap on the GPU (for example on two streams) share the array and race.
// The call synchronises its stream, so it cannot be captured into a CUDA
// graph: on a capturing stream it returns LBM_ERR_ARG before any work.
#include <cmath>
#include <cstring>

#include "lbm_obs.cuh"

namespace {

static __device__ __align__(256) double g_obs_scratch[(lbm::OBS_MAX_BLOCKS + 1) * lbm::NOBS];

// Device address of g_obs_scratch in the current context.
cudaError_t scratch_address(double **out)
{
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_obs_scratch);
    if (e != cudaSuccess) return e;
    *out = static_cast<double *>(p);
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
    cudaStream_t s = (cudaStream_t)stream;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) != cudaSuccess) return LBM_ERR_CUDA;
    if (cs != cudaStreamCaptureStatusNone) return LBM_ERR_ARG;  // the call synchronises: it cannot be captured
    double *scratch = nullptr;
    if (scratch_address(&scratch) != cudaSuccess) return LBM_ERR_CUDA;

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
