// Observables of the current fields (float-float reductions, FP64 results)
// and read-back of the gray-cell geometry results.
//
// k_obs_partial: grid-stride pass (two cells' loads in flight per thread),
//                per-thread float-float accumulators
//                (error-free FP32 sums, about 48 bits: FP64 arithmetic runs at
//                a small fraction of the FP32 rate on this part), float-float
//                warp-shuffle and shared-memory block reduction, one row of
//                float-float partials per block in the reduction scratch (a
//                pair in each double slot);
//                the last block to finish (an atomic count in the output
//                row's spare slot) sums the rows, one warp per slot: each lane
//                a fixed subset of the rows, then the warp in a fixed order
//                (deterministic), in float-float; each slot's result is
//                converted to FP64 once.
#include <cfloat>

#include "lbm_context.h"
#include "lbm_obs.cuh"

namespace lbm {


// float-float sum over the warp (lane 0 gets it)
__device__ __forceinline__ ff warp_sum_ff(ff v)
{
    for (int o = 16; o > 0; o >>= 1) {
        const ff w = {__shfl_down_sync(0xffffffffu, v.hi, o), __shfl_down_sync(0xffffffffu, v.lo, o)};
        v = ff_add(v, w);
    }
    return v;
}
__device__ __forceinline__ int warp_sum_i(int v)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ float warp_max_f(float v)
{
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_down_sync(0xffffffffu, v, o));
    return v;
}

__global__ void __launch_bounds__(OBS_BLOCK, 3) k_obs_partial(DevParams P, ObsArgs O,
                                                           const uint8_t *__restrict__ type,
                                                           const float *__restrict__ phi,
                                                           const float *__restrict__ macro,
                                                           float2 *__restrict__ partial,
                                                           double *__restrict__ out)
{
    __shared__ float2 sh[NOBS * 32];
    // slots 0-7, 9, 11 summed in float-float; 10, 12, 13 are counts
    constexpr int NS = 10;
    constexpr int slot_of[NS] = {0, 1, 2, 3, 4, 5, 6, 7, 9, 11};
    ff s[NS];
#pragma unroll
    for (int k = 0; k < NS; ++k) s[k] = ff{0.f, 0.f};
    int cin = 0, cout = 0, bad = 0;
    const int n = P.n;
    float umax = 0.0f;
    const float pcx = O.cx, pcy = O.cy, pcz = O.cz, rin2 = O.rin2, rout2 = O.rout2, Gf = O.G;
    const bool probe = O.probe != 0;  // some cell can fall inside or outside
    // cells c0 + k stride, k < UNR, per pass: all their loads are issued before
    // any is used (the fields of solid cells are read and ignored), so a pass
    // waits on memory once; the cells are summed in the grid-stride order.
    // Their coordinates advance by the stride's (x, y, z) steps with carries
    // (no division per cell).
    constexpr int UNR = 2;
    const long long stride = (long long)gridDim.x * blockDim.x;
    const int nx = P.nx, ny = P.ny;
    const int sx = (int)(stride % nx);
    const long long sq = stride / nx;
    const int sy = (int)(sq % ny), sz = (int)(sq / ny);
    const long long cstart = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    int x = (int)(cstart % nx), y = (int)((cstart / nx) % ny), z = (int)(cstart / ((long long)nx * ny));
    for (long long c0 = cstart; c0 < n; c0 += UNR * stride) {
        uint8_t tk[UNR];
        float fk[UNR][7];
#pragma unroll
        for (int k = 0; k < UNR; ++k) {
            const long long ck = c0 + k * stride;
            tk[k] = CELL_SOLID;
            if (ck < n) {
                tk[k] = type[ck];
#pragma unroll
                for (int q = 0; q < 6; ++q) fk[k][q] = macro[(size_t)q * n + ck];
                fk[k][6] = phi[ck];
            }
        }
#pragma unroll
        for (int k = 0; k < UNR; ++k) {
            const uint8_t t = tk[k];
            const int cxk = x, cyk = y, czk = z;
            // the next cell of this thread
            x += sx;
            const int carx = x >= nx;
            x -= carx ? nx : 0;
            y += sy + carx;
            const int cary = y >= ny;
            y -= cary ? ny : 0;
            z += sz + cary;
            if (t == CELL_SOLID) continue;
            // per-cell terms in FP32 (products of FP32 fields, one rounding each)
            const float ra = fk[k][0], rb = fk[k][1];
            const float u0 = fk[k][2], u1 = fk[k][3], u2 = fk[k][4];
            const float sw = fk[k][5];
            if (!isfinite(ra) || !isfinite(rb) || !isfinite(u0) || !isfinite(u1) || !isfinite(u2)) {
                ++bad;
                continue;
            }
            s[0] = ff_add_f(s[0], ra);
            s[1] = ff_add_f(s[1], rb);
            // saturation weight: phi in gray cells, 1 in pores, reservoirs left out
            const float phc = t == CELL_GRAY ? fk[k][6] : (t == CELL_PORE ? 1.0f : 0.0f);
            s[2] = ff_add_f(s[2], phc * sw);
            s[3] = ff_add_f(s[3], phc);
            if (cxk == nx - 1) s[4] = ff_add_f(s[4], u0);
            s[5] = ff_add_f(s[5], u0);
            s[6] = ff_add_f(s[6], u1);
            s[7] = ff_add_f(s[7], u2);
            umax = fmaxf(umax, sqrtf(u0 * u0 + u1 * u1 + u2 * u2));
            if (probe) {  // uniform: the pressure probe is set
                const float dx = cxk - pcx, dy = cyk - pcy, dz = czk - pcz;
                const float r2 = dx * dx + dy * dy + dz * dz;
                const float pr = (ra + rb) * (1.0f / 3.0f) + Gf * ra * rb;
                if (r2 < rin2) { s[8] = ff_add_f(s[8], pr); ++cin; }
                if (r2 > rout2) { s[9] = ff_add_f(s[9], pr); ++cout; }
            }
        }
    }
    // warp and block levels in float-float and integers, all on the FP32
    // pipe (a few FP64 operations per block, times hundreds of blocks, had
    // kept the FP64 pipe a third busy); counts stay exact as float-float
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int k = 0; k < NS; ++k) {
        const ff v = warp_sum_ff(s[k]);
        if (lane == 0) sh[slot_of[k] * 32 + warp] = make_float2(v.hi, v.lo);
    }
    umax = warp_max_f(umax);
    cin = warp_sum_i(cin);
    cout = warp_sum_i(cout);
    bad = warp_sum_i(bad);
    if (lane == 0) {
        sh[8 * 32 + warp] = make_float2(umax, 0.f);
        sh[10 * 32 + warp] = make_float2((float)cin, 0.f);  // a warp counts far fewer than 2^24 cells: exact
        sh[12 * 32 + warp] = make_float2((float)cout, 0.f);
        sh[13 * 32 + warp] = make_float2((float)bad, 0.f);
        sh[14 * 32 + warp] = make_float2(0.f, 0.f);
        sh[15 * 32 + warp] = make_float2(0.f, 0.f);
    }
    __syncthreads();
    if (warp == 0) {
        for (int k = 0; k < NOBS; ++k) {
            const float2 x = lane < nw ? sh[k * 32 + lane] : make_float2(0.f, 0.f);
            ff v = {x.x, x.y};
            if (k == SLOT_MAX) v.hi = warp_max_f(v.hi);
            else v = warp_sum_ff(v);
            if (lane == 0) partial[(size_t)blockIdx.x * NOBS + k] = make_float2(v.hi, v.lo);
        }
    }

    // ---- the block that finishes last sums the rows into out ----
    // Thread 0 wrote this block's row; the fence makes it visible device-wide
    // before the count, and the last block to count reads every row from L2.
    // The count wraps to zero at the last block (atomicInc), so even a count
    // left over by a reduction that raced with another on the same scratch
    // cannot outlive one call.
    __shared__ unsigned int s_last;
    unsigned int *done = reinterpret_cast<unsigned int *>(out + SLOT_COUNTER);
    if (threadIdx.x == 0) {
        __threadfence();
        s_last = atomicInc(done, gridDim.x - 1) == gridDim.x - 1 ? 1u : 0u;
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    // warp w sums slots w, w + nw, ...: lanes over a fixed subset of the rows,
    // then the warp in a fixed order (deterministic)
    // (a lane's rows are loaded together, then summed in row order)
    constexpr int RPL = (OBS_MAX_BLOCKS + 31) / 32;
    for (int k = warp; k < NOBS; k += nw) {
        float2 pv[RPL];
#pragma unroll
        for (int t = 0; t < RPL; ++t) {
            const int b = lane + 32 * t;
            pv[t] = b < (int)gridDim.x ? __ldcg(&partial[(size_t)b * NOBS + k]) : make_float2(0.f, 0.f);
        }
        ff v = {0.f, 0.f};
#pragma unroll
        for (int t = 0; t < RPL; ++t) {
            if (k == SLOT_MAX) v.hi = fmaxf(v.hi, pv[t].x);
            else v = ff_add(v, ff{pv[t].x, pv[t].y});
        }
        if (k == SLOT_MAX) v.hi = warp_max_f(v.hi);
        else v = warp_sum_ff(v);
        // the counter's slot goes back to zero for the next reduction
        if (lane == 0) out[k] = k == SLOT_COUNTER ? 0.0 : (double)v.hi + (double)v.lo;
    }
}

int obs_blocks(int n)
{
    // a few resident blocks per SM; each thread then sums tens of cells
    int b = (n + 8 * OBS_BLOCK - 1) / (8 * OBS_BLOCK);
    return b < OBS_MAX_BLOCKS ? (b < 1 ? 1 : b) : OBS_MAX_BLOCKS;
}

// Fills host_out16 (synchronises the stream).  red must hold
// (obs_blocks(n) + 1) * NOBS doubles, zero when allocated (the completion
// counter of each reduction lives in its output row and returns to zero).
cudaError_t launch_observables(lbm_ctx *ctx, double *host_out16) { return launch_observables(ctx, host_out16, true); }

cudaError_t launch_observables(lbm_ctx *ctx, double *host_out16, bool sync)
{
    const lbm_params &p = ctx->p;
    const ObsArgs O = obs_args(p.probe_center, p.probe_r_in, p.probe_r_out, p.G, ctx->n);
    const int nb = obs_blocks(ctx->n);
    float2 *partial = reinterpret_cast<float2 *>(ctx->red);  // a float-float pair per double slot
    double *out = ctx->red + (size_t)nb * NOBS;
    cudaEvent_t e0;
    prof_begin(ctx, "k_obs_partial", &e0);
    k_obs_partial<<<nb, OBS_BLOCK, 0, ctx->stream>>>(ctx->dp, O, ctx->type, ctx->phi, ctx->macro, partial, out);
    prof_end(ctx, "k_obs_partial", e0);
    ctx->launches += 1;
    cudaError_t err = cudaGetLastError();
    if (err != cudaSuccess) return err;
    err = cudaMemcpyAsync(host_out16, out, NOBS * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream);
    if (err != cudaSuccess) return err;
    return sync ? cudaStreamSynchronize(ctx->stream) : cudaSuccess;
}

__global__ void k_static_out(int n, const uint8_t *__restrict__ type, const GrayRec *__restrict__ gray,
                             float *__restrict__ kinv, float *__restrict__ pcs, float *__restrict__ swirr,
                             float *__restrict__ sores)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n) return;
    float k6[6] = {0, 0, 0, 0, 0, 0}, p = 0.f, si = 0.f, so = 0.f;
    if (type[c] == CELL_GRAY) {
        const GrayRec r = gray[c];
        const float ik = r.a.w, vx = r.a.x, vy = r.a.y, vz = r.a.z;
        k6[0] = ik * (1.f + vx * vx);
        k6[1] = ik * (1.f + vy * vy);
        k6[2] = ik * (1.f + vz * vz);
        k6[3] = ik * vx * vy;
        k6[4] = ik * vx * vz;
        k6[5] = ik * vy * vz;
        p = r.b.x;
        si = r.b.y;
        so = r.b.z;
    }
    if (kinv)
        for (int k = 0; k < 6; ++k) kinv[(size_t)k * n + c] = k6[k];
    if (pcs) pcs[c] = p;
    if (swirr) swirr[c] = si;
    if (sores) sores[c] = so;
}

cudaError_t launch_static_out(lbm_ctx *ctx, float *kinv6, float *pcs, float *swirr, float *sores)
{
    cudaEvent_t e0;
    prof_begin(ctx, "k_static_out", &e0);
    k_static_out<<<(ctx->n + 255) / 256, 256, 0, ctx->stream>>>(ctx->n, ctx->type, ctx->gray, kinv6, pcs,
                                                                 swirr, sores);
    prof_end(ctx, "k_static_out", e0);
    ctx->launches += 1;
    return cudaGetLastError();
}

}  // namespace lbm
