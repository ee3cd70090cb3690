// Shared declarations of the observable reduction (lbm_obs.cu): float-float
// sums on the FP32 pipe, FP64 results.
#pragma once

#include <cmath>

#include "lbm_common.cuh"

namespace lbm {

constexpr int NOBS = 16;
// slots: 0,1 mass; 2 sum phi_c Sw; 3 sum phi_c; 4 outlet u_x; 5..7 sum u;
//        8 max |u|; 9 sum p inside; 10 count inside; 11 sum p outside;
//        12 count outside; 13 non-finite count
constexpr int SLOT_MAX = 8;
constexpr int SLOT_COUNTER = 15;  // of the output row: blocks done (zero between reductions)
constexpr int OBS_BLOCK = 256;
constexpr int OBS_MAX_BLOCKS = 456;  // 3 resident blocks on each of 152 SMs

// Pressure probe in FP32 (the kernels do no FP64 arithmetic per thread):
// centre, squared inner and outer radii, G; probe = 0 when no cell can fall
// inside the inner or outside the outer sphere.
struct ObsArgs {
    float cx, cy, cz, rin2, rout2, G;
    int probe;
};
inline ObsArgs obs_args(const double c[3], double r_in, double r_out, double G, long long n)
{
    ObsArgs O;
    O.cx = (float)c[0];
    O.cy = (float)c[1];
    O.cz = (float)c[2];
    O.rin2 = (float)(r_in * r_in);
    O.rout2 = (float)std::fmin(r_out * r_out, 3.0e38);
    O.G = (float)G;
    O.probe = (r_in * r_in > 0.0 || r_out * r_out < 3.0 * (double)n * (double)n) ? 1 : 0;
    return O;
}

// Grid-stride pass over the [6][n] fields (rhoA, rhoB, ux, uy, uz, Sw): one
// row of NOBS float-float partials (hi, lo) per block in `partial`; the last
// block to finish sums the rows in a fixed order into out[NOBS] (FP64).
// out[SLOT_COUNTER] must be zero at launch and is zero again at exit.
__global__ void __launch_bounds__(OBS_BLOCK, 3) k_obs_partial(DevParams P, ObsArgs O, const uint8_t *__restrict__ type,
                              const float *__restrict__ phi, const float *__restrict__ macro,
                              float2 *__restrict__ partial, double *__restrict__ out);

int obs_blocks(int n);

}  // namespace lbm
