// Shared declarations of the FP64 observable reduction (lbm_obs.cu).
#pragma once

#include "lbm_common.cuh"

namespace lbm {

constexpr int NOBS = 16;
// slots: 0,1 mass; 2 sum phi_c Sw; 3 sum phi_c; 4 outlet u_x; 5..7 sum u;
//        8 max |u|; 9 sum p inside; 10 count inside; 11 sum p outside;
//        12 count outside; 13 non-finite count
constexpr int SLOT_MAX = 8;
constexpr int OBS_BLOCK = 256;
constexpr int OBS_MAX_BLOCKS = 608;
constexpr int OBS_FINAL_THREADS = NOBS * 32;  // k_obs_final: one warp per slot

struct ObsArgs {
    double cx, cy, cz, rin2, rout2, G;
};

// Grid-stride pass over the [6][n] fields (rhoA, rhoB, ux, uy, uz, Sw): one
// row of NOBS partials per block in `partial`.
__global__ void __launch_bounds__(OBS_BLOCK) k_obs_partial(DevParams P, ObsArgs O, const uint8_t *__restrict__ type,
                              const float *__restrict__ phi, const float *__restrict__ macro,
                              double *__restrict__ partial);
// One block of OBS_FINAL_THREADS: sums the nblocks rows of `partial` in a fixed
// order into out[NOBS].
__global__ void __launch_bounds__(OBS_FINAL_THREADS) k_obs_final(const double *__restrict__ partial, int nblocks,
                                                                double *__restrict__ out);

int obs_blocks(int n);

}  // namespace lbm
