// Internal definitions shared by the CUDA translation units of the library.
// D3Q19 velocity set, device-side parameter block, gray-cell record and
// small index helpers.  Nothing here is visible through the C ABI.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/lbm.h"

namespace lbm {

constexpr int Q = 19;
constexpr int MAX_TYPES = LBM_MAX_PORE_TYPES;

// D3Q19 velocities: rest, the six faces (+x,-x,+y,-y,+z,-z), then the twelve
// edges in opposite pairs.  opp(i) = i+1 for odd i, i-1 for even i >= 2.
__host__ __device__ constexpr int cx(int i)
{
    constexpr int t[Q] = {0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0};
    return t[i];
}
__host__ __device__ constexpr int cy(int i)
{
    constexpr int t[Q] = {0, 0, 0, 1, -1, 0, 0, 1, -1, -1, 1, 0, 0, 0, 0, 1, -1, 1, -1};
    return t[i];
}
__host__ __device__ constexpr int cz(int i)
{
    constexpr int t[Q] = {0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, -1, -1, 1, 1, -1, -1, 1};
    return t[i];
}
__host__ __device__ constexpr int opp(int i) { return i == 0 ? 0 : ((i & 1) ? i + 1 : i - 1); }
__host__ __device__ constexpr float wgt(int i)
{
    return i == 0 ? (1.0f / 3.0f) : (i <= 6 ? (1.0f / 18.0f) : (1.0f / 36.0f));
}
__host__ __device__ constexpr double wgt_d(int i)
{
    return i == 0 ? (1.0 / 3.0) : (i <= 6 ? (1.0 / 18.0) : (1.0 / 36.0));
}

// Runtime constants of one pore type's curves, in FP32.
struct Curve {
    float swr;
    float inv_1m_swr;      // 1 / (1 - swr)
    float neg_inv_lambda;  // -1 / lambda
    float nw, nn;          // Corey exponents (wetting, non-wetting)
    float thomeer_k;       // Thomeer Pc: -G log2(10); 0 selects Brooks-Corey
};
constexpr float LOG2_10 = 3.32192809488736234787f;

// Parameter block passed by value to every kernel.
struct DevParams {
    int nx, ny, nz;
    int per[3];
    int n;                 // number of cells
    float omega_fac[2];    // 1 - 1/tau
    float nu[2];           // (tau - 1/2)/3
    float G, G_lo;         // Shan-Chen coupling as float-float
    float kappa;
    float csf_coef[2];     // 1 / (phi_avg * phi_max)
    int csf_everywhere;
    float rho_wall[2];
    float accel[2][3];
    int wet;
    float r_lo, inv_r_span;
    float s_lo, s_hi, at_cut, eps_n, kr_min;
    float at_wall;         // Atwood number of the wall densities
    float rho0[2];         // shift of the 16-bit storages: f_i - w_i rho0
    float held[2][2][2];   // inlet [0] / outlet [1] densities (A, B) as float-float (hi, lo)
    float mss;             // mass-sink-source rate m (0: off)
    float mss_ib, mss_inv; // interface indicator: bulk value I_b = 4 r_lo r_hi and 1/(1 - I_b)
    int storage;           // enum lbm_storage
    Curve curve[MAX_TYPES];
};

// Gray-cell record: 32 bytes, read only where the cell type is gray.
//   a = (v.x, v.y, v.z, 1/K0), v = sqrt(aniso - 1) e1 (zero if isotropic),
//       so that K^-1 = (1/K0)(I + v v^T);
//   b = (lamL*pd, Sw_irr, So_res, meta) with meta bits 0-7 the pore type,
//       bit 8 the wet flag and bit 9 "has switched at least once".
struct __align__(16) GrayRec {
    float4 a;
    float4 b;
};
constexpr unsigned META_WET = 1u << 8;
constexpr unsigned META_SWITCHED = 1u << 9;

enum : uint8_t {
    CELL_PORE = LBM_CELL_PORE,
    CELL_SOLID = LBM_CELL_SOLID,
    CELL_GRAY = LBM_CELL_GRAY,
    CELL_INLET = LBM_CELL_INLET,
    CELL_OUTLET = LBM_CELL_OUTLET
};
// Reservoir (pressure) cell: held at the inlet or outlet densities.
__host__ __device__ __forceinline__ bool is_held(int t) { return t == CELL_INLET || t == CELL_OUTLET; }

// Neighbour coordinate along one axis: wrapped when periodic, -1 outside.
__device__ __forceinline__ int axis_nb(int v, int d, int n, int periodic)
{
    int w = v + d;
    if (w < 0) return periodic ? w + n : -1;
    if (w >= n) return periodic ? w - n : -1;
    return w;
}

}  // namespace lbm
