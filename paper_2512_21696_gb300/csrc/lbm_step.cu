// Time-step kernels of the two-component D3Q19 pseudo-potential LB model.
//
// Population storage (F32), per component a and cell x:
//   slot 0      the rest population f_0 in 2^-30 fixed point (int32), so that
//               its update is an exact integer add and the differences
//               f_0(y) - f_0(x) between cells are exact;
//   slots 1..18 the deviations g_i = f_i - 3 w_i f_0 in FP32.
// Pulling f_i(x) = f*_i(x - c_i) then gives, relative to the puller's own rest
// population, h_i = f_i(x) - 3 w_i f_0(x) = g_i(s) + 3 w_i (f_0(s) - f_0(x))
// with s = x - c_i, and every moment is a sum of small numbers:
//     rho = 3 f_0 + drho (drho = sum h_i),  j = sum c_i h_i,
//     sum c c f = sum c c h + f_0 I.
// The density stencils use rho(y) - rho(x) = 3 (f_0(y) - f_0(x)) +
// (drho(y) - drho(x)), again exact or small.  The post-collision deviations
// are written in closed form from the moments, so FP32 rounding acts on
// O(u, F, Pi_neq) quantities instead of on O(w rho) ones; the rounding
// residual of the rest population is carried into the moving populations.
// Mathematically the state is the same as plain populations.
//
// One step is two launches:
//   k_density  - pull and zeroth moment: drho^A, drho^B of every fluid cell,
//                the source of the density stencils;
//   k_collide  - pull again, residual update, forces (Shan-Chen, CSF Eq. 4,
//                Eq. 1 capillary + tensorial viscous with the semi-implicit
//                velocity), regularised collision with the Eq. 3 force term,
//                store.
#include "lbm_context.h"

namespace lbm {

constexpr float FIX_ONE = 1073741824.0f;            // 2^30
constexpr float FIX_INV = 9.313225746154785e-10f;    // 2^-30
constexpr double FIX_ONE_D = 1073741824.0;

// 3 w_i for the moving populations (faces 1/6, edges 1/12).
__host__ __device__ constexpr float w3(int i) { return i <= 6 ? (1.0f / 6.0f) : (1.0f / 12.0f); }

// Exact difference of two fixed-point rest populations, as a float.
__device__ __forceinline__ float fix_diff(int a, int b) { return (float)(a - b) * FIX_INV; }

// ---- float-float (unevaluated sum hi + lo) arithmetic ----------------------
// Used where physically large, nearly cancelling terms meet: at interfaces the
// Shan-Chen force (~0.1) balances the pressure part of j (~0.05) and u is
// their O(1e-3) residual.  Error-free transformations of Knuth (two-sum) and
// Dekker (fast two-sum) and FMA-based products.
struct ff {
    float hi, lo;
};
__device__ __forceinline__ ff two_sum(float a, float b)
{
    const float s = a + b;
    const float bb = s - a;
    return {s, (a - (s - bb)) + (b - bb)};
}
__device__ __forceinline__ ff fast_two_sum(float a, float b)
{
    const float s = a + b;
    return {s, b - (s - a)};
}
__device__ __forceinline__ ff ff_add(ff x, ff y)
{
    const ff s = two_sum(x.hi, y.hi);
    return fast_two_sum(s.hi, s.lo + (x.lo + y.lo));
}
__device__ __forceinline__ ff ff_add_f(ff x, float y)
{
    const ff s = two_sum(x.hi, y);
    return fast_two_sum(s.hi, s.lo + x.lo);
}
__device__ __forceinline__ ff ff_mul(ff x, ff y)
{
    const float p = x.hi * y.hi;
    float e = fmaf(x.hi, y.hi, -p);
    e = fmaf(x.hi, y.lo, fmaf(x.lo, y.hi, e));
    return fast_two_sum(p, e);
}
__device__ __forceinline__ ff ff_scale(ff x, float pow2) { return {x.hi * pow2, x.lo * pow2}; }
// Exact value v * pow2 of an integer (|v| < 2^48) as float-float.
__device__ __forceinline__ ff ff_from_ll(long long v, float pow2)
{
    const float hi = (float)v;
    const float lo = (float)(v - (long long)hi);
    return {hi * pow2, lo * pow2};
}
// 1/12 as float-float.
constexpr float TWELFTH_HI = (float)(1.0 / 12.0);
constexpr float TWELFTH_LO = (float)(1.0 / 12.0 - (double)(float)(1.0 / 12.0));
// v * 2^-30 / 12 for an integer sum v of weighted rest-population differences.
__device__ __forceinline__ ff ff_twelfth(long long v) { return ff_mul(ff_from_ll(v, FIX_INV), {TWELFTH_HI, TWELFTH_LO}); }

__device__ __forceinline__ void cell_xyz(int c, const DevParams &P, int &x, int &y, int &z)
{
    x = c % P.nx;
    const int t = c / P.nx;
    y = t % P.ny;
    z = t / P.ny;
}

struct Axes {
    int xs[3], ys[3], zs[3];
};

__device__ __forceinline__ Axes axes_of(const DevParams &P, int x, int y, int z)
{
    Axes A;
    A.xs[0] = axis_nb(x, -1, P.nx, P.per[0]);
    A.xs[1] = x;
    A.xs[2] = axis_nb(x, 1, P.nx, P.per[0]);
    A.ys[0] = axis_nb(y, -1, P.ny, P.per[1]);
    A.ys[1] = y;
    A.ys[2] = axis_nb(y, 1, P.ny, P.per[1]);
    A.zs[0] = axis_nb(z, -1, P.nz, P.per[2]);
    A.zs[1] = z;
    A.zs[2] = axis_nb(z, 1, P.nz, P.per[2]);
    return A;
}

// Linear index of x + c_i, or -1 outside a non-periodic axis.
__device__ __forceinline__ int nb_index(const DevParams &P, const Axes &A, int i)
{
    const int X = A.xs[cx(i) + 1], Y = A.ys[cy(i) + 1], Z = A.zs[cz(i) + 1];
    return (X < 0 || Y < 0 || Z < 0) ? -1 : X + P.nx * (Y + P.ny * Z);
}

// ---------------------------------------------------------------------------
// Initial state: equilibrium of (rhoA, rhoB, u), evaluated in FP64 once.
// ---------------------------------------------------------------------------
__global__ void k_init(DevParams P, const float *__restrict__ rhoA, const float *__restrict__ rhoB,
                       const float *__restrict__ u, const uint8_t *__restrict__ type,
                       float *__restrict__ f, float *__restrict__ drho, float *__restrict__ macro,
                       GrayRec *__restrict__ gray)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    const int n = P.n;
    if (c >= n) return;
    const uint8_t t = type[c];
    if (t == CELL_SOLID) {
        for (int k = 0; k < 2 * Q; ++k) f[(size_t)k * n + c] = 0.0f;
        drho[c] = 0.0f;
        drho[n + c] = 0.0f;
        for (int k = 0; k < 6; ++k) macro[(size_t)k * n + c] = 0.0f;
        return;
    }
    double uv[3] = {0.0, 0.0, 0.0};
    if (u) {
        uv[0] = u[c];
        uv[1] = u[(size_t)n + c];
        uv[2] = u[(size_t)2 * n + c];
    }
    const double uu = uv[0] * uv[0] + uv[1] * uv[1] + uv[2] * uv[2];
    const double r[2] = {(double)rhoA[c], (double)rhoB[c]};
    for (int a = 0; a < 2; ++a) {
        float *fa = f + (size_t)a * Q * n;
        const double f0 = r[a] / 3.0 - 0.5 * r[a] * uu;  // feq_0 = w_0 rho (1 - 3u^2/2)
        const long long q = llrint(f0 * FIX_ONE_D);
        const double r0 = f0 - (double)q / FIX_ONE_D;
        reinterpret_cast<int *>(fa)[c] = (int)q;
#pragma unroll
        for (int i = 1; i < Q; ++i) {
            const double cu = cx(i) * uv[0] + cy(i) * uv[1] + cz(i) * uv[2];
            const double g = wgt_d(i) * (r[a] * (3.0 * cu + 4.5 * cu * cu) + 3.0 * r0);
            fa[(size_t)i * n + c] = (float)g;
        }
        drho[(size_t)a * n + c] = (float)(r[a] - 3.0 * (double)q / FIX_ONE_D);
    }
    const double rw = r[P.wet], rn = r[1 - P.wet];
    double s = ((rw / (rw + rn)) - (double)P.r_lo) * (double)P.inv_r_span;
    s = s < 0.0 ? 0.0 : (s > 1.0 ? 1.0 : s);
    macro[c] = (float)r[0];
    macro[(size_t)n + c] = (float)r[1];
    macro[(size_t)2 * n + c] = (float)uv[0];
    macro[(size_t)3 * n + c] = (float)uv[1];
    macro[(size_t)4 * n + c] = (float)uv[2];
    macro[(size_t)5 * n + c] = (float)s;
    if (t == CELL_GRAY) {
        unsigned meta = __float_as_uint(gray[c].b.w) & 0xffu;
        if (s >= 0.5) meta |= META_WET;
        gray[c].b.w = __uint_as_float(meta);
    }
}

// ---------------------------------------------------------------------------
// Density deviations of the current step: drho = rho - 3 f_0 (pull + sum).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_density(DevParams P, const float *__restrict__ f,
                                                 const uint8_t *__restrict__ type,
                                                 float *__restrict__ drho)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    const int n = P.n;
    if (c >= n) return;
    if (type[c] == CELL_SOLID) return;
    int x, y, z;
    cell_xyz(c, P, x, y, z);
    const Axes A = axes_of(P, x, y, z);
    int nb[Q];
    unsigned wall = 0;
#pragma unroll
    for (int i = 1; i < Q; ++i) {
        nb[i] = nb_index(P, A, i);
        if (nb[i] < 0 || type[nb[i]] == CELL_SOLID) wall |= 1u << i;
    }
#pragma unroll
    for (int a = 0; a < 2; ++a) {
        const float *fa = f + (size_t)a * Q * n;
        const int *fi = reinterpret_cast<const int *>(fa);
        const int f0 = fi[c];
        float acc = 0.0f;
        long long id = 0;  // 12 * sum_i w3_i (f0(s) - f0(x)) in 2^-30 units
#pragma unroll
        for (int i = 1; i < Q; ++i) {
            const int o = opp(i);
            if (wall & (1u << o)) {
                acc += fa[(size_t)o * n + c];
            } else {
                const int s = nb[o];
                acc += fa[(size_t)i * n + s];
                id += (long long)(fi[s] - f0) * (i <= 6 ? 2 : 1);
            }
        }
        drho[(size_t)a * n + c] = ff_add_f(ff_twelfth(id), acc).hi;
    }
}

// rho^a(y) - rho^a(x) for a fluid neighbour y of the fluid cell x.
__device__ __forceinline__ float rho_diff(const int *__restrict__ fi, const float *__restrict__ dr, int y, int x)
{
    return 3.0f * fix_diff(fi[y], fi[x]) + (dr[y] - dr[x]);
}

// Unit normals of grad(phi^A) = grad(rho^B) and grad(phi^B) = grad(rho^A) at
// the fluid cell m = (X, Y, Z).
__device__ __forceinline__ void normals_at(const DevParams &P, const int *__restrict__ fiA,
                                           const int *__restrict__ fiB, const float *__restrict__ drA,
                                           const float *__restrict__ drB, const uint8_t *__restrict__ type,
                                           int X, int Y, int Z, float nA[3], float nB[3])
{
    const Axes A = axes_of(P, X, Y, Z);
    const int m = X + P.nx * (Y + P.ny * Z);
    const float rAm = 3.0f * (float)fiA[m] * FIX_INV + drA[m];
    const float rBm = 3.0f * (float)fiB[m] * FIX_INV + drB[m];
    float gA[3] = {0.f, 0.f, 0.f}, gB[3] = {0.f, 0.f, 0.f};
#pragma unroll
    for (int k = 1; k < Q; ++k) {
        const int mk = nb_index(P, A, k);
        float dA, dB;
        if (mk < 0 || type[mk] == CELL_SOLID) {
            dA = P.rho_wall[0] - rAm;
            dB = P.rho_wall[1] - rBm;
        } else {
            dA = rho_diff(fiA, drA, mk, m);
            dB = rho_diff(fiB, drB, mk, m);
        }
        const float w = w3(k);
        if (cx(k)) { gA[0] += w * cx(k) * dB; gB[0] += w * cx(k) * dA; }
        if (cy(k)) { gA[1] += w * cy(k) * dB; gB[1] += w * cy(k) * dA; }
        if (cz(k)) { gA[2] += w * cz(k) * dB; gB[2] += w * cz(k) * dA; }
    }
    const float mA = fmaxf(sqrtf(gA[0] * gA[0] + gA[1] * gA[1] + gA[2] * gA[2]), P.eps_n);
    const float mB = fmaxf(sqrtf(gB[0] * gB[0] + gB[1] * gB[1] + gB[2] * gB[2]), P.eps_n);
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        nA[d] = gA[d] / mA;
        nB[d] = gB[d] / mB;
    }
}

// ---------------------------------------------------------------------------
// Forces + collision.
// ---------------------------------------------------------------------------
template <bool MACRO>
__global__ void __launch_bounds__(256) k_collide(DevParams P, const float *__restrict__ fin,
                                                 float *__restrict__ fout,
                                                 const uint8_t *__restrict__ type,
                                                 const float *__restrict__ drho,
                                                 GrayRec *__restrict__ gray,
                                                 float *__restrict__ macro)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    const int n = P.n;
    if (c >= n) return;
    const uint8_t t = type[c];
    if (t == CELL_SOLID) {
        if (MACRO)
            for (int k = 0; k < 6; ++k) macro[(size_t)k * n + c] = 0.0f;
        return;
    }
    int x, y, z;
    cell_xyz(c, P, x, y, z);
    const Axes A = axes_of(P, x, y, z);
    int nb[Q];
    unsigned wall = 0;
#pragma unroll
    for (int i = 1; i < Q; ++i) {
        nb[i] = nb_index(P, A, i);
        if (nb[i] < 0 || type[nb[i]] == CELL_SOLID) wall |= 1u << i;
    }
    const int *fiA = reinterpret_cast<const int *>(fin);
    const int *fiB = reinterpret_cast<const int *>(fin + (size_t)Q * n);
    const float *drA = drho, *drB = drho + n;

    // ---- moments of the pulled populations, per component ----------------
    // h_i = g_i(s) + w3_i (f0(s) - f0(x)): the g parts are summed in FP32, the
    // rest-population parts exactly in 64-bit integers (weights 12 w3 = 2 on
    // faces, 1 on edges) and converted once.
    int f0i[2];
    float dr[2], S[2][6];
    ff rho_ff[2], j_ff[3] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
    long long ij[2][3];
#pragma unroll
    for (int a = 0; a < 2; ++a) {
        const float *fa = fin + (size_t)a * Q * n;
        const int *fi = a ? fiB : fiA;
        const int f0 = fi[c];
        float d = 0.f, j0 = 0.f, j1 = 0.f, j2 = 0.f;
        float sxx = 0.f, syy = 0.f, szz = 0.f, sxy = 0.f, sxz = 0.f, syz = 0.f;
        long long Id = 0, Ij0 = 0, Ij1 = 0, Ij2 = 0, Ixx = 0, Iyy = 0, Izz = 0, Ixy = 0, Ixz = 0, Iyz = 0;
#pragma unroll
        for (int i = 1; i < Q; ++i) {
            const int o = opp(i);
            float g;
            long long D = 0;
            if (wall & (1u << o)) {
                g = fa[(size_t)o * n + c];
            } else {
                const int sidx = nb[o];
                g = fa[(size_t)i * n + sidx];
                D = (long long)(fi[sidx] - f0) * (i <= 6 ? 2 : 1);
            }
            d += g;
            Id += D;
            if (cx(i)) { j0 += cx(i) * g; sxx += g; Ij0 += cx(i) * D; Ixx += D; }
            if (cy(i)) { j1 += cy(i) * g; syy += g; Ij1 += cy(i) * D; Iyy += D; }
            if (cz(i)) { j2 += cz(i) * g; szz += g; Ij2 += cz(i) * D; Izz += D; }
            if (cx(i) && cy(i)) { sxy += cx(i) * cy(i) * g; Ixy += cx(i) * cy(i) * D; }
            if (cx(i) && cz(i)) { sxz += cx(i) * cz(i) * g; Ixz += cx(i) * cz(i) * D; }
            if (cy(i) && cz(i)) { syz += cy(i) * cz(i) * g; Iyz += cy(i) * cz(i) * D; }
        }
        f0i[a] = f0;
        const ff dff = ff_add_f(ff_twelfth(Id), d);
        dr[a] = dff.hi;
        rho_ff[a] = ff_add(ff_from_ll(3LL * f0, FIX_INV), dff);
        j_ff[0] = ff_add(j_ff[0], ff_add_f(ff_twelfth(Ij0), j0));
        j_ff[1] = ff_add(j_ff[1], ff_add_f(ff_twelfth(Ij1), j1));
        j_ff[2] = ff_add(j_ff[2], ff_add_f(ff_twelfth(Ij2), j2));
        ij[a][0] = Ij0; ij[a][1] = Ij1; ij[a][2] = Ij2;
        S[a][0] = ff_add_f(ff_twelfth(Ixx), sxx).hi;
        S[a][1] = ff_add_f(ff_twelfth(Iyy), syy).hi;
        S[a][2] = ff_add_f(ff_twelfth(Izz), szz).hi;
        S[a][3] = ff_add_f(ff_twelfth(Ixy), sxy).hi;
        S[a][4] = ff_add_f(ff_twelfth(Ixz), sxz).hi;
        S[a][5] = ff_add_f(ff_twelfth(Iyz), syz).hi;
    }
    const float r[2] = {rho_ff[0].hi, rho_ff[1].hi};
    const float rt = r[0] + r[1];
    const bool is_gray = (t == CELL_GRAY);
    const int w = P.wet;

    // ---- density stencils: grad(rho^a) for the Shan-Chen force and CSF, and
    //      grad(At) in gray cells.  The rest-population part of grad(rho^a)
    //      is (1/4) 2^-30 sum_i 12 w3_i c_i (f0(x+c_i) - f0(x)) = -2^-32 Ij^a
    //      (the same differences the pull used); the drho part is summed in
    //      FP32; walls contribute rho_wall - rho(x). ----------------------------
    float gfA[3] = {0.f, 0.f, 0.f}, gfB[3] = {0.f, 0.f, 0.f}, gAt[3] = {0.f, 0.f, 0.f};
    const float drcA = drA[c], drcB = drB[c];
#pragma unroll
    for (int i = 1; i < Q; ++i) {
        const int m = nb[i];
        float eA, eB;  // FP32 parts of rho^a(x+c_i) - rho^a(x)
        if (wall & (1u << i)) {
            eA = P.rho_wall[0] - r[0];
            eB = P.rho_wall[1] - r[1];
        } else {
            eA = drA[m] - drcA;
            eB = drB[m] - drcB;
        }
        const float wi = w3(i);
        if (cx(i)) { gfA[0] += wi * cx(i) * eA; gfB[0] += wi * cx(i) * eB; }
        if (cy(i)) { gfA[1] += wi * cy(i) * eA; gfB[1] += wi * cy(i) * eB; }
        if (cz(i)) { gfA[2] += wi * cz(i) * eA; gfB[2] += wi * cz(i) * eB; }
        if (is_gray) {
            float nA, nB;
            if (wall & (1u << i)) {
                nA = P.rho_wall[0];
                nB = P.rho_wall[1];
            } else {
                nA = r[0] + 3.0f * fix_diff(fiA[m], f0i[0]) + eA;
                nB = r[1] + 3.0f * fix_diff(fiB[m], f0i[1]) + eB;
            }
            const float nw = w == 0 ? nA : nB, nn = w == 0 ? nB : nA;
            const float den = nw + nn;
            const float At = den > 0.f ? (nw - nn) / den : 0.f;
            if (cx(i)) gAt[0] += wi * cx(i) * At;
            if (cy(i)) gAt[1] += wi * cy(i) * At;
            if (cz(i)) gAt[2] += wi * cz(i) * At;
        }
    }
    // grad(rho^A), grad(rho^B) in float-float; phi^A = rho^B, phi^B = rho^A
    ff grA[3], grB[3];
    float gA[3], gB[3];  // grad(phi^A) = grad(rho^B), grad(phi^B) = grad(rho^A) in FP32
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        grA[d] = ff_add_f(ff_from_ll(-ij[0][d], FIX_INV * 0.25f), gfA[d]);
        grB[d] = ff_add_f(ff_from_ll(-ij[1][d], FIX_INV * 0.25f), gfB[d]);
        gA[d] = grB[d].hi;
        gB[d] = grA[d].hi;
    }
    // Shan-Chen force in float-float: F^A = -G rho^A grad(rho^B), F^B = -G rho^B grad(rho^A)
    const ff Gff = {P.G, P.G_lo};
    ff Fsc[2][3];
    float F[2][3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        Fsc[0][d] = ff_mul(Gff, ff_mul(rho_ff[0], grB[d]));
        Fsc[1][d] = ff_mul(Gff, ff_mul(rho_ff[1], grA[d]));
        Fsc[0][d].hi = -Fsc[0][d].hi; Fsc[0][d].lo = -Fsc[0][d].lo;
        Fsc[1][d].hi = -Fsc[1][d].hi; Fsc[1][d].lo = -Fsc[1][d].lo;
        F[0][d] = r[0] * P.accel[0][d];  // the remaining (small) force terms, FP32
        F[1][d] = r[1] * P.accel[1][d];
    }

    // ---- CSF (Eq. 4) --------------------------------------------------------
    if (P.kappa != 0.0f && (P.csf_everywhere || is_gray)) {
        float divA = 0.f, divB = 0.f;
        for (int i = 1; i < Q; ++i) {
            if (wall & (1u << i)) continue;  // unit normals vanish at walls
            float nA[3], nB[3];
            normals_at(P, fiA, fiB, drA, drB, type, A.xs[cx(i) + 1], A.ys[cy(i) + 1], A.zs[cz(i) + 1], nA, nB);
            const float wi = w3(i);
            divA += wi * (cx(i) * nA[0] + cy(i) * nA[1] + cz(i) * nA[2]);
            divB += wi * (cx(i) * nB[0] + cy(i) * nB[1] + cz(i) * nB[2]);
        }
        const float kA = P.kappa * (-divA) * r[0] * P.csf_coef[0];
        const float kB = P.kappa * (-divB) * r[1] * P.csf_coef[1];
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            F[0][d] += kA * gA[d];
            F[1][d] += kB * gB[d];
        }
    }

    // ---- residual state, saturation, Eq. 1 forces and velocity -------------
    const float rw = r[w], rn = r[1 - w];
    float s = (rw / rt - P.r_lo) * P.inv_r_span;
    s = fminf(fmaxf(s, 0.f), 1.f);
    float sw = s;
    float u[3];
    if (is_gray) {
        const float4 ga = gray[c].a;
        const float4 gb = gray[c].b;
        unsigned meta = __float_as_uint(gb.w);
        bool wetf = meta & META_WET;
        bool swd = meta & META_SWITCHED;
        bool changed = false;
        if (wetf && s < P.s_lo) {
            wetf = false; swd = true; changed = true;
        } else if (!wetf && s > P.s_hi) {
            wetf = true; swd = true; changed = true;
        }
        if (changed) {
            meta = (meta & 0xffu) | (wetf ? META_WET : 0u) | META_SWITCHED;
            reinterpret_cast<float *>(gray + c)[7] = __uint_as_float(meta);
        }
        const float Rw = (swd && !wetf) ? gb.y : 0.f;
        const float Ro = (swd && wetf) ? gb.z : 0.f;
        sw = Rw + (1.f - Rw - Ro) * s;
        const Curve cv = P.curve[meta & 0xffu];

        // capillary term of Eq. 1: -Pc(Sw) rho_r n H, H = |grad At|/2
        const float At_c = (rw - rn) / (rw + rn);
        const float mag = sqrtf(gAt[0] * gAt[0] + gAt[1] * gAt[1] + gAt[2] * gAt[2]);
        const float H = (fabsf(At_c) <= P.at_cut) ? 0.5f * mag : 0.f;
        if (H > 0.f) {
            const float se_c = fminf(fmaxf((sw - cv.swr) * cv.inv_1m_swr, 1e-2f), 1.f);
            const float Pc = gb.x * powf(se_c, cv.neg_inv_lambda);
            const float k = -Pc * H / fmaxf(mag, P.eps_n);
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                F[0][d] += k * (r[0] / rt) * gAt[d];
                F[1][d] += k * (r[1] / rt) * gAt[d];
            }
        }
        // viscous term of Eq. 1 with K^-1 = (1/K0)(I + v v^T) (Eq. 7)
        const float se_k = fminf(fmaxf((sw - cv.swr) * cv.inv_1m_swr, 0.f), 1.f);
        const float kr_w = powf(se_k, cv.nw), kr_n = powf(1.f - se_k, cv.nn);
        const float coef = rw * P.nu[w] / fmaxf(kr_w, P.kr_min) + rn * P.nu[1 - w] / fmaxf(kr_n, P.kr_min);
        const float rk = coef * ga.w;  // coef / K0
        const float v[3] = {ga.x, ga.y, ga.z};
        // (rho I + R/2) u = j + F/2 with R = rk (I + v v^T): Sherman-Morrison
        float b[3];
#pragma unroll
        for (int d = 0; d < 3; ++d)
            b[d] = ff_add_f(ff_add(j_ff[d], ff_scale(ff_add(Fsc[0][d], Fsc[1][d]), 0.5f)),
                            0.5f * (F[0][d] + F[1][d])).hi;
        const float al = rt + 0.5f * rk, be = 0.5f * rk;
        const float vb = v[0] * b[0] + v[1] * b[1] + v[2] * b[2];
        const float vv = v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
        const float q = be * vb / (al + be * vv);
#pragma unroll
        for (int d = 0; d < 3; ++d) u[d] = (b[d] - q * v[d]) / al;
        const float vu = v[0] * u[0] + v[1] * u[1] + v[2] * u[2];
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            const float Ru = rk * (u[d] + v[d] * vu);
            F[0][d] -= (r[0] / rt) * Ru;
            F[1][d] -= (r[1] / rt) * Ru;
        }
    } else {
#pragma unroll
        for (int d = 0; d < 3; ++d)
            u[d] = ff_add_f(ff_add(j_ff[d], ff_scale(ff_add(Fsc[0][d], Fsc[1][d]), 0.5f)),
                            0.5f * (F[0][d] + F[1][d])).hi / rt;
    }
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        F[0][d] += Fsc[0][d].hi;
        F[1][d] += Fsc[1][d].hi;
    }

    // ---- regularised collision, written as rest population + deviations ---
    const float uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
#pragma unroll
    for (int a = 0; a < 2; ++a) {
        const float om = P.omega_fac[a];
        const float ra = r[a];
        const float *Fa = F[a];
        const float uF = u[0] * Fa[0] + u[1] * Fa[1] + u[2] * Fa[2];
        const float d3 = dr[a] * (1.0f / 3.0f);
        // Pi1 = sum c c h - (drho/3) I - rho u u + (uF + Fu)/2
        const float Pxx = S[a][0] - d3 - ra * u[0] * u[0] + u[0] * Fa[0];
        const float Pyy = S[a][1] - d3 - ra * u[1] * u[1] + u[1] * Fa[1];
        const float Pzz = S[a][2] - d3 - ra * u[2] * u[2] + u[2] * Fa[2];
        const float Pxy = S[a][3] - ra * u[0] * u[1] + 0.5f * (u[0] * Fa[1] + Fa[0] * u[1]);
        const float Pxz = S[a][4] - ra * u[0] * u[2] + 0.5f * (u[0] * Fa[2] + Fa[0] * u[2]);
        const float Pyz = S[a][5] - ra * u[1] * u[2] + 0.5f * (u[1] * Fa[2] + Fa[1] * u[2]);
        const float trP = Pxx + Pyy + Pzz;
        // f*_0 - f_0 = drho/3 - rho u^2/2 - om tr(Pi1)/2 - u.F/2, added exactly in
        // fixed point; the sub-grid residual goes into the moving populations.
        const float d0 = d3 - 0.5f * ra * uu - 0.5f * om * trP - 0.5f * uF;
        const float xq = d0 * FIX_ONE;
        const float qf = rintf(xq);
        const float res = (xq - qf) * FIX_INV;
        float *fo = fout + (size_t)a * Q * n;
        reinterpret_cast<int *>(fo)[c] = f0i[a] + (int)qf;
#pragma unroll
        for (int i = 1; i < Q; ++i) {
            const float cu = cx(i) * u[0] + cy(i) * u[1] + cz(i) * u[2];
            const float cF = cx(i) * Fa[0] + cy(i) * Fa[1] + cz(i) * Fa[2];
            float cPc = 0.f;
            if (cx(i)) cPc += Pxx;
            if (cy(i)) cPc += Pyy;
            if (cz(i)) cPc += Pzz;
            if (cx(i) && cy(i)) cPc += 2.0f * cx(i) * cy(i) * Pxy;
            if (cx(i) && cz(i)) cPc += 2.0f * cx(i) * cz(i) * Pxz;
            if (cy(i) && cz(i)) cPc += 2.0f * cy(i) * cz(i) * Pyz;
            const float g = wgt(i) * (ra * (3.0f * cu + 4.5f * cu * cu) + 4.5f * om * cPc + 1.5f * cF +
                                      4.5f * cu * cF + 3.0f * res);
            fo[(size_t)i * n + c] = g;
        }
    }
    if (MACRO) {
        macro[c] = r[0];
        macro[(size_t)n + c] = r[1];
        macro[(size_t)2 * n + c] = u[0];
        macro[(size_t)3 * n + c] = u[1];
        macro[(size_t)4 * n + c] = u[2];
        macro[(size_t)5 * n + c] = sw;
    }
}

// ---------------------------------------------------------------------------
// Launch wrappers
// ---------------------------------------------------------------------------
static inline dim3 grid_for(int n, int block) { return dim3((unsigned)((n + block - 1) / block)); }

cudaError_t launch_init(lbm_ctx *ctx, const float *rhoA, const float *rhoB, const float *u)
{
    cudaEvent_t e0;
    prof_begin(ctx, "k_init", &e0);
    k_init<<<grid_for(ctx->n, 256), 256, 0, ctx->stream>>>(ctx->dp, rhoA, rhoB, u, ctx->type,
                                                          ctx->f[ctx->cur], ctx->rho, ctx->macro,
                                                          ctx->gray);
    prof_end(ctx, "k_init", e0);
    ctx->launches += 1;
    return cudaGetLastError();
}

cudaError_t launch_density(lbm_ctx *ctx)
{
    cudaEvent_t e0;
    prof_begin(ctx, "k_density", &e0);
    k_density<<<grid_for(ctx->n, 256), 256, 0, ctx->stream>>>(ctx->dp, ctx->f[ctx->cur], ctx->type,
                                                             ctx->rho);
    prof_end(ctx, "k_density", e0);
    ctx->launches += 1;
    return cudaGetLastError();
}

cudaError_t launch_collide(lbm_ctx *ctx, bool write_macro)
{
    const float *fin = ctx->f[ctx->cur];
    float *fout = ctx->f[1 - ctx->cur];
    cudaEvent_t e0;
    prof_begin(ctx, "k_collide", &e0);
    if (write_macro)
        k_collide<true><<<grid_for(ctx->n, 256), 256, 0, ctx->stream>>>(
            ctx->dp, fin, fout, ctx->type, ctx->rho, ctx->gray, ctx->macro);
    else
        k_collide<false><<<grid_for(ctx->n, 256), 256, 0, ctx->stream>>>(
            ctx->dp, fin, fout, ctx->type, ctx->rho, ctx->gray, ctx->macro);
    prof_end(ctx, "k_collide", e0);
    ctx->launches += 1;
    ctx->cur = 1 - ctx->cur;
    return cudaGetLastError();
}

}  // namespace lbm
