// Time-step kernels of the two-component D3Q19 pseudo-potential LB model.
//
// Population storage (F32): for each component a and cell x the rest
// population f_0 is kept as is and every moving population as the deviation
//     g_i = f_i - 3 w_i f_0      (i = 1..18).
// Pulling f_i(x) = f*_i(x - c_i) then gives, relative to the puller's own rest
// population, h_i = f_i(x) - 3 w_i f_0(x) = g_i(s) + 3 w_i (f_0(s) - f_0(x))
// with s = x - c_i, and every moment is a sum of small numbers:
//     rho = 3 f_0 + sum h_i,   j = sum c_i h_i,   sum c c f = sum c c h + f_0 I.
// The post-collision deviations are written in closed form from the moments,
// so FP32 rounding acts on O(u, F, Pi_neq) quantities instead of on O(w rho)
// ones.  Mathematically the state is the same as plain populations.
//
// One step is two launches:
//   k_density  - pull, moments, rho^A / rho^B of every cell (solid cells hold
//                the virtual wall densities), the source of the stencils;
//   k_collide  - pull again, residual update, forces (Shan-Chen, CSF Eq. 4,
//                Eq. 1 capillary + tensorial viscous with the semi-implicit
//                velocity), regularised collision with the Eq. 3 force term,
//                store.
#include <cstdio>

#include "lbm_context.h"

namespace lbm {

__device__ __forceinline__ void cell_xyz(int c, const DevParams &P, int &x, int &y, int &z)
{
    x = c % P.nx;
    int t = c / P.nx;
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
    int X = A.xs[cx(i) + 1], Y = A.ys[cy(i) + 1], Z = A.zs[cz(i) + 1];
    return (X < 0 || Y < 0 || Z < 0) ? -1 : X + P.nx * (Y + P.ny * Z);
}

// ---------------------------------------------------------------------------
// Initial state: equilibrium of (rhoA, rhoB, u), evaluated in FP64 once.
// ---------------------------------------------------------------------------
__global__ void k_init(DevParams P, const float *__restrict__ rhoA, const float *__restrict__ rhoB,
                       const float *__restrict__ u, const uint8_t *__restrict__ type,
                       float *__restrict__ f, float *__restrict__ rho, float *__restrict__ macro,
                       GrayRec *__restrict__ gray)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    const int n = P.n;
    if (c >= n) return;
    const uint8_t t = type[c];
    if (t == CELL_SOLID) {
        for (int k = 0; k < 2 * Q; ++k) f[(size_t)k * n + c] = 0.0f;
        rho[c] = P.rho_wall[0];
        rho[n + c] = P.rho_wall[1];
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
        const float f0s = (float)f0;
        const double r0 = f0 - (double)f0s;
        fa[c] = f0s;
#pragma unroll
        for (int i = 1; i < Q; ++i) {
            const double cu = cx(i) * uv[0] + cy(i) * uv[1] + cz(i) * uv[2];
            const double g = wgt_d(i) * (r[a] * (3.0 * cu + 4.5 * cu * cu) + 3.0 * r0);
            fa[(size_t)i * n + c] = (float)g;
        }
        rho[(size_t)a * n + c] = (float)r[a];
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
// Densities of the current step (pull + zeroth moment).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_density(DevParams P, const float *__restrict__ f,
                                                 const uint8_t *__restrict__ type,
                                                 float *__restrict__ rho)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    const int n = P.n;
    if (c >= n) return;
    if (type[c] == CELL_SOLID) {
        rho[c] = P.rho_wall[0];
        rho[n + c] = P.rho_wall[1];
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
#pragma unroll
    for (int a = 0; a < 2; ++a) {
        const float *fa = f + (size_t)a * Q * n;
        const float f0 = fa[c];
        float acc = 0.0f;
#pragma unroll
        for (int i = 1; i < Q; ++i) {
            const int o = opp(i);
            float h;
            if (wall & (1u << o)) {
                h = fa[(size_t)o * n + c];
            } else {
                const int s = nb[o];
                h = fa[(size_t)i * n + s] + 3.0f * wgt(i) * (fa[s] - f0);
            }
            acc += h;
        }
        rho[(size_t)a * n + c] = 3.0f * f0 + acc;
    }
}

// Unit normals of grad(phi^A) = grad(rho^B) and grad(phi^B) = grad(rho^A) at
// the fluid cell (X, Y, Z).
__device__ __forceinline__ void normals_at(const DevParams &P, const float *__restrict__ rho, int X,
                                           int Y, int Z, float nA[3], float nB[3])
{
    const Axes A = axes_of(P, X, Y, Z);
    float gA[3] = {0.f, 0.f, 0.f}, gB[3] = {0.f, 0.f, 0.f};
#pragma unroll
    for (int k = 1; k < Q; ++k) {
        const int m = nb_index(P, A, k);
        const float rA = m < 0 ? P.rho_wall[0] : rho[m];
        const float rB = m < 0 ? P.rho_wall[1] : rho[P.n + m];
        const float w3 = 3.0f * wgt(k);
        gA[0] += w3 * cx(k) * rB; gA[1] += w3 * cy(k) * rB; gA[2] += w3 * cz(k) * rB;
        gB[0] += w3 * cx(k) * rA; gB[1] += w3 * cy(k) * rA; gB[2] += w3 * cz(k) * rA;
    }
    const float mA = fmaxf(sqrtf(gA[0] * gA[0] + gA[1] * gA[1] + gA[2] * gA[2]), P.eps_n);
    const float mB = fmaxf(sqrtf(gB[0] * gB[0] + gB[1] * gB[1] + gB[2] * gB[2]), P.eps_n);
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
                                                 const float *__restrict__ rho,
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

    // ---- moments of the pulled populations, per component ----------------
    float f0[2], dr[2], jm[2][3], S[2][6];
#pragma unroll
    for (int a = 0; a < 2; ++a) {
        const float *fa = fin + (size_t)a * Q * n;
        const float f0a = fa[c];
        float d = 0.f, j0 = 0.f, j1 = 0.f, j2 = 0.f;
        float sxx = 0.f, syy = 0.f, szz = 0.f, sxy = 0.f, sxz = 0.f, syz = 0.f;
#pragma unroll
        for (int i = 1; i < Q; ++i) {
            const int o = opp(i);
            float h;
            if (wall & (1u << o)) {
                h = fa[(size_t)o * n + c];
            } else {
                const int s = nb[o];
                h = fa[(size_t)i * n + s] + 3.0f * wgt(i) * (fa[s] - f0a);
            }
            d += h;
            if (cx(i)) { j0 += cx(i) * h; sxx += h; }
            if (cy(i)) { j1 += cy(i) * h; syy += h; }
            if (cz(i)) { j2 += cz(i) * h; szz += h; }
            if (cx(i) && cy(i)) sxy += cx(i) * cy(i) * h;
            if (cx(i) && cz(i)) sxz += cx(i) * cz(i) * h;
            if (cy(i) && cz(i)) syz += cy(i) * cz(i) * h;
        }
        f0[a] = f0a;
        dr[a] = d;
        jm[a][0] = j0; jm[a][1] = j1; jm[a][2] = j2;
        S[a][0] = sxx; S[a][1] = syy; S[a][2] = szz; S[a][3] = sxy; S[a][4] = sxz; S[a][5] = syz;
    }
    const float r[2] = {3.0f * f0[0] + dr[0], 3.0f * f0[1] + dr[1]};
    const float rt = r[0] + r[1];
    const float jt[3] = {jm[0][0] + jm[1][0], jm[0][1] + jm[1][1], jm[0][2] + jm[1][2]};
    const bool is_gray = (t == CELL_GRAY);
    const int w = P.wet;

    // ---- density stencils: grad(phi^a) with phi^A = rho^B, phi^B = rho^A;
    //      grad(At) in gray cells --------------------------------------------
    float gA[3] = {0.f, 0.f, 0.f}, gB[3] = {0.f, 0.f, 0.f}, gAt[3] = {0.f, 0.f, 0.f};
#pragma unroll
    for (int i = 1; i < Q; ++i) {
        const int m = nb[i];
        const float nA = m < 0 ? P.rho_wall[0] : rho[m];
        const float nB = m < 0 ? P.rho_wall[1] : rho[n + m];
        const float w3 = 3.0f * wgt(i);
        if (cx(i)) { gA[0] += w3 * cx(i) * nB; gB[0] += w3 * cx(i) * nA; }
        if (cy(i)) { gA[1] += w3 * cy(i) * nB; gB[1] += w3 * cy(i) * nA; }
        if (cz(i)) { gA[2] += w3 * cz(i) * nB; gB[2] += w3 * cz(i) * nA; }
        if (is_gray) {
            const float nw = w == 0 ? nA : nB, nn = w == 0 ? nB : nA;
            const float den = nw + nn;
            const float At = den > 0.f ? (nw - nn) / den : 0.f;
            if (cx(i)) gAt[0] += w3 * cx(i) * At;
            if (cy(i)) gAt[1] += w3 * cy(i) * At;
            if (cz(i)) gAt[2] += w3 * cz(i) * At;
        }
    }

    float F[2][3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        F[0][d] = -P.G * r[0] * gA[d] + r[0] * P.accel[0][d];
        F[1][d] = -P.G * r[1] * gB[d] + r[1] * P.accel[1][d];
    }

    // ---- CSF (Eq. 4) --------------------------------------------------------
    if (P.kappa != 0.0f && (P.csf_everywhere || is_gray)) {
        float divA = 0.f, divB = 0.f;
        for (int i = 1; i < Q; ++i) {
            if (wall & (1u << i)) continue;  // unit normals vanish at walls
            float nA[3], nB[3];
            normals_at(P, rho, A.xs[cx(i) + 1], A.ys[cy(i) + 1], A.zs[cz(i) + 1], nA, nB);
            const float w3 = 3.0f * wgt(i);
            divA += w3 * (cx(i) * nA[0] + cy(i) * nA[1] + cz(i) * nA[2]);
            divB += w3 * (cx(i) * nB[0] + cy(i) * nB[1] + cz(i) * nB[2]);
        }
        const float kA = P.kappa * (-divA) * r[0] * P.csf_coef[0];
        const float kB = P.kappa * (-divB) * r[1] * P.csf_coef[1];
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            F[0][d] += kA * gA[d];
            F[1][d] += kB * gB[d];
        }
    }

    // ---- residual state, saturation ----------------------------------------
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

        // capillary term of Eq. 1: -Pc(Sw) rho_r n H
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
        // (rho I + R/2) u = j + F/2, R = rk (I + v v^T): Sherman-Morrison
        float b[3];
#pragma unroll
        for (int d = 0; d < 3; ++d) b[d] = jt[d] + 0.5f * (F[0][d] + F[1][d]);
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
        for (int d = 0; d < 3; ++d) u[d] = (jt[d] + 0.5f * (F[0][d] + F[1][d])) / rt;
    }

    // ---- regularised collision, written as deviations ----------------------
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
        const float d0 = d3 - 0.5f * ra * uu - 0.5f * om * trP - 0.5f * uF;
        const float f0n = f0[a] + d0;
        const float res = (f0[a] - f0n) + d0;  // exact rounding residual of f0n
        float *fo = fout + (size_t)a * Q * n;
        fo[c] = f0n;
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
