// Two-dimensional variant of the step on D2Q9 (one plane, nz = 1), for the
// paper's two-dimensional experiments (Sec. III: the droplet of Sec. III.A,
// the random-porosity and fibre cases): the physics of the D3Q19 path --
// Shan-Chen force, Eq. 4 surface-tension control, Eq. 1 capillary and
// tensorial viscous terms in gray cells, the residual update of Eq. 5 /
// Fig. 6, the regularised forced collision, halfway bounce-back and the
// reservoir cells -- with the nine-velocity set (weights 4/9, 1/9, 1/36,
// cs^2 = 1/3).
//
// Storage (F32, push form like the 3-D F32 layout): per component, slot 0 of
// a cell holds its rest population f_0 in 2^-30 fixed point (int32); slot i
// (1..8) holds g_i = f_i - r_i f_0(s), the population that arrived from the
// source s = x - c_i relative to the source's rest population (s = x after a
// bounce-back), r_i = w_i / w_0 = 1/4 on faces, 1/16 on diagonals.  Then
// rho = f_0 / w_0 + sum_i g_i + sum_i r_i (f_0(s_i) - f_0(x)); the last sum is
// kept exactly in 64-bit integers with weights 16 r_i = 4, 1.  The force
// balance j + F_sc/2, where large terms nearly cancel at interfaces, is
// formed in float-float.  Two launches per step: densities (drho = rho -
// f_0/w_0 and the Atwood number of every fluid cell), then forces, collision
// and the push of the new populations.
#include "lbm_cell.cuh"
#include "lbm_context.h"

namespace lbm {
namespace d2 {

constexpr int Q = 9;
__host__ __device__ constexpr int cx(int i)
{
    constexpr int t[Q] = {0, 1, -1, 0, 0, 1, -1, 1, -1};
    return t[i];
}
__host__ __device__ constexpr int cy(int i)
{
    constexpr int t[Q] = {0, 0, 0, 1, -1, 1, -1, -1, 1};
    return t[i];
}
// opposite pairs (1,2), (3,4), (5,6), (7,8)
__host__ __device__ constexpr int opp(int i) { return i == 0 ? 0 : ((i & 1) ? i + 1 : i - 1); }
__host__ __device__ constexpr float wgt(int i) { return i == 0 ? 4.0f / 9.0f : (i <= 4 ? 1.0f / 9.0f : 1.0f / 36.0f); }
__host__ __device__ constexpr double wgt_d(int i) { return i == 0 ? 4.0 / 9.0 : (i <= 4 ? 1.0 / 9.0 : 1.0 / 36.0); }
// r_i = w_i / w_0 and its integer form 16 r_i
__host__ __device__ constexpr float rr(int i) { return i <= 4 ? 0.25f : 0.0625f; }
__host__ __device__ constexpr int r16(int i) { return i <= 4 ? 4 : 1; }
constexpr float FIX16 = FIX_INV * 0.0625f;  // 2^-34: exact scale of the 16 r_i sums
constexpr float FIX4 = FIX_INV * 0.25f;     // 2^-32: exact scale of 9 f_0 = 4 f_0 / w_0

__device__ __forceinline__ int nb(const DevParams &P, int x, int y, int dx, int dy)
{
    int X = x + dx, Y = y + dy;
    if (X < 0 || X >= P.nx) {
        if (!P.per[0]) return -1;
        X = X < 0 ? X + P.nx : X - P.nx;
    }
    if (Y < 0 || Y >= P.ny) {
        if (!P.per[1]) return -1;
        Y = Y < 0 ? Y + P.ny : Y - P.ny;
    }
    return X + P.nx * Y;
}

// rho - f_0/w_0 of a reservoir cell (float-float)
__device__ __forceinline__ ff held_dev2(ff rho, int f0) { return ff_add(rho, ff_from_ll(-9LL * f0, FIX4)); }

__device__ __forceinline__ float atwood2(int w, int f0A, int f0B, float drA, float drB)
{
    const float rA = fmaf((float)f0A, 2.25f * FIX_INV, drA), rB = fmaf((float)f0B, 2.25f * FIX_INV, drB);
    const float nw = w == 0 ? rA : rB, nn = w == 0 ? rB : rA;
    const float den = nw + nn;
    return den > 0.f ? __fdividef(nw - nn, den) : 0.f;
}

// ---------------------------------------------------------------------------
// Initial state: equilibrium of (rhoA, rhoB, u), FP64 once, pushed like a step.
__global__ void k2_init(DevParams P, const float *__restrict__ rhoA, const float *__restrict__ rhoB,
                        const float *__restrict__ u, const uint8_t *__restrict__ type, float *__restrict__ f,
                        float *__restrict__ macro, GrayRec *__restrict__ gray)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    const int n = P.n;
    if (c >= n) return;
    const uint8_t t = type[c];
    if (t == CELL_SOLID) {
        for (int a = 0; a < 2; ++a) {
            reinterpret_cast<int *>(f + (size_t)a * Q * n)[c] = 0;
            for (int i = 1; i < Q; ++i) f[((size_t)a * Q + i) * n + c] = 0.0f;
        }
        for (int k = 0; k < 6; ++k) macro[(size_t)k * n + c] = 0.0f;
        return;
    }
    const int x = c % P.nx, y = c / P.nx;
    const double ux = u ? (double)u[c] : 0.0, uy = u ? (double)u[(size_t)n + c] : 0.0;
    const double uu = ux * ux + uy * uy;
    const double r[2] = {(double)rhoA[c], (double)rhoB[c]};
    for (int a = 0; a < 2; ++a) {
        float *fa = f + (size_t)a * Q * n;
        const double f0 = wgt_d(0) * r[a] * (1.0 - 1.5 * uu);
        const long long q = llrint(f0 * FIX_ONE_D);
        const double res = f0 - (double)q / FIX_ONE_D;
        reinterpret_cast<int *>(fa)[c] = (int)q;
        for (int i = 1; i < Q; ++i) {
            // f_i^eq - r_i f_0q = w_i rho (3 cu + 4.5 cu^2) + r_i res
            const double cu = cx(i) * ux + cy(i) * uy;
            const double g = wgt_d(i) * r[a] * (3.0 * cu + 4.5 * cu * cu) + (double)rr(i) * res;
            const int m = nb(P, x, y, cx(i), cy(i));
            const bool wl = m < 0 || type[m] == CELL_SOLID;
            fa[wl ? (size_t)opp(i) * n + c : (size_t)i * n + m] = (float)g;
        }
    }
    const double rw = r[P.wet], rn = r[1 - P.wet];
    double s = ((rw / (rw + rn)) - (double)P.r_lo) * (double)P.inv_r_span;
    s = s < 0.0 ? 0.0 : (s > 1.0 ? 1.0 : s);
    macro[c] = (float)r[0];
    macro[(size_t)n + c] = (float)r[1];
    macro[(size_t)2 * n + c] = (float)ux;
    macro[(size_t)3 * n + c] = (float)uy;
    macro[(size_t)4 * n + c] = 0.0f;
    macro[(size_t)5 * n + c] = (float)s;
    if (t == CELL_GRAY) {
        unsigned meta = __float_as_uint(gray[c].b.w) & 0xffu;
        if (s >= 0.5) meta |= META_WET;
        gray[c].b.w = __uint_as_float(meta);
    }
}

// ---------------------------------------------------------------------------
// drho = rho - f_0/w_0 of both components and the Atwood number.
__global__ void __launch_bounds__(256) k2_density(DevParams P, const float *__restrict__ f,
                                                  const uint8_t *__restrict__ type, float *__restrict__ drho)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    const int n = P.n;
    if (c >= n) return;
    const uint8_t t = type[c];
    if (t == CELL_SOLID) return;
    const int x = c % P.nx, y = c / P.nx;
    int nbi[Q];
    unsigned wall = 0;
#pragma unroll
    for (int i = 1; i < Q; ++i) {
        nbi[i] = nb(P, x, y, cx(i), cy(i));
        if (nbi[i] < 0 || type[nbi[i]] == CELL_SOLID) wall |= 1u << i;
    }
    int f0s[2];
#pragma unroll
    for (int a = 0; a < 2; ++a) {
        const float *fa = f + (size_t)a * Q * n;
        const int *fi = reinterpret_cast<const int *>(fa);
        const int f0 = fi[c];
        f0s[a] = f0;
        float acc = 0.0f;
        long long id = 0;
#pragma unroll
        for (int i = 1; i < Q; ++i) {
            const int o = opp(i);  // the source x - c_i is x + c_o
            acc += fa[(size_t)i * n + c];
            if (!(wall & (1u << o))) id += (long long)(fi[nbi[o]] - f0) * r16(i);
        }
        ff v = ff_add_f(ff_from_ll(id, FIX16), acc);
        if (is_held(t)) v = held_dev2(held_rho(P.held, t, a), f0);
        drho[(size_t)a * n + c] = v.hi;
    }
    drho[(size_t)2 * n + c] = atwood2(P.wet, f0s[0], f0s[1], drho[c], drho[n + c]);
}

// ---------------------------------------------------------------------------
// Forces, residual update, velocity, regularised collision and push.
template <bool MACRO>
__global__ void __launch_bounds__(256) k2_collide(DevParams P, const float *__restrict__ fin, float *__restrict__ fout,
                                                  const uint8_t *__restrict__ type, const float *__restrict__ drho,
                                                  GrayRec *__restrict__ gray, float *__restrict__ macro)
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
    const int x = c % P.nx, y = c / P.nx;
    int nbi[Q];
    unsigned wall = 0;
#pragma unroll
    for (int i = 1; i < Q; ++i) {
        nbi[i] = nb(P, x, y, cx(i), cy(i));
        if (nbi[i] < 0 || type[nbi[i]] == CELL_SOLID) wall |= 1u << i;
    }
    const bool held = is_held(t);
    const bool is_gray = t == CELL_GRAY;
    const int w = P.wet;

    // ---- moments of the pulled populations (relative to the own f_0) -------
    int f0i[2];
    ff rho[2], dr[2], j[2][2];
    long long Ij[2][2];
    float S[2][3];  // xx, yy, xy
#pragma unroll
    for (int a = 0; a < 2; ++a) {
        const float *fa = fin + (size_t)a * Q * n;
        const int *fi = reinterpret_cast<const int *>(fa);
        const int f0 = fi[c];
        f0i[a] = f0;
        float d = 0.f, jx = 0.f, jy = 0.f, sxx = 0.f, syy = 0.f, sxy = 0.f;
        long long Id = 0, Ix = 0, Iy = 0;
#pragma unroll
        for (int i = 1; i < Q; ++i) {
            const int o = opp(i);
            const float g = fa[(size_t)i * n + c];
            const int d0 = (wall & (1u << o)) ? 0 : fi[nbi[o]] - f0;
            const long long D = (long long)d0 * r16(i);
            const float h = fmaf(rr(i) * FIX_INV, (float)d0, g);
            d += g;
            Id += D;
            if (cx(i)) { jx += cx(i) * g; Ix += cx(i) * D; sxx += h; }
            if (cy(i)) { jy += cy(i) * g; Iy += cy(i) * D; syy += h; }
            if (cx(i) && cy(i)) sxy += cx(i) * cy(i) * h;
        }
        if (held) {  // reservoir: held density at rest, no force
            rho[a] = held_rho(P.held, t, a);
            dr[a] = held_dev2(rho[a], f0);
            j[a][0] = j[a][1] = ff{0.f, 0.f};
            Ij[a][0] = Ij[a][1] = 0;
            S[a][0] = S[a][1] = dr[a].hi * (1.0f / 3.0f);
            S[a][2] = 0.f;
        } else {
            dr[a] = ff_add_f(ff_from_ll(Id, FIX16), d);
            rho[a] = ff_add(ff_from_ll(9LL * f0, FIX4), dr[a]);
            j[a][0] = ff_add_f(ff_from_ll(Ix, FIX16), jx);
            j[a][1] = ff_add_f(ff_from_ll(Iy, FIX16), jy);
            Ij[a][0] = Ix;
            Ij[a][1] = Iy;
            S[a][0] = sxx;
            S[a][1] = syy;
            S[a][2] = sxy;
        }
    }
    const float r[2] = {rho[0].hi, rho[1].hi};
    const float rt = r[0] + r[1];

    // ---- density stencils: gradients (Shan-Chen), Hessians (Eq. 4), grad At ----
    const bool csf = !held && P.kappa != 0.0f && (P.csf_everywhere || is_gray);
    const float drc[2] = {drho[c], drho[n + c]};
    float gf[2][2] = {{0.f, 0.f}, {0.f, 0.f}}, gAt[2] = {0.f, 0.f};
    float hm[2][3] = {{0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}}, hl[2] = {0.f, 0.f};  // sum w c c d, sum w d
    const int *fiA = reinterpret_cast<const int *>(fin);
    const int *fiB = reinterpret_cast<const int *>(fin + (size_t)Q * n);
#pragma unroll
    for (int i = 1; i < Q; ++i) {
        const int m = nbi[i];
        const bool wl = wall & (1u << i);
        float e[2];
#pragma unroll
        for (int a = 0; a < 2; ++a) e[a] = wl ? P.rho_wall[a] - r[a] : drho[(size_t)a * n + m] - drc[a];
        const float w3i = 3.0f * wgt(i);
#pragma unroll
        for (int a = 0; a < 2; ++a) {
            if (cx(i)) gf[a][0] += w3i * cx(i) * e[a];
            if (cy(i)) gf[a][1] += w3i * cy(i) * e[a];
        }
        if (is_gray) {
            const float at = wl ? P.at_wall : drho[(size_t)2 * n + m];
            if (cx(i)) gAt[0] += w3i * cx(i) * at;
            if (cy(i)) gAt[1] += w3i * cy(i) * at;
        }
        if (csf) {
#pragma unroll
            for (int a = 0; a < 2; ++a) {
                const int *fi = a ? fiB : fiA;
                const float dd = wl ? e[a] : 2.25f * fix_diff(fi[m], f0i[a]) + e[a];
                const float wd = wgt(i) * dd;
                hl[a] += wd;
                if (cx(i)) hm[a][0] += wd;
                if (cy(i)) hm[a][1] += wd;
                if (cx(i) && cy(i)) hm[a][2] += cx(i) * cy(i) * wd;
            }
        }
    }
    // grad(rho^a) in float-float: the rest-population part is
    // 3 sum_i w_i c_i (f_0(x+c_i) - f_0(x)) / w_0 = -3 * 2^-34 Ij
    ff gr[2][2];
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int d = 0; d < 2; ++d) gr[a][d] = held ? ff{0.f, 0.f} : ff_add_f(ff_from_ll(-3LL * Ij[a][d], FIX16), gf[a][d]);
    // Shan-Chen: F^A = -G rho^A grad(rho^B), F^B = -G rho^B grad(rho^A)
    const ff Gff = {P.G, P.G_lo};
    ff Fsc[2][2];
#pragma unroll
    for (int d = 0; d < 2; ++d) {
        Fsc[0][d] = ff_mul(Gff, ff_mul(rho[0], gr[1][d]));
        Fsc[1][d] = ff_mul(Gff, ff_mul(rho[1], gr[0][d]));
        for (int a = 0; a < 2; ++a) {
            Fsc[a][d].hi = -Fsc[a][d].hi;
            Fsc[a][d].lo = -Fsc[a][d].lo;
        }
    }
    float F[2][3] = {{0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}};
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int d = 0; d < 2; ++d) F[a][d] = held ? 0.f : r[a] * P.accel[a][d];
    ff Bmix[2];
#pragma unroll
    for (int d = 0; d < 2; ++d)
        Bmix[d] = ff_add(ff_add(j[0][d], j[1][d]), ff_scale(ff_add(Fsc[0][d], Fsc[1][d]), 0.5f));

    // Eq. 4: kappa (-div n^a) (grad phi^a / phi_avg) (rho^a / phi_max), phi^A = rho^B;
    // div n = tr(H)/s - g.H.g/s^3 with the plane's moment Hessian H = 9 M - 3 L I
    if (csf) {
#pragma unroll
        for (int a = 0; a < 2; ++a) {
            const int b = 1 - a;
            const float g[2] = {gr[b][0].hi, gr[b][1].hi};
            const float Hxx = 9.f * hm[b][0] - 3.f * hl[b], Hyy = 9.f * hm[b][1] - 3.f * hl[b], Hxy = 9.f * hm[b][2];
            const float gHg = g[0] * (Hxx * g[0] + 2.f * Hxy * g[1]) + g[1] * Hyy * g[1];
            const float is = rsqrtf(g[0] * g[0] + g[1] * g[1] + P.eps_n * P.eps_n);
            const float div = is * ((Hxx + Hyy) - gHg * is * is);
            const float k = P.kappa * (-div) * r[a] * P.csf_coef[a];
            F[a][0] += k * g[0];
            F[a][1] += k * g[1];
        }
    }

    // ---- residual state, saturation, Eq. 1 forces and velocity --------------
    const float rw = r[w], rn = r[1 - w];
    float s = (rw / rt - P.r_lo) * P.inv_r_span;
    s = fminf(fmaxf(s, 0.f), 1.f);
    float sw = s;
    float u[2] = {0.f, 0.f};
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
        const float irt = __fdividef(1.0f, rt);
        const float At_c = __fdividef(rw - rn, rw + rn);
        const float mag = sqrtf(gAt[0] * gAt[0] + gAt[1] * gAt[1]);
        const float H = (fabsf(At_c) <= P.at_cut) ? 0.5f * mag : 0.f;
        if (H > 0.f) {  // capillary term of Eq. 1: -Pc(Sw) rho_r n H
            const float se_c = fminf(fmaxf((sw - cv.swr) * cv.inv_1m_swr, 1e-2f), 1.f);
            const float pw = cv.thomeer_k != 0.f ? exp2f(fminf(cv.thomeer_k / log1pf(-se_c), LOG2_10))
                                                 : __powf(se_c, cv.neg_inv_lambda);
            const float k = __fdividef(-gb.x * pw * H, fmaxf(mag, P.eps_n)) * irt;
            for (int d = 0; d < 2; ++d) {
                F[0][d] += k * r[0] * gAt[d];
                F[1][d] += k * r[1] * gAt[d];
            }
        }
        // viscous term with K^-1 = (1/K0)(I + v v^T) (Eq. 7; v in the plane),
        // (rho I + R/2) u = j + F/2 by Sherman-Morrison
        const float se_k = fminf(fmaxf((sw - cv.swr) * cv.inv_1m_swr, 0.f), 1.f);
        const float kr_w = se_k > 0.f ? __powf(se_k, cv.nw) : 0.f;
        const float kr_n = se_k < 1.f ? __powf(1.f - se_k, cv.nn) : 0.f;
        const float coef = __fdividef(rw * P.nu[w], fmaxf(kr_w, P.kr_min)) +
                           __fdividef(rn * P.nu[1 - w], fmaxf(kr_n, P.kr_min));
        const float rk = coef * ga.w;
        const float v[2] = {ga.x, ga.y};
        float b[2];
        for (int d = 0; d < 2; ++d) b[d] = ff_add_f(Bmix[d], 0.5f * (F[0][d] + F[1][d])).hi;
        const float al = rt + 0.5f * rk, be = 0.5f * rk;
        const float vb = v[0] * b[0] + v[1] * b[1];
        const float vv = v[0] * v[0] + v[1] * v[1] + ga.z * ga.z;
        const float q = __fdividef(be * vb, al + be * vv);
        const float ial = __fdividef(1.0f, al);
        for (int d = 0; d < 2; ++d) u[d] = (b[d] - q * v[d]) * ial;
        const float vu = v[0] * u[0] + v[1] * u[1];
        for (int d = 0; d < 2; ++d) {
            const float Ru = rk * (u[d] + v[d] * vu) * irt;
            F[0][d] -= r[0] * Ru;
            F[1][d] -= r[1] * Ru;
        }
    } else if (!held) {
        for (int d = 0; d < 2; ++d) u[d] = ff_add_f(Bmix[d], 0.5f * (F[0][d] + F[1][d])).hi / rt;
    }
#pragma unroll
    for (int d = 0; d < 2; ++d) {
        F[0][d] += Fsc[0][d].hi;
        F[1][d] += Fsc[1][d].hi;
    }

    // ---- regularised collision and push --------------------------------------
    const float uu = u[0] * u[0] + u[1] * u[1];
    // mass-sink-source: dm = m I from the non-wetting to the wetting component
    float dm = 0.f;
    if (!held && P.mss != 0.f) {
        const float it = __fdividef(1.0f, rt);
        dm = P.mss * fmaxf((4.0f * (rw * it) * (rn * it) - P.mss_ib) * P.mss_inv, 0.f);
    }
    auto tgt = [&](int i) -> size_t {
        return (wall & (1u << i)) ? (size_t)opp(i) * n + c : (size_t)i * n + nbi[i];
    };
#pragma unroll
    for (int a = 0; a < 2; ++a) {
        const float om = P.omega_fac[a];
        const float ra = r[a];
        const float *Fa = F[a];
        const float uF = u[0] * Fa[0] + u[1] * Fa[1];
        const float d3 = dr[a].hi * (1.0f / 3.0f);
        // Pi1 = sum c c h - (drho/3) I - rho u u + (uF + Fu)/2
        const float Pxx = S[a][0] - d3 - ra * u[0] * u[0] + u[0] * Fa[0];
        const float Pyy = S[a][1] - d3 - ra * u[1] * u[1] + u[1] * Fa[1];
        const float Pxy = S[a][2] - ra * u[0] * u[1] + 0.5f * (u[0] * Fa[1] + Fa[0] * u[1]);
        // f*_0 - f_r = w_0 drho - (2/3)(rho u^2 + om tr(Pi1) + u.F)
        const float d0 = (4.0f / 9.0f) * (dr[a].hi + (a == w ? dm : -dm)) -
                         (2.0f / 3.0f) * (ra * uu + om * (Pxx + Pyy) + uF);
        const float xq = d0 * FIX_ONE;
        const float qf = rintf(xq);
        float *fo = fout + (size_t)a * Q * n;
        reinterpret_cast<int *>(fo)[c] = f0i[a] + (int)qf;
        const float res = (xq - qf) * FIX_INV;
        // f*_i - r_i f*_0 = E +- O for the opposite pairs (i, i+1)
#pragma unroll
        for (int i = 1; i < Q; i += 2) {
            const float cu = cx(i) * u[0] + cy(i) * u[1];
            const float cF = cx(i) * Fa[0] + cy(i) * Fa[1];
            float cPc = 0.f;
            if (cx(i)) cPc += Pxx;
            if (cy(i)) cPc += Pyy;
            if (cx(i) && cy(i)) cPc += 2.0f * cx(i) * cy(i) * Pxy;
            const float E = wgt(i) * (4.5f * ra * cu * cu + 4.5f * om * cPc + 4.5f * cu * cF + 2.25f * res);
            const float O = wgt(i) * (3.0f * ra * cu + 1.5f * cF);
            fo[tgt(i)] = E + O;
            fo[tgt(i + 1)] = E - O;
        }
    }
    if (MACRO) {
        macro[c] = r[0];
        macro[(size_t)n + c] = r[1];
        macro[(size_t)2 * n + c] = u[0];
        macro[(size_t)3 * n + c] = u[1];
        macro[(size_t)4 * n + c] = 0.0f;
        macro[(size_t)5 * n + c] = sw;
    }
}

}  // namespace d2

static unsigned grid256(int n) { return (unsigned)((n + 255) / 256); }

cudaError_t launch_d2q9_init(lbm_ctx *ctx, const float *rhoA, const float *rhoB, const float *u)
{
    cudaEvent_t e0;
    prof_begin(ctx, "k2_init", &e0);
    d2::k2_init<<<grid256(ctx->n), 256, 0, ctx->stream>>>(ctx->dp, rhoA, rhoB, u, ctx->type, ctx->f[ctx->cur],
                                                          ctx->macro, ctx->gray);
    prof_end(ctx, "k2_init", e0);
    ctx->launches += 1;
    return cudaGetLastError();
}

cudaError_t launch_d2q9_step(lbm_ctx *ctx, bool write_macro)
{
    const float *fin = ctx->f[ctx->cur];
    float *fout = ctx->f[1 - ctx->cur];
    cudaEvent_t e0;
    prof_begin(ctx, "k2_density", &e0);
    d2::k2_density<<<grid256(ctx->n), step_block(ctx, 256), 0, ctx->stream>>>(ctx->dp, fin, ctx->type, ctx->rho);
    prof_end(ctx, "k2_density", e0);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    ctx->launches += 1;
    prof_begin(ctx, "k2_collide", &e0);
    const dim3 blk = step_block(ctx, 256);
    if (write_macro)
        d2::k2_collide<true><<<grid256(ctx->n), blk, 0, ctx->stream>>>(ctx->dp, fin, fout, ctx->type, ctx->rho,
                                                                      ctx->gray, ctx->macro);
    else
        d2::k2_collide<false><<<grid256(ctx->n), blk, 0, ctx->stream>>>(ctx->dp, fin, fout, ctx->type, ctx->rho,
                                                                       ctx->gray, ctx->macro);
    prof_end(ctx, "k2_collide", e0);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;  // nothing ran: the state stays in buffer cur
    ctx->launches += 1;
    ctx->cur = 1 - ctx->cur;
    return cudaSuccess;
}

}  // namespace lbm
