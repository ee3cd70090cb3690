// Hand-written discrete adjoint of the time step with respect to the
// populations and, through the gray-cell constants of the geometry
// precompute, the per-cell porosity (Eqs. 1 and 4-7).
//
// One adjoint step (going backwards, step n):
//   k_adj_cell   per fluid cell x (one thread per entry of a list of the
//                fluid cells, in groups of consecutive cells with each
//                group's plain pore cells first, then its gray cells, each
//                section whole warps, so that a warp takes one branch of the
//                gray-cell terms and no lane idles on a solid cell):
//                recomputes the cell's forward map in FP32
//                from the stored state of step n, takes the adjoints of its 38
//                outputs from lam^{n+1} at their push targets (own part plus
//                the target cell's gathered neighbour term), and runs the
//                map in reverse: moments, regularised collision with the
//                Eq. 3 force term, semi-implicit velocity (Sherman-Morrison),
//                drag, capillary term, residual saturation, CSF curvature,
//                Shan-Chen.  It writes the adjoint of its own arrived
//                populations, the adjoints of its 18 neighbours' densities
//                (one slot per direction, contrib[b][i][x]) and accumulates
//                the adjoints of its gray constants (v = sqrt(a-1) e1, 1/K0,
//                lamL*pd, Sw_irr, So_res);
//   k_adj_finish V^n(y) = sum_i contrib[b][i][y - c_i], the neighbour term,
//                the same on every slot of y (rho = sum f), so stored once
//                per cell and component and added where lam^n is read: the
//                adjoint of a push is a pull, so the neighbour terms are
//                gathered in a fixed order (no atomics; the gradient does not
//                depend on the scheduling).
// After the last adjoint step k_geom_adjoint chains the gray constants to phi
// (Kozeny-Carman, Leverett, the residual crossings and the principal axis,
// d e1 = sum_{k != 1} e_k (e_k^T dM e1)/(mu1 - mu_k)), in FP64.
// Piecewise-constant parts (residual hysteresis, the H(At) cut-off, clamps
// and floors) contribute their active branch only.
#include <algorithm>
#include <cmath>
#include <vector>

#include "lbm_context.h"
#include "lbm_host.h"

using namespace lbm_host;

namespace lbm {

// Adjoint seeds of the loss on the last step's fields.
struct AdjSeed {
    int on;        // seeds apply in this step
    float lux;     // dL/du_x on the plane x = nx - 1
    float lsw;     // dL/dSw = lsw * phi_c on non-solid cells
};

__device__ __forceinline__ float adj_phi_c(uint8_t t, float ph) { return t == CELL_GRAY ? ph : 1.0f; }

// Pc / Pe of a curve at the clamped normalised saturation se and its
// derivative in se: Brooks-Corey se^(-1/lambda); Thomeer
// 2^min(k / ln(1 - se), log2 10) (derivative pw ln2 k / (ln(1 - se)^2 (1 - se))
// below the cap, 0 on it; 1 with derivative 0 at se = 1, where the clamp
// stops the adjoint anyway).
__device__ __forceinline__ float pc_shape(const Curve &cv, float se, float &dpw)
{
    if (cv.thomeer_k != 0.f) {
        const float om = 1.f - se;
        if (!(om > 0.f)) {
            dpw = 0.f;
            return 1.f;
        }
        const float L = log1pf(-se);
        const float E = cv.thomeer_k / L;
        if (E >= LOG2_10) {
            dpw = 0.f;
            return 10.f;
        }
        const float pw = exp2f(E);
        dpw = pw * 0.69314718f * cv.thomeer_k / (L * L * om);
        return pw;
    }
    const float pw = powf(se, cv.neg_inv_lambda);
    dpw = cv.neg_inv_lambda * pw / se;
    return pw;
}

template <int N>
__device__ __forceinline__ float dotn(const float *a, const float *b)
{
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < N; ++k) s += a[k] * b[k];
    return s;
}

// symmetric 3x3 from [xx, yy, zz, xy, xz, yz]
__device__ __forceinline__ void symv(const float S[6], const float v[3], float out[3])
{
    out[0] = S[0] * v[0] + S[3] * v[1] + S[4] * v[2];
    out[1] = S[3] * v[0] + S[1] * v[1] + S[5] * v[2];
    out[2] = S[4] * v[0] + S[5] * v[1] + S[2] * v[2];
}
// c^T S c for lattice direction i
__device__ __forceinline__ float cSc(int i, const float S[6])
{
    return cx(i) * cx(i) * S[0] + cy(i) * cy(i) * S[1] + cz(i) * cz(i) * S[2] +
           2.f * (cx(i) * cy(i) * S[3] + cx(i) * cz(i) * S[4] + cy(i) * cz(i) * S[5]);
}

// v[k] += x for a runtime index k of a two-element array, as selects (an
// indexed access would put the array in local memory)
__device__ __forceinline__ void add_at(float (&v)[2], int k, float x)
{
    v[0] += k == 0 ? x : 0.f;
    v[1] += k == 1 ? x : 0.f;
}

__global__ void __launch_bounds__(128, 3) k_adj_cell(DevParams P, const float *__restrict__ fin,
                                                  const float *__restrict__ rhob, const uint8_t *__restrict__ type,
                                                  const float *__restrict__ phi, const GrayRec *__restrict__ gray,
                                                  const float *__restrict__ lam_next,
                                                  const float *__restrict__ v_next, float *__restrict__ lam_out,
                                                  float *__restrict__ contrib, double *__restrict__ gacc,
                                                  AdjSeed seed, const int *__restrict__ cells, int ncells)
{
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= ncells) return;
    const int c = cells[e];
    if (c < 0) return;
    const int n = P.n;
    const uint8_t t = type[c];
    const int x = c % P.nx, y = (c / P.nx) % P.ny, z = c / (P.nx * P.ny);
    int nb[Q];
    unsigned wall = 0;
#pragma unroll
    for (int i = 1; i < Q; ++i) {
        const int X = axis_nb(x, cx(i), P.nx, P.per[0]), Y = axis_nb(y, cy(i), P.ny, P.per[1]),
                  Z = axis_nb(z, cz(i), P.nz, P.per[2]);
        nb[i] = (X < 0 || Y < 0 || Z < 0) ? -1 : X + P.nx * (Y + P.ny * Z);
        if (nb[i] < 0 || type[nb[i]] == CELL_SOLID) wall |= 1u << i;
    }
    const int *fi = reinterpret_cast<const int *>(fin);
    // ---------------- forward recomputation (FP32, plain populations) -------
    float f[2][Q];
    float rho[2], j[2][3], Pm[2][6];
#pragma unroll
    for (int a = 0; a < 2; ++a) {
        const int f0 = fi[(size_t)a * Q * n + c];
        f[a][0] = (float)f0 * FIX_INV;
        rho[a] = f[a][0];
        j[a][0] = j[a][1] = j[a][2] = 0.f;
#pragma unroll
        for (int k = 0; k < 6; ++k) Pm[a][k] = 0.f;
#pragma unroll
        for (int i = 1; i < Q; ++i) {
            const int o = opp(i);
            const int fs = (wall & (1u << o)) ? f0 : fi[(size_t)a * Q * n + nb[o]];
            const float v = fin[(size_t)a * Q * n + (size_t)i * n + c] + w3(i) * ((float)fs * FIX_INV);
            f[a][i] = v;
            rho[a] += v;
            j[a][0] += cx(i) * v;
            j[a][1] += cy(i) * v;
            j[a][2] += cz(i) * v;
            Pm[a][0] += cx(i) * cx(i) * v;
            Pm[a][1] += cy(i) * cy(i) * v;
            Pm[a][2] += cz(i) * cz(i) * v;
            Pm[a][3] += cx(i) * cy(i) * v;
            Pm[a][4] += cx(i) * cz(i) * v;
            Pm[a][5] += cy(i) * cz(i) * v;
        }
    }
    // neighbour densities seen by the stencils and their Atwood numbers
    float rn[2][Q], at[Q];
#pragma unroll
    for (int i = 1; i < Q; ++i) {
        if (wall & (1u << i)) {
            rn[0][i] = P.rho_wall[0];
            rn[1][i] = P.rho_wall[1];
            at[i] = P.at_wall;
        } else {
            const int m = nb[i];
            rn[0][i] = (float)fi[m] * (3.0f * FIX_INV) + rhob[m];
            rn[1][i] = (float)fi[(size_t)Q * n + m] * (3.0f * FIX_INV) + rhob[n + m];
            at[i] = rhob[2 * (size_t)n + m];
        }
    }
    const float rt = rho[0] + rho[1];
    float grad[2][3];
#pragma unroll
    for (int b = 0; b < 2; ++b)
#pragma unroll
        for (int d = 0; d < 3; ++d) grad[b][d] = 0.f;
#pragma unroll
    for (int i = 1; i < Q; ++i)
#pragma unroll
        for (int b = 0; b < 2; ++b) {
            grad[b][0] += w3(i) * cx(i) * rn[b][i];
            grad[b][1] += w3(i) * cy(i) * rn[b][i];
            grad[b][2] += w3(i) * cz(i) * rn[b][i];
        }
    const bool is_gray = t == CELL_GRAY;
    const bool csf = P.kappa != 0.0f && (P.csf_everywhere || is_gray);
    float Fp[2][3];  // forces before the drag
    float Hs[2][6], trH[2], sN[2], gHg[2], dv[2];  // CSF intermediates per component (a: H of rho^{1-a})
#pragma unroll
    for (int a = 0; a < 2; ++a) {
        const float *g = grad[1 - a];
#pragma unroll
        for (int d = 0; d < 3; ++d) Fp[a][d] = -P.G * rho[a] * g[d] + rho[a] * P.accel[a][d];
        if (csf) {
            const int b = 1 - a;
            float M6[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f}, Lw = 0.f;
#pragma unroll
            for (int i = 1; i < Q; ++i) {
                const float wd = wgt(i) * (rn[b][i] - rho[b]);
                Lw += wd;
                M6[0] += cx(i) * cx(i) * wd;
                M6[1] += cy(i) * cy(i) * wd;
                M6[2] += cz(i) * cz(i) * wd;
                M6[3] += cx(i) * cy(i) * wd;
                M6[4] += cx(i) * cz(i) * wd;
                M6[5] += cy(i) * cz(i) * wd;
            }
#pragma unroll
            for (int k = 0; k < 3; ++k) Hs[a][k] = 9.f * M6[k] - 3.f * Lw;
#pragma unroll
            for (int k = 3; k < 6; ++k) Hs[a][k] = 9.f * M6[k];
            trH[a] = Hs[a][0] + Hs[a][1] + Hs[a][2];
            float Hg[3];
            symv(Hs[a], g, Hg);
            gHg[a] = dotn<3>(g, Hg);
            sN[a] = sqrtf(dotn<3>(g, g) + P.eps_n * P.eps_n);
            dv[a] = trH[a] / sN[a] - gHg[a] / (sN[a] * sN[a] * sN[a]);
            const float kc = P.kappa * (-dv[a]) * P.csf_coef[a] * rho[a];
#pragma unroll
            for (int d = 0; d < 3; ++d) Fp[a][d] += kc * g[d];
        }
    }
    const int w = P.wet;
    const float nu_w = w ? P.nu[1] : P.nu[0], nu_n = w ? P.nu[0] : P.nu[1];
    const float rw = w ? rho[1] : rho[0], rn_ = w ? rho[0] : rho[1];
    const float s_raw = (rw / rt - P.r_lo) * P.inv_r_span;
    const float s = fminf(fmaxf(s_raw, 0.f), 1.f);
    float sw = s, Rw = 0.f, Ro = 0.f;
    // gray quantities
    float gv[3] = {0.f, 0.f, 0.f}, iK0 = 0.f, pcs = 0.f;
    float gAt[3] = {0.f, 0.f, 0.f}, mag = 0.f, Hh = 0.f, mden = 1.f, Pc = 0.f, kcap = 0.f, se_c = 0.f;
    float se_k = 0.f, krw = 0.f, krn = 0.f, coef = 0.f, rk = 0.f;
    bool swd = false, wetf = false;
    Curve cv{};
    if (is_gray) {
        const GrayRec gr = gray[c];
        gv[0] = gr.a.x;
        gv[1] = gr.a.y;
        gv[2] = gr.a.z;
        iK0 = gr.a.w;
        pcs = gr.b.x;
        const unsigned meta = __float_as_uint(gr.b.w);
        wetf = meta & META_WET;
        swd = meta & META_SWITCHED;
        Rw = (swd && !wetf) ? gr.b.y : 0.f;
        Ro = (swd && wetf) ? gr.b.z : 0.f;
        sw = Rw + (1.f - Rw - Ro) * s;
        cv = P.curve[meta & 0xffu];
#pragma unroll
        for (int i = 1; i < Q; ++i) {
            gAt[0] += w3(i) * cx(i) * at[i];
            gAt[1] += w3(i) * cy(i) * at[i];
            gAt[2] += w3(i) * cz(i) * at[i];
        }
        mag = sqrtf(dotn<3>(gAt, gAt));
        const float At_c = (rw - rn_) / rt;
        Hh = (fabsf(At_c) <= P.at_cut) ? 0.5f * mag : 0.f;
        if (Hh > 0.f) {
            se_c = fminf(fmaxf((sw - cv.swr) * cv.inv_1m_swr, 1e-2f), 1.f);
            float pw_unused;
            Pc = pcs * pc_shape(cv, se_c, pw_unused);
            mden = fmaxf(mag, P.eps_n);
            kcap = -Pc * Hh / (mden * rt);
#pragma unroll
            for (int a = 0; a < 2; ++a)
#pragma unroll
                for (int d = 0; d < 3; ++d) Fp[a][d] += kcap * rho[a] * gAt[d];
        }
        se_k = fminf(fmaxf((sw - cv.swr) * cv.inv_1m_swr, 0.f), 1.f);
        krw = powf(se_k, cv.nw);
        krn = powf(1.f - se_k, cv.nn);
        coef = rw * nu_w / fmaxf(krw, P.kr_min) + rn_ * nu_n / fmaxf(krn, P.kr_min);
        rk = coef * iK0;
    }
    float bb[3], u[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) bb[d] = j[0][d] + j[1][d] + 0.5f * (Fp[0][d] + Fp[1][d]);
    float al = 1.f, be = 0.f;
    if (is_gray) {
        al = rt + 0.5f * rk;
        be = 0.5f * rk;
        const float q = be * dotn<3>(gv, bb) / (al + be * dotn<3>(gv, gv));
#pragma unroll
        for (int d = 0; d < 3; ++d) u[d] = (bb[d] - q * gv[d]) / al;
    } else {
#pragma unroll
        for (int d = 0; d < 3; ++d) u[d] = bb[d] / rt;
    }
    float Ru[3] = {0.f, 0.f, 0.f}, F[2][3];
    const float vu = dotn<3>(gv, u);
    if (is_gray)
#pragma unroll
        for (int d = 0; d < 3; ++d) Ru[d] = rk * (u[d] + gv[d] * vu);
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int d = 0; d < 3; ++d) F[a][d] = Fp[a][d] - (is_gray ? (rho[a] / rt) * Ru[d] : 0.f);

    // ---------------- reverse ----------------------------------------------
    float lrho[2] = {0.f, 0.f}, lj[3] = {0.f, 0.f, 0.f}, lP[2][6], lF[2][3], lu[3] = {0.f, 0.f, 0.f};
    const float uu = dotn<3>(u, u);
#pragma unroll
    for (int a = 0; a < 2; ++a) {
        // adjoints of the 19 outputs at their push targets
        float L0 = 0.f, L1[3] = {0.f, 0.f, 0.f}, L2[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            size_t tg;
            int tc = c;  // the target cell
            if (i == 0) tg = c;
            else if (wall & (1u << i)) tg = (size_t)opp(i) * n + c;
            else {
                tc = nb[i];
                tg = (size_t)i * n + tc;
            }
            const float li = wgt(i) * (lam_next[(size_t)a * Q * n + tg] + v_next[(size_t)a * n + tc]);
            L0 += li;
            L1[0] += cx(i) * li;
            L1[1] += cy(i) * li;
            L1[2] += cz(i) * li;
            L2[0] += cx(i) * cx(i) * li;
            L2[1] += cy(i) * cy(i) * li;
            L2[2] += cz(i) * cz(i) * li;
            L2[3] += cx(i) * cy(i) * li;
            L2[4] += cx(i) * cz(i) * li;
            L2[5] += cy(i) * cz(i) * li;
        }
        const float om = P.omega_fac[a];
        float L2u[3];
        symv(L2, u, L2u);
        // lambda_Pi = 4.5 om (L2 - L0 I / 3)
        float lPi[6];
#pragma unroll
        for (int k = 0; k < 6; ++k) lPi[k] = 4.5f * om * L2[k];
#pragma unroll
        for (int k = 0; k < 3; ++k) lPi[k] -= 1.5f * om * L0;
        float lPiu[3], lPiF[3];
        symv(lPi, u, lPiu);
        symv(lPi, F[a], lPiF);
        float L2F[3];
        symv(L2, F[a], L2F);
        lrho[a] += L0 + 3.f * dotn<3>(u, L1) + 4.5f * dotn<3>(u, L2u) - 1.5f * uu * L0;
        lrho[a] += -(lPi[0] + lPi[1] + lPi[2]) * (1.0f / 3.0f) - dotn<3>(u, lPiu);
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            lF[a][d] = 1.5f * L1[d] + 4.5f * L2u[d] - 1.5f * L0 * u[d] + lPiu[d];
            lu[d] += rho[a] * (3.f * L1[d] + 9.f * L2u[d] - 3.f * L0 * u[d]) + 4.5f * L2F[d] - 1.5f * L0 * F[a][d] -
                     2.f * rho[a] * lPiu[d] + lPiF[d];
        }
#pragma unroll
        for (int k = 0; k < 6; ++k) lP[a][k] = lPi[k];
    }
    float lsw = 0.f;
    if (seed.on) {
        if (x == P.nx - 1) lu[0] += seed.lux;
        lsw += seed.lsw * adj_phi_c(t, phi[c]);
    }
    float lrt = 0.f, lrk = 0.f, lv[3] = {0.f, 0.f, 0.f}, lFp[2][3];
    // drag: F = Fp - (rho_a/rt) Ru, Ru = rk (u + v (v.u))
    if (is_gray) {
        float lRu[3];
#pragma unroll
        for (int d = 0; d < 3; ++d) lRu[d] = -(rho[0] * lF[0][d] + rho[1] * lF[1][d]) / rt;
#pragma unroll
        for (int a = 0; a < 2; ++a) {
            const float RuF = dotn<3>(Ru, lF[a]);
            lrho[a] += -RuF / rt;
            lrt += rho[a] * RuF / (rt * rt);
        }
        const float vlRu = dotn<3>(gv, lRu);
        float uvv[3];
#pragma unroll
        for (int d = 0; d < 3; ++d) uvv[d] = u[d] + gv[d] * vu;
        lrk += dotn<3>(lRu, uvv);
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            lu[d] += rk * (lRu[d] + gv[d] * vlRu);
            lv[d] += rk * (vu * lRu[d] + vlRu * u[d]);
        }
    }
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int d = 0; d < 3; ++d) lFp[a][d] = lF[a][d];
    // velocity
    float lb[3];
    if (is_gray) {
        // (al I + be v v^T) u = b: lb = A^-1 lu, lA = -lb u^T
        const float q = be * dotn<3>(gv, lu) / (al + be * dotn<3>(gv, gv));
#pragma unroll
        for (int d = 0; d < 3; ++d) lb[d] = (lu[d] - q * gv[d]) / al;
        const float lal = -dotn<3>(lb, u);
        const float vz = dotn<3>(gv, lb);
        const float lbe = -vz * vu;
#pragma unroll
        for (int d = 0; d < 3; ++d) lv[d] += -be * (vu * lb[d] + vz * u[d]);
        lrt += lal;
        lrk += 0.5f * lal + 0.5f * lbe;
    } else {
#pragma unroll
        for (int d = 0; d < 3; ++d) lb[d] = lu[d] / rt;
        lrt += -dotn<3>(u, lu) / rt;
    }
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        lj[d] = lb[d];
        lFp[0][d] += 0.5f * lb[d];
        lFp[1][d] += 0.5f * lb[d];
    }
    float lrn[2][Q], lat[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        lrn[0][i] = lrn[1][i] = 0.f;
        lat[i] = 0.f;
    }
    float lgk[5] = {0.f, 0.f, 0.f, 0.f, 0.f};  // 1/K0, pcs, Sw_irr, So_res (and spare)
    if (is_gray) {
        // rk = coef / K0
        const float lcoef = lrk * iK0;
        lgk[0] += lrk * coef;
        const float mw = fmaxf(krw, P.kr_min), mn = fmaxf(krn, P.kr_min);
        add_at(lrho, w, lcoef * nu_w / mw);
        add_at(lrho, 1 - w, lcoef * nu_n / mn);
        const float lkrw = krw > P.kr_min ? -lcoef * rw * nu_w / (mw * mw) : 0.f;
        const float lkrn = krn > P.kr_min ? -lcoef * rn_ * nu_n / (mn * mn) : 0.f;
        float lsek = 0.f;
        if (se_k > 0.f) lsek += lkrw * cv.nw * powf(se_k, cv.nw - 1.f);
        if (se_k < 1.f) lsek += -lkrn * cv.nn * powf(1.f - se_k, cv.nn - 1.f);
        const float sek_raw = (sw - cv.swr) * cv.inv_1m_swr;
        if (sek_raw > 0.f && sek_raw < 1.f) lsw += lsek * cv.inv_1m_swr;
        // capillary: Fp += k rho_a gAt, k = -Pc Hh / (mden rt)
        if (Hh > 0.f) {
            float lk = 0.f, lgat[3] = {0.f, 0.f, 0.f};
#pragma unroll
            for (int a = 0; a < 2; ++a) {
                const float gl = dotn<3>(gAt, lFp[a]);
                lk += rho[a] * gl;
                lrho[a] += kcap * gl;
#pragma unroll
                for (int d = 0; d < 3; ++d) lgat[d] += kcap * rho[a] * lFp[a][d];
            }
            const float lPc = -lk * Hh / (mden * rt);
            const float lHh = -lk * Pc / (mden * rt);
            const float lm = lk * Pc * Hh / (mden * mden * rt);
            lrt += lk * Pc * Hh / (mden * rt * rt);
            const float lmag = 0.5f * lHh + (mag > P.eps_n ? lm : 0.f);
            if (mag > 0.f)
#pragma unroll
                for (int d = 0; d < 3; ++d) lgat[d] += lmag * gAt[d] / mag;
            // Pc = pcs pw(se_c)
            float dpw;
            const float pw = pc_shape(cv, se_c, dpw);
            lgk[1] += lPc * pw;
            const float lsec = lPc * pcs * dpw;
            const float sec_raw = (sw - cv.swr) * cv.inv_1m_swr;
            if (sec_raw > 1e-2f && sec_raw < 1.f) lsw += lsec * cv.inv_1m_swr;
#pragma unroll
            for (int i = 1; i < Q; ++i)
                if (!(wall & (1u << i))) lat[i] = w3(i) * (cx(i) * lgat[0] + cy(i) * lgat[1] + cz(i) * lgat[2]);
        }
        // sw = Rw + (1 - Rw - Ro) s
        if (swd && !wetf) lgk[2] += lsw * (1.f - s);
        if (swd && wetf) lgk[3] += -lsw * s;
        lsw *= (1.f - Rw - Ro);
    }
    // s = clamp((rho_w/rt - r_lo) / span)
    if (s_raw > 0.f && s_raw < 1.f) {
        const float ls = lsw * P.inv_r_span;
        add_at(lrho, w, ls / rt);
        lrt += -ls * rw / (rt * rt);
    }
    float lgrad[2][3] = {{0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}};
#pragma unroll
    for (int a = 0; a < 2; ++a) {
        const float *g = grad[1 - a];
        // body and Shan-Chen
        lrho[a] += dotn<3>(P.accel[a], lFp[a]) - P.G * dotn<3>(g, lFp[a]);
#pragma unroll
        for (int d = 0; d < 3; ++d) lgrad[1 - a][d] += -P.G * rho[a] * lFp[a][d];
        if (csf) {
            const int b = 1 - a;
            const float kc = P.kappa * P.csf_coef[a];
            const float gl = dotn<3>(g, lFp[a]);
            const float ldiv = -kc * rho[a] * gl;
            lrho[a] += kc * (-dv[a]) * gl;
            float lg[3];
#pragma unroll
            for (int d = 0; d < 3; ++d) lg[d] = kc * (-dv[a]) * rho[a] * lFp[a][d];
            const float s3 = sN[a] * sN[a] * sN[a];
            const float ltr = ldiv / sN[a];
            const float lgHg = -ldiv / s3;
            const float ls = ldiv * (-trH[a] / (sN[a] * sN[a]) + 3.f * gHg[a] / (s3 * sN[a]));
            float Hg[3];
            symv(Hs[a], g, Hg);
#pragma unroll
            for (int d = 0; d < 3; ++d) lg[d] += 2.f * lgHg * Hg[d] + ls * g[d] / sN[a];
            // lambda_H = lgHg g g^T + ltr I  -> per direction q_i = w_i (9 c.lH.c - 3 tr lH)
            float lH[6] = {lgHg * g[0] * g[0] + ltr, lgHg * g[1] * g[1] + ltr, lgHg * g[2] * g[2] + ltr,
                           lgHg * g[0] * g[1], lgHg * g[0] * g[2], lgHg * g[1] * g[2]};
            const float trl = lH[0] + lH[1] + lH[2];
#pragma unroll
            for (int i = 1; i < Q; ++i) {
                const float qi = wgt(i) * (9.f * cSc(i, lH) - 3.f * trl);
                if (!(wall & (1u << i))) lrn[b][i] += qi;
                lrho[b] -= qi;
            }
#pragma unroll
            for (int d = 0; d < 3; ++d) lgrad[b][d] += lg[d];
        }
    }
    // grad[b] = sum_i 3 w_i c_i rn[b][i]
#pragma unroll
    for (int i = 1; i < Q; ++i)
        if (!(wall & (1u << i)))
#pragma unroll
            for (int b = 0; b < 2; ++b)
                lrn[b][i] += w3(i) * (cx(i) * lgrad[b][0] + cy(i) * lgrad[b][1] + cz(i) * lgrad[b][2]);
    // Atwood numbers of the neighbours: At = (rw - rn)/(rw + rn)
    if (is_gray)
#pragma unroll
        for (int i = 1; i < Q; ++i)
            if (!(wall & (1u << i)) && lat[i] != 0.f) {
                const float a_w = w ? rn[1][i] : rn[0][i], a_n = w ? rn[0][i] : rn[1][i], den = a_w + a_n;
                if (den > 0.f) {
                    const float dw = lat[i] * 2.f * a_n / (den * den), dn = -lat[i] * 2.f * a_w / (den * den);
                    lrn[0][i] += w ? dn : dw;
                    lrn[1][i] += w ? dw : dn;
                }
            }
    lrho[0] += lrt;
    lrho[1] += lrt;
    // own populations: rho_a = sum f, j = sum c f (both components), P_a = sum c c f
#pragma unroll
    for (int a = 0; a < 2; ++a) {
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const float v = lrho[a] + cx(i) * lj[0] + cy(i) * lj[1] + cz(i) * lj[2] + cSc(i, lP[a]);
            lam_out[(size_t)a * Q * n + (size_t)i * n + c] = v;
        }
    }
    // the adjoint of neighbour x + c_i's density, read back by that neighbour
    // (zero towards walls, which have no density)
#pragma unroll
    for (int i = 1; i < Q; ++i) {
        const bool wl = wall & (1u << i);
        contrib[(size_t)i * n + c] = wl ? 0.f : lrn[0][i];
        contrib[(size_t)(Q + i) * n + c] = wl ? 0.f : lrn[1][i];
    }
    if (is_gray) {
        double *gk = gacc + (size_t)8 * c;
        gk[0] += (double)lv[0];
        gk[1] += (double)lv[1];
        gk[2] += (double)lv[2];
        gk[3] += (double)lgk[0];
        gk[4] += (double)lgk[1];
        gk[5] += (double)lgk[2];
        gk[6] += (double)lgk[3];
    }
}

__global__ void k_adj_finish(DevParams P, const uint8_t *__restrict__ type, float *__restrict__ vout,
                             const float *__restrict__ contrib)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    const int n = P.n;
    if (c >= n) return;
    const bool solid = type[c] == CELL_SOLID;
    const int x = c % P.nx, y = (c / P.nx) % P.ny, z = c / (P.nx * P.ny);
    float v[2] = {0.f, 0.f};
    if (!solid) {
        // the fluid neighbours x - c_i that pushed into this cell along c_i
#pragma unroll
        for (int i = 1; i < Q; ++i) {
            const int X = axis_nb(x, -cx(i), P.nx, P.per[0]), Y = axis_nb(y, -cy(i), P.ny, P.per[1]),
                      Z = axis_nb(z, -cz(i), P.nz, P.per[2]);
            if (X < 0 || Y < 0 || Z < 0) continue;
            const int s = X + P.nx * (Y + P.ny * Z);
            if (type[s] == CELL_SOLID) continue;
            v[0] += contrib[(size_t)i * n + s];
            v[1] += contrib[(size_t)(Q + i) * n + s];
        }
    }
    vout[c] = v[0];
    vout[(size_t)n + c] = v[1];
}

// d S / d phi_c = (Sw_c - S) / sum(phi) at gray cells (the weights of the
// saturation average), times dL/dS.
__global__ void k_sat_weight_grad(int n, const uint8_t *__restrict__ type, const float *__restrict__ macro,
                                  double dLdS, double S, double sumphi, double *__restrict__ dphi)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n || type[c] != CELL_GRAY) return;
    dphi[c] += dLdS * ((double)macro[(size_t)5 * n + c] - S) / sumphi;
}

// ---- geometry precompute in reverse (FP64) ----------------------------------
struct CurveTableA {
    lbm_constitutive c[MAX_TYPES];
};

__device__ __forceinline__ int nbr3(const DevParams &P, int x, int y, int z, int dx, int dy, int dz)
{
    const int X = axis_nb(x, dx, P.nx, P.per[0]), Y = axis_nb(y, dy, P.ny, P.per[1]),
              Z = axis_nb(z, dz, P.nz, P.per[2]);
    return (X < 0 || Y < 0 || Z < 0) ? -1 : X + P.nx * (Y + P.ny * Z);
}
__device__ __forceinline__ double phi_at(const uint8_t *__restrict__ type, const float *__restrict__ phi, int m)
{
    if (m < 0) return 0.0;
    const uint8_t t = type[m];
    return t == CELL_PORE ? 1.0 : (t == CELL_SOLID ? 0.0 : (double)phi[m]);
}
__device__ __forceinline__ void add_phi(const uint8_t *__restrict__ type, double *__restrict__ dphi, int m, double v)
{
    if (m >= 0 && type[m] == CELL_GRAY && v != 0.0) atomicAdd(&dphi[m], v);
}

// Cyclic Jacobi eigen-decomposition of a symmetric 3x3 matrix: eigenvalues
// mu[k] and eigenvectors V[:, k].
__device__ void jacobi3(const double Min[3][3], double mu[3], double V[3][3])
{
    double A[3][3];
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) {
            A[r][c] = Min[r][c];
            V[r][c] = (r == c) ? 1.0 : 0.0;
        }
    for (int sweep = 0; sweep < 32; ++sweep) {
        const double off = A[0][1] * A[0][1] + A[0][2] * A[0][2] + A[1][2] * A[1][2];
        const double dia = A[0][0] * A[0][0] + A[1][1] * A[1][1] + A[2][2] * A[2][2];
        if (off == 0.0 || off <= 1e-34 * dia) break;
        for (int p = 0; p < 2; ++p)
            for (int q = p + 1; q < 3; ++q) {
                const double apq = A[p][q];
                if (apq == 0.0) continue;
                const double theta = 0.5 * (A[q][q] - A[p][p]) / apq;
                const double t = copysign(1.0, theta) / (fabs(theta) + sqrt(theta * theta + 1.0));
                const double cs = 1.0 / sqrt(t * t + 1.0), sn = t * cs, tau = sn / (1.0 + cs);
                const int r = 3 - p - q;
                const double arp = A[r][p], arq = A[r][q];
                A[p][p] -= t * apq;
                A[q][q] += t * apq;
                A[p][q] = A[q][p] = 0.0;
                A[r][p] = A[p][r] = arp - sn * (arq + tau * arp);
                A[r][q] = A[q][r] = arq + sn * (arp - tau * arq);
                for (int k = 0; k < 3; ++k) {
                    const double vkp = V[k][p], vkq = V[k][q];
                    V[k][p] = vkp - sn * (vkq + tau * vkp);
                    V[k][q] = vkq + sn * (vkp - tau * vkq);
                }
            }
    }
    for (int k = 0; k < 3; ++k) mu[k] = A[k][k];
}

__global__ void k_geom_adjoint(DevParams P, CurveTableA T, double c_g, const uint8_t *__restrict__ type,
                               const float *__restrict__ phi, const GrayRec *__restrict__ gray,
                               const double *__restrict__ gacc, double *__restrict__ dphi)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= P.n || type[c] != CELL_GRAY) return;
    const double *gk = gacc + (size_t)8 * c;
    const int pt = (int)(__float_as_uint(gray[c].b.w) & 0xffu);
    const lbm_constitutive cv = T.c[pt];
    const double ph = (double)phi[c];
    // 1/K0, lamL*pd, Sw_irr, So_res as functions of phi_c
    const double d2 = cv.kc_d * cv.kc_d;
    const double K0 = d2 * ph * ph * ph / (180.0 * (1.0 - ph) * (1.0 - ph));
    const double dK0 = d2 * ph * ph * (3.0 - ph) / (180.0 * (1.0 - ph) * (1.0 - ph) * (1.0 - ph));
    const double kref = d2 * cv.phi_ref * cv.phi_ref * cv.phi_ref / (180.0 * (1.0 - cv.phi_ref) * (1.0 - cv.phi_ref));
    const double lamL = sqrt((kref / cv.phi_ref) * ph / K0);
    // lamL^2 = C phi / K0  ->  dlamL = lamL/2 (1/phi - K0'/K0)
    const double dlam = 0.5 * lamL * (1.0 / ph - dK0 / K0);
    double g = gk[3] * (-dK0 / (K0 * K0)) + gk[4] * cv.pd * dlam;
    // Sw(f) = swr + (1 - swr) Se(x), x = f / lamL: Brooks-Corey Se = min(1, x^-lambda),
    // dSe/dlamL = lambda Se / lamL below 1; Thomeer Se = 1 - exp(-G/u), u = log10 x,
    // dSe/dlamL = exp(-G/u) G / (u^2 lamL ln 10) above entry; 0 where Se = 1
    auto dse_dlam = [&](double f) {
        const double x = f / lamL;
        if (cv.thomeer_g > 0.0) {
            if (x <= 1.0) return 0.0;
            const double u = log10(x), e = exp(-cv.thomeer_g / u);
            return e * cv.thomeer_g / (u * u * lamL * log(10.0));
        }
        const double se = pow(x, -cv.lambda);
        return se < 1.0 ? cv.lambda * se / lamL : 0.0;
    };
    g += gk[5] * (1.0 - cv.swr) * dse_dlam(cv.pc_ref_max_f) * dlam;
    g += -gk[6] * (1.0 - cv.swr) * dse_dlam(cv.pc_ref_min_f) * dlam;
    atomicAdd(&dphi[c], g);
    // principal axis: v = sqrt(a - 1) e1(M), M = H H + c_g grad grad^T
    const double lv2 = gk[0] * gk[0] + gk[1] * gk[1] + gk[2] * gk[2];
    if (lv2 == 0.0 || cv.aniso <= 1.0) return;
    const int x = c % P.nx, y = (c / P.nx) % P.ny, z = c / (P.nx * P.ny);
    double gr[3] = {0.0, 0.0, 0.0};
    for (int i = 1; i < Q; i += 2) {  // opposite pairs, as in the forward geometry
        const double v = phi_at(type, phi, nbr3(P, x, y, z, cx(i), cy(i), cz(i))) -
                         phi_at(type, phi, nbr3(P, x, y, z, -cx(i), -cy(i), -cz(i)));
        gr[0] += 3.0 * wgt_d(i) * cx(i) * v;
        gr[1] += 3.0 * wgt_d(i) * cy(i) * v;
        gr[2] += 3.0 * wgt_d(i) * cz(i) * v;
    }
    double H[3][3];
    int nbp[3][3][4];  // stencil cells of the cross terms (pp, pm, mp, mm)
    int nba[3][2];     // +e_a, -e_a
    for (int a = 0; a < 3; ++a) {
        int ea[3] = {0, 0, 0};
        ea[a] = 1;
        nba[a][0] = nbr3(P, x, y, z, ea[0], ea[1], ea[2]);
        nba[a][1] = nbr3(P, x, y, z, -ea[0], -ea[1], -ea[2]);
        H[a][a] = phi_at(type, phi, nba[a][0]) - 2.0 * ph + phi_at(type, phi, nba[a][1]);
        for (int b = a + 1; b < 3; ++b) {
            int eb[3] = {0, 0, 0};
            eb[b] = 1;
            nbp[a][b][0] = nbr3(P, x, y, z, ea[0] + eb[0], ea[1] + eb[1], ea[2] + eb[2]);
            nbp[a][b][1] = nbr3(P, x, y, z, ea[0] - eb[0], ea[1] - eb[1], ea[2] - eb[2]);
            nbp[a][b][2] = nbr3(P, x, y, z, eb[0] - ea[0], eb[1] - ea[1], eb[2] - ea[2]);
            nbp[a][b][3] = nbr3(P, x, y, z, -ea[0] - eb[0], -ea[1] - eb[1], -ea[2] - eb[2]);
            H[a][b] = H[b][a] = 0.25 * (phi_at(type, phi, nbp[a][b][0]) - phi_at(type, phi, nbp[a][b][1]) -
                                        phi_at(type, phi, nbp[a][b][2]) + phi_at(type, phi, nbp[a][b][3]));
        }
    }
    double M[3][3];
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b)
            M[a][b] = H[a][0] * H[0][b] + H[a][1] * H[1][b] + H[a][2] * H[2][b] + c_g * gr[a] * gr[b];
    double mu[3], V[3][3];
    jacobi3(M, mu, V);
    int top = 0;
    for (int k = 1; k < 3; ++k)
        if (mu[k] > mu[top]) top = k;
    double second = -INFINITY;
    for (int k = 0; k < 3; ++k)
        if (k != top && mu[k] > second) second = mu[k];
    if (mu[top] - second <= 1e-12 * fmax(mu[top], 1e-30)) return;  // isotropic: no axis
    double e1[3] = {V[0][top], V[1][top], V[2][top]};
    // the stored v used the same eigenvector sign; align lambda_e1 with it
    const double sa = sqrt(cv.aniso - 1.0);
    const float4 ga = gray[c].a;
    const double dot = e1[0] * ga.x + e1[1] * ga.y + e1[2] * ga.z;
    if (dot < 0.0)
        for (int d = 0; d < 3; ++d) e1[d] = -e1[d];
    const double le[3] = {sa * gk[0], sa * gk[1], sa * gk[2]};
    // lambda_M = sym(sum_{k != top} (le . e_k)/(mu_top - mu_k) e_k e1^T)
    double lM[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
    for (int k = 0; k < 3; ++k) {
        if (k == top) continue;
        const double gap = mu[top] - mu[k];
        if (!(gap > 0.0)) continue;
        const double ck = (le[0] * V[0][k] + le[1] * V[1][k] + le[2] * V[2][k]) / gap;
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) lM[a][b] += 0.5 * ck * (V[a][k] * e1[b] + e1[a] * V[b][k]);
    }
    // M = H H + c_g g g^T: lH = lM H + H lM, lg = 2 c_g lM g
    double lH[3][3], lg[3];
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
            double s = 0.0;
            for (int k = 0; k < 3; ++k) s += lM[a][k] * H[k][b] + H[a][k] * lM[k][b];
            lH[a][b] = s;
        }
    for (int a = 0; a < 3; ++a) lg[a] = 2.0 * c_g * (lM[a][0] * gr[0] + lM[a][1] * gr[1] + lM[a][2] * gr[2]);
    // scatter to the stencil's porosities
    for (int i = 1; i < Q; ++i)
        add_phi(type, dphi, nbr3(P, x, y, z, cx(i), cy(i), cz(i)),
                3.0 * wgt_d(i) * (cx(i) * lg[0] + cy(i) * lg[1] + cz(i) * lg[2]));
    for (int a = 0; a < 3; ++a) {
        add_phi(type, dphi, nba[a][0], lH[a][a]);
        add_phi(type, dphi, nba[a][1], lH[a][a]);
        atomicAdd(&dphi[c], -2.0 * lH[a][a]);
        for (int b = a + 1; b < 3; ++b) {
            const double v = 0.25 * (lH[a][b] + lH[b][a]);
            add_phi(type, dphi, nbp[a][b][0], v);
            add_phi(type, dphi, nbp[a][b][1], -v);
            add_phi(type, dphi, nbp[a][b][2], -v);
            add_phi(type, dphi, nbp[a][b][3], v);
        }
    }
}

}  // namespace lbm

// ---------------------------------------------------------------------------
// Driver: forward with checkpoints, loss, then backwards segment by segment.
// ---------------------------------------------------------------------------
namespace {

// cells per group of the adjoint's cell list (measured on the 96^3 gradient
// against groups of 2^10 ... 2^19 cells and one group for the whole lattice)
constexpr int ADJ_GROUP = 65536;

struct DevBuf {
    void *p = nullptr;
    ~DevBuf()
    {
        if (p) cudaFree(p);
    }
};

}  // namespace

extern "C" int lbm_adjoint_run(lbm_ctx *ctx, const lbm_loss *L, int nsteps, int ckpt, float *dL_dphi, int mem,
                               double *out3)
{
    using namespace lbm;
    if (!ctx || !L || nsteps < 1 || ckpt < 1 || !dL_dphi) return LBM_ERR_ARG;
    if (mem != LBM_MEM_HOST && mem != LBM_MEM_DEVICE) return LBM_ERR_ARG;
    if (!(L->q_target != 0.0) || !std::isfinite(L->q_target) || !std::isfinite(L->s_target)) return LBM_ERR_ARG;
    if (ctx->p.storage != LBM_STORAGE_F32 || ctx->view || ctx->n_held > 0 || ctx->p.lattice != LBM_LATTICE_D3Q19 ||
        ctx->mss != 0.0)
        return LBM_ERR_ARG;
    if (!ctx->has_fields) return LBM_ERR_STATE;
    DeviceGuard dg(ctx->dev);
    if (!dg.ok) return LBM_ERR_CUDA;
    const int n = ctx->n;
    const size_t pb = pop_bytes(ctx), gb = (size_t)n * sizeof(GrayRec);
    const int nseg = (nsteps + ckpt - 1) / ckpt;
    cudaStream_t s = ctx->stream;
    // checkpoints (state + gray records at each segment start), one segment of
    // states (ckpt + 1) and gray snapshots (ckpt), adjoint buffers
    DevBuf ck_f, ck_g, seg_f, seg_g, seg_r, lam0, lam1, vb0, vb1, acc, gacc, dphi, fin_f, fin_g;
    LBM_CUDA(cudaMalloc(&ck_f.p, pb * nseg));
    LBM_CUDA(cudaMalloc(&ck_g.p, gb * nseg));
    LBM_CUDA(cudaMalloc(&seg_f.p, pb * (ckpt + 1)));
    LBM_CUDA(cudaMalloc(&seg_g.p, gb * ckpt));
    LBM_CUDA(cudaMalloc(&seg_r.p, 3 * (size_t)n * sizeof(float) * ckpt));  // densities of each replayed state
    LBM_CUDA(cudaMalloc(&lam0.p, pb));
    LBM_CUDA(cudaMalloc(&lam1.p, pb));
    LBM_CUDA(cudaMalloc(&vb0.p, 2 * (size_t)n * sizeof(float)));  // neighbour terms V[2][n]
    LBM_CUDA(cudaMalloc(&vb1.p, 2 * (size_t)n * sizeof(float)));
    LBM_CUDA(cudaMalloc(&acc.p, 2 * Q * (size_t)n * sizeof(float)));  // contrib[2][Q][n]
    LBM_CUDA(cudaMalloc(&gacc.p, 8 * (size_t)n * sizeof(double)));
    LBM_CUDA(cudaMalloc(&dphi.p, (size_t)n * sizeof(double)));
    LBM_CUDA(cudaMalloc(&fin_f.p, pb));
    LBM_CUDA(cudaMalloc(&fin_g.p, gb));
    char *ckf = (char *)ck_f.p, *ckg = (char *)ck_g.p, *sf = (char *)seg_f.p, *sg = (char *)seg_g.p;
    float *const sr = (float *)seg_r.p;
    float *const f_save[2] = {ctx->f[0], ctx->f[1]};
    const int cur_save = ctx->cur;
    const long long steps0 = ctx->steps;
    auto restore_ptrs = [&]() {
        ctx->f[0] = f_save[0];
        ctx->f[1] = f_save[1];
        ctx->rho_cap = nullptr;
    };
    // ---- forward with checkpoints ----
    for (int k = 0; k < nsteps; ++k) {
        if (k % ckpt == 0) {
            LBM_CUDA(cudaMemcpyAsync(ckf + pb * (k / ckpt), ctx->f[ctx->cur], pb, cudaMemcpyDeviceToDevice, s));
            LBM_CUDA(cudaMemcpyAsync(ckg + gb * (k / ckpt), ctx->gray, gb, cudaMemcpyDeviceToDevice, s));
        }
        LBM_CUDA(launch_fused(ctx, k == nsteps - 1));
    }
    ctx->steps = steps0 + nsteps;
    LBM_CUDA(cudaMemcpyAsync(fin_f.p, ctx->f[ctx->cur], pb, cudaMemcpyDeviceToDevice, s));
    LBM_CUDA(cudaMemcpyAsync(fin_g.p, ctx->gray, gb, cudaMemcpyDeviceToDevice, s));
    const int cur_final = ctx->cur;
    // ---- loss ----
    double v[NOBS_HOST];
    LBM_CUDA(launch_observables(ctx, v));
    const double q = v[4] / ((double)ctx->p.ny * ctx->p.nz);
    const double sumphi = v[3], S = v[3] > 0 ? v[2] / v[3] : 0.0;
    const double loss = (q - L->q_target) * (q - L->q_target) / (L->q_target * L->q_target) +
                        (S - L->s_target) * (S - L->s_target);
    const double dLdq = 2.0 * (q - L->q_target) / (L->q_target * L->q_target);
    const double dLdS = 2.0 * (S - L->s_target);
    AdjSeed seed;
    seed.on = 1;
    seed.lux = (float)(dLdq / ((double)ctx->p.ny * ctx->p.nz));
    seed.lsw = (float)(sumphi > 0 ? dLdS / sumphi : 0.0);
    LBM_CUDA(cudaMemsetAsync(lam0.p, 0, pb, s));
    LBM_CUDA(cudaMemsetAsync(lam1.p, 0, pb, s));
    LBM_CUDA(cudaMemsetAsync(vb0.p, 0, 2 * (size_t)n * sizeof(float), s));
    LBM_CUDA(cudaMemsetAsync(vb1.p, 0, 2 * (size_t)n * sizeof(float), s));
    LBM_CUDA(cudaMemsetAsync(acc.p, 0, 2 * Q * (size_t)n * sizeof(float), s));
    LBM_CUDA(cudaMemsetAsync(gacc.p, 0, 8 * (size_t)n * sizeof(double), s));
    LBM_CUDA(cudaMemsetAsync(dphi.p, 0, (size_t)n * sizeof(double), s));
    const dim3 grid((n + 127) / 128);
    // the fluid cells, group by group of ADJ_GROUP consecutive cells: in each
    // group the plain pore (and other non-gray) cells first, then the gray
    // cells, each in index order and each section padded to whole warps.  A
    // warp then takes one side of the gray-cell branches, and the warps of
    // one group, which run at about the same time, share the cache lines of
    // that group's slots.
    std::vector<uint8_t> ht((size_t)n);
    LBM_CUDA(cudaMemcpyAsync(ht.data(), ctx->type, (size_t)n, cudaMemcpyDeviceToHost, s));
    LBM_CUDA(cudaStreamSynchronize(s));
    std::vector<int> hl;
    hl.reserve((size_t)n);
    for (int g0 = 0; g0 < n; g0 += ADJ_GROUP) {
        const int g1 = std::min(n, g0 + ADJ_GROUP);
        for (int pass = 0; pass < 2; ++pass) {
            for (int c = g0; c < g1; ++c)
                if (ht[c] != CELL_SOLID && ((ht[c] == CELL_GRAY) == (pass == 1))) hl.push_back(c);
            while (hl.size() % 32) hl.push_back(-1);  // whole warps per section (-1: no cell)
        }
    }
    const int ncells = (int)hl.size();
    DevBuf cells;
    LBM_CUDA(cudaMalloc(&cells.p, std::max<size_t>(1, hl.size()) * sizeof(int)));
    if (ncells > 0)
        LBM_CUDA(cudaMemcpyAsync(cells.p, hl.data(), hl.size() * sizeof(int), cudaMemcpyHostToDevice, s));
    const dim3 grid_cells((unsigned)std::max(1, (ncells + 127) / 128));
    if (sumphi > 0)
        k_sat_weight_grad<<<grid, 128, 0, s>>>(n, ctx->type, ctx->macro, dLdS, S, sumphi, (double *)dphi.p);
    float *lam_next = (float *)lam0.p, *lam_cur = (float *)lam1.p;
    float *v_next = (float *)vb0.p, *v_cur = (float *)vb1.p;
    // ---- backwards, segment by segment ----
    int rc = LBM_OK;
    for (int sgi = nseg - 1; sgi >= 0 && rc == LBM_OK; --sgi) {
        const int k0 = sgi * ckpt, k1 = std::min(nsteps, k0 + ckpt);
        cudaError_t e = cudaMemcpyAsync(sf, ckf + pb * sgi, pb, cudaMemcpyDeviceToDevice, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(ctx->gray, ckg + gb * sgi, gb, cudaMemcpyDeviceToDevice, s);
        // recompute the segment, keeping every state, the gray records each
        // step used and the densities each step formed (the same values as
        // the density pass of the two-launch path)
        for (int k = k0; k < k1 && e == cudaSuccess; ++k) {
            ctx->f[0] = (float *)(sf + pb * (k - k0));
            ctx->f[1] = (float *)(sf + pb * (k - k0 + 1));
            ctx->cur = 0;
            ctx->rho_cap = sr + 3 * (size_t)n * (k - k0);
            e = launch_fused(ctx, false);
            ctx->rho_cap = nullptr;
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(sg + gb * (k - k0), ctx->gray, gb, cudaMemcpyDeviceToDevice, s);
        }
        for (int k = k1 - 1; k >= k0 && e == cudaSuccess; --k) {
            ctx->f[0] = (float *)(sf + pb * (k - k0));
            ctx->cur = 0;
            AdjSeed sk = seed;
            sk.on = (k == nsteps - 1);
            k_adj_cell<<<grid_cells, 128, 0, s>>>(ctx->dp, ctx->f[0], sr + 3 * (size_t)n * (k - k0), ctx->type,
                                                    ctx->phi, (const GrayRec *)(sg + gb * (k - k0)), lam_next, v_next,
                                                    lam_cur, (float *)acc.p, (double *)gacc.p, sk,
                                                    (const int *)cells.p, ncells);
            k_adj_finish<<<grid, 128, 0, s>>>(ctx->dp, ctx->type, v_cur, (const float *)acc.p);
            e = cudaGetLastError();
            ctx->launches += 2;
            std::swap(lam_next, lam_cur);
            std::swap(v_next, v_cur);
        }
        if (e != cudaSuccess) rc = cuda_fail(e, "lbm_adjoint_run backward");
    }
    restore_ptrs();
    if (rc != LBM_OK) return rc;
    // ---- chain the gray constants to phi ----
    CurveTableA T;
    for (int k = 0; k < MAX_TYPES; ++k) T.c[k] = ctx->curves[k];
    k_geom_adjoint<<<grid, 128, 0, s>>>(ctx->dp, T, ctx->p.c_g, ctx->type, ctx->phi, (const GrayRec *)ckg,
                                        (const double *)gacc.p, (double *)dphi.p);
    LBM_CUDA(cudaGetLastError());
    ctx->launches += 1;
    // ---- the context ends at the forward's final state ----
    ctx->cur = cur_final;
    (void)cur_save;
    LBM_CUDA(cudaMemcpyAsync(ctx->f[ctx->cur], fin_f.p, pb, cudaMemcpyDeviceToDevice, s));
    LBM_CUDA(cudaMemcpyAsync(ctx->gray, fin_g.p, gb, cudaMemcpyDeviceToDevice, s));
    // the fields of the final step (the recomputation did not write them)
    std::vector<double> hd((size_t)n);
    LBM_CUDA(cudaMemcpyAsync(hd.data(), dphi.p, (size_t)n * sizeof(double), cudaMemcpyDeviceToHost, s));
    LBM_CUDA(cudaStreamSynchronize(s));
    std::vector<float> hf((size_t)n);
    for (int c = 0; c < n; ++c) hf[c] = (float)hd[c];
    if (mem == LBM_MEM_HOST)
        std::copy(hf.begin(), hf.end(), dL_dphi);
    else
        LBM_CUDA(cudaMemcpy(dL_dphi, hf.data(), (size_t)n * sizeof(float), cudaMemcpyHostToDevice));
    if (out3) {
        out3[0] = loss;
        out3[1] = q;
        out3[2] = S;
    }
    return LBM_OK;
}
