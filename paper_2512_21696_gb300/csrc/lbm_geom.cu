// Geometry precompute of the gray cells, in FP64 on the device (runs once
// per lbm_set_geometry).
//
// Per gray cell (Eqs. 5-7 and the abstract's "Hessian and gradient of the
// local porosity"):
//   grad(phi)  isotropic D3Q19 stencil (1/cs^2) sum_i w_i phi(x+c_i) c_i,
//              summed as central differences over opposite pairs;
//   Hessian    second differences along the axes, four-point cross terms;
//   M = H H + c_g grad(phi) grad(phi)^T; its top eigenvector e1 is the axis
//   of lowest permeability, K = B diag(K0/a, K0, K0) B^T, so
//   K^-1 = (1/K0)(I + (a-1) e1 e1^T); ties (mu1 - mu2 <= 1e-12 mu1) fall back
//   to isotropic; pore types with a = 1 skip the axis (K^-1 = I / K0);
//   K0 (Kozeny-Carman), Leverett factor lamL (Eq. 5), and the residual
//   amounts from the crossings of Pc(Sw; phi) with pc_ref_max_f*pd and
//   pc_ref_min_f*pd (Fig. 6).
// The eigen-decomposition uses cyclic Jacobi rotations in FP64, which keep
// exact ties exact (grid-aligned neighbourhoods often give them).
#include <cmath>

#include "lbm_context.h"

namespace lbm {

struct CurveTable {
    lbm_constitutive c[MAX_TYPES];
};

__device__ __forceinline__ double phi_of(const uint8_t *__restrict__ type, const float *__restrict__ phi,
                                         int m)
{
    if (m < 0) return 0.0;
    const uint8_t t = type[m];
    return t == CELL_PORE ? 1.0 : (t == CELL_SOLID ? 0.0 : (double)phi[m]);
}

__device__ __forceinline__ int nbr(const DevParams &P, int x, int y, int z, int dx, int dy, int dz)
{
    const int X = axis_nb(x, dx, P.nx, P.per[0]);
    const int Y = axis_nb(y, dy, P.ny, P.per[1]);
    const int Z = axis_nb(z, dz, P.nz, P.per[2]);
    return (X < 0 || Y < 0 || Z < 0) ? -1 : X + P.nx * (Y + P.ny * Z);
}

__device__ __forceinline__ double kozeny(const lbm_constitutive &cv, double phi)
{
    return cv.kc_d * cv.kc_d * phi * phi * phi / (180.0 * (1.0 - phi) * (1.0 - phi));
}

// Top eigenvector of a symmetric 3x3 matrix by cyclic Jacobi rotations
// (Rutishauser's formulation); returns false when the two largest
// eigenvalues tie (mu1 - mu2 <= 1e-12 mu1), i.e. no preferred axis.
__device__ bool top_eigvec(const double Min[3][3], double e[3])
{
    double A[3][3], V[3][3];
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
                const int r = 3 - p - q;  // the third index
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
    int top = 0;
    for (int k = 1; k < 3; ++k)
        if (A[k][k] > A[top][top]) top = k;
    double second = -INFINITY;
    for (int k = 0; k < 3; ++k)
        if (k != top && A[k][k] > second) second = A[k][k];
    const double mu1 = A[top][top];
    if (mu1 - second <= 1e-12 * fmax(mu1, 1e-30)) return false;
    for (int d = 0; d < 3; ++d) e[d] = V[d][top];
    return true;
}

__global__ void k_geometry(DevParams P, CurveTable T, double c_g, const uint8_t *__restrict__ type,
                           const float *__restrict__ phi, const uint8_t *__restrict__ ptype,
                           GrayRec *__restrict__ gray)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= P.n) return;
    if (type[c] != CELL_GRAY) return;
    const int x = c % P.nx, y = (c / P.nx) % P.ny, z = c / (P.nx * P.ny);
    const double ph = (double)phi[c];
    const int pt = ptype ? (int)ptype[c] : 0;
    const lbm_constitutive cv = T.c[pt];
    double e[3] = {0.0, 0.0, 0.0};
    bool axis = false;
    // the axis matters only where the pore type is anisotropic: with a = 1,
    // K^-1 = I / K0 whatever e1 is, so the stencils and the eigenvector are skipped
    if (cv.aniso != 1.0) {
        // central differences over the opposite pairs (i odd, opp(i) = i + 1): a
        // flat neighbourhood gives exactly zero, never round-off with an axis
        double g[3] = {0.0, 0.0, 0.0};
        for (int i = 1; i < Q; i += 2) {
            const double v = phi_of(type, phi, nbr(P, x, y, z, cx(i), cy(i), cz(i))) -
                             phi_of(type, phi, nbr(P, x, y, z, -cx(i), -cy(i), -cz(i)));
            g[0] += 3.0 * wgt_d(i) * cx(i) * v;
            g[1] += 3.0 * wgt_d(i) * cy(i) * v;
            g[2] += 3.0 * wgt_d(i) * cz(i) * v;
        }
        double H[3][3];
        for (int a = 0; a < 3; ++a) {
            int ea[3] = {0, 0, 0};
            ea[a] = 1;
            H[a][a] = phi_of(type, phi, nbr(P, x, y, z, ea[0], ea[1], ea[2])) - 2.0 * ph +
                      phi_of(type, phi, nbr(P, x, y, z, -ea[0], -ea[1], -ea[2]));
            for (int b = a + 1; b < 3; ++b) {
                int eb[3] = {0, 0, 0};
                eb[b] = 1;
                const double pp = phi_of(type, phi, nbr(P, x, y, z, ea[0] + eb[0], ea[1] + eb[1], ea[2] + eb[2]));
                const double pm = phi_of(type, phi, nbr(P, x, y, z, ea[0] - eb[0], ea[1] - eb[1], ea[2] - eb[2]));
                const double mp = phi_of(type, phi, nbr(P, x, y, z, eb[0] - ea[0], eb[1] - ea[1], eb[2] - ea[2]));
                const double mm = phi_of(type, phi, nbr(P, x, y, z, -ea[0] - eb[0], -ea[1] - eb[1], -ea[2] - eb[2]));
                H[a][b] = H[b][a] = 0.25 * (pp - pm - mp + mm);
            }
        }
        double M[3][3];
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b)
                M[a][b] = H[a][0] * H[0][b] + H[a][1] * H[1][b] + H[a][2] * H[2][b] + c_g * g[a] * g[b];
        axis = top_eigvec(M, e);
    }
    const double sa = axis ? sqrt(cv.aniso - 1.0) : 0.0;
    const double K0 = kozeny(cv, ph);
    const double kref = kozeny(cv, cv.phi_ref);
    const double lamL = sqrt((kref / cv.phi_ref) / (K0 / ph));
    // Se where the curve crosses f Pd, x = f / lamL = Pc / Pe: Brooks-Corey
    // x^(-lambda); Thomeer 1 - exp(-G / log10 x) above entry; 1 at or below entry
    auto se_at = [&](double f) {
        const double x = f / lamL;
        if (cv.thomeer_g > 0.0) return x <= 1.0 ? 1.0 : 1.0 - exp(-cv.thomeer_g / log10(x));
        return fmin(pow(x, -cv.lambda), 1.0);
    };
    const double se_max = se_at(cv.pc_ref_max_f);
    const double se_min = se_at(cv.pc_ref_min_f);
    const double sw_irr = cv.swr + (1.0 - cv.swr) * se_max;
    const double so_res = 1.0 - (cv.swr + (1.0 - cv.swr) * se_min);
    GrayRec rec;
    rec.a = make_float4((float)(sa * e[0]), (float)(sa * e[1]), (float)(sa * e[2]), (float)(1.0 / K0));
    rec.b = make_float4((float)(lamL * cv.pd), (float)sw_irr, (float)so_res,
                        __uint_as_float((unsigned)pt & 0xffu));
    gray[c] = rec;
}

cudaError_t launch_geometry(lbm_ctx *ctx, const uint8_t *ptype)
{
    CurveTable T;
    for (int k = 0; k < MAX_TYPES; ++k) T.c[k] = ctx->curves[k];
    cudaEvent_t e0;
    prof_begin(ctx, "k_geometry", &e0);
    k_geometry<<<(ctx->n + 127) / 128, 128, 0, ctx->stream>>>(ctx->dp, T, ctx->p.c_g, ctx->type, ctx->phi,
                                                               ptype, ctx->gray);
    prof_end(ctx, "k_geometry", e0);
    ctx->launches += 1;
    return cudaGetLastError();
}

}  // namespace lbm
