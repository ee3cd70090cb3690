// Time-step kernels of the two-component D3Q19 pseudo-potential LB model.
//
// Population storage (F32, push form; see lbm_cell.cuh): the buffer holds the
// streamed state; slot 0 is the rest population f_0 in 2^-30 fixed point
// (int32), slot i the arrived population relative to its source's rest
// population.  Moments and density stencils are formed from small numbers and
// exact integer differences of f_0; post-collision populations are written
// into the neighbours' slots (bounce-back into the cell's own opposite slot).
// Mathematically the state is the same as plain populations.
//
// One step is two launches:
//   k_density  - pull and zeroth moment: drho^A, drho^B of every fluid cell,
//                the source of the density stencils;
//   k_collide  - own slots again, residual update, forces (Shan-Chen, CSF Eq. 4,
//                Eq. 1 capillary + tensorial viscous with the semi-implicit
//                velocity), regularised collision with the Eq. 3 force term,
//                store.
#include "lbm_cell.cuh"
#include "lbm_context.h"

namespace lbm {

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

// Fields of the initial state and the residual flag of gray cells (wet where
// s >= 1/2).
__device__ __forceinline__ void init_fields_out(const DevParams &P, int c, uint8_t t, const double r[2],
                                                const double uv[3], float *__restrict__ macro,
                                                GrayRec *__restrict__ gray)
{
    const int n = P.n;
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
// Initial state: equilibrium of (rhoA, rhoB, u), evaluated in FP64 once.
// ---------------------------------------------------------------------------
template <class LY>
__global__ void k_init(DevParams P, const float *__restrict__ rhoA, const float *__restrict__ rhoB,
                       const float *__restrict__ u, const uint8_t *__restrict__ type, LY ly,
                       float *__restrict__ drho, float *__restrict__ macro, GrayRec *__restrict__ gray)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    const int n = P.n;
    if (c >= n) return;
    const uint8_t t = type[c];
    if (t == CELL_SOLID) {
        for (int a = 0; a < 2; ++a) {
            ly.rest_out(a, c, 0);
            for (int i = 1; i < Q; ++i) ly.mov_out(a, (size_t)i * n + c, 0.0f);
        }
        drho[c] = 0.0f;
        drho[n + c] = 0.0f;
        drho[(size_t)2 * n + c] = P.at_wall;
        for (int k = 0; k < 6; ++k) macro[(size_t)k * n + c] = 0.0f;
        return;
    }
    int x, y, z;
    cell_xyz(c, P, x, y, z);
    const Axes A = axes_of(P, x, y, z);
    double uv[3] = {0.0, 0.0, 0.0};
    if (u) {
        uv[0] = u[c];
        uv[1] = u[(size_t)n + c];
        uv[2] = u[(size_t)2 * n + c];
    }
    const double uu = uv[0] * uv[0] + uv[1] * uv[1] + uv[2] * uv[2];
    const double r[2] = {(double)rhoA[c], (double)rhoB[c]};
    for (int a = 0; a < 2; ++a) {
        const double f0 = r[a] / 3.0 - 0.5 * r[a] * uu;  // feq_0 = w_0 rho (1 - 3u^2/2)
        const long long q = llrint(f0 * FIX_ONE_D);
        const double r0 = f0 - (double)q / FIX_ONE_D;
        ly.rest_out(a, c, (int)q);
        // the equilibrium populations, streamed: direction i goes to x + c_i,
        // or back into the cell's own opposite slot when x + c_i is solid
#pragma unroll
        for (int i = 1; i < Q; ++i) {
            const double cu = cx(i) * uv[0] + cy(i) * uv[1] + cz(i) * uv[2];
            const double g = wgt_d(i) * (r[a] * (3.0 * cu + 4.5 * cu * cu) + 3.0 * r0);
            const int m = nb_index(P, A, i);
            const bool wl = m < 0 || type[m] == CELL_SOLID;
            ly.mov_out(a, wl ? (size_t)opp(i) * n + c : (size_t)i * n + m, (float)g);
        }
        drho[(size_t)a * n + c] = 0.0f;
    }
    init_fields_out(P, c, t, r, uv, macro, gray);
}

// Initial state in a shifted 16-bit storage: h_i = f^eq_i - w_i rho0, pushed
// like the F32 state.
template <class H>
__global__ void k_init_lp(DevParams P, const float *__restrict__ rhoA, const float *__restrict__ rhoB,
                          const float *__restrict__ u, const uint8_t *__restrict__ type,
                          typename H::T *__restrict__ f, float *__restrict__ macro, GrayRec *__restrict__ gray)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    const int n = P.n;
    if (c >= n) return;
    const uint8_t t = type[c];
    if (t == CELL_SOLID) {
        for (int k = 0; k < 2 * Q; ++k) f[(size_t)k * n + c] = H::st(0.0f);
        for (int k = 0; k < 6; ++k) macro[(size_t)k * n + c] = 0.0f;
        return;
    }
    int x, y, z;
    cell_xyz(c, P, x, y, z);
    const Axes A = axes_of(P, x, y, z);
    double uv[3] = {0.0, 0.0, 0.0};
    if (u) {
        uv[0] = u[c];
        uv[1] = u[(size_t)n + c];
        uv[2] = u[(size_t)2 * n + c];
    }
    const double uu = uv[0] * uv[0] + uv[1] * uv[1] + uv[2] * uv[2];
    const double r[2] = {(double)rhoA[c], (double)rhoB[c]};
    for (int a = 0; a < 2; ++a) {
        typename H::T *fa = f + (size_t)a * Q * n;
        const double r0 = (double)P.rho0[a];
        fa[c] = H::st((float)(wgt_d(0) * (r[a] * (1.0 - 1.5 * uu) - r0)));
#pragma unroll
        for (int i = 1; i < Q; ++i) {
            const double cu = cx(i) * uv[0] + cy(i) * uv[1] + cz(i) * uv[2];
            const double h = wgt_d(i) * (r[a] * (1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * uu) - r0);
            const int m = nb_index(P, A, i);
            const bool wl = m < 0 || type[m] == CELL_SOLID;
            fa[wl ? (size_t)opp(i) * n + c : (size_t)i * n + m] = H::st((float)h);
        }
    }
    init_fields_out(P, c, t, r, uv, macro, gray);
}

// ---------------------------------------------------------------------------
// Density deviations of the current step: drho = rho - 3 f_0 (own slots).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_density(DevParams P, const float *__restrict__ f,
                                                 const uint8_t *__restrict__ type,
                                                 float *__restrict__ drho)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    const int n = P.n;
    if (c >= n) return;
    const uint8_t t = type[c];
    if (t == CELL_SOLID) return;
    if (is_held(t)) {  // reservoir: the held densities
        for (int a = 0; a < 2; ++a)
            drho[(size_t)a * n + c] =
                held_dev(held_rho(P.held, t, a), reinterpret_cast<const int *>(f + (size_t)a * Q * n)[c]).hi;
        drho[(size_t)2 * n + c] = atwood_of(P.wet, reinterpret_cast<const int *>(f)[c],
                                            reinterpret_cast<const int *>(f + (size_t)Q * n)[c], drho[c],
                                            drho[n + c]);
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
        const int *fi = reinterpret_cast<const int *>(fa);
        const int f0 = fi[c];
        float acc = 0.0f;
        long long id = 0;  // 12 * sum_i w3_i (f0(s) - f0(x)) in 2^-30 units
#pragma unroll
        for (int i = 1; i < Q; ++i) {
            const int o = opp(i);
            acc += fa[(size_t)i * n + c];
            if (!(wall & (1u << o))) id += (long long)(fi[nb[o]] - f0) * w12(i);
        }
        drho[(size_t)a * n + c] = ff_add_f(ff_twelfth(id), acc).hi;
    }
    drho[(size_t)2 * n + c] = atwood_of(P.wet, reinterpret_cast<const int *>(f)[c],
                                        reinterpret_cast<const int *>(f + (size_t)Q * n)[c], drho[c], drho[n + c]);
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
    int f0i[2];
    CompMom M[2];
#pragma unroll
    for (int a = 0; a < 2; ++a) {
        const float *fa = fin + (size_t)a * Q * n;
        const int *fi = a ? fiB : fiA;
        const int f0 = fi[c];
        PullSums p;
        pull_zero(p);
#pragma unroll
        for (int i = 1; i < Q; ++i) {
            const int o = opp(i);  // the source x - c_i is x + c_o
            pull_add(p, i, fa[(size_t)i * n + c], (wall & (1u << o)) ? 0 : fi[nb[o]] - f0);
        }
        f0i[a] = f0;
        M[a] = finish_moments(p, f0);
        if (is_held(t)) {  // reservoir: held density at rest, no force
            const ff rh = held_rho(P.held, t, a);
            M[a] = held_moments(rh, held_dev(rh, f0));
        }
    }
    const bool held = is_held(t);
    const float r[2] = {M[0].rho.hi, M[1].rho.hi};
    const bool is_gray = (t == CELL_GRAY);

    // ---- density stencils: FP32 parts of grad(rho^a) (drho differences; walls
    //      contribute rho_wall - rho(x)), grad(At) in gray cells, and the
    //      Hessians of rho^A, rho^B where Eq. 4 applies ------------------------
    const bool csf = !held && P.kappa != 0.0f && (P.csf_everywhere || is_gray);
    float gf[2][3] = {{0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}}, gAt[3] = {0.f, 0.f, 0.f};
    HessSum hA, hB;
    hess_zero(hA);
    hess_zero(hB);
    const float drcA = drA[c], drcB = drB[c];
#pragma unroll
    for (int i = 1; i < Q; ++i) {
        const int m = nb[i];
        const bool wl = wall & (1u << i);
        const float eA = wl ? P.rho_wall[0] - r[0] : drA[m] - drcA;
        const float eB = wl ? P.rho_wall[1] - r[1] : drB[m] - drcB;
        stencil_add(i, eA, eB, gf);
        if (is_gray) atwood_add(i, wl ? P.at_wall : drho[(size_t)2 * n + m], gAt);
        if (csf) {
            const float dA = wl ? eA : 3.0f * fix_diff(fiA[m], f0i[0]) + eA;
            const float dB = wl ? eB : 3.0f * fix_diff(fiB[m], f0i[1]) + eB;
            hess_add(hA, i, dA);
            hess_add(hB, i, dB);
        }
    }
    auto tgt = [&](int i) -> size_t {
        return (wall & (1u << i)) ? (size_t)opp(i) * n + c : (size_t)i * n + nb[i];
    };
    float acc[2][3];
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            acc[a][d] = held ? 0.f : P.accel[a][d];
            if (held) gf[a][d] = 0.f;
        }
    StoreRest<LayF32> st{LayF32{fin, fout, n}, c, {f0i[0], f0i[1]}};
    collide_store<MACRO>(P, acc, held ? 0.f : P.mss, t, c, n, st, M, gf, gAt, csf, hA, hB, gray, macro, tgt);
}

// ---------------------------------------------------------------------------
// Launch wrappers
// ---------------------------------------------------------------------------
static inline dim3 grid_for(int n, int block) { return dim3((unsigned)((n + block - 1) / block)); }

cudaError_t launch_init(lbm_ctx *ctx, const float *rhoA, const float *rhoB, const float *u)
{
    cudaEvent_t e0;
    prof_begin(ctx, "k_init", &e0);
    if (ctx->p.storage == LBM_STORAGE_F16S)
        k_init_lp<H16><<<grid_for(ctx->n, 256), 256, 0, ctx->stream>>>(
            ctx->dp, rhoA, rhoB, u, ctx->type, reinterpret_cast<__half *>(ctx->f[ctx->cur]), ctx->macro, ctx->gray);
    else if (ctx->p.storage == LBM_STORAGE_BF16S)
        k_init_lp<B16><<<grid_for(ctx->n, 256), 256, 0, ctx->stream>>>(
            ctx->dp, rhoA, rhoB, u, ctx->type, reinterpret_cast<__nv_bfloat16 *>(ctx->f[ctx->cur]), ctx->macro,
            ctx->gray);
    else if (ctx->p.storage == LBM_STORAGE_F16R)
        k_init<<<grid_for(ctx->n, 256), 256, 0, ctx->stream>>>(ctx->dp, rhoA, rhoB, u, ctx->type,
                                                              lay_r16<LayF16R>(ctx, ctx->cur, ctx->cur), ctx->rho,
                                                              ctx->macro, ctx->gray);
    else if (ctx->p.storage == LBM_STORAGE_BF16R)
        k_init<<<grid_for(ctx->n, 256), 256, 0, ctx->stream>>>(ctx->dp, rhoA, rhoB, u, ctx->type,
                                                              lay_r16<LayB16R>(ctx, ctx->cur, ctx->cur), ctx->rho,
                                                              ctx->macro, ctx->gray);
    else
        k_init<<<grid_for(ctx->n, 256), 256, 0, ctx->stream>>>(
            ctx->dp, rhoA, rhoB, u, ctx->type, LayF32{ctx->f[ctx->cur], ctx->f[ctx->cur], ctx->n}, ctx->rho,
            ctx->macro, ctx->gray);
    prof_end(ctx, "k_init", e0);
    ctx->launches += 1;
    return cudaGetLastError();
}

cudaError_t launch_density(lbm_ctx *ctx)
{
    cudaEvent_t e0;
    prof_begin(ctx, "k_density", &e0);
    k_density<<<grid_for(ctx->n, 256), step_block(ctx, 256), 0, ctx->stream>>>(ctx->dp, ctx->f[ctx->cur],
                                                                              ctx->type, ctx->rho);
    prof_end(ctx, "k_density", e0);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    ctx->launches += 1;
    return cudaSuccess;
}

cudaError_t launch_collide(lbm_ctx *ctx, bool write_macro)
{
    const float *fin = ctx->f[ctx->cur];
    float *fout = ctx->f[1 - ctx->cur];
    cudaEvent_t e0;
    prof_begin(ctx, "k_collide", &e0);
    const dim3 blk = step_block(ctx, 256);
    if (write_macro)
        k_collide<true><<<grid_for(ctx->n, 256), blk, 0, ctx->stream>>>(
            ctx->dp, fin, fout, ctx->type, ctx->rho, ctx->gray, ctx->macro);
    else
        k_collide<false><<<grid_for(ctx->n, 256), blk, 0, ctx->stream>>>(
            ctx->dp, fin, fout, ctx->type, ctx->rho, ctx->gray, ctx->macro);
    prof_end(ctx, "k_collide", e0);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;  // nothing ran: the state stays in buffer cur
    ctx->launches += 1;
    ctx->cur = 1 - ctx->cur;
    return cudaSuccess;
}

}  // namespace lbm
