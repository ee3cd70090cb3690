// Per-cell arithmetic of the time step, shared by the two-launch path
// (k_density + k_collide) and the fused rolling-window kernel, so that both
// compute bit-identical states.
//
// Storage convention (F32), push form: the buffer holds the streamed
// (pre-collision) state.  Per component, slot 0 of cell x is the rest
// population f_0(x) in 2^-30 fixed point (int32); slot i (1..18) of x holds
// g_i = f_i(x) - 3 w_i f_0(s) in FP32, the population that arrived from the
// source s = x - c_i relative to the source's rest population (s = x itself
// after a bounce-back at a solid source).  Relative to the cell's own rest
// population the arrived population is h_i = g_i + w3_i (f_0(s) - f_0(x)),
// w3_i = 3 w_i.  The g parts are summed in FP32; the rest-population parts
// exactly in 64-bit integers with weights 12 w3_i (2 on faces, 1 on edges) and
// converted once.  Each cell reads only its own slots (coalesced) and writes
// its post-collision populations into the slots of its neighbours.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "lbm_common.cuh"

namespace lbm {

constexpr float FIX_ONE = 1073741824.0f;          // 2^30
constexpr float FIX_INV = 9.313225746154785e-10f;  // 2^-30
constexpr double FIX_ONE_D = 1073741824.0;

// 3 w_i for the moving populations (faces 1/6, edges 1/12).
__host__ __device__ constexpr float w3(int i) { return i <= 6 ? (1.0f / 6.0f) : (1.0f / 12.0f); }
// 12 w3_i: the integer weight of a rest-population difference.
__host__ __device__ constexpr int w12(int i) { return i <= 6 ? 2 : 1; }

// Difference of two fixed-point rest populations, as a float.
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
// Exact value v * pow2 of an integer (|v| < 2^47) as float-float: the upper
// and lower 24-bit halves convert exactly, two-sum normalises.
__device__ __forceinline__ ff ff_from_ll(long long v, float pow2)
{
    const int vh = (int)(v >> 24);
    const int vl = (int)(v & 0xffffff);
    const ff s = fast_two_sum((float)vh * 16777216.0f, (float)vl);
    return {s.hi * pow2, s.lo * pow2};
}
constexpr float TWELFTH_HI = (float)(1.0 / 12.0);
constexpr float TWELFTH_LO = (float)(1.0 / 12.0 - (double)(float)(1.0 / 12.0));
// v * 2^-30 / 12 for an integer sum v of weighted rest-population differences.
__device__ __forceinline__ ff ff_twelfth(long long v) { return ff_mul(ff_from_ll(v, FIX_INV), {TWELFTH_HI, TWELFTH_LO}); }

// ---- pull sums --------------------------------------------------------------
// The zeroth and first moments carry the exact integer sums (they feed the
// float-float force balance); the second moments, which enter only through
// the (1 - 1/tau) regularised part, are summed from h in FP32.
struct PullSums {
    float d, j0, j1, j2, sxx, syy, szz, sxy, sxz, syz;
    long long Id, Ij0, Ij1, Ij2;
};
__device__ __forceinline__ void pull_zero(PullSums &p)
{
    p.d = p.j0 = p.j1 = p.j2 = p.sxx = p.syy = p.szz = p.sxy = p.sxz = p.syz = 0.f;
    p.Id = p.Ij0 = p.Ij1 = p.Ij2 = 0;
}
// Adds direction i: g = g_i at the source (or the bounce-back value), d0 the
// rest-population difference f_0(s) - f_0(x) in fixed point (0 at walls).
// WITH_D = false skips the zeroth moment (when the density pass already has it).
template <bool WITH_D = true>
__device__ __forceinline__ void pull_add(PullSums &p, int i, float g, int d0)
{
    const long long D = (long long)d0 * w12(i);
    const float h = fmaf(w3(i) * FIX_INV, (float)d0, g);
    if (WITH_D) {
        p.d += g;
        p.Id += D;
    }
    if (cx(i)) { p.j0 += cx(i) * g; p.sxx += h; p.Ij0 += cx(i) * D; }
    if (cy(i)) { p.j1 += cy(i) * g; p.syy += h; p.Ij1 += cy(i) * D; }
    if (cz(i)) { p.j2 += cz(i) * g; p.szz += h; p.Ij2 += cz(i) * D; }
    if (cx(i) && cy(i)) p.sxy += cx(i) * cy(i) * h;
    if (cx(i) && cz(i)) p.sxz += cx(i) * cz(i) * h;
    if (cy(i) && cz(i)) p.syz += cy(i) * cz(i) * h;
}

// Moments of one component at one cell.
struct CompMom {
    float dr;          // rho - 3 f_0 (FP32)
    ff rho;            // rho (float-float)
    ff j[3];           // momentum of this component (float-float)
    float S[6];        // sum c c h: xx, yy, zz, xy, xz, yz (FP32)
    long long Ij[3];   // integer part of j, also gives grad(rho) below
};
// rho - 3 f_0 in float-float from the sums of the pulled g and of the
// weighted rest-population differences (the density pass's value).
__device__ __forceinline__ ff density_dev(long long Id, float d) { return ff_add_f(ff_twelfth(Id), d); }

// Moments from the pull sums; dff = rho - 3 f_0 as float-float.
__device__ __forceinline__ CompMom finish_moments_d(const PullSums &p, int f0, ff dff)
{
    CompMom m;
    m.dr = dff.hi;
    m.rho = ff_add(ff_from_ll(3LL * f0, FIX_INV), dff);
    m.j[0] = ff_add_f(ff_twelfth(p.Ij0), p.j0);
    m.j[1] = ff_add_f(ff_twelfth(p.Ij1), p.j1);
    m.j[2] = ff_add_f(ff_twelfth(p.Ij2), p.j2);
    m.Ij[0] = p.Ij0;
    m.Ij[1] = p.Ij1;
    m.Ij[2] = p.Ij2;
    m.S[0] = p.sxx;
    m.S[1] = p.syy;
    m.S[2] = p.szz;
    m.S[3] = p.sxy;
    m.S[4] = p.sxz;
    m.S[5] = p.syz;
    return m;
}
__device__ __forceinline__ CompMom finish_moments(const PullSums &p, int f0)
{
    return finish_moments_d(p, f0, density_dev(p.Id, p.d));
}

// ---- reservoir (pressure) cells ---------------------------------------------
// An inlet / outlet cell holds its prescribed densities at rest: its moments
// are the held density, no momentum and the second moment of the rest
// equilibrium, so that the collision returns that equilibrium.
__device__ __forceinline__ ff held_rho(const float (&held)[2][2][2], int t, int a)
{
    // a select, not an index, so that the parameter block stays out of local memory
    return t == CELL_OUTLET ? ff{held[1][a][0], held[1][a][1]} : ff{held[0][a][0], held[0][a][1]};
}
// rho - 3 f_0 of a reservoir cell whose stored rest population is f0.
__device__ __forceinline__ ff held_dev(ff rho, int f0) { return ff_add(rho, ff_from_ll(-3LL * f0, FIX_INV)); }
// Moments relative to a reference rest population f_r with dff = rho - 3 f_r.
__device__ __forceinline__ CompMom held_moments(ff rho, ff dff)
{
    CompMom m;
    m.dr = dff.hi;
    m.rho = rho;
    const float d3 = dff.hi * (1.0f / 3.0f);  // sum c c (f^eq - 3 w f_r) = (rho - 3 f_r)/3 I
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        m.j[d] = {0.f, 0.f};
        m.Ij[d] = 0;
        m.S[d] = d3;
        m.S[3 + d] = 0.f;
    }
    return m;
}

// Accumulates the FP32 parts of grad(rho^a) (e = rho^a(x+c_i) - rho^a(x)
// without the rest-population part) and, in gray cells, grad(At) with the
// neighbour densities nA, nB.
__device__ __forceinline__ void stencil_add(int i, float eA, float eB, float gf[2][3])
{
    const float wi = w3(i);
    if (cx(i)) { gf[0][0] += wi * cx(i) * eA; gf[1][0] += wi * cx(i) * eB; }
    if (cy(i)) { gf[0][1] += wi * cy(i) * eA; gf[1][1] += wi * cy(i) * eB; }
    if (cz(i)) { gf[0][2] += wi * cz(i) * eA; gf[1][2] += wi * cz(i) * eB; }
}
// Atwood number At = (rho^w - rho^n)/(rho^w + rho^n) of a fluid cell from its
// fixed-point rest populations and drho; evaluated once per cell and step
// (approximate division, 2 ulp) and read by the gray-cell stencils.
__device__ __forceinline__ float atwood_of(int w, int f0A, int f0B, float drA, float drB)
{
    const float rA = fmaf((float)f0A, 3.0f * FIX_INV, drA), rB = fmaf((float)f0B, 3.0f * FIX_INV, drB);
    const float nw = w == 0 ? rA : rB, nn = w == 0 ? rB : rA;
    const float den = nw + nn;
    return den > 0.f ? __fdividef(nw - nn, den) : 0.f;
}
__device__ __forceinline__ void atwood_add(int i, float At, float gAt[3])
{
    const float wi = w3(i);
    if (cx(i)) gAt[0] += wi * cx(i) * At;
    if (cy(i)) gAt[1] += wi * cy(i) * At;
    if (cz(i)) gAt[2] += wi * cz(i) * At;
}

// Moment Hessian of a density: H = 9 M - 3 L I with M = sum_i w_i c_i c_i d_i
// and L = sum_i w_i d_i, d_i = rho(x + c_i) - rho(x) (i.e. (1/cs^4) sum_i
// w_i (c_i c_i - cs^2 I) d_i).  M is kept as xx, yy, zz, xy, xz, yz.
struct HessSum {
    float m[6], l;
};
__device__ __forceinline__ void hess_zero(HessSum &h)
{
    h.m[0] = h.m[1] = h.m[2] = h.m[3] = h.m[4] = h.m[5] = h.l = 0.f;
}
__device__ __forceinline__ void hess_add(HessSum &h, int i, float d)
{
    const float wd = wgt(i) * d;
    h.l += wd;
    if (cx(i)) h.m[0] += wd;
    if (cy(i)) h.m[1] += wd;
    if (cz(i)) h.m[2] += wd;
    if (cx(i) && cy(i)) h.m[3] += cx(i) * cy(i) * wd;
    if (cx(i) && cz(i)) h.m[4] += cx(i) * cz(i) * wd;
    if (cy(i) && cz(i)) h.m[5] += cy(i) * cz(i) * wd;
}
// Divergence of the regularised normal g / s, s = sqrt(|g|^2 + eps^2):
// tr(H)/s - g.H.g/s^3 (Eq. 4's curvature).
__device__ __forceinline__ float normal_divergence(const float g[3], const HessSum &h, float eps)
{
    const float Hxx = 9.f * h.m[0] - 3.f * h.l, Hyy = 9.f * h.m[1] - 3.f * h.l, Hzz = 9.f * h.m[2] - 3.f * h.l;
    const float Hxy = 9.f * h.m[3], Hxz = 9.f * h.m[4], Hyz = 9.f * h.m[5];
    const float gHg = g[0] * (Hxx * g[0] + 2.f * (Hxy * g[1] + Hxz * g[2])) + g[1] * (Hyy * g[1] + 2.f * Hyz * g[2]) +
                      g[2] * Hzz * g[2];
    const float s2 = g[0] * g[0] + g[1] * g[1] + g[2] * g[2] + eps * eps;
    const float is = rsqrtf(s2);
    return is * ((Hxx + Hyy + Hzz) - gHg * is * is);
}

// ---- shifted 16-bit storage (FP16 / BF16) -----------------------------------
// Slot i of cell x holds f_i - w_i rho0 (i = 0..18, push form as in F32); all
// arithmetic is FP32.
struct H16 {
    using T = __half;
    static __device__ __forceinline__ float ld(T v) { return __half2float(v); }
    static __device__ __forceinline__ T st(float x) { return __float2half_rn(x); }
};
struct B16 {
    using T = __nv_bfloat16;
    static __device__ __forceinline__ float ld(T v) { return __bfloat162float(v); }
    static __device__ __forceinline__ T st(float x) { return __float2bfloat16_rn(x); }
};

// Moments of one component from its 19 shifted 16-bit slots h_i = f_i - w_i rho0,
// relative to the reference rest population f_r = rho/3 (so dr = 0 and
// S = sum c c h + (rho0 - rho)/3 I).  rho = rho0 + sum_i h_i.
template <class H>
__device__ __forceinline__ CompMom moments_lp(const typename H::T *__restrict__ fa, size_t n, float rho0)
{
    float s = H::ld(fa[0]);
    float j0 = 0.f, j1 = 0.f, j2 = 0.f, sxx = 0.f, syy = 0.f, szz = 0.f, sxy = 0.f, sxz = 0.f, syz = 0.f;
#pragma unroll
    for (int i = 1; i < Q; ++i) {
        const float h = H::ld(fa[(size_t)i * n]);
        s += h;
        if (cx(i)) { j0 += cx(i) * h; sxx += h; }
        if (cy(i)) { j1 += cy(i) * h; syy += h; }
        if (cz(i)) { j2 += cz(i) * h; szz += h; }
        if (cx(i) && cy(i)) sxy += cx(i) * cy(i) * h;
        if (cx(i) && cz(i)) sxz += cx(i) * cz(i) * h;
        if (cy(i) && cz(i)) syz += cy(i) * cz(i) * h;
    }
    CompMom m;
    const float rho = rho0 + s;
    const float dd = (rho0 - rho) * (1.0f / 3.0f);
    m.dr = 0.f;
    m.rho = {rho, 0.f};
    m.j[0] = {j0, 0.f};
    m.j[1] = {j1, 0.f};
    m.j[2] = {j2, 0.f};
    m.S[0] = sxx + dd;
    m.S[1] = syy + dd;
    m.S[2] = szz + dd;
    m.S[3] = sxy;
    m.S[4] = sxz;
    m.S[5] = syz;
    m.Ij[0] = m.Ij[1] = m.Ij[2] = 0;
    return m;
}
// rho of one component from its 19 slots (same summation order as moments_lp).
template <class H>
__device__ __forceinline__ float density_lp(const typename H::T *__restrict__ fa, size_t n, float rho0)
{
    float s = H::ld(fa[0]);
#pragma unroll
    for (int i = 1; i < Q; ++i) s += H::ld(fa[(size_t)i * n]);
    return rho0 + s;
}
__device__ __forceinline__ float atwood_rho(int w, float rA, float rB)
{
    const float nw = w == 0 ? rA : rB, nn = w == 0 ? rB : rA;
    const float den = nw + nn;
    return den > 0.f ? __fdividef(nw - nn, den) : 0.f;
}
// Store of the post-collision state in a shifted 16-bit layout.
template <class H>
struct StoreLP {
    typename H::T *fout;
    int n, c;
    float f0r[2];   // reference rest populations rho/3
    float rho0[2];
    float fnew[2];  // new rest populations
    __device__ __forceinline__ float rest(int a, float d0)
    {
        fnew[a] = f0r[a] + d0;
        fout[(size_t)a * Q * n + c] = H::st(fnew[a] - rho0[a] * (1.0f / 3.0f));
        return 0.f;
    }
    __device__ __forceinline__ void pair(int a, int i, size_t ti, size_t tj, float E, float O)
    {
        const float b = w3(i) * fnew[a] - wgt(i) * rho0[a];
        typename H::T *fo = fout + (size_t)a * Q * n;
        fo[ti] = H::st(b + E + O);
        fo[tj] = H::st(b + E - O);
    }
};

// Shape of the lattice a march works on: sizes, cell count (the slot stride)
// and body acceleration (per run in a batch, P's otherwise).
struct Geo {
    int nx, ny, nz, n;
    float accel[2][3];
    float held[2][2][2];  // reservoir densities, as DevParams::held
    float mss;            // mass-sink-source rate, as DevParams::mss
};
__device__ __forceinline__ Geo geo_of(const DevParams &P)
{
    Geo G;
    G.nx = P.nx;
    G.ny = P.ny;
    G.nz = P.nz;
    G.n = P.n;
    for (int a = 0; a < 2; ++a)
        for (int d = 0; d < 3; ++d) G.accel[a][d] = P.accel[a][d];
    for (int k = 0; k < 8; ++k) (&G.held[0][0][0])[k] = (&P.held[0][0][0])[k];
    G.mss = P.mss;
    return G;
}

// One lattice of a batch (see k_fused_batch): its shape, the work items it
// contributes, its offsets in the batch buffers and its body acceleration.
struct BatchRun {
    int nx, ny, nz, n;
    int tiles_x, ncol, zchunks, item0;
    long long cell_off;  // first cell of the run in the per-cell arrays
    long long pop_off;   // byte offset of the run in each population buffer
    float accel[2][3];
    float held[2][2][2];  // reservoir densities of the run
    float mss;            // mass-sink-source rate of the run
};

// ---- rest-referenced layouts ----------------------------------------------
// The state of a cell is its rest population f_0 (int32, 2^-30 fixed point)
// and the 18 arrived populations relative to their sources' rest populations,
// g_i = f_i - 3 w_i f_0(s).  LayF32 keeps g in FP32 in slots 1..18 of
// [a][19][n] (slot 0 holds the int32 f_0); LayR16 keeps f_0 in an int32 array
// [2][n] followed by g * 2^GS in 16 bits, [2][18][n].  g is small (the
// velocity and non-equilibrium parts only), which is what makes 16 bits
// usable; the power-of-two scale keeps FP16 values out of its subnormal range.
struct LayF32 {
    const float *in;
    float *out;
    int n;
    __device__ __forceinline__ int rest_in(int a, int g) const
    {
        return reinterpret_cast<const int *>(in)[(size_t)a * Q * n + g];
    }
    __device__ __forceinline__ float mov_in(int a, int i, int g) const
    {
        return in[(size_t)a * Q * n + (size_t)i * n + g];
    }
    __device__ __forceinline__ void rest_out(int a, int c, int v) const
    {
        reinterpret_cast<int *>(out)[(size_t)a * Q * n + c] = v;
    }
    // slot = i n + cell, i >= 1
    __device__ __forceinline__ void mov_out(int a, size_t slot, float v) const { out[(size_t)a * Q * n + slot] = v; }
    // view of the population buffers of an n-cell lattice starting at in / out
    __host__ __device__ static LayF32 make(const void *in, void *out, int n)
    {
        return LayF32{reinterpret_cast<const float *>(in), reinterpret_cast<float *>(out), n};
    }
};
template <class H, int GS>
struct LayR16 {
    const int *rin;
    const typename H::T *min;
    int *rout;
    typename H::T *mout;
    int n;
    static constexpr float SC = (float)(1 << GS), ISC = 1.0f / (float)(1 << GS);
    __device__ __forceinline__ int rest_in(int a, int g) const { return rin[(size_t)a * n + g]; }
    __device__ __forceinline__ float mov_in(int a, int i, int g) const
    {
        return H::ld(min[((size_t)a * (Q - 1) + (i - 1)) * n + g]) * ISC;
    }
    __device__ __forceinline__ void rest_out(int a, int c, int v) const { rout[(size_t)a * n + c] = v; }
    __device__ __forceinline__ void mov_out(int a, size_t slot, float v) const
    {
        mout[(size_t)a * (Q - 1) * n + slot - n] = H::st(v * SC);
    }
    __host__ __device__ static LayR16 make(const void *in, void *out, int n)
    {
        using E = typename H::T;
        const char *pi = reinterpret_cast<const char *>(in);
        char *po = reinterpret_cast<char *>(out);
        return LayR16{reinterpret_cast<const int *>(pi), reinterpret_cast<const E *>(pi + 2 * (size_t)n * sizeof(int)),
                      reinterpret_cast<int *>(po), reinterpret_cast<E *>(po + 2 * (size_t)n * sizeof(int)), n};
    }
};
using LayF16R = LayR16<H16, 12>;
using LayB16R = LayR16<B16, 0>;

// Store of the post-collision state of one cell in a rest-referenced layout:
// the new rest population f_0 + d0 is added in fixed point, its sub-grid
// residual goes into the moving populations (returned to the caller, which
// adds 3 w_i res to each); direction i stores E + O, its opposite E - O.
template <class LY>
struct StoreRest {
    LY ly;
    int c;
    int f0i[2];
    __device__ __forceinline__ float rest(int a, float d0)
    {
        const float xq = d0 * FIX_ONE;
        const float qf = rintf(xq);
        ly.rest_out(a, c, f0i[a] + (int)qf);
        return (xq - qf) * FIX_INV;
    }
    __device__ __forceinline__ void pair(int a, int i, size_t ti, size_t tj, float E, float O)
    {
        ly.mov_out(a, ti, E + O);
        ly.mov_out(a, tj, E - O);
    }
};

// Forces, residual update, velocity and the regularised collision of one
// fluid cell, then the store of the new state through st (and of the fields
// if MACRO).  The moments are relative to a reference rest population f_r:
// M.dr = rho - 3 f_r and M.S = sum_i c_i c_i (f_i - 3 w_i f_r); the stored
// post-collision populations are f*_0 = f_r + d0 and
// f*_i = 3 w_i f*_0 + E_i +- O_i.
//   acc  body acceleration per component (F = rho acc);
//   M    the cell's moments;
//   gf   FP32 parts of grad(rho^A), grad(rho^B); gAt grad(At) (gray cells);
//   csf  whether Eq. 4 applies here; hA, hB the Hessian sums of rho^A, rho^B.
//   tgt  tgt(i): offset within a component's array where direction i goes,
//        i n + (index of x + c_i), or opp(i) n + c when x + c_i is solid.
//   ga, gb the cell's gray record (read by the caller, so that the load can be
//        issued early; only used in gray cells), gray the array it came from
//        (the residual flag is written back there on a transition).
template <bool MACRO, class Store, class Target>
__device__ __forceinline__ void collide_store_g(const DevParams &P, const float (&acc)[2][3], float mss, uint8_t t,
                                                int c, int n,
                                                Store &st,
                                                const CompMom M[2], const float gf[2][3], const float gAt[3],
                                                bool csf, const HessSum &hA, const HessSum &hB, const float4 ga,
                                                const float4 gb, GrayRec *__restrict__ gray,
                                                float *__restrict__ macro, const Target &tgt)
{
    const float r[2] = {M[0].rho.hi, M[1].rho.hi};
    const float rt = r[0] + r[1];
    const bool is_gray = (t == CELL_GRAY);
    const int w = P.wet;

    // grad(rho^A), grad(rho^B) in float-float: the rest-population part is
    // (1/4) 2^-30 sum_i w12_i c_i (f0(x+c_i) - f0(x)) = -2^-32 Ij
    ff grA[3], grB[3];
    float gA[3], gB[3];  // grad(phi^A) = grad(rho^B), grad(phi^B) = grad(rho^A)
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        grA[d] = ff_add_f(ff_from_ll(-M[0].Ij[d], FIX_INV * 0.25f), gf[0][d]);
        grB[d] = ff_add_f(ff_from_ll(-M[1].Ij[d], FIX_INV * 0.25f), gf[1][d]);
        gA[d] = grB[d].hi;
        gB[d] = grA[d].hi;
    }
    // Shan-Chen force in float-float: F^A = -G rho^A grad(rho^B), F^B = -G rho^B grad(rho^A)
    const ff Gff = {P.G, P.G_lo};
    ff Fsc[2][3];
    float F[2][3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        Fsc[0][d] = ff_mul(Gff, ff_mul(M[0].rho, grB[d]));
        Fsc[1][d] = ff_mul(Gff, ff_mul(M[1].rho, grA[d]));
        Fsc[0][d].hi = -Fsc[0][d].hi; Fsc[0][d].lo = -Fsc[0][d].lo;
        Fsc[1][d].hi = -Fsc[1][d].hi; Fsc[1][d].lo = -Fsc[1][d].lo;
        F[0][d] = r[0] * acc[0][d];  // the remaining (small) force terms, FP32
        F[1][d] = r[1] * acc[1][d];
    }
    // the cancelling part of the momentum balance, j + F_sc/2, in float-float;
    // the remaining forces are added to it in FP32 below
    ff Bmix[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        Bmix[d] = ff_add(ff_add(M[0].j[d], M[1].j[d]), ff_scale(ff_add(Fsc[0][d], Fsc[1][d]), 0.5f));
    }
    const float FscA[3] = {Fsc[0][0].hi, Fsc[0][1].hi, Fsc[0][2].hi};
    const float FscB[3] = {Fsc[1][0].hi, Fsc[1][1].hi, Fsc[1][2].hi};
    // CSF, Eq. 4: kappa (-div n^a) (grad phi^a / phi_avg) (rho^a / phi_max),
    // phi^A = rho^B and phi^B = rho^A
    if (csf) {
        const float divA = normal_divergence(gA, hB, P.eps_n);
        const float divB = normal_divergence(gB, hA, P.eps_n);
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

        // capillary term of Eq. 1: -Pc(Sw) rho_r n H, H = |grad At|/2.  The
        // gray-cell terms are smooth coefficients of the balance, evaluated
        // with approximate division and the exp2/log2 power (a few ulp).
        const float irt = __fdividef(1.0f, rt);
        const float At_c = __fdividef(rw - rn, rw + rn);
        const float mag = sqrtf(gAt[0] * gAt[0] + gAt[1] * gAt[1] + gAt[2] * gAt[2]);
        const float H = (fabsf(At_c) <= P.at_cut) ? 0.5f * mag : 0.f;
        if (H > 0.f) {
            const float se_c = fminf(fmaxf((sw - cv.swr) * cv.inv_1m_swr, 1e-2f), 1.f);
            // Pc / Pe: Brooks-Corey Se^(-1/lambda), or Thomeer
            // 10^min(-G / ln(1 - Se), 1) = 2^min(k / ln(1 - Se), log2 10) (1 at Se = 1); ln(1 - Se)
            // by log1pf, accurate where Se is small and the quotient steep
            const float pw = cv.thomeer_k != 0.f ? exp2f(fminf(cv.thomeer_k / log1pf(-se_c), LOG2_10))
                                                 : __powf(se_c, cv.neg_inv_lambda);
            const float Pc = gb.x * pw;
            const float k = __fdividef(-Pc * H, fmaxf(mag, P.eps_n)) * irt;
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                F[0][d] += k * r[0] * gAt[d];
                F[1][d] += k * r[1] * gAt[d];
            }
        }
        // viscous term of Eq. 1 with K^-1 = (1/K0)(I + v v^T) (Eq. 7)
        const float se_k = fminf(fmaxf((sw - cv.swr) * cv.inv_1m_swr, 0.f), 1.f);
        const float kr_w = se_k > 0.f ? __powf(se_k, cv.nw) : 0.f;
        const float kr_n = se_k < 1.f ? __powf(1.f - se_k, cv.nn) : 0.f;
        const float coef = __fdividef(rw * P.nu[w], fmaxf(kr_w, P.kr_min)) +
                           __fdividef(rn * P.nu[1 - w], fmaxf(kr_n, P.kr_min));
        const float rk = coef * ga.w;  // coef / K0
        const float v[3] = {ga.x, ga.y, ga.z};
        // (rho I + R/2) u = j + F/2 with R = rk (I + v v^T): Sherman-Morrison
        float b[3];
#pragma unroll
        for (int d = 0; d < 3; ++d) b[d] = ff_add_f(Bmix[d], 0.5f * (F[0][d] + F[1][d])).hi;
        const float al = rt + 0.5f * rk, be = 0.5f * rk;
        const float vb = v[0] * b[0] + v[1] * b[1] + v[2] * b[2];
        const float vv = v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
        const float q = __fdividef(be * vb, al + be * vv);
        const float ial = __fdividef(1.0f, al);
#pragma unroll
        for (int d = 0; d < 3; ++d) u[d] = (b[d] - q * v[d]) * ial;
        const float vu = v[0] * u[0] + v[1] * u[1] + v[2] * u[2];
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            const float Ru = rk * (u[d] + v[d] * vu) * irt;
            F[0][d] -= r[0] * Ru;
            F[1][d] -= r[1] * Ru;
        }
    } else {
#pragma unroll
        for (int d = 0; d < 3; ++d) u[d] = ff_add_f(Bmix[d], 0.5f * (F[0][d] + F[1][d])).hi / rt;
    }
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        F[0][d] += FscA[d];
        F[1][d] += FscB[d];
    }

    // ---- regularised collision, written as rest population + deviations ---
    const float uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    // mass-sink-source: dm = m I moved from the non-wetting to the wetting
    // component as rest equilibrium, I = max(0, (4 r_w r_n - I_b)/(1 - I_b))
    float dm = 0.f;
    if (mss != 0.f) {
        const float it = __fdividef(1.0f, rt);
        dm = mss * fmaxf((4.0f * (rw * it) * (rn * it) - P.mss_ib) * P.mss_inv, 0.f);
    }
#pragma unroll
    for (int a = 0; a < 2; ++a) {
        const float om = P.omega_fac[a];
        const float ra = r[a];
        const float *Fa = F[a];
        const float *S = M[a].S;
        const float uF = u[0] * Fa[0] + u[1] * Fa[1] + u[2] * Fa[2];
        const float d3 = M[a].dr * (1.0f / 3.0f);
        // Pi1 = sum c c h - (drho/3) I - rho u u + (uF + Fu)/2
        const float Pxx = S[0] - d3 - ra * u[0] * u[0] + u[0] * Fa[0];
        const float Pyy = S[1] - d3 - ra * u[1] * u[1] + u[1] * Fa[1];
        const float Pzz = S[2] - d3 - ra * u[2] * u[2] + u[2] * Fa[2];
        const float Pxy = S[3] - ra * u[0] * u[1] + 0.5f * (u[0] * Fa[1] + Fa[0] * u[1]);
        const float Pxz = S[4] - ra * u[0] * u[2] + 0.5f * (u[0] * Fa[2] + Fa[0] * u[2]);
        const float Pyz = S[5] - ra * u[1] * u[2] + 0.5f * (u[1] * Fa[2] + Fa[1] * u[2]);
        const float trP = Pxx + Pyy + Pzz;
        // f*_0 - f_r = drho/3 - rho u^2/2 - om tr(Pi1)/2 - u.F/2
        const float d0 = d3 - 0.5f * ra * uu - 0.5f * om * trP - 0.5f * uF + (a == w ? dm : -dm) * (1.0f / 3.0f);
        const float res = st.rest(a, d0);
        // opposite pairs (i, i+1): cu, cF change sign, cPc does not, so
        // g_i = E + O and g_{i+1} = E - O
#pragma unroll
        for (int i = 1; i < Q; i += 2) {
            const float cu = cx(i) * u[0] + cy(i) * u[1] + cz(i) * u[2];
            const float cF = cx(i) * Fa[0] + cy(i) * Fa[1] + cz(i) * Fa[2];
            float cPc = 0.f;
            if (cx(i)) cPc += Pxx;
            if (cy(i)) cPc += Pyy;
            if (cz(i)) cPc += Pzz;
            if (cx(i) && cy(i)) cPc += 2.0f * cx(i) * cy(i) * Pxy;
            if (cx(i) && cz(i)) cPc += 2.0f * cx(i) * cz(i) * Pxz;
            if (cy(i) && cz(i)) cPc += 2.0f * cy(i) * cz(i) * Pyz;
            const float E = wgt(i) * (4.5f * ra * cu * cu + 4.5f * om * cPc + 4.5f * cu * cF + 3.0f * res);
            const float O = wgt(i) * (3.0f * ra * cu + 1.5f * cF);
            st.pair(a, i, tgt(i), tgt(i + 1), E, O);
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

// The same with the gray record read here.
template <bool MACRO, class Store, class Target>
__device__ __forceinline__ void collide_store(const DevParams &P, const float (&acc)[2][3], float mss, uint8_t t,
                                              int c, int n,
                                              Store &st,
                                              const CompMom M[2], const float gf[2][3], const float gAt[3],
                                              bool csf, const HessSum &hA, const HessSum &hB,
                                              GrayRec *__restrict__ gray, float *__restrict__ macro,
                                              const Target &tgt)
{
    float4 ga = make_float4(0.f, 0.f, 0.f, 0.f), gb = ga;
    if (t == CELL_GRAY) {
        ga = gray[c].a;
        gb = gray[c].b;
    }
    collide_store_g<MACRO>(P, acc, mss, t, c, n, st, M, gf, gAt, csf, hA, hB, ga, gb, gray, macro, tgt);
}

}  // namespace lbm
