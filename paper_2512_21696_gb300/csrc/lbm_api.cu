// C-ABI entry points (include/lbm.h): validation, buffer ownership, stream
// handling and the launch sequence of a time step.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "lbm_context.h"
#include "lbm_host.h"

namespace lbm {
void drop_graphs(lbm_ctx *ctx)
{
    for (auto &gx : ctx->graph) {
        if (gx) cudaGraphExecDestroy(gx);
        gx = nullptr;
    }
}
}  // namespace lbm

namespace lbm_host {

thread_local char g_last_cuda_error[256] = "";

int cuda_fail(cudaError_t e, const char *where)
{
    std::snprintf(g_last_cuda_error, sizeof(g_last_cuda_error), "%s: %s", where, cudaGetErrorString(e));
    (void)cudaGetLastError();  // a non-sticky error must not surface again at a later launch check
    return e == cudaErrorMemoryAllocation ? LBM_ERR_OOM : LBM_ERR_CUDA;
}

// Device buffer that is freed on scope exit (used for staging host inputs).
struct Staging {
    void *ptr = nullptr;
    ~Staging()
    {
        if (ptr) cudaFree(ptr);
    }
};

bool valid_curve(const lbm_constitutive &c)
{
    return c.kc_d > 0 && c.pd > 0 && c.lambda > 0 && c.swr >= 0 && c.swr < 1 && c.nw > 0 && c.nn > 0 &&
           c.phi_ref > 0 && c.phi_ref < 1 && c.pc_ref_max_f > 0 && c.pc_ref_min_f > 0 && c.aniso >= 1 &&
           std::isfinite(c.aniso) && c.thomeer_g >= 0 && std::isfinite(c.thomeer_g);
}

// Bytes of one population buffer: 2 components x 19 slots x n cells.
size_t pop_bytes(const lbm_ctx *ctx)
{
    const size_t n = (size_t)ctx->n;
    if (ctx->p.lattice == LBM_LATTICE_D2Q9) return 2 * 9 * n * sizeof(float);
    switch (ctx->p.storage) {
    case LBM_STORAGE_F32: return 2 * lbm::Q * n * sizeof(float);
    case LBM_STORAGE_F16R:
    case LBM_STORAGE_BF16R: return 2 * n * sizeof(int) + 2 * (lbm::Q - 1) * n * sizeof(uint16_t);
    default: return 2 * lbm::Q * n * sizeof(uint16_t);
    }
}

void fill_device_params(lbm_ctx *ctx)
{
    lbm::drop_graphs(ctx);  // the kernels take these parameters by value
    const lbm_params &p = ctx->p;
    lbm::DevParams &d = ctx->dp;
    d.nx = p.nx;
    d.ny = p.ny;
    d.nz = p.nz;
    for (int k = 0; k < 3; ++k) d.per[k] = p.periodic[k] ? 1 : 0;
    if (p.lattice == LBM_LATTICE_D2Q9) d.per[2] = 1;  // one plane: z-invariant stencils of the geometry pass
    d.n = ctx->n;
    for (int a = 0; a < 2; ++a) {
        d.omega_fac[a] = (float)(1.0 - 1.0 / p.tau[a]);
        d.nu[a] = (float)((p.tau[a] - 0.5) / 3.0);
        d.csf_coef[a] = (float)(1.0 / (p.phi_avg[a] * p.phi_max[a]));
        d.rho_wall[a] = (float)p.rho_wall[a];
        for (int k = 0; k < 3; ++k) d.accel[a][k] = (float)p.body_accel[a][k];
    }
    d.G = (float)p.G;
    d.G_lo = (float)(p.G - (double)d.G);
    d.kappa = (float)p.kappa_csf;
    d.csf_everywhere = p.csf_everywhere ? 1 : 0;
    d.wet = p.wet_idx;
    const double r_lo = p.rho_lo / (p.rho_hi + p.rho_lo), r_hi = p.rho_hi / (p.rho_hi + p.rho_lo);
    d.r_lo = (float)r_lo;
    d.inv_r_span = (float)(1.0 / (r_hi - r_lo));
    d.s_lo = (float)p.s_lo;
    d.s_hi = (float)p.s_hi;
    d.at_cut = (float)p.at_cut;
    d.eps_n = (float)p.eps_n;
    d.kr_min = (float)p.kr_min;
    d.rho0[0] = d.rho0[1] = (float)(0.5 * (p.rho_hi + p.rho_lo));
    for (int side = 0; side < 2; ++side)
        for (int a = 0; a < 2; ++a) {
            const double v = ctx->rho_held[side][a];
            d.held[side][a][0] = (float)v;
            d.held[side][a][1] = (float)(v - (double)(float)v);
        }
    d.mss = (float)ctx->mss;
    d.mss_ib = (float)(4.0 * r_lo * r_hi);
    d.mss_inv = (float)(1.0 / (1.0 - 4.0 * r_lo * r_hi));
    d.storage = p.storage;
    {
        const double ww = p.rho_wall[p.wet_idx], wn = p.rho_wall[1 - p.wet_idx];
        d.at_wall = ww + wn > 0 ? (float)((ww - wn) / (ww + wn)) : 0.0f;
    }
    for (int k = 0; k < LBM_MAX_PORE_TYPES; ++k) {
        const lbm_constitutive &c = ctx->curves[k];
        d.curve[k].swr = (float)c.swr;
        d.curve[k].inv_1m_swr = (float)(1.0 / (1.0 - c.swr));
        d.curve[k].neg_inv_lambda = (float)(-1.0 / c.lambda);
        d.curve[k].nw = (float)c.nw;
        d.curve[k].nn = (float)c.nn;
        // Thomeer: 10^(-G / ln(1 - Se)) = 2^(k / ln(1 - Se)), k = -G log2(10)
        d.curve[k].thomeer_k = c.thomeer_g > 0 ? (float)(-c.thomeer_g * std::log2(10.0)) : 0.0f;
    }
}

void default_held(lbm_ctx *ctx)
{
    for (int side = 0; side < 2; ++side) {
        ctx->rho_held[side][0] = ctx->p.rho_hi;
        ctx->rho_held[side][1] = ctx->p.rho_lo;
    }
}

int stage_in(const void *src, size_t bytes, int mem, cudaStream_t s, Staging &st, const void **dev)
{
    if (mem == LBM_MEM_DEVICE) {
        *dev = src;
        return LBM_OK;
    }
    if (mem != LBM_MEM_HOST) return LBM_ERR_ARG;
    LBM_CUDA(cudaMalloc(&st.ptr, bytes));
    LBM_CUDA(cudaMemcpyAsync(st.ptr, src, bytes, cudaMemcpyHostToDevice, s));
    *dev = st.ptr;
    return LBM_OK;
}

int validate_params(const lbm_params *p)
{
    if (!p) return LBM_ERR_ARG;
    const long long n = (long long)p->nx * p->ny * p->nz;
    if (p->nx < 1 || p->ny < 1 || p->nz < 1 || n > (long long)INT32_MAX / 8) return LBM_ERR_ARG;
    if (!(p->tau[0] > 0.5 && p->tau[1] > 0.5)) return LBM_ERR_ARG;
    if (!(p->rho_hi > p->rho_lo && p->rho_lo > 0.0 && p->rho_hi <= 4.0)) return LBM_ERR_ARG;
    if (!(p->phi_avg[0] > 0 && p->phi_avg[1] > 0 && p->phi_max[0] > 0 && p->phi_max[1] > 0)) return LBM_ERR_ARG;
    if (p->wet_idx != 0 && p->wet_idx != 1) return LBM_ERR_ARG;
    if (!(p->s_lo >= 0 && p->s_lo < p->s_hi && p->s_hi <= 1)) return LBM_ERR_ARG;
    if (!(p->eps_n > 0 && p->kr_min > 0 && p->at_cut >= 0 && p->c_g >= 0)) return LBM_ERR_ARG;
    if (p->storage < LBM_STORAGE_F32 || p->storage > LBM_STORAGE_BF16R) return LBM_ERR_ARG;
    if (p->lattice != LBM_LATTICE_D3Q19 && p->lattice != LBM_LATTICE_D2Q9) return LBM_ERR_ARG;
    if (p->lattice == LBM_LATTICE_D2Q9 && (p->nz != 1 || p->storage != LBM_STORAGE_F32)) return LBM_ERR_ARG;
    for (int a = 0; a < 2; ++a)
        for (int k = 0; k < 3; ++k)
            if (!std::isfinite(p->body_accel[a][k])) return LBM_ERR_ARG;
    return LBM_OK;
}

}  // namespace lbm_host
using namespace lbm_host;

namespace lbm {

void prof_begin(lbm_ctx *ctx, const char *, cudaEvent_t *ev)
{
    *ev = nullptr;
    if (!ctx->profiling) return;
    if (cudaEventCreate(ev) != cudaSuccess) {
        *ev = nullptr;
        return;
    }
    cudaEventRecord(*ev, ctx->stream);
}

void prof_end(lbm_ctx *ctx, const char *name, cudaEvent_t ev0)
{
    if (!ctx->profiling || !ev0) return;
    cudaEvent_t ev1;
    if (cudaEventCreate(&ev1) != cudaSuccess) return;
    cudaEventRecord(ev1, ctx->stream);
    ctx->prof.push_back({name, ev0, ev1});
}

}  // namespace lbm

extern "C" {

const char *lbm_strerror(int code)
{
    switch (code) {
    case LBM_OK: return "ok";
    case LBM_ERR_ARG: return "invalid argument";
    case LBM_ERR_CUDA: return "CUDA runtime error";
    case LBM_ERR_OOM: return "out of memory";
    case LBM_ERR_NUMERIC: return "non-finite or negative density";
    case LBM_ERR_TIMEOUT: return "device wait timed out";
    case LBM_ERR_STATE: return "call out of order";
    default: return "unknown status";
    }
}

const char *lbm_last_cuda_error(void) { return g_last_cuda_error; }

int lbm_abi_version(void) { return LBM_ABI_VERSION; }

size_t lbm_struct_size(int which)
{
    switch (which) {
    case 0: return sizeof(lbm_params);
    case 1: return sizeof(lbm_constitutive);
    case 2: return sizeof(lbm_obs);
    case 3: return sizeof(lbm_kernel_stat);
    default: return 0;
    }
}

int lbm_default_params(lbm_params *p, int nx, int ny, int nz)
{
    if (!p || nx < 1 || ny < 1 || nz < 1) return LBM_ERR_ARG;
    std::memset(p, 0, sizeof(*p));
    p->nx = nx;
    p->ny = ny;
    p->nz = nz;
    p->periodic[0] = p->periodic[1] = p->periodic[2] = 1;
    p->tau[0] = p->tau[1] = 1.0;
    p->rho_hi = 1.0;
    p->rho_lo = 0.03;
    for (int a = 0; a < 2; ++a) {
        p->phi_avg[a] = 0.5 * (p->rho_hi + p->rho_lo);
        p->phi_max[a] = p->rho_hi;
        p->rho_wall[a] = 0.5 * (p->rho_hi + p->rho_lo);
    }
    p->wet_idx = 1;
    p->s_lo = 0.1;
    p->s_hi = 0.9;
    p->at_cut = 0.95;
    p->eps_n = 1e-4 * p->rho_hi;
    p->kr_min = 1e-6;
    p->c_g = 1.0;
    p->storage = LBM_STORAGE_F32;
    p->stream = nullptr;
    p->probe_center[0] = 0.5 * (nx - 1);
    p->probe_center[1] = 0.5 * (ny - 1);
    p->probe_center[2] = 0.5 * (nz - 1);
    p->probe_r_in = 0.0;
    p->probe_r_out = INFINITY;
    p->lattice = LBM_LATTICE_D3Q19;
    return LBM_OK;
}

int lbm_default_constitutive(lbm_constitutive *c)
{
    if (!c) return LBM_ERR_ARG;
    c->kc_d = 1.0;
    c->pd = 0.02;
    c->lambda = 2.0;
    c->swr = 0.15;
    c->nw = 3.0;
    c->nn = 2.0;
    c->phi_ref = 0.35;
    c->pc_ref_max_f = 3.5;
    c->pc_ref_min_f = 0.575;
    c->aniso = 1.0;
    c->thomeer_g = 0.0;
    return LBM_OK;
}

int lbm_create(lbm_ctx **out, const lbm_params *p)
{
    if (!out) return LBM_ERR_ARG;
    *out = nullptr;
    const int vr = validate_params(p);
    if (vr != LBM_OK) return vr;
    const long long n = (long long)p->nx * p->ny * p->nz;

    lbm_ctx *ctx = new (std::nothrow) lbm_ctx();
    if (!ctx) return LBM_ERR_OOM;
    ctx->p = *p;
    ctx->n = (int)n;
    ctx->stream = (cudaStream_t)p->stream;
    if (cudaGetDevice(&ctx->dev) != cudaSuccess) {
        delete ctx;
        return cuda_fail(cudaGetLastError(), "cudaGetDevice");
    }
    for (int k = 0; k < LBM_MAX_PORE_TYPES; ++k) lbm_default_constitutive(&ctx->curves[k]);
    default_held(ctx);
    fill_device_params(ctx);
    const size_t N = (size_t)n;
    cudaError_t e = cudaSuccess;
    for (int b = 0; b < 2 && e == cudaSuccess; ++b) {
        e = cudaMalloc(&ctx->f[b], pop_bytes(ctx));
        if (e == cudaSuccess) e = cudaMemset(ctx->f[b], 0, pop_bytes(ctx));  // solid cells' slots stay zero
    }
    if (e == cudaSuccess) e = cudaMalloc(&ctx->type, N);
    if (e == cudaSuccess) e = cudaMalloc(&ctx->phi, N * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&ctx->gray, N * sizeof(lbm::GrayRec));
    if (e == cudaSuccess) e = cudaMalloc(&ctx->rho, 3 * N * sizeof(float));  // drho^A, drho^B, At
    if (e == cudaSuccess) e = cudaMalloc(&ctx->macro, 6 * N * sizeof(float));
    ctx->red_blocks = lbm::obs_blocks(ctx->n);
    if (e == cudaSuccess) e = cudaMalloc(&ctx->red, (size_t)(ctx->red_blocks + 1) * lbm::NOBS_HOST * sizeof(double));
    // zero: the reduction's completion count starts there
    if (e == cudaSuccess) e = cudaMemset(ctx->red, 0, (size_t)(ctx->red_blocks + 1) * lbm::NOBS_HOST * sizeof(double));
    // the published-density march: wall masks, published densities, progress counters (zero)
    if (e == cudaSuccess) e = cudaMalloc(&ctx->wmask, N * sizeof(uint32_t));
    if (e == cudaSuccess) e = cudaMalloc(&ctx->pub, N * sizeof(float2));
    if (e == cudaSuccess) e = cudaMemset(ctx->pub, 0, N * sizeof(float2));
    if (e == cudaSuccess) e = cudaMalloc(&ctx->prog, lbm::MARCH_PROG_LEN * sizeof(unsigned));
    if (e == cudaSuccess) e = cudaMemset(ctx->prog, 0, lbm::MARCH_PROG_LEN * sizeof(unsigned));
    if (e == cudaSuccess) ctx->prog_len = lbm::MARCH_PROG_LEN;

    if (e != cudaSuccess) {
        int code = cuda_fail(e, "lbm_create allocation");
        lbm_destroy(ctx);
        return code;
    }
    *out = ctx;
    return LBM_OK;
}

int lbm_destroy(lbm_ctx *ctx)
{
    if (!ctx) return LBM_OK;
    if (ctx->view) return LBM_ERR_ARG;  // owned by its batch
    DeviceGuard g(ctx->dev);
    for (auto &r : ctx->prof) {
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
    }
    lbm::drop_graphs(ctx);
    if (ctx->cap) cudaStreamDestroy(ctx->cap);
    cudaFree(ctx->f[0]);
    cudaFree(ctx->f[1]);
    cudaFree(ctx->type);
    cudaFree(ctx->phi);
    cudaFree(ctx->gray);
    cudaFree(ctx->rho);
    cudaFree(ctx->macro);
    cudaFree(ctx->red);
    cudaFree(ctx->wmask);
    cudaFree(ctx->pub);
    cudaFree(ctx->prog);
    delete ctx;
    return LBM_OK;
}

int lbm_set_constitutive(lbm_ctx *ctx, int pore_type, const lbm_constitutive *c)
{
    if (!ctx || !c || pore_type < 0 || pore_type >= LBM_MAX_PORE_TYPES) return LBM_ERR_ARG;
    if (!valid_curve(*c)) return LBM_ERR_ARG;
    ctx->curves[pore_type] = *c;
    fill_device_params(ctx);
    return LBM_OK;
}

int lbm_set_geometry(lbm_ctx *ctx, const uint8_t *type, const float *phi, const uint8_t *pore_type, int mem)
{
    if (!ctx || !type || !phi) return LBM_ERR_ARG;
    if (mem != LBM_MEM_HOST && mem != LBM_MEM_DEVICE) return LBM_ERR_ARG;
    DeviceGuard g(ctx->dev);
    if (!g.ok) return LBM_ERR_CUDA;
    const size_t N = (size_t)ctx->n;
    // Validate on the host (one-time cost): device inputs are copied down.
    std::vector<uint8_t> ht(N), hp8(pore_type ? N : 0);
    std::vector<float> hphi(N);
    if (mem == LBM_MEM_DEVICE) {
        LBM_CUDA(cudaMemcpyAsync(ht.data(), type, N, cudaMemcpyDeviceToHost, ctx->stream));
        LBM_CUDA(cudaMemcpyAsync(hphi.data(), phi, N * sizeof(float), cudaMemcpyDeviceToHost, ctx->stream));
        if (pore_type) LBM_CUDA(cudaMemcpyAsync(hp8.data(), pore_type, N, cudaMemcpyDeviceToHost, ctx->stream));
        LBM_CUDA(cudaStreamSynchronize(ctx->stream));
    } else {
        std::memcpy(ht.data(), type, N);
        std::memcpy(hphi.data(), phi, N * sizeof(float));
        if (pore_type) std::memcpy(hp8.data(), pore_type, N);
    }
    long long held = 0;
    for (size_t c = 0; c < N; ++c) {
        const uint8_t t = ht[c];
        if (t > LBM_CELL_OUTLET) return LBM_ERR_ARG;
        if (t == LBM_CELL_GRAY) {
            if (!(hphi[c] > 0.0f && hphi[c] < 1.0f)) return LBM_ERR_ARG;
        } else {
            hphi[c] = t == LBM_CELL_SOLID ? 0.0f : 1.0f;
        }
        held += lbm::is_held(t) ? 1 : 0;
        if (pore_type && hp8[c] >= LBM_MAX_PORE_TYPES) return LBM_ERR_ARG;
    }
    ctx->n_held = held;
    LBM_CUDA(cudaMemcpyAsync(ctx->type, ht.data(), N, cudaMemcpyHostToDevice, ctx->stream));
    LBM_CUDA(cudaMemcpyAsync(ctx->phi, hphi.data(), N * sizeof(float), cudaMemcpyHostToDevice, ctx->stream));
    Staging pt;
    const uint8_t *dpt = nullptr;
    if (pore_type) {
        LBM_CUDA(cudaMalloc(&pt.ptr, N));
        LBM_CUDA(cudaMemcpyAsync(pt.ptr, hp8.data(), N, cudaMemcpyHostToDevice, ctx->stream));
        dpt = (const uint8_t *)pt.ptr;
    }
    LBM_CUDA(cudaMemsetAsync(ctx->gray, 0, N * sizeof(lbm::GrayRec), ctx->stream));
    fill_device_params(ctx);
    LBM_CUDA(lbm::launch_geometry(ctx, dpt));
    LBM_CUDA(lbm::launch_wallmask(ctx));
    LBM_CUDA(cudaStreamSynchronize(ctx->stream));
    ctx->has_geometry = true;
    ctx->has_fields = false;
    return LBM_OK;
}

int lbm_set_pressure(lbm_ctx *ctx, const double rho_in[2], const double rho_out[2])
{
    if (!ctx || !rho_in || !rho_out) return LBM_ERR_ARG;
    for (const double *r : {rho_in, rho_out}) {
        if (!std::isfinite(r[0]) || !std::isfinite(r[1]) || r[0] < 0.0 || r[1] < 0.0 || !(r[0] + r[1] > 0.0))
            return LBM_ERR_ARG;
    }
    for (int a = 0; a < 2; ++a) {
        ctx->rho_held[0][a] = rho_in[a];
        ctx->rho_held[1][a] = rho_out[a];
    }
    fill_device_params(ctx);
    if (ctx->owner) lbm::batch_runs_changed(ctx->owner);
    return LBM_OK;
}

int lbm_set_mss(lbm_ctx *ctx, double rate)
{
    if (!ctx || !std::isfinite(rate)) return LBM_ERR_ARG;
    ctx->mss = rate;
    fill_device_params(ctx);
    if (ctx->owner) lbm::batch_runs_changed(ctx->owner);
    return LBM_OK;
}

int lbm_mss_to_saturation(lbm_ctx *ctx, double target, double gain, double max_rate, double tol, int check_every,
                          int max_steps, int *steps_done)
{
    if (!ctx || !steps_done || !(target >= 0.0 && target <= 1.0) || !(gain > 0.0) || !(max_rate > 0.0) ||
        !(tol > 0.0) || check_every < 1 || max_steps < 1 || !std::isfinite(gain) || !std::isfinite(max_rate))
        return LBM_ERR_ARG;
    if (!ctx->has_fields) return LBM_ERR_STATE;
    int done = 0, rc = LBM_OK;
    bool reached = false;
    lbm_obs o;
    while (rc == LBM_OK) {
        rc = lbm_observables(ctx, &o);
        if (rc != LBM_OK) break;
        const double err = target - o.sat;
        reached = std::fabs(err) <= tol;
        if (reached || done >= max_steps) break;
        rc = lbm_set_mss(ctx, std::max(-max_rate, std::min(max_rate, gain * err)));
        const int m = std::min(check_every, max_steps - done);
        if (rc == LBM_OK) rc = lbm_step(ctx, m);
        done += m;
    }
    const int off = lbm_set_mss(ctx, 0.0);
    *steps_done = done;
    if (rc != LBM_OK) return rc;
    if (off != LBM_OK) return off;
    return reached ? LBM_OK : LBM_ERR_TIMEOUT;
}

int lbm_pressure_levels(lbm_ctx *ctx, int nlevels, const double *rho_in, const double *rho_out, int check_every,
                        double sat_tol, int max_steps, double *sat, int *steps)
{
    if (!ctx || nlevels < 1 || !rho_in || !rho_out || check_every < 1 || !(sat_tol >= 0.0) || max_steps < 1 ||
        !sat || !steps)
        return LBM_ERR_ARG;
    for (int k = 0; k < 2 * nlevels; k += 2)
        for (const double *r : {rho_in + k, rho_out + k})
            if (!std::isfinite(r[0]) || !std::isfinite(r[1]) || r[0] < 0.0 || r[1] < 0.0 || !(r[0] + r[1] > 0.0))
                return LBM_ERR_ARG;
    if (!ctx->has_fields || ctx->n_held == 0) return LBM_ERR_STATE;
    bool all = true;
    for (int k = 0; k < nlevels; ++k) {
        int rc = lbm_set_pressure(ctx, rho_in + 2 * k, rho_out + 2 * k);
        lbm_obs o;
        if (rc == LBM_OK) rc = lbm_observables(ctx, &o);
        if (rc != LBM_OK) return rc;
        double prev = o.sat;
        int done = 0;
        bool steady = false;
        while (done < max_steps && !steady) {
            const int m = std::min(check_every, max_steps - done);
            rc = lbm_step(ctx, m);
            if (rc == LBM_OK) rc = lbm_observables(ctx, &o);
            if (rc != LBM_OK) return rc;
            done += m;
            steady = std::fabs(o.sat - prev) <= sat_tol;
            prev = o.sat;
        }
        sat[k] = o.sat;
        steps[k] = done;
        all = all && steady;
    }
    return all ? LBM_OK : LBM_ERR_TIMEOUT;
}

int lbm_init_fields(lbm_ctx *ctx, const float *rhoA, const float *rhoB, const float *u, int mem)
{
    if (!ctx || !rhoA || !rhoB) return LBM_ERR_ARG;
    if (!ctx->has_geometry) return LBM_ERR_STATE;
    DeviceGuard g(ctx->dev);
    if (!g.ok) return LBM_ERR_CUDA;
    const size_t N = (size_t)ctx->n;
    Staging sa, sb, su;
    const void *da, *db, *du = nullptr;
    int rc;
    if ((rc = stage_in(rhoA, N * sizeof(float), mem, ctx->stream, sa, &da)) != LBM_OK) return rc;
    if ((rc = stage_in(rhoB, N * sizeof(float), mem, ctx->stream, sb, &db)) != LBM_OK) return rc;
    if (u && (rc = stage_in(u, 3 * N * sizeof(float), mem, ctx->stream, su, &du)) != LBM_OK) return rc;
    lbm::drop_graphs(ctx);
    ctx->cur = 0;
    if (ctx->p.lattice == LBM_LATTICE_D2Q9)
        LBM_CUDA(lbm::launch_d2q9_init(ctx, (const float *)da, (const float *)db, (const float *)du));
    else
        LBM_CUDA(lbm::launch_init(ctx, (const float *)da, (const float *)db, (const float *)du));
    if (mem == LBM_MEM_HOST) LBM_CUDA(cudaStreamSynchronize(ctx->stream));
    ctx->steps = 0;
    ctx->has_fields = true;
    return LBM_OK;
}

// One step: its kernels on ctx->stream (fields written if write_macro).
static cudaError_t step_once(lbm_ctx *ctx, bool write_macro)
{
    cudaError_t e;
    if (ctx->p.lattice == LBM_LATTICE_D2Q9) {
        e = lbm::launch_d2q9_step(ctx, write_macro);
    } else if (ctx->p.storage == LBM_STORAGE_F16S || ctx->p.storage == LBM_STORAGE_BF16S) {
        e = lbm::launch_fused_lp(ctx, write_macro);
    } else if (ctx->path == 1 && ctx->p.storage == LBM_STORAGE_F32) {
        e = lbm::launch_density(ctx);
        if (e == cudaSuccess) e = lbm::launch_collide(ctx, write_macro);
    } else {
        e = lbm::launch_fused(ctx, write_macro);
    }
    if (e == cudaSuccess) ctx->steps += 1;
    return e;
}

// Captures GRAPH_STEPS steps (no field output) from the current buffer parity
// on the private stream; nothing runs.  Returns false, with the context as
// before, when the capture or instantiation fails.
static bool capture_steps(lbm_ctx *ctx)
{
    if (!ctx->cap && cudaStreamCreateWithFlags(&ctx->cap, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    const cudaStream_t user = ctx->stream;
    const int cur0 = ctx->cur;
    const long long steps0 = ctx->steps, launches0 = ctx->launches;
    ctx->stream = ctx->cap;
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamBeginCapture(ctx->cap, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        for (int k = 0; k < lbm::GRAPH_STEPS && e == cudaSuccess; ++k) e = step_once(ctx, false);
        const cudaError_t ce = cudaStreamEndCapture(ctx->cap, &graph);
        if (e == cudaSuccess) e = ce;
    }
    ctx->stream = user;
    const long long per_replay = ctx->launches - launches0;
    ctx->cur = cur0;  // nothing ran: the state is where it was
    ctx->steps = steps0;
    ctx->launches = launches0;
    cudaGraphExec_t exec = nullptr;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
        cudaGetLastError();  // capture errors leave the context usable
        return false;
    }
    ctx->graph[cur0] = exec;
    ctx->graph_launches = per_replay;
    return true;
}

int lbm_step(lbm_ctx *ctx, int nsteps)
{
    if (!ctx || nsteps < 0) return LBM_ERR_ARG;
    if (!ctx->has_fields) return LBM_ERR_STATE;
    DeviceGuard g(ctx->dev);
    if (!g.ok) return LBM_ERR_CUDA;
    int k = 0;
    // small lattices: after one direct step (which also resolves each
    // kernel's launch configuration), replay GRAPH_STEPS-step graphs while
    // more than GRAPH_STEPS steps remain; the last steps, which write the
    // fields, run directly.  A caller capturing its own stream gets direct
    // launches (a capture of ours inside theirs could invalidate it).
    // The march (tiles 5, 6) is a cooperative launch and steps directly.
    bool replay = !ctx->view && !ctx->profiling && !ctx->graph_off && ctx->n <= lbm::GRAPH_MAX_CELLS &&
                  ctx->tile != 5 && ctx->tile != 6 && nsteps > lbm::GRAPH_STEPS + 1;
    if (replay) {
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        if (cudaStreamIsCapturing(ctx->stream, &cs) != cudaSuccess) {
            cudaGetLastError();
            cs = cudaStreamCaptureStatusActive;
        }
        replay = cs == cudaStreamCaptureStatusNone;
    }
    if (replay) {
        LBM_CUDA(step_once(ctx, false));
        k = 1;
        while (nsteps - k > lbm::GRAPH_STEPS) {
            if (!ctx->graph[ctx->cur] && !capture_steps(ctx)) {
                ctx->graph_off = true;
                break;
            }
            LBM_CUDA(cudaGraphLaunch(ctx->graph[ctx->cur], ctx->stream));
            ctx->steps += lbm::GRAPH_STEPS;
            ctx->launches += ctx->graph_launches;
            k += lbm::GRAPH_STEPS;  // even: the state is back in buffer cur
        }
    }
    for (; k < nsteps; ++k) LBM_CUDA(step_once(ctx, k == nsteps - 1));
    return LBM_OK;
}

int lbm_observables(lbm_ctx *ctx, lbm_obs *out)
{
    if (!ctx || !out) return LBM_ERR_ARG;
    if (!ctx->has_fields) return LBM_ERR_STATE;
    DeviceGuard g(ctx->dev);
    if (!g.ok) return LBM_ERR_CUDA;
    double v[LBM_OBS_RAW];
    LBM_CUDA(lbm::launch_observables(ctx, v));
    v[lbm::NOBS_HOST] = (double)ctx->steps;
    int timed_out = 0;
    LBM_CUDA(lbm::march_take_error(ctx, &timed_out));
    if (timed_out) return LBM_ERR_TIMEOUT;
    return lbm_obs_decode(ctx, v, out);
}

int lbm_observables_async(lbm_ctx *ctx, double *raw)
{
    if (!ctx || !raw) return LBM_ERR_ARG;
    if (!ctx->has_fields) return LBM_ERR_STATE;
    DeviceGuard g(ctx->dev);
    if (!g.ok) return LBM_ERR_CUDA;
    raw[lbm::NOBS_HOST] = (double)ctx->steps;
    LBM_CUDA(lbm::launch_observables(ctx, raw, false));
    return LBM_OK;
}

int lbm_obs_decode(lbm_ctx *ctx, const double *v, lbm_obs *out)
{
    if (!ctx || !v || !out) return LBM_ERR_ARG;
    const lbm_params &p = ctx->p;
    out->mass[0] = v[0];
    out->mass[1] = v[1];
    out->sat = v[3] > 0 ? v[2] / v[3] : 0.0;
    out->flux_out = v[4] / ((double)p.ny * p.nz);
    for (int d = 0; d < 3; ++d) out->flux_vol[d] = v[5 + d] / (double)ctx->n;
    out->max_u = v[8];
    out->dp = (v[10] > 0 ? v[9] / v[10] : 0.0) - (v[12] > 0 ? v[11] / v[12] : 0.0);
    out->nan_count = (long long)v[13];
    out->step = (long long)v[lbm::NOBS_HOST];
    return out->nan_count > 0 ? LBM_ERR_NUMERIC : LBM_OK;
}

int lbm_get_fields(lbm_ctx *ctx, float *rhoA, float *rhoB, float *u, float *sw, int mem)
{
    if (!ctx) return LBM_ERR_ARG;
    if (mem != LBM_MEM_HOST && mem != LBM_MEM_DEVICE) return LBM_ERR_ARG;
    if (!ctx->has_fields) return LBM_ERR_STATE;
    DeviceGuard g(ctx->dev);
    if (!g.ok) return LBM_ERR_CUDA;
    const size_t N = (size_t)ctx->n;
    const cudaMemcpyKind kind = mem == LBM_MEM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
    if (rhoA) LBM_CUDA(cudaMemcpyAsync(rhoA, ctx->macro, N * sizeof(float), kind, ctx->stream));
    if (rhoB) LBM_CUDA(cudaMemcpyAsync(rhoB, ctx->macro + N, N * sizeof(float), kind, ctx->stream));
    if (u) LBM_CUDA(cudaMemcpyAsync(u, ctx->macro + 2 * N, 3 * N * sizeof(float), kind, ctx->stream));
    if (sw) LBM_CUDA(cudaMemcpyAsync(sw, ctx->macro + 5 * N, N * sizeof(float), kind, ctx->stream));
    if (mem == LBM_MEM_HOST) LBM_CUDA(cudaStreamSynchronize(ctx->stream));
    int timed_out = 0;
    LBM_CUDA(lbm::march_take_error(ctx, &timed_out));
    if (timed_out) return LBM_ERR_TIMEOUT;
    return LBM_OK;
}

int lbm_get_static(lbm_ctx *ctx, float *kinv, float *pc_scale, float *sw_irr, float *so_res, int mem)
{
    if (!ctx) return LBM_ERR_ARG;
    if (mem != LBM_MEM_HOST && mem != LBM_MEM_DEVICE) return LBM_ERR_ARG;
    if (!ctx->has_geometry) return LBM_ERR_STATE;
    DeviceGuard g(ctx->dev);
    if (!g.ok) return LBM_ERR_CUDA;
    const size_t N = (size_t)ctx->n;
    if (mem == LBM_MEM_DEVICE) {
        LBM_CUDA(lbm::launch_static_out(ctx, kinv, pc_scale, sw_irr, so_res));
        return LBM_OK;
    }
    Staging st;
    LBM_CUDA(cudaMalloc(&st.ptr, 9 * N * sizeof(float)));
    float *d = (float *)st.ptr;
    LBM_CUDA(lbm::launch_static_out(ctx, d, d + 6 * N, d + 7 * N, d + 8 * N));
    if (kinv) LBM_CUDA(cudaMemcpyAsync(kinv, d, 6 * N * sizeof(float), cudaMemcpyDeviceToHost, ctx->stream));
    if (pc_scale) LBM_CUDA(cudaMemcpyAsync(pc_scale, d + 6 * N, N * sizeof(float), cudaMemcpyDeviceToHost, ctx->stream));
    if (sw_irr) LBM_CUDA(cudaMemcpyAsync(sw_irr, d + 7 * N, N * sizeof(float), cudaMemcpyDeviceToHost, ctx->stream));
    if (so_res) LBM_CUDA(cudaMemcpyAsync(so_res, d + 8 * N, N * sizeof(float), cudaMemcpyDeviceToHost, ctx->stream));
    LBM_CUDA(cudaStreamSynchronize(ctx->stream));
    return LBM_OK;
}

// Checkpoint layout: [int64 magic][int64 n][int64 steps][int64 storage]
// [populations 38 n slots of the storage][gray records n * 32 B][macro 6 n float].
static size_t state_bytes(const lbm_ctx *ctx)
{
    const size_t N = (size_t)ctx->n;
    return 4 * sizeof(long long) + pop_bytes(ctx) + N * sizeof(lbm::GrayRec) + 6 * N * sizeof(float);
}
static const long long STATE_MAGIC = 0x4c424d3253544154LL;  // "LBM2STAT"

int lbm_state_size(lbm_ctx *ctx, size_t *bytes)
{
    if (!ctx || !bytes) return LBM_ERR_ARG;
    *bytes = state_bytes(ctx);
    return LBM_OK;
}

int lbm_save_state(lbm_ctx *ctx, void *buf, size_t bytes)
{
    if (!ctx || !buf || bytes < state_bytes(ctx)) return LBM_ERR_ARG;
    if (!ctx->has_fields) return LBM_ERR_STATE;
    DeviceGuard g(ctx->dev);
    if (!g.ok) return LBM_ERR_CUDA;
    const size_t N = (size_t)ctx->n;
    long long *hdr = (long long *)buf;
    hdr[0] = STATE_MAGIC;
    hdr[1] = ctx->n;
    hdr[2] = ctx->steps;
    hdr[3] = ctx->p.storage;
    char *p = (char *)buf + 4 * sizeof(long long);
    LBM_CUDA(cudaMemcpyAsync(p, ctx->f[ctx->cur], pop_bytes(ctx), cudaMemcpyDeviceToHost, ctx->stream));
    p += pop_bytes(ctx);
    LBM_CUDA(cudaMemcpyAsync(p, ctx->gray, N * sizeof(lbm::GrayRec), cudaMemcpyDeviceToHost, ctx->stream));
    p += N * sizeof(lbm::GrayRec);
    LBM_CUDA(cudaMemcpyAsync(p, ctx->macro, 6 * N * sizeof(float), cudaMemcpyDeviceToHost, ctx->stream));
    LBM_CUDA(cudaStreamSynchronize(ctx->stream));
    return LBM_OK;
}

int lbm_load_state(lbm_ctx *ctx, const void *buf, size_t bytes)
{
    if (!ctx || !buf || bytes < state_bytes(ctx)) return LBM_ERR_ARG;
    if (!ctx->has_geometry) return LBM_ERR_STATE;
    const long long *hdr = (const long long *)buf;
    if (hdr[0] != STATE_MAGIC || hdr[1] != ctx->n || hdr[3] != ctx->p.storage) return LBM_ERR_ARG;
    DeviceGuard g(ctx->dev);
    if (!g.ok) return LBM_ERR_CUDA;
    const size_t N = (size_t)ctx->n;
    const char *p = (const char *)buf + 4 * sizeof(long long);
    lbm::drop_graphs(ctx);
    ctx->cur = 0;
    LBM_CUDA(cudaMemcpyAsync(ctx->f[0], p, pop_bytes(ctx), cudaMemcpyHostToDevice, ctx->stream));
    p += pop_bytes(ctx);
    LBM_CUDA(cudaMemcpyAsync(ctx->gray, p, N * sizeof(lbm::GrayRec), cudaMemcpyHostToDevice, ctx->stream));
    p += N * sizeof(lbm::GrayRec);
    LBM_CUDA(cudaMemcpyAsync(ctx->macro, p, 6 * N * sizeof(float), cudaMemcpyHostToDevice, ctx->stream));
    LBM_CUDA(cudaStreamSynchronize(ctx->stream));
    ctx->steps = hdr[2];
    ctx->has_fields = true;
    return LBM_OK;
}

int lbm_profile(lbm_ctx *ctx, int enable)
{
    if (!ctx) return LBM_ERR_ARG;
    DeviceGuard g(ctx->dev);
    for (auto &r : ctx->prof) {
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
    }
    ctx->prof.clear();
    ctx->profiling = enable != 0;
    lbm::drop_graphs(ctx);
    return LBM_OK;
}

int lbm_profile_read(lbm_ctx *ctx, lbm_kernel_stat *out, int max, int *count)
{
    if (!ctx || !count || (max > 0 && !out)) return LBM_ERR_ARG;
    DeviceGuard g(ctx->dev);
    if (!g.ok) return LBM_ERR_CUDA;
    LBM_CUDA(cudaStreamSynchronize(ctx->stream));
    std::vector<lbm_kernel_stat> acc;
    for (auto &r : ctx->prof) {
        float ms = 0.f;
        LBM_CUDA(cudaEventElapsedTime(&ms, r.a, r.b));
        lbm_kernel_stat *slot = nullptr;
        for (auto &s : acc)
            if (std::strncmp(s.name, r.name, sizeof(s.name)) == 0) slot = &s;
        if (!slot) {
            lbm_kernel_stat s{};
            std::snprintf(s.name, sizeof(s.name), "%s", r.name);
            acc.push_back(s);
            slot = &acc.back();
        }
        slot->launches += 1;
        slot->total_ms += ms;
    }
    *count = (int)acc.size();
    for (int k = 0; k < max && k < (int)acc.size(); ++k) out[k] = acc[k];
    return LBM_OK;
}

int lbm_set_kernel(lbm_ctx *ctx, int path, int tile)
{
    if (!ctx || path < 0 || path > 1 || tile < 0 || tile > 8) return LBM_ERR_ARG;
    ctx->path = path;
    ctx->tile = tile;
    lbm::drop_graphs(ctx);
    return LBM_OK;
}

int lbm_get_kernel(lbm_ctx *ctx, int *path, int *tile)
{
    if (!ctx || !path || !tile) return LBM_ERR_ARG;
    DeviceGuard g(ctx->dev);
    if (!g.ok) return LBM_ERR_CUDA;
    *path = ctx->path;
    *tile = ctx->path == 0 ? lbm::fused_tile_in_use(ctx) : ctx->tile;
    return LBM_OK;
}

int lbm_inject_launch_failures(lbm_ctx *ctx, int count)
{
    if (!ctx || count < 0) return LBM_ERR_ARG;
    ctx->fail_launches = count;
    lbm::drop_graphs(ctx);  // replays would bypass the launchers
    return LBM_OK;
}

int lbm_launch_count(lbm_ctx *ctx, long long *count)
{
    if (!ctx || !count) return LBM_ERR_ARG;
    *count = ctx->launches;
    return LBM_OK;
}

}  // extern "C"
