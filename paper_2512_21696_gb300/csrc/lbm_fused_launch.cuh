// The fused step kernel of one lattice and its launch, shared by the
// translation units that instantiate its tile shapes (lbm_fused.cu: the
// default shapes and the automatic choice; lbm_fused_alt.cu: the other
// selectable shapes; lbm_fused_f16r.cu, lbm_fused_bf16r.cu: the 16-bit
// rest-referenced layouts; compiled in parallel).
//
// Work items are (column, z-chunk) with the items of one chunk consecutive, so
// the CTAs of a wave march neighbouring columns through the same planes at the
// same time and the halo reads hit lines their neighbours have just brought
// into L2.  The march itself is fused_item (lbm_fused.cuh).
#pragma once

#include <algorithm>

#include "lbm_context.h"
#include "lbm_fused.cuh"

namespace lbm {

template <int TX, int TY, int MINB, bool MACRO, bool EXT, class LY, bool CAP = false>
__global__ void __launch_bounds__(TX *TY, MINB)
    k_fused(DevParams P, int zchunks, LY ly, const uint8_t *__restrict__ type, GrayRec *__restrict__ gray,
            float *__restrict__ macro, float *__restrict__ cap)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const Geo G = geo_of(P);
    const int tiles_x = (P.nx + TX - 1) / TX, tiles_y = (P.ny + TY - 1) / TY;
    const int ncol = tiles_x * tiles_y;
    for (int item = blockIdx.x; item < ncol * zchunks; item += gridDim.x) {
        const int col = item % ncol, chunk = item / ncol;
        const int za = (int)((long long)P.nz * chunk / zchunks);
        const int zb = (int)((long long)P.nz * (chunk + 1) / zchunks);
        if (za >= zb) continue;
        fused_item<TX, TY, MACRO, EXT, LY, CAP>(P, G, ly, type, gray, macro, (col % tiles_x) * TX,
                                                (col / tiles_x) * TY, za, zb, smem_raw, cap);
    }
}

// ---------------------------------------------------------------------------
// Resident CTAs of one instantiation on the context's device (resolved once
// per device; also sets the kernel's dynamic shared-memory limit).
template <int TX, int TY, int MINB, bool MACRO, bool EXT, class LY, bool CAP = false>
static cudaError_t fused_slots(lbm_ctx *ctx, int *slots)
{
    auto kern = k_fused<TX, TY, MINB, MACRO, EXT, LY, CAP>;
    const size_t smem = Tiles<TX, TY>::smem();
    static int cached_slots[64] = {};  // resident CTAs per device
    const int dev = ctx->dev < 64 ? ctx->dev : 63;
    if (!cached_slots[dev]) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        int per_sm = 0, sms = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, TX * TY, smem);
        if (e != cudaSuccess) return e;
        e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->dev);
        if (e != cudaSuccess) return e;
        cached_slots[dev] = std::max(per_sm, 1) * sms;
    }
    *slots = cached_slots[dev];
    return cudaSuccess;
}

// z-chunks per column so that one wave of resident CTAs covers the grid
static int fused_zchunks(const lbm_params &p, int tx, int ty, int slots)
{
    const long long ncol = (long long)((p.nx + tx - 1) / tx) * ((p.ny + ty - 1) / ty);
    return (int)std::max<long long>(1, std::min<long long>(slots / ncol, p.nz));
}

template <int TX, int TY, int MINB, bool MACRO, bool EXT, class LY, bool CAP = false>
static cudaError_t launch_fused_t(lbm_ctx *ctx, LY ly)
{
    auto kern = k_fused<TX, TY, MINB, MACRO, EXT, LY, CAP>;
    const size_t smem = Tiles<TX, TY>::smem();
    int slots = 0;
    cudaError_t es = fused_slots<TX, TY, MINB, MACRO, EXT, LY, CAP>(ctx, &slots);
    if (es != cudaSuccess) return es;
    const long long ncol = (long long)((ctx->p.nx + TX - 1) / TX) * ((ctx->p.ny + TY - 1) / TY);
    const int zchunks = fused_zchunks(ctx->p, TX, TY, slots);
    const long long grid = std::min<long long>(ncol * zchunks, slots);
    cudaEvent_t e0;
    prof_begin(ctx, "k_fused", &e0);
    kern<<<(unsigned)grid, step_block(ctx, TX * TY), smem, ctx->stream>>>(ctx->dp, zchunks, ly, ctx->type,
                                                                        ctx->gray, ctx->macro, ctx->rho_cap);
    prof_end(ctx, "k_fused", e0);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;  // nothing ran: the state stays in buffer cur
    ctx->launches += 1;
    ctx->cur = 1 - ctx->cur;
    return cudaSuccess;
}

// Geometries with reservoir cells, or a mass-sink-source rate, run the
// instantiation that handles them; the others keep the plain march.
template <int TX, int TY, int MINB, class LY>
static cudaError_t launch_fused_tile(lbm_ctx *ctx, bool write_macro, LY ly)
{
    if (ctx->n_held > 0 || ctx->mss != 0.0)
        return write_macro ? launch_fused_t<TX, TY, MINB, true, true>(ctx, ly)
                           : launch_fused_t<TX, TY, MINB, false, true>(ctx, ly);
    return write_macro ? launch_fused_t<TX, TY, MINB, true, false>(ctx, ly)
                       : launch_fused_t<TX, TY, MINB, false, false>(ctx, ly);
}

// The automatic choice (tile 8) among 2 (32x8, two CTAs per SM), 4 (64x8)
// and 7 (64x7): the grid of each is one wave of z-chunked columns, and its
// step lasts about (planes per chunk + the 2 halo planes) x the time a
// resident CTA takes per plane, times the waves.  Per-plane times of the
// three shapes on a GB300 (F32, 2070 MHz), fitted to the 128^3 drainage and
// 192^3 fibre-bundle steps (32x8: 12.26 and 12.59 us measured; 64x8: 12.24 and
// 12.19; 64x7: 11.8 and 11.7, then 11.26 on 128^3 with the density pass's
// sub-partition order): 12.45, 12.2 and 11.3 us.  64x7 wins where its
// extra columns fill the SMs (128^3: 152 items on 152 slots, against 128 of
// 152 for 64x8 and 256 of 304 for 32x8), 64x8 where both fill them (192^3);
// lattices whose width is not a multiple of 64 keep 32x8.
// (a template, so that only the translation unit that calls it instantiates
// the candidates' kernels)
template <int UNUSED = 0>
static int auto_tile(lbm_ctx *ctx)
{
    if (ctx->auto_tile >= 0) return ctx->auto_tile;
    struct Cand {
        int tile, tx, ty;
        double t_plane;
        int slots;
    } cand[3] = {{2, 32, 8, 12.45, 0}, {4, 64, 8, 12.2, 0}, {7, 64, 7, 11.3, 0}};
    if (fused_slots<32, 8, 2, false, false, LayF32>(ctx, &cand[0].slots) != cudaSuccess ||
        fused_slots<64, 8, 1, false, false, LayF32>(ctx, &cand[1].slots) != cudaSuccess ||
        fused_slots<64, 7, 1, false, false, LayF32>(ctx, &cand[2].slots) != cudaSuccess) {
        cudaGetLastError();
        return 2;  // not cached: the launch itself reports any error
    }
    int best = 2;
    double best_t = 0.0;
    for (const Cand &cd : cand) {
        // the per-plane times hold for full-width tiles: a 64-wide tile on a
        // lattice that is not a multiple of 64 wide idles part of its warps
        if (cd.tx != 32 && ctx->p.nx % cd.tx != 0) continue;
        const long long ncol = (long long)((ctx->p.nx + cd.tx - 1) / cd.tx) * ((ctx->p.ny + cd.ty - 1) / cd.ty);
        const int zch = fused_zchunks(ctx->p, cd.tx, cd.ty, cd.slots);
        const long long items = ncol * zch;
        const long long waves = (items + cd.slots - 1) / cd.slots;
        const double t = (double)waves * ((ctx->p.nz + zch - 1) / zch + 2) * cd.t_plane;
        if (best_t == 0.0 || t < best_t * 0.99) {  // a clear gain only; ties keep the earlier shape
            best = cd.tile;
            best_t = t;
        }
    }
    ctx->auto_tile = best;
    return best;
}

// Tiles 0 (32x8, one CTA per SM), 1 (32x16) and 3 (32x12), in lbm_fused_alt.cu.
cudaError_t launch_fused_alt(lbm_ctx *ctx, int tile, bool write_macro, const LayF32 &ly);
// The rest-referenced 16-bit layouts on tiles 2, 4 and 7 (any other tile runs
// 2), one translation unit per layout (lbm_fused_f16r.cu, lbm_fused_bf16r.cu).
template <class LY>
static cudaError_t launch_r16_tile(lbm_ctx *ctx, int tile, bool write_macro, LY ly)
{
    switch (tile) {
    case 4: return launch_fused_tile<64, 8, 1>(ctx, write_macro, ly);
    case 7: return launch_fused_tile<64, 7, 1>(ctx, write_macro, ly);
    default: return launch_fused_tile<32, 8, 2>(ctx, write_macro, ly);
    }
}
cudaError_t launch_fused_f16r(lbm_ctx *ctx, int tile, bool write_macro);
cudaError_t launch_fused_bf16r(lbm_ctx *ctx, int tile, bool write_macro);

}  // namespace lbm
