// Fused time step of one lattice: one launch per step.
//
// Work items are (column, z-chunk) with the items of one chunk consecutive, so
// the CTAs of a wave march neighbouring columns through the same planes at the
// same time and the halo reads hit lines their neighbours have just brought
// into L2.  The march itself is fused_item (lbm_fused.cuh).
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
template <int TX, int TY, int MINB, bool MACRO, bool EXT, class LY, bool CAP = false>
static cudaError_t launch_fused_t(lbm_ctx *ctx, LY ly)
{
    auto kern = k_fused<TX, TY, MINB, MACRO, EXT, LY, CAP>;
    const size_t smem = Tiles<TX, TY>::smem();
    // launch configuration, resolved once per device
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
    // z-chunks per column so that one wave of resident CTAs covers the grid
    const long long ncol = (long long)((ctx->p.nx + TX - 1) / TX) * ((ctx->p.ny + TY - 1) / TY);
    const int slots = cached_slots[dev];
    const int zchunks = (int)std::max<long long>(1, std::min<long long>(slots / ncol, ctx->p.nz));
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

// Tile variants: 0 = 32x8 (one CTA per SM, no register cap), 1 = 32x16
// (128 registers), 2 = 32x8 with two CTAs per SM (128 registers), 3 = 32x12
// (168 registers), 4 = 64x8 (128 registers).
// The rest-referenced 16-bit layouts run the default tile.
cudaError_t launch_fused(lbm_ctx *ctx, bool write_macro)
{
    if (ctx->rho_cap) {  // the adjoint's replay: plain F32 steps that also store their densities
        if (ctx->p.storage != LBM_STORAGE_F32 || write_macro || ctx->n_held > 0 || ctx->mss != 0.0)
            return cudaErrorInvalidValue;
        return launch_fused_t<32, 8, 2, false, false, LayF32, true>(ctx, LayF32{ctx->f[ctx->cur], ctx->f[1 - ctx->cur],
                                                                            ctx->n});
    }
    if (ctx->tile == 5 || ctx->tile == 6) {  // the published-density march where it applies, else tile 2
        bool ran = false;
        const cudaError_t e = launch_march(ctx, write_macro, &ran);
        if (e != cudaSuccess || ran) return e;
    }
    if (ctx->p.storage == LBM_STORAGE_F16R)
        return launch_fused_tile<32, 8, 2>(ctx, write_macro, lay_r16<LayF16R>(ctx, ctx->cur, 1 - ctx->cur));
    if (ctx->p.storage == LBM_STORAGE_BF16R)
        return launch_fused_tile<32, 8, 2>(ctx, write_macro, lay_r16<LayB16R>(ctx, ctx->cur, 1 - ctx->cur));
    const LayF32 ly{ctx->f[ctx->cur], ctx->f[1 - ctx->cur], ctx->n};
    switch (ctx->tile) {
    case 1: return launch_fused_tile<32, 16, 1>(ctx, write_macro, ly);
    case 2: return launch_fused_tile<32, 8, 2>(ctx, write_macro, ly);
    case 3: return launch_fused_tile<32, 12, 1>(ctx, write_macro, ly);
    case 4: return launch_fused_tile<64, 8, 1>(ctx, write_macro, ly);

    default: return launch_fused_tile<32, 8, 1>(ctx, write_macro, ly);
    }
}

}  // namespace lbm
