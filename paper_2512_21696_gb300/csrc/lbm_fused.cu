// Fused time step of one lattice: one launch per step (the kernel and its
// launch are in lbm_fused_launch.cuh).
#include "lbm_fused_launch.cuh"

namespace lbm {

// Tile variants: 0 = 32x8 (one CTA per SM, no register cap), 1 = 32x16
// (128 registers), 2 = 32x8 with two CTAs per SM (128 registers), 3 = 32x12
// (168 registers), 4 = 64x8 (128 registers), 7 = 64x7 (one CTA per SM),
// 8 = the automatic choice above (the default).
// The rest-referenced 16-bit layouts run tiles 2, 4 and 7 (others run 2).
int fused_tile_in_use(lbm_ctx *ctx)
{
    int tile = ctx->tile;
    if (tile == 8) tile = auto_tile<>(ctx);
    if (ctx->p.storage == LBM_STORAGE_F16S || ctx->p.storage == LBM_STORAGE_BF16S) return tile == 7 ? 7 : 2;
    if ((ctx->p.storage == LBM_STORAGE_F16R || ctx->p.storage == LBM_STORAGE_BF16R) && tile != 4 && tile != 7)
        return 2;
    return tile;
}

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
    int tile = ctx->tile;
    if (tile == 8) tile = auto_tile<>(ctx);
    else if (tile == 5 || tile == 6) tile = 2;  // where the march does not apply
    if (ctx->p.storage == LBM_STORAGE_F16R) return launch_fused_f16r(ctx, tile, write_macro);
    if (ctx->p.storage == LBM_STORAGE_BF16R) return launch_fused_bf16r(ctx, tile, write_macro);
    const LayF32 ly{ctx->f[ctx->cur], ctx->f[1 - ctx->cur], ctx->n};
    switch (tile) {
    case 2: return launch_fused_tile<32, 8, 2>(ctx, write_macro, ly);
    case 4: return launch_fused_tile<64, 8, 1>(ctx, write_macro, ly);
    case 7: return launch_fused_tile<64, 7, 1>(ctx, write_macro, ly);
    default: return launch_fused_alt(ctx, tile, write_macro, ly);
    }
}

}  // namespace lbm
