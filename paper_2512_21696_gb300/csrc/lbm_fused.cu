// Fused time step of one lattice: one launch per step (the kernel and its
// launch are in lbm_fused_launch.cuh).
#include "lbm_fused_launch.cuh"

namespace lbm {

// The automatic choice (tile 8) among 2 (32x8, two CTAs per SM), 4 (64x8)
// and 7 (64x7): the grid of each is one wave of z-chunked columns, and its
// step lasts about (planes per chunk + the 2 halo planes) x the time a
// resident CTA takes per plane, times the waves.  Per-plane times of the
// three shapes on a GB300 (F32, 2070 MHz), fitted to the 128^3 drainage and
// 192^3 fibre-bundle steps (32x8: 12.26 and 12.59 us measured; 64x8: 12.24 and
// 12.19; 64x7: 11.8 and 11.7): 12.45, 12.2 and 11.8 us.  64x7 wins where its
// extra columns fill the SMs (128^3: 152 items on 152 slots, against 128 of
// 152 for 64x8 and 256 of 304 for 32x8), 64x8 where both fill them (192^3);
// lattices whose width is not a multiple of 64 keep 32x8.
static int auto_tile(lbm_ctx *ctx)
{
    if (ctx->auto_tile >= 0) return ctx->auto_tile;
    struct Cand {
        int tile, tx, ty;
        double t_plane;
        int slots;
    } cand[3] = {{2, 32, 8, 12.45, 0}, {4, 64, 8, 12.2, 0}, {7, 64, 7, 11.8, 0}};
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

// Tile variants: 0 = 32x8 (one CTA per SM, no register cap), 1 = 32x16
// (128 registers), 2 = 32x8 with two CTAs per SM (128 registers), 3 = 32x12
// (168 registers), 4 = 64x8 (128 registers), 7 = 64x7 (one CTA per SM),
// 8 = the automatic choice above (the default).
// The rest-referenced 16-bit layouts run tiles 2, 4 and 7 (others run 2).
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
    if (tile == 8) tile = auto_tile(ctx);
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
