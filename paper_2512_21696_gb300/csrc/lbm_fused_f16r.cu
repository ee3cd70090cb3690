// The fused step on the rest-referenced F16R layout: the F32 march with
// 16-bit deviations, on the tile shapes of the automatic choice (a
// translation unit of its own, compiled in parallel with the others).
#include "lbm_fused_launch.cuh"

namespace lbm {

cudaError_t launch_fused_f16r(lbm_ctx *ctx, int tile, bool write_macro)
{
    return launch_r16_tile(ctx, tile, write_macro, lay_r16<LayF16R>(ctx, ctx->cur, 1 - ctx->cur));
}

}  // namespace lbm
