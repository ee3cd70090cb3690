// The selectable tile shapes that the automatic choice does not use: 0 (32x8,
// one CTA per SM, no register cap), 1 (32x16, 128 registers) and 3 (32x12,
// 168 registers).  A translation unit of their own, so that they compile in
// parallel with the default shapes.
#include "lbm_fused_launch.cuh"

namespace lbm {

cudaError_t launch_fused_alt(lbm_ctx *ctx, int tile, bool write_macro, const LayF32 &ly)
{
    switch (tile) {
    case 1: return launch_fused_tile<32, 16, 1>(ctx, write_macro, ly);
    case 3: return launch_fused_tile<32, 12, 1>(ctx, write_macro, ly);
    default: return launch_fused_tile<32, 8, 1>(ctx, write_macro, ly);
    }
}

}  // namespace lbm
