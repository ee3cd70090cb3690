// Fused time step for the shifted 16-bit storages (FP16 / BF16).
//
// Slot i of cell x holds f_i - w_i rho0 (push form, like F32); every moment
// and force is formed in FP32 from the converted slots, and the post-
// collision populations are shifted and rounded once on store.  The march is
// the one of the F32 kernel with a single ring: the populations are absolute
// (shifted by a constant), so a cell needs no rest population of its
// sources.
//   den ring (4 planes, tile + 1-cell halo): rho^A, rho^B, type, global index
//   and the Atwood number of the current time level.
// Per iteration with lead plane L: densities of the den region at plane L,
// one barrier, then forces + collision of the tile at plane L - 1 (own slots
// again, from L2) with the push of the new populations.
#include <algorithm>

#include "lbm_cell.cuh"
#include "lbm_context.h"

namespace lbm {

struct DenLP {
    float rA, rB, at;
    int type;
};

template <int TX, int TY>
struct TilesLP {
    static constexpr int NT = TX * TY;
    static constexpr int DX = TX + 2, DY = TY + 2, DN = DX * DY;
    static constexpr size_t smem() { return 4 * DN * (sizeof(DenLP) + sizeof(int)); }  // four-plane ring
};

__device__ __forceinline__ int wrap_lp(int v, int n, int per)
{
    if (v >= 0 && v < n) return v;
    if (!per) return -1;
    v %= n;
    return v < 0 ? v + n : v;
}
// slot of plane p in the four-plane ring (also for negative p: two's complement)
__device__ __forceinline__ int ring4_lp(int p) { return p & 3; }

template <int TX, int TY, int MINB, bool MACRO, class H>
__global__ void __launch_bounds__(TX *TY, MINB)
    k_fused_lp(DevParams P, int zchunks, const typename H::T *__restrict__ fin, typename H::T *__restrict__ fout,
               const uint8_t *__restrict__ type, GrayRec *__restrict__ gray, float *__restrict__ macro)
{
    using T = TilesLP<TX, TY>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    DenLP *den = reinterpret_cast<DenLP *>(smem_raw);        // [4][DN]
    int *dgi = reinterpret_cast<int *>(den + 4 * T::DN);     // [4][DN] global index (-1 solid)

    const int n = P.n;
    const int tid = threadIdx.x;
    // the den region's entries beyond the first pass go first to the warps of
    // the SM sub-partitions holding fewer collision warps (warp w runs on
    // partition w % 4; the identity for warp counts that are multiples of 4)
    const int tid_late = [&] {
        constexpr int NW = T::NT / 32;
        const int w = tid >> 5;
        const int load_w = (NW - (w & 3) + 3) >> 2;
        int idx = 0;
#pragma unroll
        for (int v = 0; v < NW; ++v) {
            const int load_v = (NW - (v & 3) + 3) >> 2;
            idx += (load_v < load_w || (load_v == load_w && v < w)) ? 1 : 0;
        }
        return idx * 32 + (tid & 31);
    }();
    const int tiles_x = (P.nx + TX - 1) / TX, tiles_y = (P.ny + TY - 1) / TY;
    const int ncol = tiles_x * tiles_y;

    for (int item = blockIdx.x; item < ncol * zchunks; item += gridDim.x) {
        const int col = item % ncol, chunk = item / ncol;
        const int za = (int)((long long)P.nz * chunk / zchunks);
        const int zb = (int)((long long)P.nz * (chunk + 1) / zchunks);
        if (za >= zb) continue;
        const int x0 = (col % tiles_x) * TX, y0 = (col / tiles_x) * TY;

        // densities of every den cell (tile + 1-cell halo) at plane L
        auto densities = [&](int L) {
            DenLP *dd = den + ring4_lp(L) * T::DN;
            int *dg = dgi + ring4_lp(L) * T::DN;
            const int gz = wrap_lp(L, P.nz, P.per[2]);
            for (int e = tid, pass = 1; e < T::DN; e = pass++ * T::NT + tid_late) {
                const int gx = wrap_lp(x0 - 1 + e % T::DX, P.nx, P.per[0]);
                const int gy = wrap_lp(y0 - 1 + e / T::DX, P.ny, P.per[1]);
                DenLP dc = {0.f, 0.f, P.at_wall, CELL_SOLID};
                int g = -1;
                if (gx >= 0 && gy >= 0 && gz >= 0) {
                    const int gi = gx + P.nx * (gy + P.ny * gz);
                    dc.type = type[gi];
                    if (dc.type != CELL_SOLID) {
                        g = gi;
                        if (is_held(dc.type)) {  // reservoir: the held densities
                            dc.rA = held_rho(P.held, dc.type, 0).hi;
                            dc.rB = held_rho(P.held, dc.type, 1).hi;
                        } else {
                            dc.rA = density_lp<H>(fin + g, n, P.rho0[0]);
                            dc.rB = density_lp<H>(fin + (size_t)Q * n + g, n, P.rho0[1]);
                        }
                        dc.at = atwood_rho(P.wet, dc.rA, dc.rB);
                    }
                }
                dd[e] = dc;
                dg[e] = g;
            }
        };

        // forces + collision of the tile at plane z
        auto collide = [&](int z) {
            const int ux = tid % TX, uy = tid / TX;
            if (x0 + ux >= P.nx || y0 + uy >= P.ny) return;
            const DenLP *d0p = den + ring4_lp(z - 1) * T::DN;
            const DenLP *d1 = den + ring4_lp(z) * T::DN;
            const DenLP *d2 = den + ring4_lp(z + 1) * T::DN;
            const int *g0 = dgi + ring4_lp(z - 1) * T::DN;
            const int *g1 = dgi + ring4_lp(z) * T::DN;
            const int *g2 = dgi + ring4_lp(z + 1) * T::DN;
            const int dk = (ux + 1) + T::DX * (uy + 1);
            const DenLP me = d1[dk];
            if (me.type == CELL_SOLID) {
                if (MACRO) {
                    const int gc = (x0 + ux) + P.nx * ((y0 + uy) + P.ny * z);
                    for (int q = 0; q < 6; ++q) macro[(size_t)q * n + gc] = 0.0f;
                }
                return;
            }
            const int c = g1[dk];
            unsigned wall = 0;
#pragma unroll
            for (int i = 1; i < Q; ++i) {
                const DenLP &nd = (cz(i) < 0 ? d0p : (cz(i) > 0 ? d2 : d1))[dk + cx(i) + T::DX * cy(i)];
                if (nd.type == CELL_SOLID) wall |= 1u << i;
            }
            CompMom M[2];
            const uint8_t t = (uint8_t)me.type;
            const bool held = is_held(t);
            if (held) {  // reservoir: held density at rest (reference rho/3), no force
                M[0] = held_moments(ff{me.rA, 0.f}, ff{0.f, 0.f});
                M[1] = held_moments(ff{me.rB, 0.f}, ff{0.f, 0.f});
            } else {
                M[0] = moments_lp<H>(fin + c, n, P.rho0[0]);
                M[1] = moments_lp<H>(fin + (size_t)Q * n + c, n, P.rho0[1]);
            }
            const float r[2] = {M[0].rho.hi, M[1].rho.hi};
            const bool is_gray = (t == CELL_GRAY);
            const bool csf = !held && P.kappa != 0.0f && (P.csf_everywhere || is_gray);
            float gf[2][3] = {{0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}}, gAt[3] = {0.f, 0.f, 0.f};
            HessSum hA, hB;
            hess_zero(hA);
            hess_zero(hB);
#pragma unroll
            for (int i = 1; i < Q; ++i) {
                const DenLP &nd = (cz(i) < 0 ? d0p : (cz(i) > 0 ? d2 : d1))[dk + cx(i) + T::DX * cy(i)];
                const bool wl = wall & (1u << i);
                const float eA = (wl ? P.rho_wall[0] : nd.rA) - r[0];
                const float eB = (wl ? P.rho_wall[1] : nd.rB) - r[1];
                stencil_add(i, eA, eB, gf);
                if (is_gray) atwood_add(i, nd.at, gAt);
                if (csf) {
                    hess_add(hA, i, eA);
                    hess_add(hB, i, eB);
                }
            }
            auto tgt = [&](int i) -> size_t {
                if (wall & (1u << i)) return (size_t)opp(i) * n + c;
                return (size_t)i * n + (cz(i) < 0 ? g0 : (cz(i) > 0 ? g2 : g1))[dk + cx(i) + T::DX * cy(i)];
            };
            float acc[2][3];
#pragma unroll
            for (int a = 0; a < 2; ++a)
#pragma unroll
                for (int d = 0; d < 3; ++d) {
                    acc[a][d] = held ? 0.f : P.accel[a][d];
                    if (held) gf[a][d] = 0.f;
                }
            StoreLP<H> st{fout, n, c, {r[0] * (1.0f / 3.0f), r[1] * (1.0f / 3.0f)}, {P.rho0[0], P.rho0[1]}, {0.f, 0.f}};
            collide_store<MACRO>(P, acc, held ? 0.f : P.mss, t, c, n, st, M, gf, gAt, csf, hA, hB, gray, macro, tgt);
        };

        // one barrier per plane: the densities of plane L+1 go into the slot
        // of plane L-3, which the collision of plane L-2 read before the
        // barrier of plane L
        densities(za - 1);
        for (int L = za; L <= zb; ++L) {
            densities(L);
            __syncthreads();
            if (L - 1 >= za) collide(L - 1);
        }
        __syncthreads();  // the ring is reused by the next item
    }
}

// ---------------------------------------------------------------------------
template <int TX, int TY, int MINB, bool MACRO, class H>
static cudaError_t launch_lp_t(lbm_ctx *ctx)
{
    auto kern = k_fused_lp<TX, TY, MINB, MACRO, H>;
    const size_t smem = TilesLP<TX, TY>::smem();
    static int cached_slots[64] = {};
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
    const long long ncol = (long long)((ctx->p.nx + TX - 1) / TX) * ((ctx->p.ny + TY - 1) / TY);
    const int slots = cached_slots[dev];
    const int zchunks = (int)std::max<long long>(1, std::min<long long>(slots / ncol, ctx->p.nz));
    const long long grid = std::min<long long>(ncol * zchunks, slots);
    using E = typename H::T;
    const E *fin = reinterpret_cast<const E *>(ctx->f[ctx->cur]);
    E *fout = reinterpret_cast<E *>(ctx->f[1 - ctx->cur]);
    cudaEvent_t e0;
    prof_begin(ctx, "k_fused_lp", &e0);
    kern<<<(unsigned)grid, step_block(ctx, TX * TY), smem, ctx->stream>>>(ctx->dp, zchunks, fin, fout, ctx->type,
                                                                        ctx->gray, ctx->macro);
    prof_end(ctx, "k_fused_lp", e0);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;  // nothing ran: the state stays in buffer cur
    ctx->launches += 1;
    ctx->cur = 1 - ctx->cur;
    return cudaSuccess;
}

template <class H>
static cudaError_t launch_lp_h(lbm_ctx *ctx, bool write_macro)
{
    if (fused_tile_in_use(ctx) == 7)  // the grids where 64x7 fills the SMs
        return write_macro ? launch_lp_t<64, 7, 1, true, H>(ctx) : launch_lp_t<64, 7, 1, false, H>(ctx);
    return write_macro ? launch_lp_t<32, 8, 2, true, H>(ctx) : launch_lp_t<32, 8, 2, false, H>(ctx);
}

cudaError_t launch_fused_lp(lbm_ctx *ctx, bool write_macro)
{
    return ctx->p.storage == LBM_STORAGE_BF16S ? launch_lp_h<B16>(ctx, write_macro)
                                               : launch_lp_h<H16>(ctx, write_macro);
}

}  // namespace lbm
