// Fused time step with published densities: one launch per step, every
// population read from HBM once and written once, and every cell's density
// computed once per step.
//
// The step of Eqs. 1-4 needs, before a cell can collide, the densities of its
// 18 neighbours at the same time level (Shan-Chen force, the Eq. 4 curvature,
// the gradient of the Atwood number in Eq. 1).  Each CTA owns an x-y tile of
// TX x TY columns over a chunk of z-planes and marches along z; all CTAs of
// the grid are resident at once (cooperative launch).  Per plane a CTA
//   A  sums the arrived populations of its own cells (the zeroth moment of
//      the push-form state, see lbm_cell.cuh) and publishes the two
//      densities to a global array (L2-resident) and a progress counter;
//   F  reads the densities of the 1-cell ring around its tile, owned by the
//      neighbouring tiles, from that array once their counters show the plane
//      (a bounded wait: an error flag and an early exit on timeout);
//   C  collides its own fluid cells three planes behind A, from a compacted
//      list (solid cells occupy no lane), and pushes the new populations into
//      the neighbours' slots.
// One block barrier per plane.  Every global read whose result is not needed
// at once is issued a phase ahead: the progress counters before A, the ring
// densities and the next rest populations before C (stored to shared memory
// after it), so that neither the waits on the neighbours nor their L2 round
// trips sit in front of a barrier.
// Ring densities are therefore read, not recomputed from the ring's
// populations.  The static per-cell wall mask (bits 1..18: neighbour x + c_i
// is solid or outside; bits 24..31: the cell type) replaces the type stencil.
// All per-cell arithmetic is the one of lbm_cell.cuh in the same order as the
// other kernels, so the states are bit-identical to theirs.
#include <algorithm>

#include "lbm_cell.cuh"
#include "lbm_context.h"

namespace lbm {

// ---------------------------------------------------------------------------
// Static wall mask, once per geometry.
__global__ void k_wallmask(DevParams P, const uint8_t *__restrict__ type, uint32_t *__restrict__ mask)
{
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < P.n; c += gridDim.x * blockDim.x) {
        const int x = c % P.nx, y = (c / P.nx) % P.ny, z = c / (P.nx * P.ny);
        uint32_t m = (uint32_t)type[c] << 24;
#pragma unroll
        for (int i = 1; i < Q; ++i) {
            const int xx = axis_nb(x, cx(i), P.nx, P.per[0]);
            const int yy = axis_nb(y, cy(i), P.ny, P.per[1]);
            const int zz = axis_nb(z, cz(i), P.nz, P.per[2]);
            if (xx < 0 || yy < 0 || zz < 0 || type[xx + P.nx * (yy + P.ny * zz)] == CELL_SOLID) m |= 1u << i;
        }
        mask[c] = m;
    }
}

cudaError_t launch_wallmask(lbm_ctx *ctx)
{
    if (!ctx->wmask) return cudaSuccess;
    const int grid = (int)std::min<long long>(((long long)ctx->n + 255) / 256, 152LL * 16);
    k_wallmask<<<grid, 256, 0, ctx->stream>>>(ctx->dp, ctx->type, ctx->wmask);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
constexpr uint32_t WALL_BITS = 0x7fffeu;  // bits 1..18

template <int TX, int TY>
struct MarchTile {
    static constexpr int NT = TX * TY, DX = TX + 2, DY = TY + 2, DN = DX * DY, NW = NT / 32;
    // iteration L: A(L) reads rest planes L-1..L+1 while L+3 is stored after the barrier;
    // C(L-3) reads density planes L-4..L-2 while the ring of L-1 is stored and, in a thread
    // already in the next iteration, A(L+1) writes plane L+1
    static constexpr int RP = 5;
    static constexpr int DP = 6;
    struct Smem {
        int4 den[DP][DN];        // f_0^A, f_0^B (fixed point), drho^A, drho^B (float bits)
        int2 raw[RP][DN];        // f_0^A, f_0^B of the tile and its ring
        float at[DP][DN];        // Atwood number
        float2 lo[DP][NT];       // low parts of drho^A, drho^B of the own cells
        uint32_t msk[DP][NT];    // wall masks of the own cells
        uint16_t list[DP][NT];   // own fluid cells, compacted
        int cnt[DP];
        int wcnt[2][NW];          // fluid cells per warp, by plane parity
        int abort;
    };
    static_assert(NT % 32 == 0, "whole warps");
};

__device__ __forceinline__ int mod_pos(int p, int m) { return ((p % m) + m) % m; }
__device__ __forceinline__ int wrap_or_out(int v, int n, int per)
{
    if (v >= 0 && v < n) return v;
    if (!per) return -1;
    v %= n;
    return v < 0 ? v + n : v;
}
__device__ __forceinline__ unsigned ld_relaxed(const unsigned *p)
{
    unsigned v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void fence_acquire() { asm volatile("fence.acq_rel.gpu;" ::: "memory"); }
__device__ __forceinline__ void st_release(unsigned *p, unsigned v)
{
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
constexpr unsigned long long WAIT_NS = 1000000000ull;  // a neighbour that has not moved for 1 s: give up

// Push targets of a cell at (x, y, z): i n + index of x + c_i, with the
// periodic wrap folded into per-axis steps; bounce-back into the cell's own
// opposite slot where x + c_i is solid or outside.
struct MarchTarget {
    unsigned wall;
    int c, n;
    int xm, xp, ym, yp, zm, zp;  // index steps to the -/+ neighbour along each axis
    __device__ __forceinline__ size_t operator()(int i) const
    {
        if (wall & (1u << i)) return (size_t)opp(i) * n + c;
        int t = c;
        if (cx(i) < 0) t += xm;
        if (cx(i) > 0) t += xp;
        if (cy(i) < 0) t += ym;
        if (cy(i) > 0) t += yp;
        if (cz(i) < 0) t += zm;
        if (cz(i) > 0) t += zp;
        return (size_t)i * n + t;
    }
};

// prog[0] the error flag (a wait that gave up), prog[1] the count of finished
// CTAs (the last one resets the counters), prog[2 + item] the progress of each
// work item (planes published, counted from 1).
template <int TX, int TY, int MINB, bool MACRO>
__global__ void __launch_bounds__(TX *TY, MINB)
    k_march(DevParams P, int zchunks, LayF32 ly, const uint32_t *__restrict__ wmask, GrayRec *__restrict__ gray,
            float *__restrict__ macro, float2 *__restrict__ pub, unsigned *__restrict__ prog)
{
    using T = MarchTile<TX, TY>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    typename T::Smem &S = *reinterpret_cast<typename T::Smem *>(smem_raw);
    const int nx = P.nx, ny = P.ny, nz = P.nz, n = P.n;
    const int nxy = nx * ny;
    const int tiles_x = (nx + TX - 1) / TX, tiles_y = (ny + TY - 1) / TY, ncol = tiles_x * tiles_y;
    const int item = blockIdx.x;
    const int col = item % ncol, chunk = item / ncol;
    const int tx = col % tiles_x, ty = col / tiles_x;
    const int x0 = tx * TX, y0 = ty * TY;
    const int za = (int)((long long)nz * chunk / zchunks), zb = (int)((long long)nz * (chunk + 1) / zchunks);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int ux = tid % TX, uy = tid / TX;
    const bool own_valid = x0 + ux < nx && y0 + uy < ny;
    const int own_e = (ux + 1) + T::DX * (uy + 1);
    // den entries that are not own cells: their global column (or -1 outside)
    auto entry_col = [&](int e) -> int {
        const int dx = e % T::DX, dy = e / T::DX;
        const int gx = wrap_or_out(x0 - 1 + dx, nx, P.per[0]);
        const int gy = wrap_or_out(y0 - 1 + dy, ny, P.per[1]);
        return (gx < 0 || gy < 0) ? -1 : gx + nx * gy;
    };
    auto is_own = [&](int e) -> bool {
        const int dx = e % T::DX, dy = e / T::DX;
        return dx >= 1 && dx <= TX && dy >= 1 && dy <= TY && x0 + dx - 1 < nx && y0 + dy - 1 < ny;
    };
    // neighbour work items (same z-chunk) whose cells the ring holds: polled by
    // lanes 0-7 of the last warp, which the compacted collision fills last
    int poll_item = -1;
    const int ctl = tid - (T::NT - 32);  // lane within the last warp, negative elsewhere
    if (ctl >= 0 && ctl < 8) {
        const int k = ctl < 4 ? ctl : ctl + 1;  // the 3 x 3 block without its centre
        int ntx = tx + k % 3 - 1, nty = ty + k / 3 - 1;
        bool ok = true;
        if (ntx < 0 || ntx >= tiles_x) {
            if (P.per[0]) ntx = (ntx + tiles_x) % tiles_x;
            else ok = false;
        }
        if (nty < 0 || nty >= tiles_y) {
            if (P.per[1]) nty = (nty + tiles_y) % tiles_y;
            else ok = false;
        }
        if (ok) poll_item = 2 + chunk * ncol + nty * tiles_x + ntx;
    }
    if (tid == 0) S.abort = 0;

    // rest populations of plane p (tile + ring) into registers, then the ring
    const int e0 = tid, e1 = tid + T::NT;
    int2 rv0 = {0, 0}, rv1 = {0, 0};
    auto raw_load = [&](int p) {
        const int gz = wrap_or_out(p, nz, P.per[2]);
        rv0 = rv1 = make_int2(0, 0);
        if (gz < 0) return;
        const int c0 = entry_col(e0);
        if (c0 >= 0) {
            const int g = c0 + nxy * gz;
            rv0 = make_int2(ly.rest_in(0, g), ly.rest_in(1, g));
        }
        if (e1 < T::DN) {
            const int c1 = entry_col(e1);
            if (c1 >= 0) {
                const int g = c1 + nxy * gz;
                rv1 = make_int2(ly.rest_in(0, g), ly.rest_in(1, g));
            }
        }
    };
    auto raw_store = [&](int p) {
        int2 *dst = S.raw[mod_pos(p, T::RP)];
        dst[e0] = rv0;
        if (e1 < T::DN) dst[e1] = rv1;
    };

    // ---- A: densities of the own cells at plane L, published -----------------
    unsigned fluid_ballot = 0;
    auto dens = [&](int L) {
        const int gz = wrap_or_out(L, nz, P.per[2]);
        const int sl = mod_pos(L, T::DP);
        bool fluid = false;
        if (own_valid && gz >= 0) {
            const int c = (x0 + ux) + nx * ((y0 + uy) + ny * gz);
            const uint32_t m = wmask[c];
            const int t = (int)(m >> 24);
            fluid = t != CELL_SOLID;
            S.msk[sl][tid] = m;
            int4 dv = make_int4(0, 0, 0, 0);
            float2 lv = make_float2(0.f, 0.f);
            float av = P.at_wall;
            if (fluid) {
                const int2 *r0 = S.raw[mod_pos(L - 1, T::RP)];
                const int2 *r1 = S.raw[mod_pos(L, T::RP)];
                const int2 *r2 = S.raw[mod_pos(L + 1, T::RP)];
                const int2 f0 = r1[own_e];
                ff v[2];
#pragma unroll
                for (int a = 0; a < 2; ++a) {
                    const int f0a = a ? f0.y : f0.x;
                    float acc = 0.f;
                    long long id = 0;
#pragma unroll
                    for (int i = 1; i < Q; ++i) {
                        const int o = opp(i);  // the source x - c_i is x + c_o
                        acc += ly.mov_in(a, i, c);
                        if (!(m & (1u << o))) {
                            const int2 *rp = cz(o) < 0 ? r0 : (cz(o) > 0 ? r2 : r1);
                            const int2 s = rp[own_e + cx(o) + T::DX * cy(o)];
                            id += (long long)((a ? s.y : s.x) - f0a) * w12(i);
                        }
                    }
                    v[a] = density_dev(id, acc);
                }
                dv = make_int4(f0.x, f0.y, __float_as_int(v[0].hi), __float_as_int(v[1].hi));
                lv = make_float2(v[0].lo, v[1].lo);
                av = atwood_of(P.wet, f0.x, f0.y, v[0].hi, v[1].hi);
                __stcg(&pub[c], make_float2(v[0].hi, v[1].hi));
            } else if (MACRO) {
                for (int q = 0; q < 6; ++q) macro[(size_t)q * n + c] = 0.0f;
            }
            S.den[sl][own_e] = dv;
            S.at[sl][own_e] = av;
            S.lo[sl][tid] = lv;
        }
        fluid_ballot = __ballot_sync(0xffffffffu, fluid);
        if (lane == 0) S.wcnt[L & 1][warp] = __popc(fluid_ballot);
    };
    // compacted list of the own fluid cells of plane L (after the barrier that follows A)
    auto make_list = [&](int L) {
        const int sl = mod_pos(L, T::DP);
        int off = 0, tot = 0;
#pragma unroll
        for (int w = 0; w < T::NW; ++w) {
            const int cw = S.wcnt[L & 1][w];
            off += w < warp ? cw : 0;
            tot += cw;
        }
        if (fluid_ballot & (1u << lane))
            S.list[sl][off + __popc(fluid_ballot & ((1u << lane) - 1u))] = (uint16_t)tid;
        if (tid == 0) S.cnt[sl] = tot;
    };

    // ---- F: ring densities of plane L from the neighbours' published values ----
    // issued before the collision into registers (entries tid and tid + NT),
    // stored to shared memory after it
    float2 fv0 = {0.f, 0.f}, fv1 = {0.f, 0.f};
    bool fget0 = false, fget1 = false;
    auto fetch_issue = [&](int L) {
        fget0 = fget1 = false;
        const int gz = wrap_or_out(L, nz, P.per[2]);
        if (gz < 0) return;
        if (!is_own(e0)) {
            const int cc = entry_col(e0);
            if (cc >= 0) {  // outside a non-periodic face: a wall, never read
                fv0 = __ldcg(&pub[cc + nxy * gz]);
                fget0 = true;
            }
        }
        if (e1 < T::DN && !is_own(e1)) {
            const int cc = entry_col(e1);
            if (cc >= 0) {
                fv1 = __ldcg(&pub[cc + nxy * gz]);
                fget1 = true;
            }
        }
    };
    auto fetch_store = [&](int L) {
        const int sl = mod_pos(L, T::DP);
        const int2 *rr = S.raw[mod_pos(L, T::RP)];
        if (fget0) {
            const int2 f0 = rr[e0];
            S.den[sl][e0] = make_int4(f0.x, f0.y, __float_as_int(fv0.x), __float_as_int(fv0.y));
            S.at[sl][e0] = atwood_of(P.wet, f0.x, f0.y, fv0.x, fv0.y);
        }
        if (fget1) {
            const int2 f0 = rr[e1];
            S.den[sl][e1] = make_int4(f0.x, f0.y, __float_as_int(fv1.x), __float_as_int(fv1.y));
            S.at[sl][e1] = atwood_of(P.wet, f0.x, f0.y, fv1.x, fv1.y);
        }
    };

    // ---- C: forces, collision and push of the own fluid cells at plane z ----
    auto collide = [&](int z) {
        const int sl = mod_pos(z, T::DP);
        if (tid >= S.cnt[sl]) return;
        const int q = S.list[sl][tid];
        const int qx = q % TX, qy = q / TX;
        const int e = (qx + 1) + T::DX * (qy + 1);
        const int gz = wrap_or_out(z, nz, P.per[2]);
        const int x = x0 + qx, y = y0 + qy;
        const int c = x + nx * (y + ny * gz);
        const uint32_t m = S.msk[sl][q];
        const uint8_t t = (uint8_t)(m >> 24);
        const unsigned wall = m & WALL_BITS;
        const bool is_gray = t == CELL_GRAY;
        float4 ga = make_float4(0.f, 0.f, 0.f, 0.f), gb = ga;
        if (is_gray) {  // issued first: used only after the pull and the stencils
            ga = gray[c].a;
            gb = gray[c].b;
        }
        const int4 *d0p = S.den[mod_pos(z - 1, T::DP)];
        const int4 *d1 = S.den[sl];
        const int4 *d2 = S.den[mod_pos(z + 1, T::DP)];
        const float *a0 = S.at[mod_pos(z - 1, T::DP)];
        const float *a1 = S.at[sl];
        const float *a2 = S.at[mod_pos(z + 1, T::DP)];
        const int4 dc = d1[e];
        const float2 lo = S.lo[sl][q];
        const int f0i[2] = {dc.x, dc.y};
        const float drc[2] = {__int_as_float(dc.z), __int_as_float(dc.w)};
        CompMom M[2];
#pragma unroll
        for (int a = 0; a < 2; ++a) {
            PullSums p;
            pull_zero(p);
#pragma unroll
            for (int i = 1; i < Q; ++i) {
                const int o = opp(i);  // the source x - c_i is x + c_o
                int dfi = 0;
                if (!(wall & (1u << o))) {
                    const int4 sd = (cz(o) < 0 ? d0p : (cz(o) > 0 ? d2 : d1))[e + cx(o) + T::DX * cy(o)];
                    dfi = (a ? sd.y : sd.x) - f0i[a];
                }
                pull_add<false>(p, i, ly.mov_in(a, i, c), dfi);
            }
            M[a] = finish_moments_d(p, f0i[a], a ? ff{drc[1], lo.y} : ff{drc[0], lo.x});
        }
        const float r[2] = {M[0].rho.hi, M[1].rho.hi};
        const bool csf = P.kappa != 0.0f && (P.csf_everywhere || is_gray);
        float gf[2][3] = {{0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}}, gAt[3] = {0.f, 0.f, 0.f};
        HessSum hA, hB;
        hess_zero(hA);
        hess_zero(hB);
#pragma unroll
        for (int i = 1; i < Q; ++i) {
            const int k = e + cx(i) + T::DX * cy(i);
            const int4 nd = (cz(i) < 0 ? d0p : (cz(i) > 0 ? d2 : d1))[k];
            const bool wl = wall & (1u << i);
            const float eA = wl ? P.rho_wall[0] - r[0] : __int_as_float(nd.z) - drc[0];
            const float eB = wl ? P.rho_wall[1] - r[1] : __int_as_float(nd.w) - drc[1];
            stencil_add(i, eA, eB, gf);
            if (is_gray) atwood_add(i, wl ? P.at_wall : (cz(i) < 0 ? a0 : (cz(i) > 0 ? a2 : a1))[k], gAt);
            if (csf) {
                const float dA = wl ? eA : 3.0f * fix_diff(nd.x, f0i[0]) + eA;
                const float dB = wl ? eB : 3.0f * fix_diff(nd.y, f0i[1]) + eB;
                hess_add(hA, i, dA);
                hess_add(hB, i, dB);
            }
        }
        MarchTarget tgt;
        tgt.wall = wall;
        tgt.c = c;
        tgt.n = n;
        tgt.xm = x > 0 ? -1 : nx - 1;
        tgt.xp = x < nx - 1 ? 1 : 1 - nx;
        tgt.ym = y > 0 ? -nx : nxy - nx;
        tgt.yp = y < ny - 1 ? nx : nx - nxy;
        tgt.zm = gz > 0 ? -nxy : n - nxy;
        tgt.zp = gz < nz - 1 ? nxy : nxy - n;
        float acc[2][3];
#pragma unroll
        for (int a = 0; a < 2; ++a)
#pragma unroll
            for (int d = 0; d < 3; ++d) acc[a][d] = P.accel[a][d];
        StoreRest<LayF32> st{ly, c, {f0i[0], f0i[1]}};
        collide_store_g<MACRO>(P, acc, 0.f, t, c, n, st, M, gf, gAt, csf, hA, hB, ga, gb, gray, macro, tgt);
    };

    // ---- the march -------------------------------------------------------
    // iteration L: A(L) | barrier | F(L-1) issued, C(L-3), F(L-1) stored
    for (int p = za - 2; p <= za + 1; ++p) {
        raw_load(p);
        raw_store(p);
    }
    raw_load(za + 2);
    __syncthreads();
    for (int L = za - 1; L <= zb + 2; ++L) {
        const unsigned k = (unsigned)(L - za + 2);  // progress value of plane L
        // the neighbours' progress for plane L - 1, read ahead of A
        const bool poll = poll_item >= 0 && L - 1 >= za - 1 && L - 1 <= zb;
        unsigned seen = poll ? ld_relaxed(prog + poll_item) : 0u;
        if (L <= zb) dens(L);
        else fluid_ballot = 0;
        if (poll) {
            if (seen < k - 1) {
                const unsigned long long t0 = global_ns();
                while ((seen = ld_relaxed(prog + poll_item)) < k - 1) {
                    if (global_ns() - t0 > WAIT_NS) {
                        atomicOr(prog, 1u);
                        S.abort = 1;
                        break;
                    }
                    __nanosleep(100);
                }
            }
            fence_acquire();  // the ring reads below see what the neighbour published
        }
        __syncthreads();
        if (S.abort) break;
        if (ctl == 31 && L <= zb) st_release(prog + 2 + item, k);  // after every own store of plane L
        if (L + 3 <= zb + 1) raw_store(L + 3);
        if (L <= zb) make_list(L);
        const bool fetch = L - 1 >= za - 1 && L - 1 <= zb;
        if (fetch) fetch_issue(L - 1);
        if (L + 4 <= zb + 1) raw_load(L + 4);
        if (L - 3 >= za) collide(L - 3);
        if (fetch) fetch_store(L - 1);
    }
    __syncthreads();
    if (tid == 0) {
        __threadfence();
        const unsigned done = atomicAdd(prog + 1, 1u);
        if (done == gridDim.x - 1) {  // the last CTA: counters back to zero for the next launch
            for (unsigned k = 0; k < gridDim.x; ++k) prog[2 + k] = 0u;
            prog[1] = 0u;
            __threadfence();
        }
    }
}

// ---------------------------------------------------------------------------
template <int TX, int TY, int MINB, bool MACRO>
static cudaError_t launch_march_t(lbm_ctx *ctx, bool *ran)
{
    auto kern = k_march<TX, TY, MINB, MACRO>;
    const size_t smem = sizeof(typename MarchTile<TX, TY>::Smem);
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
    const int slots = cached_slots[dev];
    const long long ncol = (long long)((ctx->p.nx + TX - 1) / TX) * ((ctx->p.ny + TY - 1) / TY);
    if (ncol > slots) {
        *ran = false;  // every work item must be resident at once
        return cudaSuccess;
    }
    const int zchunks = (int)std::max<long long>(1, std::min<long long>(slots / ncol, ctx->p.nz));
    const int items = (int)(ncol * zchunks);
    if (items + 2 > ctx->prog_len) {
        *ran = false;
        return cudaSuccess;
    }
    LayF32 ly{ctx->f[ctx->cur], ctx->f[1 - ctx->cur], ctx->n};
    DevParams dp = ctx->dp;
    const uint32_t *wm = ctx->wmask;
    GrayRec *gray = ctx->gray;
    float *macro = ctx->macro;
    float2 *pub = ctx->pub;
    unsigned *prog = ctx->prog;
    int zc = zchunks;
    void *args[] = {&dp, &zc, &ly, &wm, &gray, &macro, &pub, &prog};
    cudaEvent_t e0;
    prof_begin(ctx, "k_march", &e0);
    cudaError_t e = cudaLaunchCooperativeKernel((const void *)kern, dim3(items), step_block(ctx, TX * TY), args,
                                                smem, ctx->stream);
    prof_end(ctx, "k_march", e0);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return e;  // nothing ran: the state stays in buffer cur
    }
    ctx->launches += 1;
    ctx->cur = 1 - ctx->cur;
    *ran = true;
    return cudaSuccess;
}

// The march runs the plain F32 step (no reservoir cells, no mass-sink-source)
// of a lattice whose columns fit in one wave of resident CTAs; *ran is false
// where it does not apply (the caller runs the rolling-window kernel).
cudaError_t launch_march(lbm_ctx *ctx, bool write_macro, bool *ran)
{
    *ran = false;
    if (ctx->p.storage != LBM_STORAGE_F32 || ctx->n_held > 0 || ctx->mss != 0.0 || !ctx->wmask || !ctx->pub ||
        ctx->view)
        return cudaSuccess;
    if (ctx->tile == 6)
        return write_macro ? launch_march_t<32, 7, 2, true>(ctx, ran) : launch_march_t<32, 7, 2, false>(ctx, ran);
    return write_macro ? launch_march_t<32, 8, 2, true>(ctx, ran) : launch_march_t<32, 8, 2, false>(ctx, ran);
}

// The error flag of the march's bounded waits (cleared by the read).
cudaError_t march_take_error(lbm_ctx *ctx, int *flag)
{
    *flag = 0;
    if (!ctx->prog) return cudaSuccess;
    unsigned v = 0;
    cudaError_t e = cudaMemcpyAsync(&v, ctx->prog, sizeof(unsigned), cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e == cudaSuccess && v) {
        *flag = 1;
        e = cudaMemsetAsync(ctx->prog, 0, sizeof(unsigned), ctx->stream);
    }
    return e;
}

}  // namespace lbm
