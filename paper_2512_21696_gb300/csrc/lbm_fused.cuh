// Rolling-window march of the fused time step (shared by the one-lattice
// kernel and the batched kernel): populations cross HBM once each way.
//
// Each CTA owns an x-y tile of TX x TY columns and marches along z over a
// chunk of planes.  Two shared-memory rings follow the march:
//   raw  (4 planes, tile + 2-cell halo): cell type and fixed-point rest
//        populations, the reference of every arrived population;
//   den  (4 planes, tile + 1-cell halo): rest populations, drho, type and
//        global index of the current time level, the source of the density
//        stencils (gradients, Atwood number, Eq. 4 Hessian) and of the push
//        targets.
// With lead plane L the pipeline per iteration is
//   phase A  raw plane L+2 from HBM, and drho of the den region at plane L
//            (own slots from HBM/L2, source rest populations from the raw
//            ring)
//   barrier
//   phase B  forces + collision of the tile at plane L-1 (own slots again,
//            from L2), push of the new populations into the neighbours' slots.
// The rings hold four planes, so one barrier per plane suffices: a warp may
// still be in phase B of plane L-1 while others run phase A of plane L+1,
// and every slot phase A writes was last read before the previous barrier.
// All per-cell arithmetic is shared with the two-launch path
// (lbm_cell.cuh), so both give identical states.
#pragma once

#include "lbm_cell.cuh"

namespace lbm {

struct RawCell {
    int f0A, f0B, type, pad;
};
struct DenCell {
    int f0A, f0B;
    float drA, drB;  // rho - 3 f_0 (hi) ...
    float loA, loB;  // ... and its low part (float-float)
};
struct DenMeta {
    int type, gidx;
};

template <int TX, int TY>
struct Tiles {
    static constexpr int NT = TX * TY;
    static constexpr int RX = TX + 4, RY = TY + 4, RN = RX * RY;
    static constexpr int DX = TX + 2, DY = TY + 2, DN = DX * DY;
    static constexpr int NP = 4;  // planes per ring
    static constexpr size_t smem()
    {
        return NP * RN * sizeof(RawCell) + NP * DN * (sizeof(DenCell) + sizeof(DenMeta) + sizeof(float));
    }
};

__device__ __forceinline__ int wrap_coord(int v, int n, int per)
{
    if (v >= 0 && v < n) return v;
    if (!per) return -1;
    v %= n;
    return v < 0 ? v + n : v;
}
// slot of plane p in a four-plane ring (also for negative p: two's complement)
__device__ __forceinline__ int ring4(int p) { return p & 3; }

// One work item: the TX x TY columns at (x0, y0) over planes [za, zb) of the
// lattice of shape G (G.n is the slot stride of ly, type, gray and macro),
// physics P.  EXT compiles in the reservoir (inlet / outlet) cells and the
// mass-sink-source term; without it neither is expected.  Ends with a block
// barrier, so the rings can be reused at once.
// CAP: the densities of the tile's own cells (rho - 3 f_0 of both
// components and the Atwood number, the values the two-launch path's density
// pass writes) are also stored into cap[3][n], for the adjoint's replay.
template <int TX, int TY, bool MACRO, bool EXT, class LY, bool CAP = false>
__device__ __forceinline__ void fused_item(const DevParams &P, const Geo &G, const LY &ly,
                                           const uint8_t *__restrict__ type,
                                           GrayRec *__restrict__ gray, float *__restrict__ macro, int x0, int y0,
                                           int za, int zb, unsigned char *smem_raw, float *__restrict__ cap = nullptr)
{
    using T = Tiles<TX, TY>;
    constexpr int NP = T::NP;
    RawCell *raw = reinterpret_cast<RawCell *>(smem_raw);          // [NP][RN]
    DenCell *den = reinterpret_cast<DenCell *>(raw + NP * T::RN);  // [NP][DN]
    DenMeta *dmeta = reinterpret_cast<DenMeta *>(den + NP * T::DN); // [NP][DN]
    float *dat = reinterpret_cast<float *>(dmeta + NP * T::DN);     // [NP][DN] Atwood number
    const int n = G.n;
    const int tid = threadIdx.x;
    // The den region has more entries than the tile has threads; the entries
    // beyond the first pass go first to the warps of the SM sub-partitions
    // that hold fewer of the collision's warps (warp w runs on partition
    // w % 4): with 14 warps the collision puts 4, 4, 3 and 3 warps on the four
    // partitions, so the extra density work lands on the last two.  With a
    // warp count that is a multiple of 4 the order is the identity.
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

    // ---- phase A, first part: raw plane q (tile + 2-cell halo) ----
    auto raw_entry = [&](int q, int e) -> RawCell {
        const int gz = wrap_coord(q, G.nz, P.per[2]);
        const int rx = e % T::RX, ry = e / T::RX;
        const int gx = wrap_coord(x0 - 2 + rx, G.nx, P.per[0]);
        const int gy = wrap_coord(y0 - 2 + ry, G.ny, P.per[1]);
        RawCell rc = {0, 0, CELL_SOLID, 0};
        if (gx >= 0 && gy >= 0 && gz >= 0) {
            // the three loads are independent (one memory round trip, not
            // two); a solid cell's rest slot is never read as a population
            const int g = gx + G.nx * (gy + G.ny * gz);
            rc.type = type[g];
            const int fA = ly.rest_in(0, g), fB = ly.rest_in(1, g);
            const bool solid = rc.type == CELL_SOLID;
            rc.f0A = solid ? 0 : fA;
            rc.f0B = solid ? 0 : fB;
        }
        return rc;
    };
    auto load_raw = [&](int q) {
        RawCell *dst = raw + ring4(q) * T::RN;
        for (int e = tid; e < T::RN; e += T::NT) dst[e] = raw_entry(q, e);
    };

    // ---- phase A: drho of the den region (tile + 1-cell halo) at plane L ----
    auto densities = [&](int L) {
        const RawCell *r0 = raw + ring4(L - 1) * T::RN;
        const RawCell *r1 = raw + ring4(L) * T::RN;
        const RawCell *r2 = raw + ring4(L + 1) * T::RN;
        DenCell *dd = den + ring4(L) * T::DN;
        DenMeta *dm = dmeta + ring4(L) * T::DN;
        float *da = dat + ring4(L) * T::DN;
        const int gz = wrap_coord(L, G.nz, P.per[2]);
        for (int e = tid, pass = 1; e < T::DN; e = pass++ * T::NT + tid_late) {
            const int dx = e % T::DX, dy = e / T::DX;
            const RawCell me = r1[(dx + 1) + T::RX * (dy + 1)];
            DenCell dc = {me.f0A, me.f0B, 0.f, 0.f, 0.f, 0.f};
            int g = -1;
            if (me.type != CELL_SOLID) {
                g = wrap_coord(x0 - 1 + dx, G.nx, P.per[0]) +
                    G.nx * (wrap_coord(y0 - 1 + dy, G.ny, P.per[1]) + G.ny * gz);
                const bool held = EXT && is_held(me.type);
#pragma unroll
                for (int a = 0; a < 2; ++a) {
                    const int f0 = a ? me.f0B : me.f0A;
                    float acc = 0.f;
                    long long id = 0;
#pragma unroll
                    for (int i = 1; i < Q; ++i) {
                        const int o = opp(i);  // the source x - c_i is x + c_o
                        const RawCell *rp = cz(o) < 0 ? r0 : (cz(o) > 0 ? r2 : r1);
                        const RawCell &src = rp[(dx + 1 + cx(o)) + T::RX * (dy + 1 + cy(o))];
                        acc += ly.mov_in(a, i, g);
                        if (src.type != CELL_SOLID) id += (long long)((a ? src.f0B : src.f0A) - f0) * w12(i);
                    }
                    ff v = density_dev(id, acc);
                    if (held) v = held_dev(held_rho(G.held, me.type, a), f0);  // a reservoir's density is the held one
                    if (a) {
                        dc.drB = v.hi;
                        dc.loB = v.lo;
                    } else {
                        dc.drA = v.hi;
                        dc.loA = v.lo;
                    }
                }
            }
            dd[e] = dc;
            dm[e] = {me.type, g};
            da[e] = me.type != CELL_SOLID ? atwood_of(P.wet, dc.f0A, dc.f0B, dc.drA, dc.drB) : P.at_wall;
            if (CAP && g >= 0 && L >= za && L < zb && dx >= 1 && dx <= TX && dy >= 1 && dy <= TY &&
                x0 - 1 + dx < G.nx && y0 - 1 + dy < G.ny) {
                cap[g] = dc.drA;
                cap[(size_t)n + g] = dc.drB;
                cap[(size_t)2 * n + g] = da[e];
            }
        }
    };

    // ---- phase B: forces + collision of the tile at plane z ----
    auto collide = [&](int z) {
        const int ux = tid % TX, uy = tid / TX;
        if (x0 + ux >= G.nx || y0 + uy >= G.ny) return;
        const DenCell *d0p = den + ring4(z - 1) * T::DN;
        const DenCell *d1 = den + ring4(z) * T::DN;
        const DenCell *d2 = den + ring4(z + 1) * T::DN;
        const DenMeta *m0 = dmeta + ring4(z - 1) * T::DN;
        const DenMeta *m1 = dmeta + ring4(z) * T::DN;
        const DenMeta *m2 = dmeta + ring4(z + 1) * T::DN;
        const float *a0 = dat + ring4(z - 1) * T::DN;
        const float *a1 = dat + ring4(z) * T::DN;
        const float *a2 = dat + ring4(z + 1) * T::DN;
        const int dk = (ux + 1) + T::DX * (uy + 1);
        const DenMeta me = m1[dk];
        if (me.type == CELL_SOLID) {
            if (MACRO) {
                const int gc = (x0 + ux) + G.nx * ((y0 + uy) + G.ny * z);
                for (int q = 0; q < 6; ++q) macro[(size_t)q * n + gc] = 0.0f;
            }
            return;
        }
        const int c = me.gidx;
        const DenCell dc = d1[dk];
        unsigned wall = 0;
#pragma unroll
        for (int i = 1; i < Q; ++i) {
            const DenMeta &nm = (cz(i) < 0 ? m0 : (cz(i) > 0 ? m2 : m1))[dk + cx(i) + T::DX * cy(i)];
            if (nm.type == CELL_SOLID) wall |= 1u << i;
        }
        const int f0i[2] = {dc.f0A, dc.f0B};
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
                    const DenCell &sd = (cz(o) < 0 ? d0p : (cz(o) > 0 ? d2 : d1))[dk + cx(o) + T::DX * cy(o)];
                    dfi = (a ? sd.f0B : sd.f0A) - f0i[a];
                }
                pull_add<false>(p, i, ly.mov_in(a, i, c), dfi);
            }
            M[a] = finish_moments_d(p, f0i[a], a ? ff{dc.drB, dc.loB} : ff{dc.drA, dc.loA});
        }
        const uint8_t t = (uint8_t)me.type;
        const bool held = EXT && is_held(t);
        if (held) {  // reservoir: held density at rest, no force
            M[0] = held_moments(held_rho(G.held, t, 0), ff{dc.drA, dc.loA});
            M[1] = held_moments(held_rho(G.held, t, 1), ff{dc.drB, dc.loB});
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
            const DenCell &nd = (cz(i) < 0 ? d0p : (cz(i) > 0 ? d2 : d1))[dk + cx(i) + T::DX * cy(i)];
            const bool wl = wall & (1u << i);
            const float eA = wl ? P.rho_wall[0] - r[0] : nd.drA - dc.drA;
            const float eB = wl ? P.rho_wall[1] - r[1] : nd.drB - dc.drB;
            stencil_add(i, eA, eB, gf);
            if (is_gray) atwood_add(i, (cz(i) < 0 ? a0 : (cz(i) > 0 ? a2 : a1))[dk + cx(i) + T::DX * cy(i)], gAt);
            if (csf) {
                const float dA = wl ? eA : 3.0f * fix_diff(nd.f0A, f0i[0]) + eA;
                const float dB = wl ? eB : 3.0f * fix_diff(nd.f0B, f0i[1]) + eB;
                hess_add(hA, i, dA);
                hess_add(hB, i, dB);
            }
        }
        auto tgt = [&](int i) -> size_t {
            if (wall & (1u << i)) return (size_t)opp(i) * n + c;
            const DenMeta &tm = (cz(i) < 0 ? m0 : (cz(i) > 0 ? m2 : m1))[dk + cx(i) + T::DX * cy(i)];
            return (size_t)i * n + tm.gidx;
        };
        float acc[2][3];
#pragma unroll
        for (int a = 0; a < 2; ++a)
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                acc[a][d] = held ? 0.f : G.accel[a][d];
                if (held) gf[a][d] = 0.f;
            }
        StoreRest<LY> st{ly, c, {f0i[0], f0i[1]}};
        collide_store<MACRO>(P, acc, (EXT && !held) ? G.mss : 0.f, t, c, n, st, M, gf, gAt, csf, hA, hB, gray, macro,
                             tgt);
    };

    load_raw(za - 2);
    load_raw(za - 1);
    load_raw(za);
    __syncthreads();
    for (int L = za - 1; L <= zb; ++L) {
        if (L + 2 <= zb + 1) load_raw(L + 2);
        densities(L);
        __syncthreads();
        if (L - 1 >= za) collide(L - 1);
    }
    __syncthreads();
}

}  // namespace lbm
