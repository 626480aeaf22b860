// Red-black CG iteration on colour-compact vectors (FP32, TMA-fed).
//
// CG on the red Schur complement (Eisenstat's form of red-black symmetric Gauss-Seidel) needs the
// vectors r, p, x, q only on the black unknowns.  With nx even, the cells c = 2h and 2h+1 of a row
// form pair h = c >> 1, and each pair holds exactly one odd-parity (black) cell: the compact
// vectors store that cell's value at index h (N/2 entries), followed by the few even-parity cells
// that belong to merge groups (the "exceptions", unknowns of the black set too).  A red-black
// iteration then streams half of each vector instead of all of it: about 24 B per cell for the
// iteration kernel instead of 36.
//
// Per plane m, for a tile of 32 pairs (64 cells) x 8 RPT rows:
//   p = r + beta p_old on the pairs of the tile with a two-pair / two-row halo (compact);
//   w on the even cell of each pair of the tile with a one-cell halo: the red formula
//     w = sum_f T_f p_nb for every even cell (all its neighbours are black); an exception's w must
//     be its own p instead, which the fix-row kernel of vofp_rbc.cu puts back afterwards from the
//     differences dE that the blocks form with the exceptions' own rows;
//   t = p - sum_f T_f w_nb on the black cell of each own pair, p.t, x += alpha p_old.
// Blocks march groups of neighbouring tiles in step (RbcSplit), so that the halos they share
// come from L2.
// The even cell of pair h in row j, plane m sits at x = 2h + rho with rho = (j + m) & 1, the black
// one at 2h + 1 - rho; x-neighbours of the even cell are the black cells of pairs h - 1 + rho and
// h + rho, those of the black cell the even cells of pairs h - rho and h + 1 - rho; y- and
// z-neighbours keep x and so belong to the same pair.  Coefficients stay full-grid arrays.
#pragma once
#include "vofp_tma.cuh"

namespace vofp {

struct RbcMaps {
    CUtensorMap r, p, tx, ty, tz;
};

// The exception rows (compact entries base + e, e < ne: even cells that belong to merge groups),
// handled by the iteration kernel's blocks beside their tiles: per exception the compact index of
// the black cell behind each face (enb, the own pair and coefficient 0 where there is none) and the
// face coefficient (eT), six each in the order of the red formula; r the compact residual; dE the
// difference w_red - p_e per exception.
struct RbcExc {
    const float* r;
    const int* enb;
    const float* eT;
    float* dE;
    long long base;
    int ne;
};


constexpr size_t rbc_al(size_t b) { return (b + 127) / 128 * 128; }

// Tile of RPT x 8 rows of 32 pairs; thread (tx, ty) owns pair h0 + tx in rows j0 + ty + 8 q,
// q < RPT.
template <int RPT>
struct RbcGeomT {
    static constexpr int TH = kBY * RPT;              // rows of a tile
    static constexpr int NP = kBX;                    // pairs of a tile row (64 cells)
    static constexpr int HXC = 4;                     // compact box x origin h0 - 4 (16-byte aligned)
    static constexpr int BWC = NP + 2 * HXC;          // 40 pairs: h0-4 .. h0+35
    static constexpr int HXF = 4;                     // full-grid box x origin i0 - 4
    static constexpr int BWF = 2 * NP + 2 * HXF;      // 72 cells: i0-4 .. i0+67
    static constexpr int RN = BWC * (TH + 4);         // compact r, p_old: rows j0-2 .. j0+TH+1
    static constexpr int XN = BWF * (TH + 2);         // Tx: rows j0-1 .. j0+TH
    static constexpr int YN = BWF * (TH + 3);         // Ty: rows j0-2 .. j0+TH
    static constexpr int ZN = BWF * (TH + 2);         // Tz: rows j0-1 .. j0+TH
    static constexpr size_t oR = 0;
    static constexpr size_t oP = oR + rbc_al(RN * 4);
    static constexpr size_t oX = oP + rbc_al(RN * 4);
    static constexpr size_t oY = oX + rbc_al(XN * 4);
    static constexpr size_t oZ = oY + rbc_al(YN * 4);
    static constexpr size_t kStage = oZ + rbc_al(ZN * 4);
    static constexpr uint32_t kTx = (uint32_t)((2 * RN + XN + YN + ZN) * 4);
    // p ring plane (black cells): index xr <-> pair h0 + xr - 2 (36), row yr <-> j0 + yr - 2
    static constexpr int PW = NP + 4;
    static constexpr int PN = PW * (TH + 4);
    // w ring plane (even cells): same pair index, row yw <-> j0 + yw - 1
    static constexpr int WN = PW * (TH + 2);
    static_assert(PW % 2 == 0 && BWC % 2 == 0, "p items are formed two pairs at a time");
    static constexpr int kPItems = PN / 2;            // p items per plane: two neighbouring pairs each
    static constexpr int kPPer = (kPItems + kBX * kBY - 1) / (kBX * kBY);   // per thread
    static constexpr int kRing = 2 * NP + 2 * TH;     // even cells of the w halo ring
};
using RbcGeom = RbcGeomT<1>;

template <int NS, int RPT>
constexpr size_t cg_rbc_smem() {
    using G = RbcGeomT<RPT>;
    return 128 + NS * G::kStage + 4 * G::PN * 4 + 4 * G::WN * 4 + NS * sizeof(uint64_t);
}

// A stage of step s carries compact r and p_old of plane s+2 and Tx, Ty, Tz of plane s; a step
// forms p of plane s+2, t of plane s-2 and w of plane s, each from ring planes that earlier steps
// wrote, so that one barrier per step orders it: p and w live in rings of four planes (p: s-1 .. s+2,
// w: s-3 .. s).
template <int NS, int RPT>
__global__ void __launch_bounds__(kBX* kBY, RPT == 1 ? 3 : 2)
k_rbc_tma(const __grid_constant__ RbcMaps maps, const Dims d, const RbcSplit sp, const RbcExc ex,
          const float* __restrict__ pold,
          float* __restrict__ pnew, float* __restrict__ xv, float* __restrict__ out, CgScalars* __restrict__ sc,
          double* __restrict__ pq_part) {
    using G = RbcGeomT<RPT>;
    constexpr int PW = G::PW, BWF = G::BWF, BWC = G::BWC, TH = G::TH;
    extern __shared__ __align__(128) unsigned char rbc_smem[];
    unsigned char* base = rbc_smem + ((128u - (smem_addr(rbc_smem) & 127u)) & 127u);
    float* pring = reinterpret_cast<float*>(base + NS * G::kStage);
    float* wring = pring + 4 * G::PN;
    uint64_t* bars = reinterpret_cast<uint64_t*>(wring + 4 * G::WN);
    __shared__ double sh[32];
    const int tx = threadIdx.x, ty = threadIdx.y, tid = tx + kBX * ty;
    AccF2 acc;
    if (tid == 0) {
        for (int s = 0; s < NS; ++s) mbar_init(&bars[s], 1);
        fence_mbar_init();
    }
    __syncthreads();
    uint32_t phase = 0u, pending = 0u;
    bool bad = false;
    auto stage = [&](int s) -> unsigned char* { return base + s * G::kStage; };
    // ring planes by plane index (planes >= -8)
    auto pl = [&](int kk) -> float* { return pring + ((kk + 8) & 3) * G::PN; };
    auto wl = [&](int kk) -> float* { return wring + ((kk + 8) & 3) * G::WN; };

    // p items: item it = tid + 256 q covers ring indices 2 it and 2 it + 1 of the 36 x (TH + 4)
    // plane (row 2 it / PW, pairs 2 it % PW and the next); box index of the same pairs
    // 2 it + (BWC - PW) (2 it / PW) + 2 (both even, so each item is one 8-byte word)
    int pi_src[G::kPPer];
    bool pi_on[G::kPPer];
#pragma unroll
    for (int q = 0; q < G::kPPer; ++q) {
        const int it = tid + q * kBX * kBY;
        pi_on[q] = it < G::kPItems;
        pi_src[q] = 2 * it + (BWC - PW) * ((2 * it) / PW) + 2;
    }
    // own pair xr = tx + 2 in w rows ty + 8 q + 1; ring items (threads 0 .. 2 NP + 2 TH - 1): the
    // pairs of rows j0-1 and j0+TH, then the pairs h0-1 and h0+NP of rows j0 .. j0+TH-1
    const int xo = tx + 2;
    int rx = 0, ry = 0;
    const bool has_ring = tid < G::kRing;
    if (tid < G::NP) { rx = tid + 2; ry = 0; }
    else if (tid < 2 * G::NP) { rx = tid - G::NP + 2; ry = TH + 1; }
    else if (tid < 2 * G::NP + TH) { rx = 1; ry = 1 + (tid - 2 * G::NP); }
    else if (tid < G::kRing) { rx = PW - 2; ry = 1 + (tid - 2 * G::NP - TH); }

    // everything above is block-local set-up; the scalars and vectors come from the kernels before
    grid_dep_wait();
    const float beta = (float)sc->beta, alpha = (float)sc->alpha;
    const int nh = d.nx >> 1;
    // This block's share of the exception rows: p = r + beta p_old, x += alpha p_old, the row
    // t_e = p_e - sum_f T_f p_nb and dE_e = w_red - p_e, where w_red is the red formula the tiles
    // take at the exception's cell (same operands, same order) and p_nb the black neighbours' p
    // formed here from r and p_old exactly as the tiles form them.  Run once per block, while the
    // first stages of its first segment are in flight.
    bool exc_done = false;
    auto exception_rows = [&]() {
        const int per_b = (ex.ne + (int)gridDim.x - 1) / (int)gridDim.x;
        const int e0 = (int)blockIdx.x * per_b, e1 = min(ex.ne, e0 + per_b);
        for (int e = e0 + tid; e < e1; e += kBX * kBY) {
            const long long ie = ex.base + e;
            int nb[6];
            float T[6];
#pragma unroll
            for (int f = 0; f < 6; ++f) {
                nb[f] = ex.enb[6 * e + f];
                T[f] = ex.eT[6 * e + f];
            }
            const float po_e = pold[ie];
            const float pe = fmav(beta, po_e, ex.r[ie]);
            float p[6];
#pragma unroll
            for (int f = 0; f < 6; ++f) p[f] = fmav(beta, pold[nb[f]], ex.r[nb[f]]);
            float w = 0.0f, t = pe;
#pragma unroll
            for (int f = 0; f < 6; ++f) {
                w = fmav(T[f], p[f], w);
                t = fmav(-T[f], p[f], t);
            }
            pnew[ie] = pe;
            xv[ie] = fmav(alpha, po_e, xv[ie]);
            ex.dE[e] = w - pe;
            out[ie] = t;
            acc.add(pe, t);
        }
        exc_done = true;
    };
    const int pad = sp.pad;
    // groups of gx x gy neighbouring tiles march the same planes in the same steps (their shared
    // halo sectors then come from L2); group g, member jg of the block
    const int gsz = sp.gx * sp.gy;
    const int grp = (int)blockIdx.x / gsz, jg = (int)blockIdx.x - grp * gsz;
    const int ncx = (nh + G::NP - 1) / G::NP / sp.gx;   // group columns along x
    const long long ncols = (long long)ncx * (((d.ny + TH - 1) / TH) / sp.gy);
    // work items w = column * (nz + pad) + pad + plane of the group columns: every column starts
    // with `pad` items that stand for no plane, so that an equal split of w charges each column's
    // first segment for its prologue steps (pad = 0: the plain equal split)
    const int nzp = d.nz + pad;
    const int total = (int)ncols * nzp;
    const int w0 = min(grp * sp.per, total);
    const int w1 = min(w0 + sp.per, total);
    for (int w = w0; w < w1 && !bad;) {
        const int col = w / nzp;
        const int kp0 = w - col * nzp;
        const int kp1 = min(nzp, kp0 + (w1 - w));
        w += kp1 - kp0;
        const int k0 = max(kp0 - pad, 0), k1 = kp1 - pad;
        if (k1 <= k0) continue;   // padding only (the same for every thread of the block)
        const int h0 = ((col % ncx) * sp.gx + jg % sp.gx) * G::NP, j0 = ((col / ncx) * sp.gy + jg / sp.gx) * TH;
        const int i0 = 2 * h0;
        const int h = h0 + tx;
        const long long cplane = (long long)nh * d.ny;
        bool inside[RPT];
        long long own[RPT];   // compact index within a plane
#pragma unroll
        for (int q = 0; q < RPT; ++q) {
            const int j = j0 + ty + kBY * q;
            inside[q] = h < nh && j < d.ny;
            own[q] = inside[q] ? h + (long long)nh * j : 0;
        }
        // steps s_first .. k1 + 1: p of planes k0-2 .. k1+1 (steps s_first .. k1-1), w of planes
        // k0-1 .. k1 (steps k0-1 .. k1), t of planes k0 .. k1-1 (steps k0+2 .. k1+1); stages are
        // loaded for steps s_first .. k1
        const int s_first = k0 - 4, s_last = k1;
        auto slot = [&](int s) { return (s - s_first) % NS; };
        auto issue = [&](int s) {
            const int q = slot(s);
            pending |= 1u << q;
            if (tid == 0) {
                unsigned char* b = stage(q);
                mbar_expect_tx(&bars[q], G::kTx);
                tma_load_3d(b + G::oR, &maps.r, &bars[q], h0 - G::HXC, j0 - 2, s + 2);
                tma_load_3d(b + G::oP, &maps.p, &bars[q], h0 - G::HXC, j0 - 2, s + 2);
                tma_load_3d(b + G::oX, &maps.tx, &bars[q], i0 - G::HXF, j0 - 1, s);
                tma_load_3d(b + G::oY, &maps.ty, &bars[q], i0 - G::HXF, j0 - 2, s);
                tma_load_3d(b + G::oZ, &maps.tz, &bars[q], i0 - G::HXF, j0 - 1, s);
            }
        };
        auto wait = [&](int s) -> bool {
            const int q = slot(s);
            const bool ok = mbar_wait_bounded(&bars[q], (phase >> q) & 1u);
            phase ^= 1u << q;
            pending &= ~(1u << q);
            return ok;
        };
        // w of the even cell of pair index xr in w row yw, plane m (p ring planes P0 = m, Pu = m+1,
        // Pd = m-1); tzm: the pair's Tz of plane m-1 (both cells); tzp returns the pair's Tz of plane m
        auto w_even = [&](const unsigned char* b, int m, int xr, int yw, float2 tzm, float2& tzp, const float* P0,
                          const float* Pu, const float* Pd) -> float {
            const float* X = reinterpret_cast<const float*>(b + G::oX);
            const float* Y = reinterpret_cast<const float*>(b + G::oY);
            const float* Z = reinterpret_cast<const float*>(b + G::oZ);
            const int rho = (j0 + yw - 1 + m) & 1;
            const int yr = yw + 1, e = yr * PW + xr;
            const int xb = 2 * xr + rho;                  // full-grid box index of the even cell
            tzp = *reinterpret_cast<const float2*>(Z + yw * BWF + 2 * xr);
            float u = 0.0f;
            u = fmav(X[yw * BWF + xb], P0[e + rho], u);
            u = fmav(X[yw * BWF + xb - 1], P0[e - 1 + rho], u);
            u = fmav(Y[yr * BWF + xb], P0[e + PW], u);
            u = fmav(Y[(yr - 1) * BWF + xb], P0[e - PW], u);
            u = fmav(rho ? tzp.y : tzp.x, Pu[e], u);
            u = fmav(rho ? tzm.y : tzm.x, Pd[e], u);
            return u;
        };

        // coefficients of the own black cell kept from plane m's w step to its t step
        struct Co {
            float tx, txl, ty, tyd, tz, tzm, p;
        };
        Co sa[RPT], sb[RPT];
        float2 own_tzm[RPT];
        float xa[RPT], pa[RPT], xn[RPT], pn2[RPT];
#pragma unroll
        for (int q = 0; q < RPT; ++q) {
            sa[q] = Co{};
            sb[q] = Co{};
            own_tzm[q] = make_float2(0.f, 0.f);
            xa[q] = pa[q] = xn[q] = pn2[q] = 0.f;
        }
        float2 ring_tzm = make_float2(0.f, 0.f);

        __syncthreads();
        if (tid == 0) fence_proxy_async_smem();
        for (int s = s_first; s <= min(s_first + NS - 1, s_last); ++s) issue(s);
        if (!exc_done) exception_rows();
        for (int s = s_first; s <= k1 + 1; ++s) {
            // the slot of step s-1 is free (every thread passed the barrier that closed it)
            if (s - 1 >= s_first && s - 1 + NS <= s_last) {
                if (tid == 0) fence_proxy_async_smem();
                issue(s - 1 + NS);
            }
            // x and p_old of the own black cells of plane s-1, for its t step (the next one)
#pragma unroll
            for (int q = 0; q < RPT; ++q) {
                xn[q] = 0.f;
                pn2[q] = 0.f;
                if (s - 1 >= k0 && s - 1 < k1 && inside[q]) {
                    const long long c = (long long)(s - 1) * cplane + own[q];
                    xn[q] = xv[c];
                    pn2[q] = pold[c];
                }
            }
            bool ok = true;
            if (s <= s_last) ok = wait(s);
            const unsigned char* b = stage(slot(s));
            // A: p of plane s+2
            if (s + 2 <= k1 + 1 && ok) {
                const float* R = reinterpret_cast<const float*>(b + G::oR);
                const float* P = reinterpret_cast<const float*>(b + G::oP);
                float* op = pl(s + 2);
#pragma unroll
                for (int q = 0; q < G::kPPer; ++q)
                    if (pi_on[q]) {
                        const float2 pv = *reinterpret_cast<const float2*>(P + pi_src[q]);
                        const float2 rv = *reinterpret_cast<const float2*>(R + pi_src[q]);
                        *reinterpret_cast<float2*>(op + 2 * (tid + q * kBX * kBY)) =
                            make_float2(fmav(beta, pv.x, rv.x), fmav(beta, pv.y, rv.y));
                    }
            }
            // B: t of plane s-2 on the black cell of each own pair (w of planes s-3, s-2, s-1); the
            // rows' sums are formed together (every ring read is in bounds) and only the stores
            // and the dot product wait on whether the cell is inside the grid
            const int m = s - 2;
            if (m >= k0 && m < k1) {
                const float* W0 = wl(m);
                const float* Wu = wl(m + 1);
                const float* Wd = wl(m - 1);
                float t[RPT];
#pragma unroll
                for (int q = 0; q < RPT; ++q) {
                    const int rho = (j0 + ty + kBY * q + m) & 1;
                    const int e = (ty + kBY * q + 1) * PW + xo;
                    float u = sa[q].p;
                    u = fmav(-sa[q].tx, W0[e + 1 - rho], u);
                    u = fmav(-sa[q].txl, W0[e - rho], u);
                    u = fmav(-sa[q].ty, W0[e + PW], u);
                    u = fmav(-sa[q].tyd, W0[e - PW], u);
                    u = fmav(-sa[q].tz, Wu[e], u);
                    u = fmav(-sa[q].tzm, Wd[e], u);
                    t[q] = u;
                }
#pragma unroll
                for (int q = 0; q < RPT; ++q) {
                    if (inside[q]) {
                        const long long c = (long long)m * cplane + own[q];
                        out[c] = t[q];
                        pnew[c] = sa[q].p;
                        xv[c] = fmav(alpha, pa[q], xa[q]);
                        acc.add(sa[q].p, t[q]);
                    }
                }
            }
#pragma unroll
            for (int q = 0; q < RPT; ++q) {
                xa[q] = xn[q];
                pa[q] = pn2[q];
            }
            // C: w of plane s (even cells of the own pairs and the ring; p of planes s-1, s, s+1);
            // at plane k0-2 only the pairs' Tz is carried
            if (ok && s >= k0 - 2 && s <= k1) {
                const int mw = s;
                const float* Z = reinterpret_cast<const float*>(b + G::oZ);
                if (mw >= k0 - 1) {
                    const float* X = reinterpret_cast<const float*>(b + G::oX);
                    const float* Y = reinterpret_cast<const float*>(b + G::oY);
                    const float* P0 = pl(mw);
                    const float* Pu = pl(mw + 1);
                    const float* Pd = pl(mw - 1);
                    float* Wo = wl(mw);
                    // the own pair (cells 2 xo, 2 xo + 1 of box row yo): its even cell's w (the
                    // terms of w_even, same order) and its black cell's coefficients and p for the
                    // t step two steps later, from the coefficients of both cells read as 8-byte
                    // words. The even cell's side rho is the same for the RPT rows of a thread
                    // (kBY rows apart) and for the 32 threads of a warp (one row): a branch per
                    // warp instead of a select per operand
                    auto own_row = [&](auto rho_c, int q) {
                        constexpr int RHO = decltype(rho_c)::value;
                        const int yo = ty + kBY * q + 1;
                        const float xl = X[yo * BWF + 2 * xo - 1];
                        const float2 x2 = *reinterpret_cast<const float2*>(X + yo * BWF + 2 * xo);
                        const float2 ya = *reinterpret_cast<const float2*>(Y + yo * BWF + 2 * xo);
                        const float2 yb = *reinterpret_cast<const float2*>(Y + (yo + 1) * BWF + 2 * xo);
                        const float2 tzp = *reinterpret_cast<const float2*>(Z + yo * BWF + 2 * xo);
                        const float2 tzm = own_tzm[q];
                        const int e = (yo + 1) * PW + xo;
                        const float pc = P0[e];
                        float u = 0.0f;
                        Co co;
                        if constexpr (RHO == 1) {
                            u = fmav(x2.y, P0[e + 1], u);
                            u = fmav(x2.x, pc, u);
                            u = fmav(yb.y, P0[e + PW], u);
                            u = fmav(ya.y, P0[e - PW], u);
                            u = fmav(tzp.y, Pu[e], u);
                            u = fmav(tzm.y, Pd[e], u);
                            co = Co{x2.x, xl, yb.x, ya.x, tzp.x, tzm.x, pc};
                        } else {
                            u = fmav(x2.x, pc, u);
                            u = fmav(xl, P0[e - 1], u);
                            u = fmav(yb.x, P0[e + PW], u);
                            u = fmav(ya.x, P0[e - PW], u);
                            u = fmav(tzp.x, Pu[e], u);
                            u = fmav(tzm.x, Pd[e], u);
                            co = Co{x2.y, x2.x, yb.y, ya.y, tzp.y, tzm.y, pc};
                        }
                        Wo[yo * PW + xo] = u;
                        own_tzm[q] = tzp;
                        sa[q] = sb[q];
                        sb[q] = co;
                    };
                    static_assert(kBY % 2 == 0, "the rows of a thread share their parity");
                    if ((j0 + ty + mw) & 1) {
#pragma unroll
                        for (int q = 0; q < RPT; ++q) own_row(std::integral_constant<int, 1>{}, q);
                    } else {
#pragma unroll
                        for (int q = 0; q < RPT; ++q) own_row(std::integral_constant<int, 0>{}, q);
                    }
                    if (has_ring) {
                        float2 tzr;
                        Wo[ry * PW + rx] = w_even(b, mw, rx, ry, ring_tzm, tzr, P0, Pu, Pd);
                        ring_tzm = tzr;
                    }
                } else {
#pragma unroll
                    for (int q = 0; q < RPT; ++q)
                        own_tzm[q] = *reinterpret_cast<const float2*>(Z + (ty + kBY * q + 1) * BWF + 2 * xo);
                    if (has_ring) ring_tzm = *reinterpret_cast<const float2*>(Z + ry * BWF + 2 * rx);
                }
            } else {
#pragma unroll
                for (int q = 0; q < RPT; ++q) sa[q] = sb[q];
            }
            if (__syncthreads_or(!ok)) {
                bad = true;
                break;
            }
        }
    }
    if (bad) {
        for (int s = 0; s < NS; ++s)
            if (pending & (1u << s)) mbar_wait_bounded(&bars[s], (phase >> s) & 1u);
        if (tid == 0) atomicCAS(&sc->status, (int)VOFP_OK, (int)VOFP_ERR_DEVICE_TIMEOUT);
    }
    if (!exc_done) exception_rows();   // blocks without planes (or that stopped early)
    // this block's p.t (fixed order); the update kernel sums the blocks' partials
    const double v = warp_sum(acc.value());
    if ((tid & 31) == 0) sh[tid >> 5] = v;
    __syncthreads();
    if (tid == 0) {
        double b = 0.0;
        for (int w = 0; w < (kBX * kBY) / 32; ++w) b += sh[w];
        pq_part[blockIdx.x] = b;
    }
}

}  // namespace vofp
