// Fused red-black CG iteration (Eisenstat's form of red-black symmetric Gauss-Seidel: CG on the
// red Schur complement) with TMA-fed planes, FP32, 64 x 8 tiles, two cells per thread.
//
// Per plane m the iteration needs
//   p = r + beta p_old                      on the tile with a two-cell halo,
//   w = sum_f T_f p_nb on red cells, w = p elsewhere   on the tile with a one-cell halo,
//   t = w - sum_f T_f w_nb on the non-red rows (the Schur operator), p.t, x += alpha p_old.
// A step s forms p of plane s+2, w of plane s+1 and t of plane s-1, so a stage of the copy ring
// carries r and p_old of plane s+2 with the coefficients of plane s+1 and lives for one step; the
// coefficients the t of a plane needs stay in the registers of the thread that read them for its
// w.  Two cells per thread: every pair (i even, i+1) holds one cell of each parity, so red and
// black work is the same for every lane.  The red flag is the sign bit of the Tz copy (Tzr).
#pragma once
#include "vofp_tma.cuh"

namespace vofp {

struct RbMaps {
    CUtensorMap r, p, tx, ty, tz;
};

constexpr size_t rb_al(size_t b) { return (b + 127) / 128 * 128; }

template <int TH>
struct RbGeom {
    static constexpr int TW = 2 * kBX;                // 64 cells of a tile row; TH rows
    static constexpr int NT = kBX * TH;               // threads of a block
    static constexpr int HX = 4;                      // box x origin i0 - 4 (16-byte aligned)
    static constexpr int BW = TW + 2 * HX;            // 72: every box spans x = i0-4 .. i0+67
    static constexpr int RN = BW * (TH + 4);          // r, p_old: rows j0-2 .. j0+TH+1
    static constexpr int XN = BW * (TH + 2);          // Tx: rows j0-1 .. j0+TH
    static constexpr int YN = BW * (TH + 3);          // Ty: rows j0-2 .. j0+TH
    static constexpr int ZN = BW * (TH + 2);          // Tz (signed): rows j0-1 .. j0+TH
    static constexpr size_t oR = 0;
    static constexpr size_t oP = oR + rb_al(RN * 4);
    static constexpr size_t oX = oP + rb_al(RN * 4);
    static constexpr size_t oY = oX + rb_al(XN * 4);
    static constexpr size_t oZ = oY + rb_al(YN * 4);
    static constexpr size_t kStage = oZ + rb_al(ZN * 4);
    static constexpr uint32_t kTx = (uint32_t)((2 * RN + XN + YN + ZN) * 4);
    // p ring plane: x index xr <-> cell i0 + xr - 2, row yr <-> j0 + yr - 2 (68 x (TH+4))
    static constexpr int PW = TW + 4;
    static constexpr int PN = PW * (TH + 4);
    // w ring plane: same x index, row yw <-> j0 + yw - 1 (68 x (TH+2))
    static constexpr int WN = PW * (TH + 2);
    static constexpr int kPItems = (PW / 2) * (TH + 4);   // p pairs formed per plane
    static constexpr int kPPer = (kPItems + NT - 1) / NT; // p pairs per thread
};

template <int NS, int TH>
constexpr size_t cg_rb_tma_smem() {
    using G = RbGeom<TH>;
    return 128 + NS * G::kStage + 3 * G::PN * 4 + 3 * G::WN * 4 + NS * sizeof(uint64_t);
}

// coefficients of a thread's own pair kept from its w to its t (plane m): Tx of both cells and of
// the cell left of the pair, Ty of both cells and of the cells below, signed Tz (red flags) of
// plane m and |Tz| of plane m-1
struct RbCo {
    float2 tx, ty, tyd, tz, tzm;
    float txl;
};

template <int NS, int TH>
__global__ void __launch_bounds__(kBX* TH, TH == 8 ? 3 : 6)
k_cg_rb_tma(const __grid_constant__ RbMaps maps, const Dims d, const int per_block, const float* __restrict__ pold,
            float* __restrict__ pnew, float* __restrict__ xv, float* __restrict__ out, CgScalars* __restrict__ sc,
            double* __restrict__ partials, unsigned int* __restrict__ counter) {
    using G = RbGeom<TH>;
    constexpr int PW = G::PW, BW = G::BW, NT = G::NT, PP = G::kPPer;
    extern __shared__ __align__(128) unsigned char rb_smem[];
    unsigned char* base = rb_smem + ((128u - (smem_addr(rb_smem) & 127u)) & 127u);
    float* pring = reinterpret_cast<float*>(base + NS * G::kStage);
    float* wring = pring + 3 * G::PN;
    uint64_t* bars = reinterpret_cast<uint64_t*>(wring + 3 * G::WN);
    __shared__ double sh[32];
    const int tx = threadIdx.x, ty = threadIdx.y, tid = tx + kBX * ty;
    const float beta = (float)sc->beta, alpha = (float)sc->alpha;
    AccF2 acc;
    if (tid == 0) {
        for (int s = 0; s < NS; ++s) mbar_init(&bars[s], 1);
        fence_mbar_init();
    }
    __syncthreads();
    uint32_t phase = 0u, pending = 0u;
    bool bad = false;
    auto stage = [&](int s) -> unsigned char* { return base + s * G::kStage; };
    auto pl = [&](int kk) -> float* { return pring + ((kk + 6) % 3) * G::PN; };
    auto wl = [&](int kk) -> float* { return wring + ((kk + 6) % 3) * G::WN; };

    // this thread's p items (pairs of the 68 x 12 plane)
    int pi_dst[PP], pi_src[PP];
    bool pi_on[PP];
#pragma unroll
    for (int q = 0; q < PP; ++q) {
        const int it = tid + q * NT;
        pi_on[q] = it < G::kPItems;
        const int xr = pi_on[q] ? 2 * (it % (PW / 2)) : 0, yr = pi_on[q] ? it / (PW / 2) : 0;
        pi_dst[q] = yr * PW + xr;
        pi_src[q] = yr * BW + xr + 2;
    }
    // own pair: w/p ring x index xo, w row ty + 1; ring item of threads 0..63+2TH: a pair in the
    // rows j0-1 / j0+TH (threads 0..63) or a single cell in the columns i0-1 / i0+64
    const int xo = 2 + 2 * tx, yo = ty + 1;
    int rx = 0, ry = 0;
    const bool ring_pair = tid < 64, ring_single = tid >= 64 && tid < 64 + 2 * TH;
    if (tid < 32) { rx = 2 + 2 * tid; ry = 0; }
    else if (tid < 64) { rx = 2 + 2 * (tid - 32); ry = TH + 1; }
    else if (tid < 64 + TH) { rx = 1; ry = 1 + (tid - 64); }
    else if (tid < 64 + 2 * TH) { rx = PW - 2; ry = 1 + (tid - 64 - TH); }

    const int tiles_x = (d.nx + G::TW - 1) / G::TW;
    const long long ntiles = (long long)tiles_x * ((d.ny + TH - 1) / TH);
    const long long total = ntiles * d.nz;
    const long long w0 = min((long long)blockIdx.x * per_block, total);
    const long long w1 = min(w0 + per_block, total);
    for (long long w = w0; w < w1 && !bad;) {
        const long long tile_id = w / d.nz;
        const int k0 = int(w - tile_id * d.nz);
        const int k1 = (int)min((long long)d.nz, (long long)k0 + (w1 - w));
        w += k1 - k0;
        const int i0 = int(tile_id % tiles_x) * G::TW, j0 = int(tile_id / tiles_x) * TH;
        const int i = i0 + 2 * tx, j = j0 + ty;
        const bool inside = i < d.nx && j < d.ny;     // nx is even: both cells of the pair
        const int s_first = k0 - 4, s_last = k1 - 1;  // steps that consume a stage
        auto slot = [&](int s) { return (s - s_first) % NS; };
        // stage of step s: r and p_old of plane s+2, Tx, Ty, Tz of plane s+1
        auto issue = [&](int s) {
            const int q = slot(s);
            pending |= 1u << q;
            if (tid == 0) {
                unsigned char* b = stage(q);
                mbar_expect_tx(&bars[q], G::kTx);
                tma_load_3d(b + G::oR, &maps.r, &bars[q], i0 - G::HX, j0 - 2, s + 2);
                tma_load_3d(b + G::oP, &maps.p, &bars[q], i0 - G::HX, j0 - 2, s + 2);
                tma_load_3d(b + G::oX, &maps.tx, &bars[q], i0 - G::HX, j0 - 1, s + 1);
                tma_load_3d(b + G::oY, &maps.ty, &bars[q], i0 - G::HX, j0 - 2, s + 1);
                tma_load_3d(b + G::oZ, &maps.tz, &bars[q], i0 - G::HX, j0 - 1, s + 1);
            }
        };
        auto wait = [&](int s) -> bool {
            const int q = slot(s);
            const bool ok = mbar_wait_bounded(&bars[q], (phase >> q) & 1u);
            phase ^= 1u << q;
            pending &= ~(1u << q);
            return ok;
        };
        // w of one cell at ring x index xr, w row yw, plane m (tzm: |Tz| of plane m-1 there)
        auto w_single = [&](const unsigned char* b, int m, int xr, int yw, float tzm, float& tz_out) -> float {
            const float* X = reinterpret_cast<const float*>(b + G::oX);
            const float* Y = reinterpret_cast<const float*>(b + G::oY);
            const float* Z = reinterpret_cast<const float*>(b + G::oZ);
            const float* P0 = pl(m);
            const int yr = yw + 1, e = yr * PW + xr, xb = xr + 2;
            const float tz = Z[yw * BW + xb];
            float u = 0.0f;
            u = fmav(X[yw * BW + xb], P0[e + 1], u);
            u = fmav(X[yw * BW + xb - 1], P0[e - 1], u);
            u = fmav(Y[yr * BW + xb], P0[e + PW], u);
            u = fmav(Y[(yr - 1) * BW + xb], P0[e - PW], u);
            u = fmav(fabsf(tz), pl(m + 1)[e], u);
            u = fmav(tzm, pl(m - 1)[e], u);
            tz_out = fabsf(tz);
            return signbit(tz) ? u : P0[e];
        };
        // w of a pair at (xr even, yw); fills its coefficients
        auto w_pair = [&](const unsigned char* b, int m, int xr, int yw, float2 tzm, RbCo& co) -> float2 {
            const float* X = reinterpret_cast<const float*>(b + G::oX);
            const float* Y = reinterpret_cast<const float*>(b + G::oY);
            const float* Z = reinterpret_cast<const float*>(b + G::oZ);
            const float* P0 = pl(m);
            const int yr = yw + 1, e = yr * PW + xr, xb = xr + 2;
            co.tx = *reinterpret_cast<const float2*>(X + yw * BW + xb);
            co.txl = X[yw * BW + xb - 1];
            co.ty = *reinterpret_cast<const float2*>(Y + yr * BW + xb);
            co.tyd = *reinterpret_cast<const float2*>(Y + (yr - 1) * BW + xb);
            co.tz = *reinterpret_cast<const float2*>(Z + yw * BW + xb);
            co.tzm = tzm;
            const float2 v = *reinterpret_cast<const float2*>(P0 + e);
            const float lf = P0[e - 1], rt = P0[e + 2];
            const float2 up = *reinterpret_cast<const float2*>(P0 + e + PW);
            const float2 dn = *reinterpret_cast<const float2*>(P0 + e - PW);
            const float2 zp = *reinterpret_cast<const float2*>(pl(m + 1) + e);
            const float2 zm = *reinterpret_cast<const float2*>(pl(m - 1) + e);
            float u0 = 0.0f, u1 = 0.0f;
            u0 = fmav(co.tx.x, v.y, u0);
            u1 = fmav(co.tx.y, rt, u1);
            u0 = fmav(co.txl, lf, u0);
            u1 = fmav(co.tx.x, v.x, u1);
            u0 = fmav(co.ty.x, up.x, u0);
            u1 = fmav(co.ty.y, up.y, u1);
            u0 = fmav(co.tyd.x, dn.x, u0);
            u1 = fmav(co.tyd.y, dn.y, u1);
            u0 = fmav(fabsf(co.tz.x), zp.x, u0);
            u1 = fmav(fabsf(co.tz.y), zp.y, u1);
            u0 = fmav(tzm.x, zm.x, u0);
            u1 = fmav(tzm.y, zm.y, u1);
            return make_float2(signbit(co.tz.x) ? u0 : v.x, signbit(co.tz.y) ? u1 : v.y);
        };

        RbCo sa{}, sb{};                  // own-pair coefficients of planes s-1 and s
        float2 own_tzm = make_float2(0.f, 0.f), ring_tzm2 = make_float2(0.f, 0.f);
        float ring_tzm1 = 0.0f;
        float2 xa = make_float2(0.f, 0.f), pa = xa, xb2 = xa, pb = xa;   // x, p_old of planes s-1, s

        __syncthreads();   // the previous segment's readers are done with the stages and rings
        if (tid == 0) fence_proxy_async_smem();
        for (int s = s_first; s <= min(s_first + NS - 1, s_last); ++s) issue(s);
        for (int s = s_first; s <= k1; ++s) {
            if (s - 1 >= s_first && s - 1 + NS <= s_last) {
                if (tid == 0) fence_proxy_async_smem();
                issue(s - 1 + NS);
            }
            bool ok = true;
            if (s <= s_last) ok = wait(s);
            const unsigned char* b = stage(slot(s));
            // P1: p of plane s+2
            if (s <= s_last) {
                const float* R = reinterpret_cast<const float*>(b + G::oR);
                const float* P = reinterpret_cast<const float*>(b + G::oP);
                float* op = pl(s + 2);
#pragma unroll
                for (int q = 0; q < PP; ++q) {
                    if (!pi_on[q]) continue;
                    const float2 pv = *reinterpret_cast<const float2*>(P + pi_src[q]);
                    const float2 rv = *reinterpret_cast<const float2*>(R + pi_src[q]);
                    *reinterpret_cast<float2*>(op + pi_dst[q]) =
                        make_float2(fmav(beta, pv.x, rv.x), fmav(beta, pv.y, rv.y));
                }
            }
            // P1: t of plane s-1 on the non-red cells of the own pair
            const int m = s - 1;
            if (m >= k0 && m < k1 && inside) {
                const float* W0 = wl(m);
                const int e = yo * PW + xo;
                const float2 wv = *reinterpret_cast<const float2*>(W0 + e);
                const float wlf = W0[e - 1], wrt = W0[e + 2];
                const float2 wup = *reinterpret_cast<const float2*>(W0 + e + PW);
                const float2 wdn = *reinterpret_cast<const float2*>(W0 + e - PW);
                const float2 wzp = *reinterpret_cast<const float2*>(wl(m + 1) + e);
                const float2 wzm = *reinterpret_cast<const float2*>(wl(m - 1) + e);
                float t0 = wv.x, t1 = wv.y;
                t0 = fmav(-sa.tx.x, wv.y, t0);
                t1 = fmav(-sa.tx.y, wrt, t1);
                t0 = fmav(-sa.txl, wlf, t0);
                t1 = fmav(-sa.tx.x, wv.x, t1);
                t0 = fmav(-sa.ty.x, wup.x, t0);
                t1 = fmav(-sa.ty.y, wup.y, t1);
                t0 = fmav(-sa.tyd.x, wdn.x, t0);
                t1 = fmav(-sa.tyd.y, wdn.y, t1);
                t0 = fmav(-fabsf(sa.tz.x), wzp.x, t0);
                t1 = fmav(-fabsf(sa.tz.y), wzp.y, t1);
                t0 = fmav(-sa.tzm.x, wzm.x, t0);
                t1 = fmav(-sa.tzm.y, wzm.y, t1);
                const bool r0 = signbit(sa.tz.x), r1 = signbit(sa.tz.y);
                const long long c = (long long)m * d.plane + i + (long long)d.nx * j;
                *reinterpret_cast<float2*>(out + c) = make_float2(r0 ? 0.f : t0, r1 ? 0.f : t1);
                *reinterpret_cast<float2*>(pnew + c) = make_float2(r0 ? 0.f : wv.x, r1 ? 0.f : wv.y);
                *reinterpret_cast<float2*>(xv + c) =
                    make_float2(r0 ? xa.x : fmav(alpha, pa.x, xa.x), r1 ? xa.y : fmav(alpha, pa.y, xa.y));
                if (!r0) acc.add(wv.x, t0);
                if (!r1) acc.add(wv.y, t1);
            }
            // x and p_old of plane s+1 (for its t, two steps later)
            xa = xb2;
            pa = pb;
            xb2 = make_float2(0.f, 0.f);
            pb = xb2;
            if (s + 1 >= k0 && s + 1 < k1 && inside) {
                const long long c = (long long)(s + 1) * d.plane + i + (long long)d.nx * j;
                xb2 = *reinterpret_cast<const float2*>(xv + c);
                pb = *reinterpret_cast<const float2*>(pold + c);
            }
            if (__syncthreads_or(!ok)) {
                bad = true;
                break;
            }
            // P2: w of plane s+1 (own pair and ring); before plane k0-1 only |Tz| is carried
            if (s <= s_last && s + 1 >= k0 - 2) {
                const int mw = s + 1;
                const float* Z = reinterpret_cast<const float*>(b + G::oZ);
                if (mw >= k0 - 1) {
                    RbCo co;
                    const float2 wv = w_pair(b, mw, xo, yo, own_tzm, co);
                    *reinterpret_cast<float2*>(wl(mw) + yo * PW + xo) = wv;
                    own_tzm = make_float2(fabsf(co.tz.x), fabsf(co.tz.y));
                    sa = sb;
                    sb = co;
                    if (ring_pair) {
                        RbCo cr;
                        const float2 wr = w_pair(b, mw, rx, ry, ring_tzm2, cr);
                        *reinterpret_cast<float2*>(wl(mw) + ry * PW + rx) = wr;
                        ring_tzm2 = make_float2(fabsf(cr.tz.x), fabsf(cr.tz.y));
                    } else if (ring_single) {
                        float tzo;
                        wl(mw)[ry * PW + rx] = w_single(b, mw, rx, ry, ring_tzm1, tzo);
                        ring_tzm1 = tzo;
                    }
                } else {
                    const float2 tz = *reinterpret_cast<const float2*>(Z + yo * BW + xo + 2);
                    own_tzm = make_float2(fabsf(tz.x), fabsf(tz.y));
                    if (ring_pair) {
                        const float2 tr = *reinterpret_cast<const float2*>(Z + ry * BW + rx + 2);
                        ring_tzm2 = make_float2(fabsf(tr.x), fabsf(tr.y));
                    } else if (ring_single) {
                        ring_tzm1 = fabsf(Z[ry * BW + rx + 2]);
                    }
                }
            } else {
                sa = sb;
            }
            __syncthreads();
        }
    }
    if (bad) {
        for (int s = 0; s < NS; ++s)
            if (pending & (1u << s)) mbar_wait_bounded(&bars[s], (phase >> s) & 1u);
        if (tid == 0) atomicCAS(&sc->status, (int)VOFP_OK, (int)VOFP_ERR_DEVICE_TIMEOUT);
    }
    double tot;
    if (grid_reduce(acc.value(), partials, counter, sh, &tot)) sc->pq_raw = tot;
}

}  // namespace vofp
