// Fused red-black iteration kernel (shared-memory tiles fed by register prefetch).
#pragma once
#include "vofp_kernels.cuh"

namespace vofp {

// Red-black elimination (Eisenstat's form of red-black symmetric Gauss-Seidel).  On the scaled
// operator I - E the red block is the identity, so red unknowns are eliminated exactly:
// x_R = b_R + E_RS x_S, and CG runs on the Schur complement S = I_SS - E_SS - E_SR E_RS of the
// remaining (black and merge-group) unknowns.  An iteration forms w = E_RS p on the red cells
// and w = p on the others, and applies I - E to w on the black rows.
// Fused red-black iteration: one pass per CG iteration.
// A block (32 x 8 columns) marches planes in z.  Four rotating shared planes hold, with a 2-cell
// halo, the direction p = r + beta p_old and the coefficients Tx, Ty, Tz; three rotating planes
// hold w (w = p on black cells, w = E_RS p on red cells; 1-cell halo); a byte tile per plane
// holds the red flags.  The raw inputs of plane k+2 are prefetched into registers one step ahead.
// Step k: store plane k+2; barrier; form w of plane k+1 from shared memory; barrier; apply I - E
// to w on the black rows of plane k.
constexpr int kPX = kBX + 4, kPY = kBY + 4, kPN = kPX * kPY;

template <typename V, int PF>
__global__ void __launch_bounds__(kBX* kBY, 3)
k_cg_rb(const Dims d, const int per_block, const V* __restrict__ Tx, const V* __restrict__ Ty,
        const V* __restrict__ Tz, const uint32_t* __restrict__ red, const V* __restrict__ src,
        const V* __restrict__ pold, V* __restrict__ pnew, V* __restrict__ xv, V* __restrict__ out,
        CgScalars* __restrict__ sc, double* __restrict__ partials, unsigned int* __restrict__ counter) {
    using Acc = typename AccFor<V>::type;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    V* sm = reinterpret_cast<V*>(smem_raw);
    // [4 planes][4 fields: p, Tx, Ty, Tz][kPN] then w [3 planes][(kBY+2) x (kBX+2)]
    auto tile = [&](int kk, int f) -> V* { return sm + ((((kk + 8) & 3) * 4 + f) * kPN); };
    constexpr int WN = (kBY + 2) * (kBX + 2);
    auto wpl = [&](int kk) -> V* { return sm + 16 * kPN + ((kk + 6) % 3) * WN; };
    // red flags of the same four planes, one byte per p-tile position
    unsigned char* flags = reinterpret_cast<unsigned char*>(sm + 16 * kPN + 3 * WN);
    auto ftile = [&](int kk) -> unsigned char* { return flags + ((kk + 8) & 3) * kPN; };
    __shared__ double sh[32];
    const int tx = threadIdx.x, ty = threadIdx.y, tid = tx + kBX * ty;
    const V beta = (V)sc->beta, alpha = (V)sc->alpha;
    Acc acc;
    const int tiles_x = (d.nx + kBX - 1) / kBX;
    const long long ntiles = (long long)tiles_x * ((d.ny + kBY - 1) / kBY);
    const long long total = ntiles * d.nz;
    const long long w0 = min((long long)blockIdx.x * per_block, total);
    const long long w1 = min(w0 + per_block, total);
    for (long long w = w0; w < w1;) {
        const long long tile_id = w / d.nz;
        const int k0 = int(w - tile_id * d.nz);
        const int k1 = (int)min((long long)d.nz, (long long)k0 + (w1 - w));
        w += k1 - k0;
        const int i0 = int(tile_id % tiles_x) * kBX, j0 = int(tile_id / tiles_x) * kBY;
        const int i = i0 + tx, j = j0 + ty;
        const bool inside = i < d.nx && j < d.ny;
        const long long own = inside ? i + (long long)d.nx * j : 0;
        long long poff[2];
        bool pval[2];
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            const int e = tid + q * kBX * kBY;
            const int gi = i0 - 2 + e % kPX, gj = j0 - 2 + e / kPX;
            pval[q] = e < kPN && gi >= 0 && gi < d.nx && gj >= 0 && gj < d.ny;
            poff[q] = pval[q] ? gi + (long long)d.nx * gj : 0;
        }
        int hi = 0, hj = 0, hgi = -1, hgj = -1;
        const bool has_ring = tid < kHalo;
        if (has_ring) {
            if (tid < kBX) { hgi = i0 + tid; hgj = j0 - 1; hi = tid + 1; hj = 0; }
            else if (tid < 2 * kBX) { hgi = i0 + tid - kBX; hgj = j0 + kBY; hi = tid - kBX + 1; hj = kBY + 1; }
            else if (tid < 2 * kBX + kBY) { hgi = i0 - 1; hgj = j0 + tid - 2 * kBX; hi = 0; hj = tid - 2 * kBX + 1; }
            else { hgi = i0 + kBX; hgj = j0 + tid - 2 * kBX - kBY; hi = kBX + 1; hj = tid - 2 * kBX - kBY + 1; }
        }
        struct Raw { V r[2], p[2], x[2], y[2], z[2]; unsigned f[2]; };
        auto load_raw = [&](int kk, Raw& R) {
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                R.r[q] = R.p[q] = R.x[q] = R.y[q] = R.z[q] = V(0);
                R.f[q] = 0u;
                if (pval[q] && kk >= 0 && kk < d.nz) {
                    const long long c = (long long)kk * d.plane + poff[q];
                    R.f[q] = (red[c >> 5] >> (c & 31)) & 1u;
                    R.r[q] = src[c];
                    R.p[q] = pold[c];
                    R.x[q] = Tx[c];
                    R.y[q] = Ty[c];
                    R.z[q] = Tz[c];
                }
            }
        };
        auto store_raw = [&](int kk, const Raw& R) {
            V* P = tile(kk, 0);
            V* X = tile(kk, 1);
            V* Y = tile(kk, 2);
            V* Z = tile(kk, 3);
            unsigned char* Fl = ftile(kk);
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                const int e = tid + q * kBX * kBY;
                if (e < kPN) {
                    Fl[e] = (unsigned char)R.f[q];
                    P[e] = fmav(beta, R.p[q], R.r[q]);
                    X[e] = R.x[q];
                    Y[e] = R.y[q];
                    Z[e] = R.z[q];
                }
            }
        };
        // w of cell (gi, gj, kw) at p-tile position (px, py): red cells sum T p over their faces
        auto wval = [&](int gi, int gj, int kw, int px, int py) -> V {
            if (gi < 0 || gi >= d.nx || gj < 0 || gj >= d.ny || kw < 0 || kw >= d.nz) return V(0);
            const int e = py * kPX + px;
            const V* P = tile(kw, 0);
            if (!ftile(kw)[e]) return P[e];
            const V* X = tile(kw, 1);
            const V* Y = tile(kw, 2);
            const V* Z = tile(kw, 3);
            V u = V(0);
            u = fmav(X[e], P[e + 1], u);
            u = fmav(X[e - 1], P[e - 1], u);
            u = fmav(Y[e], P[e + kPX], u);
            u = fmav(Y[e - kPX], P[e - kPX], u);
            u = fmav(Z[e], tile(kw + 1, 0)[e], u);
            u = fmav(tile(kw - 1, 3)[e], tile(kw - 1, 0)[e], u);
            return u;
        };
        auto form_w = [&](int kw) {
            V* Wp = wpl(kw);
            Wp[(ty + 1) * (kBX + 2) + tx + 1] = wval(i, j, kw, tx + 2, ty + 2);
            if (has_ring) Wp[hj * (kBX + 2) + hi] = wval(hgi, hgj, kw, hi + 1, hj + 1);
        };

        __syncthreads();   // the previous segment's readers are done with the buffers
        {
            Raw R;
            for (int kk = k0 - 2; kk <= k0 + 1; ++kk) {
                load_raw(kk, R);
                store_raw(kk, R);
            }
        }
        __syncthreads();
        form_w(k0 - 1);
        form_w(k0);
        __syncthreads();
        Raw pre[PF];
#pragma unroll
        for (int q = 0; q < PF; ++q) {
            if (k0 + 2 + q <= k1 + 1) load_raw(k0 + 2 + q, pre[q]);
            else load_raw(-100, pre[q]);
        }
        const int eo = (ty + 2) * kPX + tx + 2;       // own p-tile position
        V tzm1 = tile(k0 - 1, 3)[eo];
        V xo = V(0), po = V(0);
        if (inside) {
            const long long c = (long long)k0 * d.plane + own;
            xo = xv[c];
            po = pold[c];
        }
        for (int k = k0; k < k1; ++k) {
            store_raw(k + 2, pre[0]);
#pragma unroll
            for (int q = 0; q < PF - 1; ++q) pre[q] = pre[q + 1];
            const int kn = k + 2 + PF;
            if (kn <= k1 + 1) load_raw(kn, pre[PF - 1]);
            V xn = V(0), pn_ = V(0);
            if (inside && k + 1 < k1) {
                const long long c = (long long)(k + 1) * d.plane + own;
                xn = xv[c];
                pn_ = pold[c];
            }
            __syncthreads();
            form_w(k + 1);
            __syncthreads();
            const V tzk = tile(k, 3)[eo];
            if (inside) {
                const long long c = (long long)k * d.plane + own;
                if (!ftile(k)[eo]) {
                    const V* Wk = wpl(k);
                    const V* X = tile(k, 1);
                    const V* Y = tile(k, 2);
                    const int wo = (ty + 1) * (kBX + 2) + tx + 1;
                    const V v = Wk[wo];
                    V t = v;
                    t = fmav(-X[eo], Wk[wo + 1], t);
                    t = fmav(-X[eo - 1], Wk[wo - 1], t);
                    t = fmav(-Y[eo], Wk[wo + kBX + 2], t);
                    t = fmav(-Y[eo - kPX], Wk[wo - kBX - 2], t);
                    t = fmav(-tzk, wpl(k + 1)[wo], t);
                    t = fmav(-tzm1, wpl(k - 1)[wo], t);
                    out[c] = t;
                    pnew[c] = tile(k, 0)[eo];
                    xv[c] = fmav(alpha, po, xo);
                    acc.add(v, t);
                }
            }
            tzm1 = tzk;
            xo = xn;
            po = pn_;
        }
    }
    double tot;
    if (grid_reduce(acc.value(), partials, counter, sh, &tot)) sc->pq_raw = tot;
}

template <typename V>
constexpr size_t cg_rb_smem() {
    return sizeof(V) * (16 * kPN + 3 * (kBY + 2) * (kBX + 2)) + 4 * kPN;
}

// Set-up and reconstruction gathers on the scaled FP64 operator (not in the iteration loop):
//   to_red = 1: for red cells    dst_c = base_c + sum_nb T_f src_nb   (others untouched)
//   to_red = 0: for non-red cells dst_c = base_c + sum over red nb of T_f src_nb, and 0 at red cells
// base may be null (0).
__global__ void __launch_bounds__(kRedThreads)
k_rb_gather(const Dims d, const double* __restrict__ Tx, const double* __restrict__ Ty,
            const double* __restrict__ Tz, const uint32_t* __restrict__ red, const double* __restrict__ src,
            const double* __restrict__ base, double* __restrict__ dst, int to_red) {
    const long long rows = (long long)d.ny * d.nz;
    auto is_red = [&](long long c) { return (red[c >> 5] >> (c & 31)) & 1u; };
    for (long long row = blockIdx.y; row < rows; row += gridDim.y) {
        const int j = int(row % d.ny), k = int(row / d.ny);
        for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < d.nx; i += gridDim.x * blockDim.x) {
            const long long c = i + (long long)d.nx * row;
            const bool rc = is_red(c);
            if (to_red && !rc) continue;
            if (!to_red && rc) {
                dst[c] = 0.0;
                continue;
            }
            double acc = base ? base[c] : 0.0;
            auto term = [&](long long n, double T) {
                if (to_red || is_red(n)) acc = fma(T, src[n], acc);
            };
            if (i > 0) term(c - 1, Tx[c - 1]);
            if (i < d.nx - 1) term(c + 1, Tx[c]);
            if (j > 0) term(c - d.nx, Ty[c - d.nx]);
            if (j < d.ny - 1) term(c + d.nx, Ty[c]);
            if (k > 0) term(c - d.plane, Tz[c - d.plane]);
            if (k < d.nz - 1) term(c + d.plane, Tz[c]);
            dst[c] = acc;
        }
    }
}

// Per merge group: q_m = sum over the group's cells of t + corr_m p_m, written to every cell of
// the group; sum over groups of corr_m p_m^2 (the part of p.A_hat p that the unit-diagonal
// stencil leaves out) goes to sc->pq_corr when `dot` is set.

}  // namespace vofp
