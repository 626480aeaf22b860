// Kernels of the conjugate-gradient loop (Sec. 1: the pressure equation is solved by
// preconditioned conjugate gradients).
//
// The loop runs on the symmetrically scaled system  S A_hat S y = S b_hat,  S = diag(A_hat)^-1/2,
// x = S y, which is the diagonally (Jacobi) preconditioned CG written so that the operator has a
// unit diagonal: no diagonal and no z = D^-1 r stream are read.  Vectors live on the full grid:
// every cell of a merge group holds the group's value (r, p, x, q expanded), so the 7-point
// stencil runs unchanged over merged cells and a small per-group kernel folds the stencil output
// into the group's row (Sec. 2.3 merging as P^T A P).
//
// Per iteration (FP64: 12 array passes, 96 bytes per cell):
//   stencil   p = r + beta p_old (shared-memory tile with halo), x += alpha p_old,
//             t = (S A S) p with unit diagonal, p.t       (reads r, p_old, x, Tx, Ty, Tz;
//                                                           writes p, x, t)
//   patch     per merge group: q_m = sum_G t + corr_m p_m, written to every cell of G; adds
//             corr_m p_m^2 to p.Ap                          (O(merged cells))
//   update    alpha = r.r / p.Ap;  r -= alpha q;  r.r over the unknowns   (reads r, q; writes r)
// Reductions: block partial sums, reduced in index order by the block that finishes last, so
// results are bitwise reproducible from run to run.
#pragma once
#include <type_traits>

#include "vofp_internal.cuh"

namespace vofp {

enum StencilMode { ST_APPLY_UNSCALED = 0, ST_APPLY_SCALED = 1, ST_CG = 2 };

// FP64 accumulator.
struct AccD {
    double s = 0.0;
    __device__ __forceinline__ void add(double a, double b) { s = fma(a, b, s); }
    __device__ __forceinline__ void add(float a, float b) { s = fma((double)a, (double)b, s); }
    __device__ __forceinline__ double value() const { return s; }
};

// FP32 compensated dot product accumulator (error-free product by FMA and error-free sum, the
// "Dot2" scheme of Ogita, Rump and Oishi, Accurate sum and dot product, SIAM J. Sci. Comput.
// 2005): the per-thread result is as accurate as if accumulated in twice FP32's precision and is
// converted to FP64 once per thread, so dot products of FP32 vectors are accumulated to FP64-level
// accuracy without FP64 arithmetic per element.
struct AccF2 {
    float s = 0.0f, c = 0.0f;
    __device__ __forceinline__ void add(float a, float b) {
        const float p = __fmul_rn(a, b);
        const float e = __fmaf_rn(a, b, -p);
        const float t = __fadd_rn(s, p);
        const float bp = __fsub_rn(t, s);
        const float err = __fadd_rn(__fsub_rn(s, __fsub_rn(t, bp)), __fsub_rn(p, bp));
        s = t;
        c = __fadd_rn(c, __fadd_rn(err, e));
    }
    __device__ __forceinline__ double value() const { return (double)s + (double)c; }
};

template <typename V>
struct AccFor;
template <>
struct AccFor<double> {
    using type = AccD;
};
template <>
struct AccFor<float> {
    using type = AccF2;
};

__device__ __forceinline__ double fmav(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ float fmav(float a, float b, float c) { return __fmaf_rn(a, b, c); }

// Reduce `part` over the grid; the last block to finish writes the sum (index order) to *out.
// Returns true in thread 0 of that block.
__device__ __forceinline__ bool grid_reduce(double part, double* partials, unsigned int* counter,
                                            double* sh, double* total) {
    __shared__ bool is_last;
    const int nt = blockDim.x * blockDim.y;
    const int tid = threadIdx.x + blockDim.x * threadIdx.y;
    const int nb = gridDim.x * gridDim.y * gridDim.z;
    const int b = blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z);
    // block sum (fixed order)
    double v = warp_sum(part);
    if ((tid & 31) == 0) sh[tid >> 5] = v;
    __syncthreads();
    if (tid == 0) {
        double s = 0.0;
        for (int w = 0; w < nt / 32; ++w) s += sh[w];
        partials[b] = s;
        __threadfence();
        unsigned int t = atomicAdd(counter, 1u);
        is_last = (t == (unsigned int)(nb - 1));
    }
    __syncthreads();
    if (!is_last) return false;
    __threadfence();
    double s = 0.0;
    for (int i = tid; i < nb; i += nt) s += __ldcg(&partials[i]);
    s = warp_sum(s);
    __syncthreads();
    if ((tid & 31) == 0) sh[tid >> 5] = s;
    __syncthreads();
    if (tid == 0) {
        double tot = 0.0;
        for (int w = 0; w < nt / 32; ++w) tot += sh[w];
        *total = tot;
        *counter = 0u;
    }
    return tid == 0;
}

// Fused direction update + stencil + dot (ST_CG), or a plain operator apply.
// A block of kBX x kBY threads marches kBX x kBY column tiles in z over its share of tile-planes.
// Plane k (with a one-cell halo) and the own columns of planes k-1 and k+1 sit in four rotating
// shared buffers (one barrier per plane); the raw inputs of planes k+1 .. k+PF are prefetched
// into registers one barrier ahead, so global loads overlap the arithmetic of the plane before.
// In ST_CG the tile holds p = r + beta p_old, computed once per loaded element (halo included)
// with the same fused multiply-add as its owning block, so neighbouring tiles agree bitwise.
constexpr int kHalo = 2 * kBX + 2 * kBY;

template <typename V>
struct StCoef {
    V txp, txm, typ, tym, tzp, xo, dg;
};

template <typename V, int MODE, int PF>
__global__ void __launch_bounds__(kBX* kBY, 4)
k_stencil(const Dims d, const int per_block, const V* __restrict__ Tx, const V* __restrict__ Ty,
          const V* __restrict__ Tz, const double* __restrict__ diag, const V* __restrict__ src,
          const V* __restrict__ pold, V* __restrict__ pnew, V* __restrict__ xv, V* __restrict__ out,
          CgScalars* __restrict__ sc, double* __restrict__ partials, unsigned int* __restrict__ counter) {
    using Acc = typename AccFor<V>::type;
    constexpr bool CG = MODE == ST_CG;
    __shared__ V tile[4][kBY + 2][kBX + 2];
    __shared__ double sh[32];
    const int tx = threadIdx.x, ty = threadIdx.y, tid = tx + kBX * ty;
    V beta = V(0), alpha = V(0);
    if (CG) {
        beta = (V)sc->beta;
        alpha = (V)sc->alpha;
    }
    Acc acc;
    // This block's share of the work: the tile-planes [w0, w1) in tile-major order, so every block
    // marches the same number of planes (one wave, no tail) in at most a few column segments.
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
        // this thread's halo element: rows j0-1 and j0+kBY, then columns i0-1 and i0+kBX
        int hi = 0, hj = 0;
        long long hoff = -1;
        const bool has_halo = tid < kHalo;
        if (has_halo) {
            int gi, gj;
            if (tid < kBX) {
                gi = i0 + tid; gj = j0 - 1; hi = tid + 1; hj = 0;
            } else if (tid < 2 * kBX) {
                gi = i0 + tid - kBX; gj = j0 + kBY; hi = tid - kBX + 1; hj = kBY + 1;
            } else if (tid < 2 * kBX + kBY) {
                gi = i0 - 1; gj = j0 + tid - 2 * kBX; hi = 0; hj = tid - 2 * kBX + 1;
            } else {
                gi = i0 + kBX; gj = j0 + tid - 2 * kBX - kBY; hi = kBX + 1; hj = tid - 2 * kBX - kBY + 1;
            }
            if (gi >= 0 && gi < d.nx && gj >= 0 && gj < d.ny) hoff = gi + (long long)d.nx * gj;
        }
        auto load = [&](int kk, V& r_, V& p_, V& hr, V& hp) {
            r_ = V(0); p_ = V(0); hr = V(0); hp = V(0);
            if (kk < 0 || kk >= d.nz) return;
            const long long base = (long long)kk * d.plane;
            if (inside) {
                r_ = src[base + own];
                if (CG) p_ = pold[base + own];
            }
            if (hoff >= 0) {
                hr = src[base + hoff];
                if (CG) hp = pold[base + hoff];
            }
        };
        auto store = [&](int b, V r_, V p_, V hr, V hp) {
            tile[b][ty + 1][tx + 1] = CG ? fmav(beta, p_, r_) : r_;
            if (has_halo) tile[b][hj][hi] = CG ? fmav(beta, hp, hr) : hr;
        };
        auto loadc = [&](int kk, StCoef<V>& c) {
            c.txp = c.txm = c.typ = c.tym = c.tzp = c.xo = c.dg = V(0);
            if (!inside || kk >= k1) return;
            const long long cc = (long long)kk * d.plane + own;
            c.txp = Tx[cc];
            c.txm = i > 0 ? Tx[cc - 1] : V(0);
            c.typ = Ty[cc];
            c.tym = j > 0 ? Ty[cc - d.nx] : V(0);
            c.tzp = Tz[cc];
            if (CG) c.xo = xv[cc];
            if (MODE == ST_APPLY_UNSCALED) c.dg = (V)diag[cc];
        };

        // the previous segment's last readers of the buffers must be done before they are refilled
        __syncthreads();
        V rr_[PF], pp_[PF], hr_[PF], hp_[PF];
        {
            V a, b, c2, e;
            load(k0 - 1, a, b, c2, e);
            store(0, a, b, c2, e);
        }
        V po_cur;
        {
            V a, c2, e;
            load(k0, a, po_cur, c2, e);
            store(1, a, po_cur, c2, e);
        }
#pragma unroll
        for (int q = 0; q < PF; ++q) {
            if (k0 + 1 + q <= k1) load(k0 + 1 + q, rr_[q], pp_[q], hr_[q], hp_[q]);
            else rr_[q] = pp_[q] = hr_[q] = hp_[q] = V(0);
        }
        StCoef<V> cc;
        loadc(k0, cc);
        V tzm1 = (inside && k0 > 0) ? Tz[(long long)(k0 - 1) * d.plane + own] : V(0);
        for (int k = k0; k < k1; ++k) {
            const int rel = k - k0 + 1;
            const int bm = (rel + 3) & 3, b0 = rel & 3, bp = (rel + 1) & 3;
            store(bp, rr_[0], pp_[0], hr_[0], hp_[0]);
            const V po_next = pp_[0];
#pragma unroll
            for (int q = 0; q < PF - 1; ++q) {
                rr_[q] = rr_[q + 1]; pp_[q] = pp_[q + 1]; hr_[q] = hr_[q + 1]; hp_[q] = hp_[q + 1];
            }
            const int kn = k + 1 + PF;
            if (kn <= k1) load(kn, rr_[PF - 1], pp_[PF - 1], hr_[PF - 1], hp_[PF - 1]);
            StCoef<V> cn;
            loadc(k + 1, cn);
            __syncthreads();
            if (inside) {
                const long long c = (long long)k * d.plane + own;
                const V v = tile[b0][ty + 1][tx + 1];
                V t = (MODE == ST_APPLY_UNSCALED) ? cc.dg * v : v;
                t = fmav(-cc.txp, tile[b0][ty + 1][tx + 2], t);
                t = fmav(-cc.txm, tile[b0][ty + 1][tx], t);
                t = fmav(-cc.typ, tile[b0][ty + 2][tx + 1], t);
                t = fmav(-cc.tym, tile[b0][ty][tx + 1], t);
                t = fmav(-cc.tzp, tile[bp][ty + 1][tx + 1], t);
                t = fmav(-tzm1, tile[bm][ty + 1][tx + 1], t);
                out[c] = t;
                if (CG) {
                    pnew[c] = v;
                    xv[c] = fmav(alpha, po_cur, cc.xo);
                    acc.add(v, t);
                }
            }
            tzm1 = cc.tzp;
            cc = cn;
            po_cur = po_next;
        }
    }
    if (CG) {
        double tot;
        if (grid_reduce(acc.value(), partials, counter, sh, &tot)) sc->pq_raw = tot;
    }
}

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
template <typename V>
__global__ void k_group_patch(int ng, const int* __restrict__ gptr, const int* __restrict__ gcells,
                              const double* __restrict__ gcorr, V* __restrict__ t,
                              const V* __restrict__ p, int dot, CgScalars* sc,
                              double* __restrict__ partials, unsigned int* __restrict__ counter) {
    __shared__ double sh[32];
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    double part = 0.0;
    if (g < ng) {
        const int b = gptr[g], e = gptr[g + 1];
        const int m = gcells[b];
        double s = 0.0;
        for (int u = b; u < e; ++u) s += (double)t[gcells[u]];
        const double pm = (double)p[m];
        const V qm = (V)(s + gcorr[g] * pm);
        for (int u = b; u < e; ++u) t[gcells[u]] = qm;
        part = gcorr[g] * pm * pm;
    }
    if (dot) {
        double tot;
        if (grid_reduce(part, partials, counter, sh, &tot)) sc->pq_corr = tot;
    }
}

__device__ __forceinline__ bool is_slave(const uint32_t* __restrict__ bits, long long c) {
    return (bits[c >> 5] >> (c & 31)) & 1u;
}

// alpha = r.r / p.Ap;  r -= alpha q;  r.r over the unknowns (cells that are not another cell's
// group member).  The last block stores rr, beta = rr_new / rr_old, alpha, counts the iteration
// and, for an inner (mixed-precision) loop, ends it when rr <= inner_rtol^2 rr0 or max_iter.
template <typename V, bool INNER>
__global__ void __launch_bounds__(kRedThreads)
k_cg_update(long long n, V* __restrict__ r, const V* __restrict__ q, const uint32_t* __restrict__ bits,
            CgScalars* sc, double* __restrict__ partials, unsigned int* __restrict__ counter,
            cudaGraphConditionalHandle handle, int use_handle) {
    using Acc = typename AccFor<V>::type;
    __shared__ double sh[32];
    __shared__ double s_alpha;
    __shared__ int s_flags;
    // the scalar step is computed once per block (FP64 division is slow on this part)
    if (threadIdx.x == 0) {
        const double rr = sc->rr;
        const double pq = sc->pq_raw + sc->pq_corr;
        // rr == 0: the residual vanished exactly (later unrolled iterations are no-ops)
        const bool ok = sc->status == VOFP_OK && (pq > 0.0) && isfinite(pq) && isfinite(rr) && rr > 0.0;
        const bool broke = !ok && !(rr == 0.0 && sc->status == VOFP_OK);
        s_alpha = ok ? rr / pq : 0.0;
        s_flags = (ok ? 1 : 0) | (broke ? 2 : 0);
    }
    __syncthreads();
    const double alpha_d = s_alpha;
    const bool broke = (s_flags & 2) != 0;
    const V alpha = (V)alpha_d;
    Acc acc;
    constexpr int VW = sizeof(V) == 8 ? 2 : 4;
    using VV = typename std::conditional<sizeof(V) == 8, double2, float4>::type;
    constexpr int UN = 4;
    const long long nv = n / VW;
    const long long stride = (long long)gridDim.x * blockDim.x;
    const V na = -alpha;
    auto upd = [&](VV& rv, const VV& qv, uint32_t w) {
        if constexpr (VW == 2) {
            rv.x = fmav(na, qv.x, rv.x);
            rv.y = fmav(na, qv.y, rv.y);
            if (!(w & 1u)) acc.add(rv.x, rv.x);
            if (!(w & 2u)) acc.add(rv.y, rv.y);
        } else {
            rv.x = fmav(na, qv.x, rv.x);
            rv.y = fmav(na, qv.y, rv.y);
            rv.z = fmav(na, qv.z, rv.z);
            rv.w = fmav(na, qv.w, rv.w);
            if (!(w & 1u)) acc.add(rv.x, rv.x);
            if (!(w & 2u)) acc.add(rv.y, rv.y);
            if (!(w & 4u)) acc.add(rv.z, rv.z);
            if (!(w & 8u)) acc.add(rv.w, rv.w);
        }
    };
    VV* rvp = reinterpret_cast<VV*>(r);
    const VV* qvp = reinterpret_cast<const VV*>(q);
    long long vi = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    for (; vi + (UN - 1) * stride < nv; vi += UN * stride) {
        VV rv[UN], qv[UN];
        uint32_t w[UN];
#pragma unroll
        for (int u = 0; u < UN; ++u) {
            rv[u] = rvp[vi + u * stride];
            qv[u] = qvp[vi + u * stride];
            const long long c0 = (vi + u * stride) * VW;
            w[u] = bits[c0 >> 5] >> (c0 & 31);
        }
#pragma unroll
        for (int u = 0; u < UN; ++u) {
            upd(rv[u], qv[u], w[u]);
            rvp[vi + u * stride] = rv[u];
        }
    }
    for (; vi < nv; vi += stride) {
        VV rv = rvp[vi];
        const VV qv = qvp[vi];
        const long long c0 = vi * VW;
        upd(rv, qv, bits[c0 >> 5] >> (c0 & 31));
        rvp[vi] = rv;
    }
    for (long long c = nv * VW + blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n; c += stride) {
        V rv = fmav(-alpha, q[c], r[c]);
        r[c] = rv;
        if (!is_slave(bits, c)) acc.add(rv, rv);
    }
    double tot;
    if (grid_reduce(acc.value(), partials, counter, sh, &tot)) {
        const double rr = sc->rr;
        sc->rr_prev = rr;
        sc->rr = tot;
        sc->beta = (rr > 0.0) ? tot / rr : 0.0;
        sc->alpha = alpha_d;
        sc->iter += 1;
        sc->iter_total += 1;
        if ((broke || !isfinite(tot)) && sc->status == VOFP_OK && !sc->timing) {
            sc->status = VOFP_ERR_BREAKDOWN;
            sc->alpha = 0.0;
            sc->beta = 0.0;
        }
        if (INNER) {
            bool stop = broke || !isfinite(tot) || tot <= sc->inner_target * sc->inner_target * sc->rr0 ||
                        sc->iter >= sc->max_iter || sc->iter_total >= sc->max_iter;
            if (stop) sc->inner_done = 1;
            if (use_handle && stop) cudaGraphSetConditional(handle, 0);
        }
    }
}

// True residual check of the FP64 loop: ||r_hat||^2 = sum over unknowns of (r_scaled / s)^2.
template <typename V>
__global__ void __launch_bounds__(kRedThreads)
k_cg_check(long long n, const V* __restrict__ r, const double* __restrict__ sq,
           const uint32_t* __restrict__ bits, CgScalars* sc, double* __restrict__ partials,
           unsigned int* __restrict__ counter, cudaGraphConditionalHandle handle, int use_handle) {
    __shared__ double sh[32];
    double acc = 0.0;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n; c += stride) {
        if (is_slave(bits, c)) continue;
        const double v = (double)r[c] * sq[c];
        acc = fma(v, v, acc);
    }
    double tot;
    if (grid_reduce(acc, partials, counter, sh, &tot)) {
        sc->rnorm2 = tot;
        bool stop = false;
        if (!isfinite(tot) || sc->status != VOFP_OK) {
            if (sc->status == VOFP_OK) sc->status = VOFP_ERR_BREAKDOWN;
            stop = true;
        } else if (tot <= sc->rtol * sc->rtol * sc->ref2) {
            stop = true;
        } else if (sc->iter >= sc->max_iter) {
            sc->status = VOFP_ERR_NOT_CONVERGED;
            stop = true;
        }
        if (stop) sc->done = 1;
        if (use_handle && stop) cudaGraphSetConditional(handle, 0);
    }
}

}  // namespace vofp
