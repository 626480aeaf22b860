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

// Programmatic dependent launch (sm_90 and later). A kernel launched with programmatic stream
// serialisation may be scheduled while the kernel before it on the stream still runs;
// griddepcontrol.wait holds it until that kernel has completed and its writes are visible (for an
// ordinary launch it returns at once), and launch_dependents lets the next kernel's blocks be
// scheduled before this grid ends. Every kernel that takes part calls the wait before it reads
// anything its predecessor wrote, so the chain stays ordered kernel by kernel.
__device__ __forceinline__ void grid_dep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void grid_dep_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

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
// At most 64 registers (four 256-thread blocks per SM), so that a grid of four blocks per SM is one
// wave.
template <typename V, bool INNER>
__global__ void __launch_bounds__(kRedThreads, 4)
k_cg_update(long long n, V* __restrict__ r, const V* __restrict__ q, const uint32_t* __restrict__ bits,
            CgScalars* sc, double* __restrict__ partials, unsigned int* __restrict__ counter,
            cudaGraphConditionalHandle handle, int use_handle, const double* __restrict__ pq_part, int npq) {
    __shared__ double sh[32];
    __shared__ double s_alpha;
    __shared__ int s_flags;
    grid_dep_wait();
    using Acc = typename AccFor<V>::type;
    constexpr int VW = sizeof(V) == 8 ? 2 : 4;
    using VV = typename std::conditional<sizeof(V) == 8, double2, float4>::type;
    constexpr int UN = 4;
    const long long nv = n / VW;
    const long long stride = (long long)gridDim.x * blockDim.x;
    VV* rvp = reinterpret_cast<VV*>(r);
    const VV* qvp = reinterpret_cast<const VV*>(q);
    long long vi = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    VV rv[UN], qv[UN];
    uint32_t w[UN];
    auto load = [&]() {
#pragma unroll
        for (int u = 0; u < UN; ++u) {
            rv[u] = rvp[vi + u * stride];
            qv[u] = qvp[vi + u * stride];
            const long long c0 = (vi + u * stride) * VW;
            w[u] = bits[c0 >> 5] >> (c0 & 31);
        }
    };
    // the first chunk's loads do not depend on alpha: issued before the scalar step, so that
    // their latency overlaps the p.Ap sum and the division
    bool full = vi + (UN - 1) * stride < nv;
    if (full) load();
    // p.Ap: with npq > 0 the kernels before left their block partials in pq_part and every block
    // sums them itself, in the same fixed order (no last-block pass in those kernels); else the
    // scalars hold it
    double pq_sum = 0.0;
    if (npq > 0) {
        const int nt = blockDim.x;
        double v = 0.0;
        for (int i = threadIdx.x; i < npq; i += nt) v += __ldcg(&pq_part[i]);
        v = warp_sum(v);
        if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
        __syncthreads();
        if (threadIdx.x == 0)
            for (int wi = 0; wi < nt / 32; ++wi) pq_sum += sh[wi];
        __syncthreads();
    }
    // the scalar step is computed once per block (FP64 division is slow on this part)
    if (threadIdx.x == 0) {
        const double rr = sc->rr;
        const double pq = npq > 0 ? pq_sum : sc->pq_raw + sc->pq_corr;
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
    const V na = -alpha;
    auto upd = [&](VV& a, const VV& b, uint32_t m) {
        if constexpr (VW == 2) {
            a.x = fmav(na, b.x, a.x);
            a.y = fmav(na, b.y, a.y);
            if (!(m & 1u)) acc.add(a.x, a.x);
            if (!(m & 2u)) acc.add(a.y, a.y);
        } else {
            a.x = fmav(na, b.x, a.x);
            a.y = fmav(na, b.y, a.y);
            a.z = fmav(na, b.z, a.z);
            a.w = fmav(na, b.w, a.w);
            if (!(m & 1u)) acc.add(a.x, a.x);
            if (!(m & 2u)) acc.add(a.y, a.y);
            if (!(m & 4u)) acc.add(a.z, a.z);
            if (!(m & 8u)) acc.add(a.w, a.w);
        }
    };
    while (full) {
#pragma unroll
        for (int u = 0; u < UN; ++u) {
            upd(rv[u], qv[u], w[u]);
            rvp[vi + u * stride] = rv[u];
        }
        vi += UN * stride;
        full = vi + (UN - 1) * stride < nv;
        if (full) load();
    }
    for (; vi < nv; vi += stride) {
        VV a = rvp[vi];
        const VV b = qvp[vi];
        const long long c0 = vi * VW;
        upd(a, b, bits[c0 >> 5] >> (c0 & 31));
        rvp[vi] = a;
    }
    for (long long c = nv * VW + blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n; c += stride) {
        V a = fmav(-alpha, q[c], r[c]);
        r[c] = a;
        if (!is_slave(bits, c)) acc.add(a, a);
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
