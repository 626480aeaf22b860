// Solve orchestration: the preconditioned CG loop of Sec. 1 as a CUDA graph with a device-side
// WHILE condition (no host round trip per iteration), FP64 or mixed-precision iterative
// refinement (FP64 outer residual and solution update, FP32 inner CG with FP64-accurate dots).
#include <algorithm>
#include <cmath>

#include "vofp_kernels.cuh"
#include "vofp_rb.cuh"

namespace vofp {
namespace {

constexpr int kNT = kRedThreads;

int stream_grid(long long n) {
    long long b = (n + kNT - 1) / kNT;
    long long cap = (long long)num_sms() * 4;
    return int(std::max(1LL, std::min(b, cap)));
}

// persistent stencil grid: 4 resident blocks per SM, each marching an equal share of tile-planes
int stencil_blocks(const vofp_ctx* c) {
    const long long tiles = (long long)ceil_div(c->d.nx, kBX) * ceil_div(c->d.ny, kBY);
    const long long total = tiles * c->d.nz;
    const long long want = (long long)num_sms() * 4;
    return (int)std::max(1LL, std::min(want, total));
}
int stencil_per_block(const vofp_ctx* c) {
    const long long tiles = (long long)ceil_div(c->d.nx, kBX) * ceil_div(c->d.ny, kBY);
    const long long total = tiles * c->d.nz;
    const int nb = stencil_blocks(c);
    return (int)((total + nb - 1) / nb);
}
dim3 stencil_grid(const vofp_ctx* c) { return dim3(stencil_blocks(c)); }

// persistent grid of the fused red-black kernel: 3 resident blocks per SM (its shared tiles of
// p and the coefficients take about 63 KB per block in FP64)
constexpr int kRbBlocksPerSm = 3;
int rb_blocks(const vofp_ctx* c) {
    const long long tiles = (long long)ceil_div(c->d.nx, kBX) * ceil_div(c->d.ny, kBY);
    return (int)std::max(1LL, std::min((long long)num_sms() * kRbBlocksPerSm, tiles * c->d.nz));
}
int rb_per_block(const vofp_ctx* c) {
    const long long tiles = (long long)ceil_div(c->d.nx, kBX) * ceil_div(c->d.ny, kBY);
    const int nb = rb_blocks(c);
    return (int)((tiles * c->d.nz + nb - 1) / nb);
}

// register prefetch depth of the stencil: deeper for FP32, whose planes carry half the bytes
template <typename V>
constexpr int stencil_pf() {
    return sizeof(V) == 8 ? 1 : 2;
}

// Opt the red-black kernel into its dynamic shared memory and prepare the TMA-fed stencil, on the
// context's device, before any graph capture.
void prepare_kernels(vofp_ctx* c) {
    if (c->kernels_prepared) return;
    cudaFuncSetAttribute(k_cg_rb<float, stencil_pf<float>()>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)cg_rb_smem<float>());
    cudaFuncSetAttribute(k_cg_rb<double, stencil_pf<double>()>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)cg_rb_smem<double>());
    prepare_tma(c);
    prepare_rb_tma(c);
    c->kernels_prepared = true;
}

// One fused CG stencil (p = r + beta p_old, x += alpha p_old, q = S A S p, p.q): the TMA-fed
// kernel where its tensor maps can be built, else the register-prefetch kernel.
template <typename V>
void launch_cg_stencil(vofp_ctx* c, cudaStream_t st, const V* Tx, const V* Ty, const V* Tz, const V* r,
                       const V* po, V* pn, V* xv, V* q) {
    if (launch_cg_tma(c, st, Tx, Ty, Tz, r, po, pn, xv, q)) return;
    launch(c, k_stencil<V, ST_CG, stencil_pf<V>()>, stencil_grid(c), dim3(kBX, kBY), st, c->d, stencil_per_block(c),
           Tx, Ty, Tz, (const double*)nullptr, r, po, pn, xv, q, c->sc, c->partials, c->counters);
}

// one fused red-black CG iteration (k_cg_rb)
template <typename V>
void launch_cg_rb(vofp_ctx* c, cudaStream_t st, const V* Tx, const V* Ty, const V* Tz, const V* r,
                  const V* po, V* pn, V* xv, V* q) {
    if constexpr (sizeof(V) == 4) {
        if (launch_cg_rb_tma(c, st, r, po, pn, xv, q)) return;
    }
    constexpr size_t smem = cg_rb_smem<V>();
    launch_smem(c, k_cg_rb<V, stencil_pf<V>()>, dim3(rb_blocks(c)), dim3(kBX, kBY), smem, st, c->d,
                rb_per_block(c), Tx, Ty, Tz, (const uint32_t*)c->red_bits, r, po, pn, xv, q, c->sc, c->partials,
                c->counters);
}

// x_t[c] = x0[root(c)] * sq[c] (scaled initial guess, expanded over groups; 0 without unknown)
__global__ void k_init_x(long long n, const double* __restrict__ x0, const int32_t* __restrict__ root,
                         const double* __restrict__ sq, double* __restrict__ xt, int zero) {
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x) {
        const int32_t r = root[c];
        xt[c] = (zero || r < 0) ? 0.0 : x0[r] * sq[c];
    }
}

// work = b; the group fold follows.  bt = s * b_hat (after the fold)
__global__ void k_copy(long long n, const double* __restrict__ a, double* __restrict__ b) {
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x)
        b[c] = a[c];
}

// sums over unknowns (root[c] == c) of b_hat and |b_hat|, and of b_hat^2
__global__ void k_bsums(long long n, const double* __restrict__ bh, const int32_t* __restrict__ root,
                        double* __restrict__ partials, unsigned int* __restrict__ counter, double* out3) {
    __shared__ double sh[32];
    double s = 0.0, a = 0.0, q = 0.0;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x) {
        if (root[c] != (int32_t)c) continue;
        const double v = bh[c];
        s += v;
        a += fabs(v);
        q = fma(v, v, q);
    }
    double t;
    if (grid_reduce(s, partials, counter, sh, &t)) out3[0] = t;
    __syncthreads();
    if (grid_reduce(a, partials + kMaxPartials / 4, counter + 1, sh, &t)) out3[1] = t;
    __syncthreads();
    if (grid_reduce(q, partials + kMaxPartials / 2, counter + 2, sh, &t)) out3[2] = t;
}

// b_hat -= shift at unknowns (all cells of a group hold the group's value)
__global__ void k_shift(long long n, double* __restrict__ bh, const int32_t* __restrict__ root, const double* shift) {
    const double sft = *shift;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x)
        if (root[c] >= 0) bh[c] -= sft;
}

__global__ void k_scale(long long n, const double* __restrict__ s, const double* __restrict__ a, double* __restrict__ out) {
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x)
        out[c] = s[c] * a[c];
}

// r = bt - q over all cells; rr = r.r over unknowns; rn2 = sum (r sq)^2 over unknowns.
// Starts a loop: alpha = beta = 0, iteration count 0.
__global__ void k_init_residual(long long n, const double* __restrict__ bt, const double* __restrict__ q,
                                const double* __restrict__ sq, const uint32_t* __restrict__ bits,
                                double* __restrict__ r, CgScalars* sc, double* __restrict__ partials,
                                unsigned int* __restrict__ counter) {
    __shared__ double sh[32];
    double a = 0.0, b = 0.0;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x) {
        const double v = bt[c] - q[c];
        r[c] = v;
        if (!is_slave(bits, c)) {
            a = fma(v, v, a);
            const double u = v * sq[c];
            b = fma(u, u, b);
        }
    }
    double t;
    if (grid_reduce(a, partials, counter, sh, &t)) {
        sc->rr = t;
        sc->rr0 = t;
    }
    __syncthreads();
    if (grid_reduce(b, partials + kMaxPartials / 2, counter + 1, sh, &t)) sc->rnorm2 = t;
}

// pending x update of the last iteration, then the unscaled solution x = s * x_t
__global__ void k_finalize_x(long long n, double* __restrict__ xt, const double* __restrict__ p,
                             const double* __restrict__ s, const CgScalars* sc, double* __restrict__ xout) {
    const double alpha = sc->alpha;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x) {
        const double v = fma(alpha, p[c], xt[c]);
        xt[c] = v;
        xout[c] = s[c] * v;
    }
}

// expand: out[c] = x[root(c)], 0 without unknown
__global__ void k_expand_gather(long long n, const double* __restrict__ x, const int32_t* __restrict__ root,
                                double* __restrict__ out) {
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x) {
        const int32_t r = root[c];
        out[c] = r < 0 ? 0.0 : x[r];
    }
}

// ||b_hat - y||^2 and ||b_hat||^2 over unknowns (b_hat and y folded: group value at the master)
__global__ void k_resid_norms(long long n, const double* __restrict__ bh, const double* __restrict__ y,
                              const int32_t* __restrict__ root, double* __restrict__ partials,
                              unsigned int* __restrict__ counter, double* out2) {
    __shared__ double sh[32];
    double a = 0.0, b = 0.0;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x) {
        if (root[c] != (int32_t)c) continue;
        const double rv = bh[c] - y[c];
        a = fma(rv, rv, a);
        b = fma(bh[c], bh[c], b);
    }
    double t;
    if (grid_reduce(a, partials, counter, sh, &t)) out2[0] = t;
    __syncthreads();
    if (grid_reduce(b, partials + kMaxPartials / 2, counter + 1, sh, &t)) out2[1] = t;
}

// mean over unknowns of x, subtracted at every cell with an unknown (all-Neumann problems)
__global__ void k_sum_unknowns(long long n, const double* __restrict__ x, const int32_t* __restrict__ root,
                               double* __restrict__ partials, unsigned int* __restrict__ counter, double* out) {
    __shared__ double sh[32];
    double a = 0.0;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x)
        if (root[c] == (int32_t)c) a += x[c];
    double t;
    if (grid_reduce(a, partials, counter, sh, &t)) *out = t;
}

__global__ void k_set_pq_inf(CgScalars* sc, int timing) {
    sc->pq_raw = INFINITY;
    sc->pq_corr = 0.0;
    sc->alpha = 0.0;
    sc->beta = 0.0;
    sc->timing = timing;
}

// v_m = sum over the group of v, written to every cell of the group
__global__ void k_group_fold_d(int ng, const int* __restrict__ gptr, const int* __restrict__ gcells,
                               double* __restrict__ v) {
    int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= ng) return;
    double sum = 0.0;
    for (int t = gptr[g]; t < gptr[g + 1]; ++t) sum += v[gcells[t]];
    for (int t = gptr[g]; t < gptr[g + 1]; ++t) v[gcells[t]] = sum;
}

// ---- mixed precision ----------------------------------------------------------------------
// Outer step of iterative refinement: r = bt - q (q = scaled A x_t, FP64), true residual check,
// and the FP32 right-hand side of the next inner solve, normalised to unit norm.
__global__ void k_outer_residual(long long n, const double* __restrict__ bt, const double* __restrict__ q,
                                 const double* __restrict__ sq, const uint32_t* __restrict__ bits,
                                 double* __restrict__ r, CgScalars* sc, double* __restrict__ partials,
                                 unsigned int* __restrict__ counter, cudaGraphConditionalHandle h_outer,
                                 cudaGraphConditionalHandle h_inner, int use_handles) {
    __shared__ double sh[32];
    double a = 0.0, b = 0.0;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x) {
        const double v = bt[c] - q[c];
        r[c] = v;
        if (!is_slave(bits, c)) {
            a = fma(v, v, a);
            const double u = v * sq[c];
            b = fma(u, u, b);
        }
    }
    double t;
    if (grid_reduce(a, partials, counter, sh, &t)) sc->rr0 = t;   // scaled residual norm^2
    __syncthreads();
    if (grid_reduce(b, partials + kMaxPartials / 2, counter + 1, sh, &t)) {
        sc->rnorm2 = t;
        bool stop = false;
        if (!isfinite(t) || sc->status != VOFP_OK) {
            if (sc->status == VOFP_OK) sc->status = VOFP_ERR_BREAKDOWN;
            stop = true;
        } else if (t <= sc->rtol * sc->rtol * sc->ref2) {
            stop = true;
        } else if (sc->iter_total >= sc->max_iter || sc->outer >= 200) {
            sc->status = VOFP_ERR_NOT_CONVERGED;
            stop = true;
        }
        sc->done = stop ? 1 : 0;
        if (!stop) sc->outer += 1;
        if (use_handles) {
            cudaGraphSetConditional(h_outer, stop ? 0u : 1u);
            cudaGraphSetConditional(h_inner, stop ? 0u : 1u);
        }
    }
}

// Inner start: rf = r / ||r||, x_f = 0, rr = rf.rf (Dot2-accumulated).  Restarted refinement:
// p_f(old) = 0, so the inner CG starts from p = rf.  Refinement that keeps the direction (a
// "reliable update" of the residual, Sleijpen and van der Vorst 1996): the FP64 residual replaces
// the recursively updated FP32 one, and the next direction is p = r_new + beta p_old with
// beta = ||r_new||^2 / r_k.r_k (r_k: the residual of the last step length), the old direction
// being rescaled from the old to the new inner units (factor scale_old / scale_new) inside beta.
__global__ void k_inner_prep(long long n, const double* __restrict__ r, const uint32_t* __restrict__ bits,
                             float* __restrict__ rf, float* __restrict__ xf, float* __restrict__ pf0,
                             CgScalars* sc, double* __restrict__ partials, unsigned int* __restrict__ counter) {
    __shared__ double sh[32];
    const double rr = sc->rr0;
    const double inv = (rr > 0.0 && !sc->done) ? 1.0 / sqrt(rr) : 0.0;
    const bool keep = sc->keep_dir && sc->dir_valid;
    AccF2 acc;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x) {
        const float v = (float)(r[c] * inv);
        rf[c] = v;
        xf[c] = 0.0f;
        if (!keep) pf0[c] = 0.0f;
        if (!is_slave(bits, c)) acc.add(v, v);
    }
    double t;
    if (grid_reduce(acc.value(), partials, counter, sh, &t)) inner_start_scalars(sc, t, rr, keep);
}

// end of an inner solve: x_f += alpha p_f (pending), x_t += ||r|| * x_f in FP64
__global__ void k_inner_finish(long long n, float* __restrict__ xf, const float* __restrict__ pf,
                               double* __restrict__ xt, const CgScalars* sc) {
    const float alpha = (float)sc->alpha;
    const double scale = sc->scale;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x) {
        const float v = __fmaf_rn(alpha, pf[c], xf[c]);
        xt[c] = fma(scale, (double)v, xt[c]);
    }
}

// dst = a + b at cells outside the red set, 0 at red cells; ||dst||^2 over cells outside `excl`
// to sc->rr0 (the reduced right-hand side of a red-black inner solve and its norm)
__global__ void k_reduced_rhs(long long n, const double* __restrict__ a, const double* __restrict__ b,
                              const uint32_t* __restrict__ red, const uint32_t* __restrict__ excl,
                              double* __restrict__ dst, CgScalars* sc, double* __restrict__ partials,
                              unsigned int* __restrict__ counter, int norm) {
    __shared__ double sh[32];
    double acc = 0.0;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x) {
        const double v = is_slave(red, c) ? 0.0 : a[c] + b[c];
        dst[c] = v;
        if (!is_slave(excl, c)) acc = fma(v, v, acc);
    }
    if (norm) {
        double t;
        if (grid_reduce(acc, partials, counter, sh, &t)) sc->rr0 = t;
    }
}

// x = s * x_t at every cell (after the red unknowns are reconstructed)
__global__ void k_unscale(long long n, const double* __restrict__ xt, const double* __restrict__ s,
                          double* __restrict__ xout) {
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x)
        xout[c] = s[c] * xt[c];
}

// end of a red-black inner solve: x_f += alpha p_f at every cell (red entries of p_f are 0)
__global__ void k_inner_xf(long long n, float* __restrict__ xf, const float* __restrict__ pf, const CgScalars* sc) {
    const float alpha = (float)sc->alpha;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x)
        xf[c] = __fmaf_rn(alpha, pf[c], xf[c]);
}

// correction d of A d = r from the reduced solution: d_S = scale x_f, d_R = r_R + scale E_RS x_f
// (FP64 coefficients); x_t += d
__global__ void __launch_bounds__(kRedThreads)
k_inner_finish_rb(const Dims d, const double* __restrict__ Tx, const double* __restrict__ Ty,
                  const double* __restrict__ Tz, const uint32_t* __restrict__ red, const float* __restrict__ xf,
                  const double* __restrict__ r, double* __restrict__ xt, const CgScalars* sc) {
    const double scale = sc->scale;
    const long long rows = (long long)d.ny * d.nz;
    for (long long row = blockIdx.y; row < rows; row += gridDim.y) {
        const int j = int(row % d.ny), k = int(row / d.ny);
        for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < d.nx; i += gridDim.x * blockDim.x) {
            const long long c = i + (long long)d.nx * row;
            if (!is_slave(red, c)) {
                xt[c] = fma(scale, (double)xf[c], xt[c]);
                continue;
            }
            double acc = 0.0;
            if (i > 0) acc = fma(Tx[c - 1], (double)xf[c - 1], acc);
            if (i < d.nx - 1) acc = fma(Tx[c], (double)xf[c + 1], acc);
            if (j > 0) acc = fma(Ty[c - d.nx], (double)xf[c - d.nx], acc);
            if (j < d.ny - 1) acc = fma(Ty[c], (double)xf[c + d.nx], acc);
            if (k > 0) acc = fma(Tz[c - d.plane], (double)xf[c - d.plane], acc);
            if (k < d.nz - 1) acc = fma(Tz[c], (double)xf[c + d.plane], acc);
            if (scale > 0.0) xt[c] += r[c] + scale * acc;
        }
    }
}

// The same with one thread per x pair of cells (nx even): a pair holds one cell of each parity,
// so every thread takes both branches in the same order and no warp splits on the colour; the
// arithmetic of each cell is the same as above (bitwise the same result).
__global__ void __launch_bounds__(kRedThreads)
k_inner_finish_rb_pairs(const Dims d, const double* __restrict__ Tx, const double* __restrict__ Ty,
                        const double* __restrict__ Tz, const uint32_t* __restrict__ red, const float* __restrict__ xf,
                        const double* __restrict__ r, double* __restrict__ xt, const CgScalars* sc) {
    const double scale = sc->scale;
    const long long rows = (long long)d.ny * d.nz;
    const int nh = d.nx >> 1;
    for (long long row = blockIdx.y; row < rows; row += gridDim.y) {
        const int j = int(row % d.ny), k = int(row / d.ny);
        for (int h = blockIdx.x * blockDim.x + threadIdx.x; h < nh; h += gridDim.x * blockDim.x) {
            const long long c0 = 2LL * h + (long long)d.nx * row;
            const double2 xt2 = *reinterpret_cast<const double2*>(xt + c0);
            const float2 xf2 = *reinterpret_cast<const float2*>(xf + c0);
            double out[2] = {xt2.x, xt2.y};
            const float own[2] = {xf2.x, xf2.y};
#pragma unroll
            for (int u = 0; u < 2; ++u) {
                const long long c = c0 + u;
                const int i = 2 * h + u;
                if (!is_slave(red, c)) {
                    out[u] = fma(scale, (double)own[u], out[u]);
                    continue;
                }
                double acc = 0.0;
                if (i > 0) acc = fma(Tx[c - 1], (double)xf[c - 1], acc);
                if (i < d.nx - 1) acc = fma(Tx[c], (double)xf[c + 1], acc);
                if (j > 0) acc = fma(Ty[c - d.nx], (double)xf[c - d.nx], acc);
                if (j < d.ny - 1) acc = fma(Ty[c], (double)xf[c + d.nx], acc);
                if (k > 0) acc = fma(Tz[c - d.plane], (double)xf[c - d.plane], acc);
                if (k < d.nz - 1) acc = fma(Tz[c], (double)xf[c + d.plane], acc);
                if (scale > 0.0) out[u] += r[c] + scale * acc;
            }
            *reinterpret_cast<double2*>(xt + c0) = make_double2(out[0], out[1]);
        }
    }
}

dim3 rows_grid(const vofp_ctx* c, int threads) {
    const long long rows = (long long)c->d.ny * c->d.nz;
    const int gx = ceil_div(c->d.nx, threads);
    return dim3(gx, (unsigned)std::max(1LL, std::min(rows, (long long)num_sms() * 32)));
}

// ---- flexible CG with the learned preconditioner -----------------------------------------
// FCG(1) (Notay 2000): each direction is made A-orthogonal to the previous one, which keeps CG's
// short recurrence valid for a preconditioner that changes from one application to the next.
// Every scalar lives in device memory; the kernels of one iteration read what the previous one
// wrote, so the inner loop runs as a CUDA graph with no host round trip.
constexpr int kFcgHist = 64;
struct FcgScalars {
    double zq;               // z . q_prev
    double pq, pr;           // p . q and p . r of the current iteration
    double pq_prev;
    double rr, rr0;          // r . r now and at the start of the inner solve
    double target2;          // the inner solve stops at rr <= target2 rr0
    double alpha, beta;
    long long k;             // iterations of the current inner solve
    long long total;         // iterations of the whole solve
    long long max_total;
    int window;              // stagnation window (iterations)
    double stag2;            // the residual must fall to stag2 (ratio squared) of rr `window` iterations before
    int done;                // inner solve finished
    int fell_back;           // stagnation, breakdown or a non-finite value
    double hist[kFcgHist];   // rr of the last iterations (ring)
};

// r_f = r * inv (FP32), x_f = 0, r_f.r_f; the inner solve's scalars
__global__ void __launch_bounds__(kNT)
k_fcg_start(long long n, const double* __restrict__ r, double inv, float* __restrict__ rf, float* __restrict__ xf,
            const uint32_t* __restrict__ bits, double* __restrict__ partials, unsigned int* __restrict__ counter,
            FcgScalars* fs, double target2, long long max_total, int window, double stag2) {
    __shared__ double sh[32];
    AccF2 acc;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x) {
        const float v = (float)(r[c] * inv);
        rf[c] = v;
        xf[c] = 0.0f;
        if (!is_slave(bits, c)) acc.add(v, v);
    }
    double t;
    if (grid_reduce(acc.value(), partials, counter, sh, &t)) {
        fs->rr = fs->rr0 = t;
        fs->target2 = target2;
        fs->k = 0;
        fs->max_total = max_total;
        fs->window = window;
        fs->stag2 = stag2;
        fs->done = (fs->total >= max_total || !(t > 0.0)) ? 1 : 0;
        fs->fell_back = 0;
        fs->pq_prev = 0.0;
        fs->beta = 0.0;
    }
}

// beta = -(z . q_prev) / (p_prev . q_prev) (0 on the first iteration)
__global__ void __launch_bounds__(kNT)
k_fcg_beta(long long n, const float* __restrict__ z, const float* __restrict__ qp, const uint32_t* __restrict__ bits,
           double* __restrict__ partials, unsigned int* __restrict__ counter, FcgScalars* fs) {
    __shared__ double sh[32];
    if (fs->done || fs->k == 0) {
        if (blockIdx.x == 0 && threadIdx.x == 0 && !fs->done) fs->beta = 0.0;
        return;
    }
    AccF2 acc;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x)
        if (!is_slave(bits, c)) acc.add(z[c], qp[c]);
    double t;
    if (grid_reduce(acc.value(), partials, counter, sh, &t)) {
        fs->zq = t;
        fs->beta = -t / fs->pq_prev;
    }
}

// p = z + beta p_prev (p = z on the first iteration: p_prev holds no direction of this solve)
__global__ void k_fcg_dir(long long n, const float* __restrict__ z, const float* __restrict__ pp,
                          float* __restrict__ p, const FcgScalars* fs) {
    if (fs->done) return;
    const bool first = fs->k == 0;
    const float beta = (float)fs->beta;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x)
        p[c] = first ? z[c] : __fmaf_rn(beta, pp[c], z[c]);
}

// p . q and p . r; alpha = p.r / p.q, or a breakdown
__global__ void __launch_bounds__(kNT)
k_fcg_dots(long long n, const float* __restrict__ p, const float* __restrict__ q, const float* __restrict__ r,
           const uint32_t* __restrict__ bits, double* __restrict__ partials, unsigned int* __restrict__ counter,
           FcgScalars* fs) {
    __shared__ double sh[32];
    if (fs->done) return;
    AccF2 a, b;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x) {
        if (is_slave(bits, c)) continue;
        a.add(p[c], q[c]);
        b.add(p[c], r[c]);
    }
    double t;
    if (grid_reduce(a.value(), partials, counter, sh, &t)) fs->pq = t;
    __syncthreads();
    if (grid_reduce(b.value(), partials + kMaxPartials / 2, counter + 1, sh, &t)) {
        fs->pr = t;
        const double pq = fs->pq;
        if (!(pq > 0.0) || !isfinite(pq) || !isfinite(t)) {
            fs->fell_back = 1;
            fs->done = 1;
        } else {
            fs->alpha = t / pq;
        }
    }
}

// x += alpha p, r -= alpha q, r.r; convergence, stagnation (residual norm down by less than 10 %
// over `window` iterations) and the iteration cap end the inner loop
__global__ void __launch_bounds__(kNT)
k_fcg_update(long long n, const float* __restrict__ p, const float* __restrict__ q, float* __restrict__ x,
             float* __restrict__ r, const uint32_t* __restrict__ bits, double* __restrict__ partials,
             unsigned int* __restrict__ counter, FcgScalars* fs, cudaGraphConditionalHandle h, int use_h) {
    __shared__ double sh[32];
    if (fs->done) {
        if (use_h && blockIdx.x == 0 && threadIdx.x == 0) cudaGraphSetConditional(h, 0u);
        return;
    }
    const float alpha = (float)fs->alpha;
    AccF2 acc;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x) {
        x[c] = __fmaf_rn(alpha, p[c], x[c]);
        const float v = __fmaf_rn(-alpha, q[c], r[c]);
        r[c] = v;
        if (!is_slave(bits, c)) acc.add(v, v);
    }
    double t;
    if (grid_reduce(acc.value(), partials, counter, sh, &t)) {
        fs->rr = t;
        fs->pq_prev = fs->pq;
        const long long k = fs->k;
        fs->k = k + 1;
        fs->total += 1;
        int done = 0;
        if (!isfinite(t)) {
            fs->fell_back = 1;
            done = 1;
        } else if (t <= fs->target2 * fs->rr0 || fs->total >= fs->max_total) {
            done = 1;
        } else if (k + 1 >= fs->window && !(t < fs->stag2 * fs->hist[(k + 1 - fs->window) % kFcgHist])) {
            fs->fell_back = 1;
            done = 1;
        }
        fs->hist[(k + 1) % kFcgHist] = t;
        if (k == 0) fs->hist[0] = fs->rr0;
        fs->done = done;
        if (use_h) cudaGraphSetConditional(h, done ? 0u : 1u);
    }
}

// Relative A-norm error of a network output z against the exact error e of the residual r
// (A e = r): L = (z - e)' A (z - e) / (e' A e) = (z'q - 2 z'r + e'r) / e'r with q = A z, over the
// unknowns (cells in no other cell's group).  out[0..2] = z'q, z'r, e'r.
__global__ void __launch_bounds__(kNT)
k_anorm_dots(long long n, const float* __restrict__ z, const float* __restrict__ q, const float* __restrict__ r,
             const float* __restrict__ e, const uint32_t* __restrict__ bits, double* __restrict__ partials,
             unsigned int* __restrict__ counter, double* out) {
    __shared__ double sh[32];
    AccF2 a, b, c2;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x) {
        if (is_slave(bits, c)) continue;
        a.add(z[c], q[c]);
        b.add(z[c], r[c]);
        c2.add(e[c], r[c]);
    }
    double t;
    if (grid_reduce(a.value(), partials, counter, sh, &t)) out[0] = t;
    __syncthreads();
    if (grid_reduce(b.value(), partials + kMaxPartials / 4, counter + 1, sh, &t)) out[1] = t;
    __syncthreads();
    if (grid_reduce(c2.value(), partials + kMaxPartials / 2, counter + 2, sh, &t)) out[2] = t;
}
// dL/dz = 2 (q - r) / e'r at the unknowns, 0 at the other cells of a group (their output is
// replaced by the master's)
__global__ void k_anorm_grad(long long n, const float* __restrict__ q, const float* __restrict__ r,
                             const uint32_t* __restrict__ bits, const double* sums, float* __restrict__ dz) {
    const double er = sums[2];
    const float f = er > 0.0 ? (float)(2.0 / er) : 0.0f;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x)
        dz[c] = is_slave(bits, c) ? 0.0f : f * (q[c] - r[c]);
}
__global__ void k_copy_f(long long n, const float* __restrict__ a, float* __restrict__ b) {
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x)
        b[c] = a[c];
}

// x_t += scale * x_f (FP64)
__global__ void k_ffold(long long n, const float* __restrict__ xf, double scale, double* __restrict__ xt) {
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x)
        xt[c] = fma(scale, (double)xf[c], xt[c]);
}

// every cell of a merge group takes its master's value (FP32)
__global__ void k_group_expand_f(int ng, const int* __restrict__ gptr, const int* __restrict__ gcells,
                                 float* __restrict__ v) {
    int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= ng) return;
    const float vm = v[gcells[gptr[g]]];
    for (int t = gptr[g] + 1; t < gptr[g + 1]; ++t) v[gcells[t]] = vm;
}

__global__ void k_to_float(long long n, const double* __restrict__ a, float* __restrict__ b) {
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x)
        b[c] = (float)a[c];
}

}  // namespace

// ---- launch helpers --------------------------------------------------------------------------

void launch_stencil_apply_unscaled(vofp_ctx* c, const double* x, double* t) {
    launch(c, k_stencil<double, ST_APPLY_UNSCALED, 1>, stencil_grid(c), dim3(kBX, kBY), c->stream, 
        c->d, stencil_per_block(c), c->Tx, c->Ty, c->Tz, c->diag, x, nullptr, nullptr, nullptr, t, c->sc, c->partials, c->counters);
}

void launch_stencil_apply_scaled(vofp_ctx* c, const double* x, double* t) {
    launch(c, k_stencil<double, ST_APPLY_SCALED, 1>, stencil_grid(c), dim3(kBX, kBY), c->stream, 
        c->d, stencil_per_block(c), c->Txs, c->Tys, c->Tzs, nullptr, x, nullptr, nullptr, nullptr, t, c->sc, c->partials, c->counters);
}

template <typename V>
void launch_group_patch(vofp_ctx* c, V* t, const V* p, bool dot) {
    if (c->ngroups == 0) return;
    launch(c, k_group_patch<V>, ceil_div(c->ngroups, kNT), kNT, c->stream, c->ngroups, c->gptr, c->gcells, c->gcorr, t, p,
                                                                        dot ? 1 : 0, c->sc, c->partials, c->counters);
}
template void launch_group_patch<double>(vofp_ctx*, double*, const double*, bool);
template void launch_group_patch<float>(vofp_ctx*, float*, const float*, bool);

namespace {

// one CG iteration on stream st (FP64 or FP32), reading p_old from `po` and writing `pn`; in
// red-black mode the red half-stencil runs first and the stencil skips red rows
template <typename V>
void launch_cg_iteration(vofp_ctx* c, cudaStream_t st, V* r, V* po, V* pn, V* xv, V* q,
                         const V* Tx, const V* Ty, const V* Tz, bool inner, bool rb,
                         cudaGraphConditionalHandle h, int use_h) {
    const uint32_t* bits = rb ? c->excl_bits : c->slave_bits;
    if (rb) {
        launch_cg_rb<V>(c, st, Tx, Ty, Tz, r, po, pn, xv, q);
    } else {
        launch_cg_stencil<V>(c, st, Tx, Ty, Tz, r, po, pn, xv, q);
    }
    if (c->ngroups > 0)
        launch(c, k_group_patch<V>, ceil_div(c->ngroups, kNT), kNT, st, c->ngroups, c->gptr, c->gcells, c->gcorr, q, pn,
               1, c->sc, c->partials, c->counters);
    if (inner)
        launch(c, k_cg_update<V, true>, stream_grid(c->d.n / (sizeof(V) == 8 ? 2 : 4) + 1), kNT, st,
               c->d.n, r, (const V*)q, bits, c->sc, c->partials, c->counters, h, use_h, (const double*)nullptr, 0);
    else
        launch(c, k_cg_update<V, false>, stream_grid(c->d.n / (sizeof(V) == 8 ? 2 : 4) + 1), kNT, st,
               c->d.n, r, (const V*)q, bits, c->sc, c->partials, c->counters, h, use_h, (const double*)nullptr, 0);
}

// kernels of one iteration (for the launch count of graph executions)
int iteration_kernels(const vofp_ctx* c, bool rb) {
    (void)rb;
    return 2 + (c->ngroups > 0 ? 1 : 0);
}

// Mixed precision, red-black: the reduced right-hand side r_S + E_SR r_R of the correction
// equation (folded over merge groups) into c->q, its norm into sc->rr0.
// k_rb_gather with to_red = 0 and no base, one thread per x pair of cells (nx even; bitwise the
// same): dst_c = sum over the red neighbours of T_f src_nb for non-red cells, 0 at red cells
__global__ void __launch_bounds__(kRedThreads)
k_rb_gather_pairs(const Dims d, const double* __restrict__ Tx, const double* __restrict__ Ty,
                  const double* __restrict__ Tz, const uint32_t* __restrict__ red, const double* __restrict__ src,
                  double* __restrict__ dst) {
    const long long rows = (long long)d.ny * d.nz;
    const int nh = d.nx >> 1;
    auto is_red = [&](long long c) { return (red[c >> 5] >> (c & 31)) & 1u; };
    for (long long row = blockIdx.y; row < rows; row += gridDim.y) {
        const int j = int(row % d.ny), k = int(row / d.ny);
        for (int h = blockIdx.x * blockDim.x + threadIdx.x; h < nh; h += gridDim.x * blockDim.x) {
            const long long c0 = 2LL * h + (long long)d.nx * row;
            double out[2];
#pragma unroll
            for (int u = 0; u < 2; ++u) {
                const long long c = c0 + u;
                const int i = 2 * h + u;
                if (is_red(c)) {
                    out[u] = 0.0;
                    continue;
                }
                double acc = 0.0;
                auto term = [&](long long n, double T) {
                    if (is_red(n)) acc = fma(T, src[n], acc);
                };
                if (i > 0) term(c - 1, Tx[c - 1]);
                if (i < d.nx - 1) term(c + 1, Tx[c]);
                if (j > 0) term(c - d.nx, Ty[c - d.nx]);
                if (j < d.ny - 1) term(c + d.nx, Ty[c]);
                if (k > 0) term(c - d.plane, Tz[c - d.plane]);
                if (k < d.nz - 1) term(c + d.plane, Tz[c]);
                out[u] = acc;
            }
            *reinterpret_cast<double2*>(dst + c0) = make_double2(out[0], out[1]);
        }
    }
}

void launch_reduced_rhs(vofp_ctx* c, cudaStream_t st) {
    if (c->d.nx % 2 == 0)
        launch(c, k_rb_gather_pairs, rows_grid(c, 2 * kNT), dim3(kNT), st, c->d, (const double*)c->Txs,
               (const double*)c->Tys, (const double*)c->Tzs, (const uint32_t*)c->red_bits, (const double*)c->r, c->q);
    else
        launch(c, k_rb_gather, rows_grid(c, kNT), dim3(kNT), st, c->d, (const double*)c->Txs, (const double*)c->Tys,
               (const double*)c->Tzs, (const uint32_t*)c->red_bits, (const double*)c->r, (const double*)nullptr, c->q,
               0);
    if (c->ngroups > 0)
        launch(c, k_group_fold_d, ceil_div(c->ngroups, kNT), kNT, st, c->ngroups, (const int*)c->gptr,
               (const int*)c->gcells, c->q);
    launch(c, k_reduced_rhs, stream_grid(c->d.n), kNT, st, c->d.n, (const double*)c->r, (const double*)c->q,
           (const uint32_t*)c->red_bits, (const uint32_t*)c->excl_bits, c->q, c->sc, c->partials, c->counters, 1);
}

vofp_status ensure_workspace(vofp_ctx* c) {
    if (c->xt) return VOFP_OK;
    const long long N = c->d.n;
    vofp_status s;
    if ((s = c->alloc(&c->xt, N)) || (s = c->alloc(&c->r, N)) || (s = c->alloc(&c->p0, N)) ||
        (s = c->alloc(&c->p1, N)) || (s = c->alloc(&c->q, N)) || (s = c->alloc(&c->bt, N)) ||
        (s = c->alloc(&c->rf, N)) || (s = c->alloc(&c->pf0, N)) || (s = c->alloc(&c->pf1, N)) ||
        (s = c->alloc(&c->qf, N)) || (s = c->alloc(&c->xf, N)))
        return s;
    VOFP_CUDA_TRY(c, cudaEventCreate(&c->ev0));
    VOFP_CUDA_TRY(c, cudaEventCreate(&c->ev1));
    return VOFP_OK;
}

// capture `fn` (launches on stream cs) into the body graph of a WHILE node
template <typename F>
vofp_status capture_into(vofp_ctx* c, cudaStream_t cs, cudaGraph_t body, F fn) {
    VOFP_CUDA_TRY(c, cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
    fn();
    cudaGraph_t out = body;
    VOFP_CUDA_TRY(c, cudaStreamEndCapture(cs, &out));
    return VOFP_OK;
}

vofp_status add_while(vofp_ctx* c, cudaGraph_t g, cudaGraphConditionalHandle* h, cudaGraph_t* body,
                      const cudaGraphNode_t* deps, size_t ndeps, cudaGraphNode_t* node, unsigned int dflt) {
    VOFP_CUDA_TRY(c, cudaGraphConditionalHandleCreate(h, g, dflt, cudaGraphCondAssignDefault));
    cudaGraphNodeParams prm = {};
    prm.type = cudaGraphNodeTypeConditional;
    prm.conditional.handle = *h;
    prm.conditional.type = cudaGraphCondTypeWhile;
    prm.conditional.size = 1;
    VOFP_CUDA_TRY(c, cudaGraphAddNode(node, g, deps, nullptr, ndeps, &prm));
    *body = prm.conditional.phGraph_out[0];
    return VOFP_OK;
}

// Launch sequences shared by the graph capture and the host-driven loop.
// FP64 body: U iterations, then the true-residual check (sets the WHILE condition).
void launch_fp64_body(vofp_ctx* c, cudaStream_t st, int U, bool rb, cudaGraphConditionalHandle h, int use_h) {
    for (int u = 0; u < U; ++u) {
        double* po = (u % 2 == 0) ? c->p0 : c->p1;
        double* pn = (u % 2 == 0) ? c->p1 : c->p0;
        launch_cg_iteration<double>(c, st, c->r, po, pn, c->xt, c->q, c->Txs, c->Tys, c->Tzs, false, rb, h, 0);
    }
    launch(c, k_cg_check<double>, stream_grid(c->d.n), kNT, st, c->d.n, (const double*)c->r, (const double*)c->sq,
           (const uint32_t*)(rb ? c->excl_bits : c->slave_bits), c->sc, c->partials, c->counters, h, use_h);
}
int fp64_body_kernels(const vofp_ctx* c, int U, bool rb) { return U * iteration_kernels(c, rb) + 1; }

// Mixed outer step, first part: FP64 residual of the full system, outer test, inner right-hand side.
void launch_outer_head(vofp_ctx* c, cudaStream_t st, bool rb, cudaGraphConditionalHandle ho,
                       cudaGraphConditionalHandle hi, int use_h) {
    launch(c, k_stencil<double, ST_APPLY_SCALED, 1>, stencil_grid(c), dim3(kBX, kBY), st, c->d, stencil_per_block(c),
           (const double*)c->Txs, (const double*)c->Tys, (const double*)c->Tzs, (const double*)nullptr,
           (const double*)c->xt, (const double*)nullptr, (double*)nullptr, (double*)nullptr, c->q, c->sc, c->partials,
           c->counters);
    if (c->ngroups > 0)
        launch(c, k_group_patch<double>, ceil_div(c->ngroups, kNT), kNT, st, c->ngroups, (const int*)c->gptr,
               (const int*)c->gcells, (const double*)c->gcorr, c->q, (const double*)c->xt, 0, c->sc, c->partials,
               c->counters);
    launch(c, k_outer_residual, stream_grid(c->d.n), kNT, st, c->d.n, (const double*)c->bt, (const double*)c->q,
           (const double*)c->sq, (const uint32_t*)c->slave_bits, c->r, c->sc, c->partials, c->counters, ho, hi, use_h);
    if (rb) {
        launch_reduced_rhs(c, st);
        if (c->rbc_ok)
            rbc_prep(c, st, c->q);
        else
            launch(c, k_inner_prep, stream_grid(c->d.n), kNT, st, c->d.n, (const double*)c->q,
                   (const uint32_t*)c->excl_bits, c->rf, c->xf, c->pf0, c->sc, c->partials, c->counters);
    } else {
        launch(c, k_inner_prep, stream_grid(c->d.n), kNT, st, c->d.n, (const double*)c->r,
               (const uint32_t*)c->slave_bits, c->rf, c->xf, c->pf0, c->sc, c->partials, c->counters);
    }
}
int outer_head_kernels(const vofp_ctx* c, bool rb) {
    const int g = c->ngroups > 0 ? 1 : 0;
    return 1 + g + 1 + (rb ? 2 + g : 0) + 1;
}
void launch_inner_body(vofp_ctx* c, cudaStream_t st, int U, bool rb, cudaGraphConditionalHandle hi, int use_h) {
    if (rb && c->rbc_ok) {
        for (int u = 0; u < U; ++u)
            rbc_iteration(c, st, (u % 2 == 0) ? c->rbc_p0 : c->rbc_p1, (u % 2 == 0) ? c->rbc_p1 : c->rbc_p0, hi, use_h);
        return;
    }
    for (int u = 0; u < U; ++u) {
        float* po = (u % 2 == 0) ? c->pf0 : c->pf1;
        float* pn = (u % 2 == 0) ? c->pf1 : c->pf0;
        launch_cg_iteration<float>(c, st, c->rf, po, pn, c->xf, c->qf, c->Txf, c->Tyf, c->Tzf, true, rb, hi, use_h);
    }
}
// Mixed outer step, last part: fold the inner solution into x_t (FP64).
void launch_outer_tail(vofp_ctx* c, cudaStream_t st, bool rb) {
    if (rb) {
        if (c->rbc_ok)
            rbc_finish_xf(c, st);
        else
            launch(c, k_inner_xf, stream_grid(c->d.n), kNT, st, c->d.n, c->xf, (const float*)c->pf0,
                   (const CgScalars*)c->sc);
        if (c->d.nx % 2 == 0)
            launch(c, k_inner_finish_rb_pairs, rows_grid(c, 2 * kNT), dim3(kNT), st, c->d, (const double*)c->Txs,
                   (const double*)c->Tys, (const double*)c->Tzs, (const uint32_t*)c->red_bits, (const float*)c->xf,
                   (const double*)c->r, c->xt, (const CgScalars*)c->sc);
        else
            launch(c, k_inner_finish_rb, rows_grid(c, kNT), dim3(kNT), st, c->d, (const double*)c->Txs,
                   (const double*)c->Tys, (const double*)c->Tzs, (const uint32_t*)c->red_bits, (const float*)c->xf,
                   (const double*)c->r, c->xt, (const CgScalars*)c->sc);
    } else {
        launch(c, k_inner_finish, stream_grid(c->d.n), kNT, st, c->d.n, c->xf, (const float*)c->pf0, c->xt,
               (const CgScalars*)c->sc);
    }
}
int outer_tail_kernels(const vofp_ctx* c, bool rb) {
    return rb ? (c->rbc_ok ? 2 + (c->rbc_ne > 0 ? 1 : 0) : 2) : 1;
}
// kernels of one mixed inner iteration
int inner_iteration_kernels(const vofp_ctx* c, bool rb) {
    if (rb && c->rbc_ok)   // iteration kernel (exception rows inside), fix rows, update
        return 2 + (c->rbc_nf + (c->rbc_gm ? c->ngroups : 0) > 0 ? 1 : 0);
    return iteration_kernels(c, rb);
}

int graph_key(int U, bool rb) { return U * 2 + (rb ? 1 : 0); }

// FP64 loop: WHILE { U x [red half-stencil (RB), stencil, patch, update]; true-residual check }
vofp_status build_graph_fp64(vofp_ctx* c, int U, bool rb) {
    if (c->graph_fp64 && c->graph_fp64_key == graph_key(U, rb)) return VOFP_OK;
    const long long launches0 = c->launches;
    if (c->graph_fp64) {
        cudaGraphExecDestroy(c->graph_fp64);
        c->graph_fp64 = nullptr;
    }
    cudaStream_t cs;
    VOFP_CUDA_TRY(c, cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    cudaGraph_t g;
    VOFP_CUDA_TRY(c, cudaGraphCreate(&g, 0));
    cudaGraphConditionalHandle h;
    cudaGraph_t body;
    cudaGraphNode_t node;
    vofp_status s = add_while(c, g, &h, &body, nullptr, 0, &node, 1u);
    if (s) return s;
    s = capture_into(c, cs, body, [&]() { launch_fp64_body(c, cs, U, rb, h, 1); });
    if (s) return s;
    VOFP_CUDA_TRY(c, cudaGraphInstantiate(&c->graph_fp64, g, 0));
    cudaGraphDestroy(g);
    cudaStreamDestroy(cs);
    c->graph_fp64_key = graph_key(U, rb);
    c->launches = launches0;
    return VOFP_OK;
}

// Mixed: WHILE_outer { FP64 residual, outer test, inner right-hand side (sets both conditions);
//                      WHILE_inner { U x FP32 iterations (inner stop) }; fold the correction }
vofp_status build_graph_mixed_once(vofp_ctx* c, int U, bool rb) {
    const long long launches0 = c->launches;
    if (c->graph_mixed) {
        cudaGraphExecDestroy(c->graph_mixed);
        c->graph_mixed = nullptr;
    }
    cudaStream_t cs;
    VOFP_CUDA_TRY(c, cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    cudaGraph_t g;
    VOFP_CUDA_TRY(c, cudaGraphCreate(&g, 0));
    cudaGraphConditionalHandle ho, hi;
    cudaGraph_t obody, ibody;
    cudaGraphNode_t onode, inode;
    vofp_status s = add_while(c, g, &ho, &obody, nullptr, 0, &onode, 1u);
    if (s) return s;
    cudaGraphNode_t last = nullptr;
    VOFP_CUDA_TRY(c, cudaGraphConditionalHandleCreate(&hi, obody, 1u, cudaGraphCondAssignDefault));
    VOFP_CUDA_TRY(c, cudaStreamBeginCaptureToGraph(cs, obody, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
    launch_outer_head(c, cs, rb, ho, hi, 1);
    {
        cudaGraph_t tmp = obody;
        VOFP_CUDA_TRY(c, cudaStreamEndCapture(cs, &tmp));
    }
    // the node captured last in the outer body is the sink: find it (the graph is a chain)
    {
        size_t nn = 0;
        VOFP_CUDA_TRY(c, cudaGraphGetNodes(obody, nullptr, &nn));
        std::vector<cudaGraphNode_t> nodes(nn);
        VOFP_CUDA_TRY(c, cudaGraphGetNodes(obody, nodes.data(), &nn));
        for (auto nd : nodes) {
            size_t no = 0;
            VOFP_CUDA_TRY(c, cudaGraphNodeGetDependentNodes(nd, nullptr, nullptr, &no));
            if (no == 0) last = nd;
        }
    }
    cudaGraphNodeParams prm = {};
    prm.type = cudaGraphNodeTypeConditional;
    prm.conditional.handle = hi;
    prm.conditional.type = cudaGraphCondTypeWhile;
    prm.conditional.size = 1;
    VOFP_CUDA_TRY(c, cudaGraphAddNode(&inode, obody, &last, nullptr, 1, &prm));
    ibody = prm.conditional.phGraph_out[0];
    s = capture_into(c, cs, ibody, [&]() { launch_inner_body(c, cs, U, rb, hi, 1); });
    if (s) return s;
    VOFP_CUDA_TRY(c, cudaStreamBeginCaptureToGraph(cs, obody, &inode, nullptr, 1, cudaStreamCaptureModeRelaxed));
    launch_outer_tail(c, cs, rb);
    {
        cudaGraph_t tmp = obody;
        VOFP_CUDA_TRY(c, cudaStreamEndCapture(cs, &tmp));
    }
    c->launches = launches0;
    const cudaError_t ie = cudaGraphInstantiate(&c->graph_mixed, g, 0);
    cudaGraphDestroy(g);
    cudaStreamDestroy(cs);
    if (ie != cudaSuccess) {
        c->graph_mixed = nullptr;
        c->set_error(std::string("cudaGraphInstantiate: ") + cudaGetErrorString(ie));
        return VOFP_ERR_CUDA;
    }
    c->graph_mixed_key = graph_key(U, rb);
    return VOFP_OK;
}

// The mixed loop's graph, with the inner iteration's kernels chained by programmatic dependent
// launch where the driver accepts that inside the conditional body; otherwise rebuilt once with
// ordinary edges (and kept so for the context).
vofp_status build_graph_mixed(vofp_ctx* c, int U, bool rb) {
    if (c->graph_mixed && c->graph_mixed_key == graph_key(U, rb)) return VOFP_OK;
    c->launch_err = cudaSuccess;
    const long long launches0 = c->launches;
    vofp_status s = build_graph_mixed_once(c, U, rb);
    if ((s != VOFP_OK || c->launch_err != cudaSuccess) && c->pdl) {
        (void)cudaGetLastError();
        c->launches = launches0;
        if (c->graph_mixed) {
            cudaGraphExecDestroy(c->graph_mixed);
            c->graph_mixed = nullptr;
        }
        c->pdl = 0;
        c->launch_err = cudaSuccess;
        s = build_graph_mixed_once(c, U, rb);
    }
    if (s == VOFP_OK && c->launch_err != cudaSuccess) {
        c->set_error(std::string("kernel launch during capture: ") + cudaGetErrorString(c->launch_err));
        s = VOFP_ERR_CUDA;
    }
    return s;
}

// b_hat (expanded over groups) into c->work, its scaled copy into c->bt; returns sums over
// unknowns of b_hat, |b_hat|, b_hat^2 (host) after optional Neumann projection.
vofp_status prepare_rhs(vofp_ctx* c, const double* b, double* sums3) {
    const long long N = c->d.n;
    cudaStream_t st = c->stream;
    launch(c, k_copy, stream_grid(N), kNT, st, N, b, c->work);
    launch_group_fold(c, c->work, false);
    double* d3 = c->partials + kMaxPartials - 8;
    launch(c, k_bsums, stream_grid(N), kNT, st, N, c->work, c->root, c->partials, c->counters, d3);
    VOFP_CUDA_TRY(c, cudaMemcpyAsync(sums3, d3, 3 * sizeof(double), cudaMemcpyDeviceToHost, st));
    VOFP_CUDA_TRY(c, cudaStreamSynchronize(st));
    if (!c->dirichlet) {
        // all-Neumann: A_hat 1 = 0, so b_hat must sum to zero (integral form, Sec. 2.3)
        if (std::fabs(sums3[0]) > 1e-12 * std::max(sums3[1], 1e-300)) {
            c->set_error("all-Neumann problem: sum of b_hat is not zero");
            return VOFP_ERR_INCOMPATIBLE_RHS;
        }
        double shift = c->n_unknowns > 0 ? sums3[0] / double(c->n_unknowns) : 0.0;
        VOFP_CUDA_TRY(c, cudaMemcpyAsync(d3 + 4, &shift, sizeof(double), cudaMemcpyHostToDevice, st));
        launch(c, k_shift, stream_grid(N), kNT, st, N, c->work, c->root, d3 + 4);
        launch(c, k_bsums, stream_grid(N), kNT, st, N, c->work, c->root, c->partials, c->counters, d3);
        VOFP_CUDA_TRY(c, cudaMemcpyAsync(sums3, d3, 3 * sizeof(double), cudaMemcpyDeviceToHost, st));
        VOFP_CUDA_TRY(c, cudaStreamSynchronize(st));
    }
    launch(c, k_scale, stream_grid(N), kNT, st, N, c->s, c->work, c->bt);
    return VOFP_OK;
}

// The same loops driven from the host: every kernel is an ordinary launch on the context
// stream and the host reads the convergence flags every U iterations.
vofp_status host_loop(vofp_ctx* c, bool mixed, bool rb, int U) {
    cudaStream_t st = c->stream;
    int flags[2] = {0, 0};
    auto read_flags = [&]() -> vofp_status {
        VOFP_CUDA_TRY(c, cudaMemcpyAsync(&flags[0], &c->sc->done, sizeof(int), cudaMemcpyDeviceToHost, st));
        VOFP_CUDA_TRY(c, cudaMemcpyAsync(&flags[1], &c->sc->inner_done, sizeof(int), cudaMemcpyDeviceToHost, st));
        VOFP_CUDA_TRY(c, cudaStreamSynchronize(st));
        return VOFP_OK;
    };
    vofp_status s;
    if (!mixed) {
        for (;;) {
            launch_fp64_body(c, st, U, rb, (cudaGraphConditionalHandle)0, 0);
            if ((s = read_flags())) return s;
            if (flags[0]) return VOFP_OK;
        }
    }
    for (;;) {
        launch_outer_head(c, st, rb, (cudaGraphConditionalHandle)0, (cudaGraphConditionalHandle)0, 0);
        if ((s = read_flags())) return s;
        if (flags[0]) return VOFP_OK;
        for (;;) {
            launch_inner_body(c, st, U, rb, (cudaGraphConditionalHandle)0, 0);
            if ((s = read_flags())) return s;
            if (flags[1]) break;
        }
        launch_outer_tail(c, st, rb);
    }
}

}  // namespace

vofp_status apply_unscaled(vofp_ctx* c, const double* x, double* y) {
    const long long N = c->d.n;
    launch(c, k_expand_gather, stream_grid(N), kNT, c->stream, N, x, c->root, c->work);
    launch_stencil_apply_unscaled(c, c->work, y);
    launch_group_fold(c, y, true);
    VOFP_CUDA_TRY(c, cudaGetLastError());
    return VOFP_OK;
}

// rel = ||b_hat - A_hat x|| / ||b_hat|| with the unscaled operator (x read at masters)
vofp_status residual(vofp_ctx* c, const double* b, const double* x, double* rel) {
    vofp_status s = ensure_workspace(c);
    if (s) return s;
    const long long N = c->d.n;
    cudaStream_t st = c->stream;
    launch(c, k_copy, stream_grid(N), kNT, st, N, b, c->q);
    launch_group_fold(c, c->q, true);
    launch(c, k_expand_gather, stream_grid(N), kNT, st, N, x, c->root, c->work);
    launch_stencil_apply_unscaled(c, c->work, c->p1);
    launch_group_fold(c, c->p1, true);
    double* d2 = c->partials + kMaxPartials - 16;
    launch(c, k_resid_norms, stream_grid(N), kNT, st, N, c->q, c->p1, c->root, c->partials, c->counters, d2);
    double h[2];
    VOFP_CUDA_TRY(c, cudaMemcpyAsync(h, d2, sizeof(h), cudaMemcpyDeviceToHost, st));
    VOFP_CUDA_TRY(c, cudaStreamSynchronize(st));
    *rel = h[1] > 0.0 ? std::sqrt(h[0] / h[1]) : std::sqrt(h[0]);
    return VOFP_OK;
}

namespace {

// The loops stop on a residual that the iteration itself carries (the recursively updated one in
// FP64 mode, an FP64 residual summed in another order in mixed mode), while the contract is on
// the residual recomputed from x at the end.  They aim a little below rtol so that the two agree
// without a restart in the usual case.
constexpr double kLoopMargin = 0.99;
// Mixed-precision refinement aims at half the tolerance: its FP32 inner solves do not minimise the
// error over the whole Krylov space as one FP64 CG does, and at the same residual its iterates
// carry about twice the error (relative L2 error per unit relative residual 175-190 against 80-100
// for FP64 CG on the 512x256x128 hull workload, condition number 3.3e6); at 0.5 rtol its error
// matches an FP64 solve to rtol.
constexpr double kMixedLoopMargin = 0.5;
// Restarts from the current iterate when the recomputed residual is still above rtol; each must
// at least halve it, else the solve reports VOFP_ERR_STAGNATED.
constexpr int kMaxRestarts = 3;

// One pass of the FP64 or mixed-precision solve from x (or 0); fills every field of *info
// (rel_residual recomputed from x) and returns the loop's own status.
vofp_status solve_pass(vofp_ctx* c, const double* b, double* x, const vofp_solve_opts* o, vofp_solve_info* info) {
    vofp_status s = ensure_workspace(c);
    if (s) return s;
    // colour-compact vectors of the red-black inner solve (built once per operator)
    if (o->mode == VOFP_MODE_MIXED && o->precond == VOFP_PRECOND_RBSGS && (s = rbc_ensure(c))) return s;
    const long long N = c->d.n;
    cudaStream_t st = c->stream;
    // Default: the FP64 loop checks its true residual every 8 iterations, and so does the mixed
    // solve's inner loop below 2^20 cells; from 2^20 cells on it tests its stop every 64. An inner
    // solve runs on to the end of its unrolled body past its target, and on large systems, where
    // one takes hundreds of iterations, that overshoot saves refinement steps (512x256x128: 2560
    // iterations in 8 steps, 290 ms, against 2640 in 12, 303 ms, testing every 8). On small ones
    // an inner solve can reach the FP32 rounding floor within 64 iterations, and the steps taken
    // there, kept as the next inner solve's direction, stalled it (a 16^3 sphere, Jacobi: 100032
    // iterations without converging).
    const int U = o->check_every > 0 ? o->check_every : (o->mode == VOFP_MODE_MIXED && N >= (1LL << 20) ? 64 : 8);
    VOFP_CUDA_TRY(c, cudaEventRecord(c->ev0, st));
    double sums[3];
    if ((s = prepare_rhs(c, b, sums))) return s;
    const bool rb = o->precond == VOFP_PRECOND_RBSGS;
    const bool mixed = o->mode == VOFP_MODE_MIXED;
    // red-black vectors keep 0 at red cells that the stencil never writes
    VOFP_CUDA_TRY(c, cudaMemsetAsync(c->p1, 0, sizeof(double) * N, st));
    VOFP_CUDA_TRY(c, cudaMemsetAsync(c->pf1, 0, sizeof(float) * N, st));
    VOFP_CUDA_TRY(c, cudaMemsetAsync(c->qf, 0, sizeof(float) * N, st));
    // scaled initial guess, r = bt - (S A S) x_t
    launch(c, k_init_x, stream_grid(N), kNT, st, N, x, c->root, c->sq, c->xt, o->x0_zero);
    const double* rhs_loop = c->bt;
    if (rb && !mixed) {
        // reduced system: b_S' = b_S + E_SR b_R (folded over groups) into c->work, and
        // S x_t = (I - E)(w) on non-red rows with w = x_t there and w_R = E_RS x_t
        launch(c, k_rb_gather, rows_grid(c, kNT), dim3(kNT), st, c->d, (const double*)c->Txs, (const double*)c->Tys,
               (const double*)c->Tzs, (const uint32_t*)c->red_bits, (const double*)c->bt, (const double*)nullptr,
               c->q, 0);
        if (c->ngroups > 0)
            launch(c, k_group_fold_d, ceil_div(c->ngroups, kNT), kNT, st, c->ngroups, (const int*)c->gptr,
                   (const int*)c->gcells, c->q);
        launch(c, k_reduced_rhs, stream_grid(N), kNT, st, N, (const double*)c->bt, (const double*)c->q,
               (const uint32_t*)c->red_bits, (const uint32_t*)c->excl_bits, c->work, c->sc, c->partials, c->counters,
               0);
        launch(c, k_copy, stream_grid(N), kNT, st, N, (const double*)c->xt, c->p1);
        launch(c, k_rb_gather, rows_grid(c, kNT), dim3(kNT), st, c->d, (const double*)c->Txs, (const double*)c->Tys,
               (const double*)c->Tzs, (const uint32_t*)c->red_bits, (const double*)c->xt, (const double*)nullptr,
               c->p1, 1);
        launch_stencil_apply_scaled(c, c->p1, c->q);
        launch_group_patch<double>(c, c->q, c->xt, false);
        rhs_loop = c->work;
        VOFP_CUDA_TRY(c, cudaMemsetAsync(c->p1, 0, sizeof(double) * N, st));
    } else {
        launch_stencil_apply_scaled(c, c->xt, c->q);
        launch_group_patch<double>(c, c->q, c->xt, false);
    }
    CgScalars h{};
    h.status = VOFP_OK;
    const double rtol_loop = (o->mode == VOFP_MODE_MIXED ? kMixedLoopMargin : kLoopMargin) * o->rtol;
    h.rtol = rtol_loop;
    // default reduction per refinement step: 0.2 when the direction is kept (a frequent FP64
    // residual keeps the FP32 recurrence close to it), 1e-3 for restarted inner solves
    h.inner_rtol = o->inner_rtol > 0 ? o->inner_rtol : (o->inner_restart ? 1e-3 : 0.2);
    h.max_iter = o->max_iter > 0 ? o->max_iter : 100000;
    h.bnorm2 = sums[2];
    h.ref2 = sums[2];
    h.keep_dir = o->inner_restart ? 0 : 1;
    h.dir_valid = 0;
    VOFP_CUDA_TRY(c, cudaMemcpyAsync(c->sc, &h, sizeof(h), cudaMemcpyHostToDevice, st));
    launch(c, k_init_residual, stream_grid(N), kNT, st, N, rhs_loop, (const double*)c->q, (const double*)c->sq,
           (const uint32_t*)((rb && !mixed) ? c->excl_bits : c->slave_bits), c->r, c->sc, c->partials, c->counters);
    VOFP_CUDA_TRY(c, cudaMemsetAsync(c->p0, 0, sizeof(double) * N, st));
    VOFP_CUDA_TRY(c, cudaMemcpyAsync(&h, c->sc, sizeof(h), cudaMemcpyDeviceToHost, st));
    VOFP_CUDA_TRY(c, cudaStreamSynchronize(st));
    if (!std::isfinite(h.rnorm2) || !std::isfinite(h.ref2) || !std::isfinite(h.rr)) {
        // a non-finite right-hand side or initial guess: report, leave x as the scaled guess
        launch(c, k_finalize_x, stream_grid(N), kNT, st, N, c->xt, c->p0, c->s, (const CgScalars*)c->sc, x);
        VOFP_CUDA_TRY(c, cudaStreamSynchronize(st));
        if (info) {
            info->status = VOFP_ERR_BREAKDOWN;
            info->rel_residual = NAN;
        }
        c->set_error("non-finite right-hand side or initial residual");
        return VOFP_ERR_BREAKDOWN;
    }
    const bool converged0 = !(h.rnorm2 > rtol_loop * rtol_loop * h.ref2);
    if (o->host_loop && !converged0) {
        if ((s = host_loop(c, mixed, rb, U))) return s;
    }
    if (mixed) {
        if (!o->host_loop && (s = build_graph_mixed(c, U, rb))) return s;
        if (!converged0 && !o->host_loop) VOFP_CUDA_TRY(c, cudaGraphLaunch(c->graph_mixed, st));
        // the mixed loop folds every inner solution into x_t itself; no pending step
        launch(c, k_set_pq_inf, 1, 1, st, c->sc, 0);
        launch(c, k_finalize_x, stream_grid(N), kNT, st, N, c->xt, (const double*)c->p0, (const double*)c->s,
               (const CgScalars*)c->sc, x);
    } else {
        if (!o->host_loop && (s = build_graph_fp64(c, U, rb))) return s;
        if (!converged0 && !o->host_loop) VOFP_CUDA_TRY(c, cudaGraphLaunch(c->graph_fp64, st));
        launch(c, k_finalize_x, stream_grid(N), kNT, st, N, c->xt, (const double*)c->p0, (const double*)c->s,
               (const CgScalars*)c->sc, x);
        if (rb) {
            // eliminated unknowns: x_R = b_R + E_RS x_S, then unscale every cell
            launch(c, k_rb_gather, rows_grid(c, kNT), dim3(kNT), st, c->d, (const double*)c->Txs,
                   (const double*)c->Tys, (const double*)c->Tzs, (const uint32_t*)c->red_bits, (const double*)c->xt,
                   (const double*)c->bt, c->xt, 1);
            launch(c, k_unscale, stream_grid(N), kNT, st, N, (const double*)c->xt, (const double*)c->s, x);
        }
    }
    if (!c->dirichlet) {
        double* d1 = c->partials + kMaxPartials - 24;
        launch(c, k_sum_unknowns, stream_grid(N), kNT, st, N, x, c->root, c->partials, c->counters, d1);
        double tot = 0.0;
        VOFP_CUDA_TRY(c, cudaMemcpyAsync(&tot, d1, sizeof(double), cudaMemcpyDeviceToHost, st));
        VOFP_CUDA_TRY(c, cudaStreamSynchronize(st));
        double mean = c->n_unknowns > 0 ? tot / double(c->n_unknowns) : 0.0;
        VOFP_CUDA_TRY(c, cudaMemcpyAsync(d1 + 2, &mean, sizeof(double), cudaMemcpyHostToDevice, st));
        launch(c, k_shift, stream_grid(N), kNT, st, N, x, c->root, d1 + 2);
    }
    VOFP_CUDA_TRY(c, cudaEventRecord(c->ev1, st));
    VOFP_CUDA_TRY(c, cudaMemcpyAsync(&h, c->sc, sizeof(h), cudaMemcpyDeviceToHost, st));
    VOFP_CUDA_TRY(c, cudaGetLastError());
    double rel = 0.0;
    if ((s = residual(c, b, x, &rel))) return s;
    float ms = 0.0f;
    VOFP_CUDA_TRY(c, cudaEventElapsedTime(&ms, c->ev0, c->ev1));
    if (!converged0 && !o->host_loop) {
        // kernels executed by the graph: whole bodies of U iterations
        if (mixed)
            c->launches += (long long)(h.outer + 1) * outer_head_kernels(c, rb) +
                           (long long)h.outer * outer_tail_kernels(c, rb) + h.iter_total * inner_iteration_kernels(c, rb);
        else
            c->launches += (h.iter_total / U) * fp64_body_kernels(c, U, rb);
    }
    const vofp_status result = (vofp_status)h.status;
    info->iterations = (int)h.iter_total;
    info->outer_iterations = o->mode == VOFP_MODE_MIXED ? h.outer : 1;
    info->rel_residual = rel;
    info->seconds = ms * 1e-3;
    info->status = result;
    info->nn_applications = 0;
    info->fell_back = 0;
    return result;
}

const char* status_text(vofp_status s) {
    switch (s) {
        case VOFP_ERR_NOT_CONVERGED: return "solve did not reach rtol within max_iter";
        case VOFP_ERR_STAGNATED: return "restarts from the iterate stopped reducing the recomputed residual";
        case VOFP_ERR_BREAKDOWN: return "CG breakdown";
        case VOFP_ERR_DEVICE_TIMEOUT: return "a bounded device-side wait ran out";
        default: return "solve failed";
    }
}

}  // namespace

// The solve of the contract: VOFP_OK only when the residual recomputed from the returned x is at
// most rtol.  A pass that stops with its own residual below rtol but the recomputed one above it
// is restarted from its iterate (a fresh true residual); VOFP_ERR_STAGNATED when a restart fails
// to halve the recomputed residual or kMaxRestarts do not reach rtol, VOFP_ERR_NOT_CONVERGED when
// max_iter runs out first.
vofp_status solve(vofp_ctx* c, const double* b, double* x, const vofp_solve_opts* o, vofp_solve_info* info) {
    prepare_kernels(c);
    if (o->mode == VOFP_MODE_FCG_NN) return solve_fcg(c, b, x, o, info);
    vofp_solve_info acc{};
    vofp_status r = solve_pass(c, b, x, o, &acc);
    const long long max_iter = o->max_iter > 0 ? o->max_iter : 100000;
    for (int restart = 0; r == VOFP_OK && !(acc.rel_residual <= o->rtol); ++restart) {
        if (acc.iterations >= max_iter) {
            r = VOFP_ERR_NOT_CONVERGED;
            break;
        }
        if (restart == kMaxRestarts) {
            r = VOFP_ERR_STAGNATED;
            break;
        }
        vofp_solve_opts o2 = *o;
        o2.x0_zero = 0;
        o2.max_iter = (int)(max_iter - acc.iterations);
        vofp_solve_info i2{};
        const double before = acc.rel_residual;
        r = solve_pass(c, b, x, &o2, &i2);
        acc.iterations += i2.iterations;
        acc.outer_iterations += i2.outer_iterations;
        acc.seconds += i2.seconds;
        acc.rel_residual = i2.rel_residual;
        if (r == VOFP_OK && !(acc.rel_residual <= o->rtol) && !(acc.rel_residual <= 0.5 * before)) {
            r = VOFP_ERR_STAGNATED;
            break;
        }
    }
    acc.status = r;
    if (info) *info = acc;
    if (r != VOFP_OK && c->err.empty()) c->set_error(status_text(r));
    return r;
}

vofp_status scaled_pair(vofp_ctx* c, const double* b, const double* x, float* r_scaled, float* x_scaled) {
    vofp_status s = ensure_workspace(c);
    if (s) return s;
    const long long N = c->d.n;
    cudaStream_t st = c->stream;
    double sums[3];
    if ((s = prepare_rhs(c, b, sums))) return s;
    launch(c, k_to_float, stream_grid(N), kNT, st, N, (const double*)c->bt, r_scaled);
    launch(c, k_init_x, stream_grid(N), kNT, st, N, x, (const int32_t*)c->root, (const double*)c->sq, c->xt, 0);
    launch(c, k_to_float, stream_grid(N), kNT, st, N, (const double*)c->xt, x_scaled);
    VOFP_CUDA_TRY(c, cudaStreamSynchronize(st));
    return VOFP_OK;
}

// FP64 refinement around a flexible CG (FCG(1)) whose preconditioner is the network; the network
// also gives the initial guess (the first step is the optimally scaled x0 = alpha NN(b)).  The
// refinement steps run on the host (a few per solve); each inner solve is one launch of a graph
// whose WHILE body holds two FCG iterations (network forward on this stream, beta, direction,
// operator apply, step length, update with the stop tests), so the inner loop has no host round
// trip.  A stagnating inner solve hands over to mixed-precision PCG from the current iterate.
vofp_status solve_fcg(vofp_ctx* c, const double* b, double* x, const vofp_solve_opts* o, vofp_solve_info* info) {
    vofp_status s = ensure_workspace(c);
    if (s) return s;
    const long long N = c->d.n;
    cudaStream_t st = c->stream;
    if (!c->qf2) {
        if ((s = c->alloc(&c->qf2, N))) return s;
    }
    if (!c->fcg) {
        if ((s = c->alloc(&c->fcg, sizeof(FcgScalars)))) return s;
        VOFP_CUDA_TRY(c, cudaMemsetAsync(c->fcg, 0, sizeof(FcgScalars), st));
    }
    FcgScalars* fs = reinterpret_cast<FcgScalars*>(c->fcg);
    vofp_nn* nn = o->nn;
    if (nn::bound_cells(nn) != N) {
        c->set_error("the network is not bound to this grid (vofp_nn_bind)");
        return VOFP_ERR_INVALID_ARG;
    }
    const int W = std::min(kFcgHist - 1, std::max(1, o->stag_window > 0 ? o->stag_window : 2));
    const double ratio = o->stag_ratio > 0.0 ? o->stag_ratio : 0.6;
    const long long max_iter = o->max_iter > 0 ? o->max_iter : 100000;
    const uint32_t* bits = c->slave_bits;
    // the network's first pass runs before any capture: it sets up its kernels and tensor maps
    if ((s = nn::forward_on(nn, st, c->rf))) {
        c->set_error(std::string("network: ") + vofp_nn_last_error(nn));
        return s;
    }
    float* z = nn::output(nn);
    auto apply_f = [&](cudaStream_t ss, const float* p, float* q) {
        launch(c, k_stencil<float, ST_APPLY_SCALED, 2>, stencil_grid(c), dim3(kBX, kBY), ss, c->d,
               stencil_per_block(c), (const float*)c->Txf, (const float*)c->Tyf, (const float*)c->Tzf,
               (const double*)nullptr, p, (const float*)nullptr, (float*)nullptr, (float*)nullptr, q, c->sc,
               c->partials, c->counters);
        if (c->ngroups > 0)
            launch(c, k_group_patch<float>, ceil_div(c->ngroups, kNT), kNT, ss, c->ngroups, (const int*)c->gptr,
                   (const int*)c->gcells, (const double*)c->gcorr, q, p, 0, c->sc, c->partials, c->counters);
    };
    // one FCG iteration: direction and step into (p, q), previous direction in (pp, qp)
    auto iteration = [&](cudaStream_t ss, float* p, float* q, const float* pp, const float* qp,
                         cudaGraphConditionalHandle h, int use_h) -> vofp_status {
        vofp_status r = nn::forward_on(nn, ss, c->rf);
        if (r) return r;
        if (c->ngroups > 0)
            launch(c, k_group_expand_f, ceil_div(c->ngroups, kNT), kNT, ss, c->ngroups, (const int*)c->gptr,
                   (const int*)c->gcells, z);
        launch(c, k_fcg_beta, stream_grid(N), kNT, ss, N, (const float*)z, qp, bits, c->partials, c->counters, fs);
        launch(c, k_fcg_dir, stream_grid(N), kNT, ss, N, (const float*)z, pp, p, (const FcgScalars*)fs);
        apply_f(ss, p, q);
        launch(c, k_fcg_dots, stream_grid(N), kNT, ss, N, (const float*)p, (const float*)q, (const float*)c->rf, bits,
               c->partials, c->counters, fs);
        launch(c, k_fcg_update, stream_grid(N), kNT, ss, N, (const float*)p, (const float*)q, c->xf, c->rf, bits,
               c->partials, c->counters, fs, h, use_h);
        return VOFP_OK;
    };
    // the inner loop's graph: WHILE { two iterations, the buffers swapping roles }
    cudaGraphExec_t ge = nullptr;
    {
        cudaStream_t cs;
        VOFP_CUDA_TRY(c, cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
        cudaGraph_t g;
        VOFP_CUDA_TRY(c, cudaGraphCreate(&g, 0));
        cudaGraphConditionalHandle h;
        cudaGraph_t body;
        cudaGraphNode_t node;
        const long long launches0 = c->launches;
        if ((s = add_while(c, g, &h, &body, nullptr, 0, &node, 1u))) return s;
        vofp_status r1 = VOFP_OK;
        s = capture_into(c, cs, body, [&]() {
            r1 = iteration(cs, c->pf0, c->qf, c->pf1, c->qf2, h, 1);
            if (!r1) r1 = iteration(cs, c->pf1, c->qf2, c->pf0, c->qf, h, 1);
        });
        c->launches = launches0;
        if (s || r1) {
            cudaGraphDestroy(g);
            cudaStreamDestroy(cs);
            c->set_error(std::string("capturing the flexible-CG loop: ") + vofp_nn_last_error(nn));
            return s ? s : r1;
        }
        const cudaError_t ie = cudaGraphInstantiate(&ge, g, 0);
        cudaGraphDestroy(g);
        cudaStreamDestroy(cs);
        if (ie != cudaSuccess) {
            c->set_error(std::string("cudaGraphInstantiate: ") + cudaGetErrorString(ie));
            return VOFP_ERR_CUDA;
        }
    }
    const int body_kernels = 2 * (nn::forward_kernels(nn) + (c->ngroups > 0 ? 2 : 1) + 5);
    VOFP_CUDA_TRY(c, cudaEventRecord(c->ev0, st));
    double sums[3];
    if ((s = prepare_rhs(c, b, sums))) {
        cudaGraphExecDestroy(ge);
        return s;
    }
    const double bnorm2 = sums[2];
    launch(c, k_init_x, stream_grid(N), kNT, st, N, x, (const int32_t*)c->root, (const double*)c->sq, c->xt,
           o->x0_zero);
    {
        FcgScalars z0{};
        VOFP_CUDA_TRY(c, cudaMemcpyAsync(fs, &z0, sizeof(z0), cudaMemcpyHostToDevice, st));
    }
    long long iters = 0, bodies = 0;
    int outer = 0, fell_back = 0;
    vofp_status result = VOFP_OK;
    for (;;) {
        // FP64 residual of the scaled system and its true (unscaled) norm
        launch_stencil_apply_scaled(c, c->xt, c->q);
        launch_group_patch<double>(c, c->q, c->xt, false);
        CgScalars h{};
        h.status = VOFP_OK;
        VOFP_CUDA_TRY(c, cudaMemcpyAsync(c->sc, &h, sizeof(h), cudaMemcpyHostToDevice, st));
        launch(c, k_init_residual, stream_grid(N), kNT, st, N, (const double*)c->bt, (const double*)c->q,
               (const double*)c->sq, bits, c->r, c->sc, c->partials, c->counters);
        VOFP_CUDA_TRY(c, cudaMemcpyAsync(&h, c->sc, sizeof(h), cudaMemcpyDeviceToHost, st));
        VOFP_CUDA_TRY(c, cudaStreamSynchronize(st));
        const double rnorm2 = h.rnorm2;
        if (!std::isfinite(rnorm2)) {
            result = VOFP_ERR_BREAKDOWN;
            break;
        }
        if (rnorm2 <= kMixedLoopMargin * kMixedLoopMargin * o->rtol * o->rtol * bnorm2) break;
        if (iters >= max_iter || outer >= 200) {
            result = VOFP_ERR_NOT_CONVERGED;
            break;
        }
        ++outer;
        const double scale = std::sqrt(h.rr);
        // each inner solve reduces its residual by inner_rtol (default 1e-3), or to 0.3 of what
        // the outer tolerance still needs, whichever is looser
        const double target = std::max(o->inner_rtol > 0 ? o->inner_rtol : 1e-3,
                                       std::min(0.5, 0.3 * kMixedLoopMargin * o->rtol * std::sqrt(bnorm2 / rnorm2)));
        launch(c, k_fcg_start, stream_grid(N), kNT, st, N, (const double*)c->r, scale > 0 ? 1.0 / scale : 0.0, c->rf,
               c->xf, bits, c->partials, c->counters, fs, target * target, max_iter, W, ratio * ratio);
        VOFP_CUDA_TRY(c, cudaGraphLaunch(ge, st));
        FcgScalars hf{};
        VOFP_CUDA_TRY(c, cudaMemcpyAsync(&hf, fs, sizeof(hf), cudaMemcpyDeviceToHost, st));
        VOFP_CUDA_TRY(c, cudaStreamSynchronize(st));
        iters = hf.total;
        bodies += std::max(1LL, (hf.k + 1) / 2);
        launch(c, k_ffold, stream_grid(N), kNT, st, N, (const float*)c->xf, scale, c->xt);
        if (hf.fell_back) {
            fell_back = 1;
            break;
        }
    }
    c->launches += bodies * body_kernels;
    cudaGraphExecDestroy(ge);
    launch(c, k_unscale, stream_grid(N), kNT, st, N, (const double*)c->xt, (const double*)c->s, x);
    VOFP_CUDA_TRY(c, cudaEventRecord(c->ev1, st));
    VOFP_CUDA_TRY(c, cudaStreamSynchronize(st));
    if ((s = nn::read_device_error(nn))) {
        c->set_error("the network's convolutions reported a bounded wait that ran out");
        return s;
    }
    float ms = 0.0f;
    VOFP_CUDA_TRY(c, cudaEventElapsedTime(&ms, c->ev0, c->ev1));
    int it_total = (int)iters, outer_total = outer;
    double seconds = ms * 1e-3;
    if (fell_back && result == VOFP_OK) {
        // plain mixed-precision PCG from the current iterate
        vofp_solve_opts o2 = *o;
        o2.mode = VOFP_MODE_MIXED;
        o2.x0_zero = 0;
        o2.max_iter = (int)std::max(1LL, max_iter - iters);
        vofp_solve_info i2{};
        result = solve(c, b, x, &o2, &i2);
        it_total += i2.iterations;
        outer_total += i2.outer_iterations;
        seconds += i2.seconds;
    }
    double rel = 0.0;
    if ((s = residual(c, b, x, &rel))) return s;
    if (result == VOFP_OK && !(rel <= o->rtol)) result = VOFP_ERR_NOT_CONVERGED;
    if (info) {
        info->iterations = it_total;
        info->outer_iterations = outer_total;
        info->rel_residual = rel;
        info->seconds = seconds;
        info->status = result;
        info->nn_applications = (int)(2 * bodies + 1);
        info->fell_back = fell_back;
    }
    if (result != VOFP_OK) c->set_error("learned-preconditioner solve did not reach rtol");
    return result;
}

// One training step of the network as a preconditioner of this operator: forward on the scaled
// residual r, q = A_scaled z (FP32, merge groups as in the solve), the relative A-norm error of z
// against the exact error e and its gradient, backward, Adam.
vofp_status nn_train_anorm(vofp_ctx* c, vofp_nn* nn, const float* r, const float* e, float lr, int update,
                           float* loss) {
    vofp_status s = ensure_workspace(c);
    if (s) return s;
    prepare_kernels(c);
    if (nn::bound_cells(nn) != c->d.n) {
        c->set_error("the network is not bound to this grid (vofp_nn_bind or vofp_nn_set_geometry)");
        return VOFP_ERR_INVALID_ARG;
    }
    if (!c->qf2) {
        if ((s = c->alloc(&c->qf2, c->d.n))) return s;
    }
    if ((s = nn::prepare_training(nn))) return s;
    const long long N = c->d.n;
    cudaStream_t st = c->stream;
    if ((s = nn::forward_on(nn, st, r))) {
        c->set_error(std::string("network: ") + vofp_nn_last_error(nn));
        return s;
    }
    float* z = c->pf0;
    launch(c, k_copy_f, stream_grid(N), kNT, st, N, (const float*)nn::output(nn), z);
    if (c->ngroups > 0)
        launch(c, k_group_expand_f, ceil_div(c->ngroups, kNT), kNT, st, c->ngroups, (const int*)c->gptr,
               (const int*)c->gcells, z);
    launch(c, k_stencil<float, ST_APPLY_SCALED, 2>, stencil_grid(c), dim3(kBX, kBY), st, c->d, stencil_per_block(c),
           (const float*)c->Txf, (const float*)c->Tyf, (const float*)c->Tzf, (const double*)nullptr, (const float*)z,
           (const float*)nullptr, (float*)nullptr, (float*)nullptr, c->qf, c->sc, c->partials, c->counters);
    if (c->ngroups > 0)
        launch(c, k_group_patch<float>, ceil_div(c->ngroups, kNT), kNT, st, c->ngroups, (const int*)c->gptr,
               (const int*)c->gcells, (const double*)c->gcorr, c->qf, (const float*)z, 0, c->sc, c->partials,
               c->counters);
    double* sums = c->partials + kMaxPartials - 48;
    launch(c, k_anorm_dots, stream_grid(N), kNT, st, N, (const float*)z, (const float*)c->qf, r, e,
           (const uint32_t*)c->slave_bits, c->partials, c->counters, sums);
    launch(c, k_anorm_grad, stream_grid(N), kNT, st, N, (const float*)c->qf, r, (const uint32_t*)c->slave_bits,
           (const double*)sums, c->qf2);
    if ((s = nn::train_from_grad_on(nn, st, c->qf2, lr, update))) {
        c->set_error(std::string("network: ") + vofp_nn_last_error(nn));
        return s;
    }
    double h[3];
    VOFP_CUDA_TRY(c, cudaMemcpyAsync(h, sums, sizeof(h), cudaMemcpyDeviceToHost, st));
    VOFP_CUDA_TRY(c, cudaStreamSynchronize(st));
    if (loss) *loss = h[2] > 0.0 ? (float)((h[0] - 2.0 * h[1] + h[2]) / h[2]) : 0.0f;
    return VOFP_OK;
}

vofp_status time_iteration_kernels(vofp_ctx* c, int precision, bool rb, int reps, float* stencil_ms,
                                   float* update_ms, float* aux_ms) {
    prepare_kernels(c);
    vofp_status s = ensure_workspace(c);
    if (s) return s;
    const cudaStream_t home = c->stream;
    cudaStream_t st = home;   // the stream the bodies launch on (the capture stream while capturing)
    const long long N = c->d.n;
    cudaEvent_t a, b2;
    cudaStream_t cs = nullptr;
    VOFP_CUDA_TRY(c, cudaEventCreate(&a));
    VOFP_CUDA_TRY(c, cudaEventCreate(&b2));
    VOFP_CUDA_TRY(c, cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    float t1 = 0.0f, t2 = 0.0f, t3 = 0.0f;
    // `reps` launches of a body captured into one graph and timed with events on the context
    // stream: device time without the host's per-launch cost
    auto timed = [&](auto&& body, float* out) -> vofp_status {
        // alpha = beta = 0 keeps every value fixed while every byte is still read and written
        launch(c, k_set_pq_inf, 1, 1, home, c->sc, 1);
        body();   // warm-up launch
        cudaError_t e = cudaStreamSynchronize(home);
        cudaGraph_t g = nullptr;
        cudaGraphExec_t ge = nullptr;
        if (e == cudaSuccess) e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeRelaxed);
        if (e == cudaSuccess) {
            const long long before = c->launches;
            st = cs;
            for (int i = 0; i < reps; ++i) body();
            st = home;
            e = cudaStreamEndCapture(cs, &g);
            c->launches += c->launches - before;   // the graph runs twice
        }
        if (e == cudaSuccess) e = cudaGraphInstantiate(&ge, g, 0);
        if (e == cudaSuccess) e = cudaGraphLaunch(ge, home);
        if (e == cudaSuccess) e = cudaEventRecord(a, home);
        if (e == cudaSuccess) e = cudaGraphLaunch(ge, home);
        if (e == cudaSuccess) e = cudaEventRecord(b2, home);
        if (e == cudaSuccess) e = cudaEventSynchronize(b2);
        if (e == cudaSuccess) e = cudaEventElapsedTime(out, a, b2);
        if (ge) cudaGraphExecDestroy(ge);
        if (g) cudaGraphDestroy(g);
        if (e != cudaSuccess) {
            c->set_error(std::string("timing graph: ") + cudaGetErrorString(e));
            return VOFP_ERR_CUDA;
        }
        *out /= reps;
        return VOFP_OK;
    };
    const uint32_t* bits = rb ? c->excl_bits : c->slave_bits;
    if (precision == 32 && rb && (s = rbc_ensure(c))) return s;
    if (precision == 32 && rb && c->rbc_ok) {
        // the colour-compact red-black iteration kernel and the update on the compact vectors
        const long long nc = c->rbc_nh + c->rbc_ne;
        auto stn = [&]() { rbc_time_kernel(c, st); };
        auto upd = [&]() {
            launch(c, k_cg_update<float, false>, stream_grid(nc / 4 + 1), kNT, st, nc, c->rbc_r,
                   (const float*)c->rbc_q, (const uint32_t*)c->rbc_bits, c->sc, c->partials, c->counters,
                   (cudaGraphConditionalHandle)0, 0, (const double*)nullptr, 0);
        };
        auto aux = [&]() { rbc_time_aux(c, st); };
        if ((s = timed(stn, &t1)) || (s = timed(upd, &t2)) || (s = timed(aux, &t3))) return s;
    } else if (precision == 32) {
        auto stn = [&]() {
            if (rb)
                launch_cg_rb<float>(c, st, c->Txf, c->Tyf, c->Tzf, c->rf, c->pf0, c->pf1, c->xf, c->qf);
            else
                launch_cg_stencil<float>(c, st, c->Txf, c->Tyf, c->Tzf, c->rf, c->pf0, c->pf1, c->xf, c->qf);
        };
        auto upd = [&]() {
            launch(c, k_cg_update<float, false>, stream_grid(N / 4 + 1), kNT, st, N, c->rf, (const float*)c->qf, bits,
                   c->sc, c->partials, c->counters, (cudaGraphConditionalHandle)0, 0, (const double*)nullptr, 0);
        };
        if ((s = timed(stn, &t1)) || (s = timed(upd, &t2))) return s;
    } else {
        auto stn = [&]() {
            if (rb)
                launch_cg_rb<double>(c, st, c->Txs, c->Tys, c->Tzs, c->r, c->p0, c->p1, c->xt, c->q);
            else
                launch_cg_stencil<double>(c, st, c->Txs, c->Tys, c->Tzs, c->r, c->p0, c->p1, c->xt, c->q);
        };
        auto upd = [&]() {
            launch(c, k_cg_update<double, false>, stream_grid(N / 2 + 1), kNT, st, N, c->r, (const double*)c->q, bits,
                   c->sc, c->partials, c->counters, (cudaGraphConditionalHandle)0, 0, (const double*)nullptr, 0);
        };
        if ((s = timed(stn, &t1)) || (s = timed(upd, &t2))) return s;
    }
    launch(c, k_set_pq_inf, 1, 1, home, c->sc, 0);
    VOFP_CUDA_TRY(c, cudaStreamSynchronize(home));
    cudaEventDestroy(a);
    cudaEventDestroy(b2);
    cudaStreamDestroy(cs);
    *stencil_ms = t1;
    *update_ms = t2;
    *aux_ms = t3;
    return VOFP_OK;
}

}  // namespace vofp
