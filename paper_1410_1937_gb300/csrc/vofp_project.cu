// Projection of the face velocities onto the discretely divergence-free field (Sec. 2.1, Eq. runge1:
// u = u* - dt (1/rho) grad p) and the check of that property: the net outward flux of every merge
// group (Sec. 2.3, the integral form over open faces) of the projected field.
//
// The face gradient uses the operator's own face coefficient reading: (p_R - p_L) over the
// half-cell resistance sum (d_L rho_L + d_R rho_R) / 2 (its inverse kept per face from the
// assembly, so the projection needs no division), so the projected fluxes satisfy the discrete
// pressure equation row by row and every group's net flux is the solver's residual.
#include <algorithm>
#include <cstring>

#include "vofp_internal.cuh"

namespace vofp {
namespace {

constexpr int kNT = 256;

struct Walls {
    int kind[6];               // VOFP_BC_* per domain face, order -x,+x,-y,+y,-z,+z
    const double* g[6];        // prescribed outward (1/rho) dp/dn on Neumann faces (or null)
};

int grid_cells(long long n) {
    long long b = (n + kNT - 1) / kNT;
    return int(std::max(1LL, std::min(b, (long long)num_sms() * 16)));
}

// u_new on an interior face between cells L and R with inverse resistance kap (0 on a closed face,
// which keeps its velocity: the pressure gradient drives no flux through it)
__device__ __forceinline__ double interior(double u, double kap, double dt, double pL, double pR) {
    return u - dt * ((pR - pL) * kap);
}
// u_new on a domain face next to cell c; `sgn` = +1 on a + face, -1 on a - face
__device__ __forceinline__ double wall(double u, double a, double dt, int kind, const double* g, long long gi,
                                       int sgn, double pc, double dc, double rc) {
    if (kind == VOFP_BC_DIRICHLET) return a > 0.0 ? u - dt * (sgn * (0.0 - pc) / (0.5 * dc * rc)) : u;
    return g ? -sgn * dt * g[gi] : 0.0;
}

// Each thread owns one cell and writes its -x, -y, -z faces, plus the + domain faces of the last
// cell of each line; a face is read and written by the same thread, so the output may alias u, v, w.
__global__ void k_project(Dims d, Walls wl, double dt, const double* __restrict__ dx, const double* __restrict__ dy,
                          const double* __restrict__ dz, const double* __restrict__ rho,
                          const double* __restrict__ axe, const double* __restrict__ aye,
                          const double* __restrict__ aze, const double* __restrict__ kx,
                          const double* __restrict__ ky, const double* __restrict__ kz, const double* __restrict__ p,
                          const double* u, const double* v, const double* w, double* uo, double* vo, double* wo) {
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < d.n;
         c += (long long)gridDim.x * blockDim.x) {
        int i, j, k;
        cell_ijk(d, c, i, j, k);
        const double pc = p[c];
        long long f = fx_idx(d, i, j, k);
        uo[f] = i > 0 ? interior(u[f], kx[c - 1], dt, p[c - 1], pc)
                      : wall(u[f], axe[f], dt, wl.kind[0], wl.g[0], j + (long long)d.ny * k, -1, pc, dx[i], rho[c]);
        if (i == d.nx - 1) {
            f = fx_idx(d, i + 1, j, k);
            uo[f] = wall(u[f], axe[f], dt, wl.kind[1], wl.g[1], j + (long long)d.ny * k, +1, pc, dx[i], rho[c]);
        }
        f = fy_idx(d, i, j, k);
        vo[f] = j > 0 ? interior(v[f], ky[c - d.nx], dt, p[c - d.nx], pc)
                      : wall(v[f], aye[f], dt, wl.kind[2], wl.g[2], i + (long long)d.nx * k, -1, pc, dy[j], rho[c]);
        if (j == d.ny - 1) {
            f = fy_idx(d, i, j + 1, k);
            vo[f] = wall(v[f], aye[f], dt, wl.kind[3], wl.g[3], i + (long long)d.nx * k, +1, pc, dy[j], rho[c]);
        }
        f = fz_idx(d, i, j, k);
        wo[f] = k > 0 ? interior(w[f], kz[c - d.plane], dt, p[c - d.plane], pc)
                      : wall(w[f], aze[f], dt, wl.kind[4], wl.g[4], i + (long long)d.nx * j, -1, pc, dz[k], rho[c]);
        if (k == d.nz - 1) {
            f = fz_idx(d, i, j, k + 1);
            wo[f] = wall(w[f], aze[f], dt, wl.kind[5], wl.g[5], i + (long long)d.nx * j, +1, pc, dz[k], rho[c]);
        }
    }
}

// net outward flux of each cell through its open faces (+ body-surface flux), 0 without unknown
__global__ void k_divergence(Dims d, const double* __restrict__ dx, const double* __restrict__ dy,
                             const double* __restrict__ dz, const double* __restrict__ axe,
                             const double* __restrict__ aye, const double* __restrict__ aze,
                             const uint8_t* __restrict__ ina, const double* __restrict__ u,
                             const double* __restrict__ v, const double* __restrict__ w,
                             const double* __restrict__ body, double* __restrict__ div) {
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < d.n;
         c += (long long)gridDim.x * blockDim.x) {
        if (ina[c]) {
            div[c] = 0.0;
            continue;
        }
        int i, j, k;
        cell_ijk(d, c, i, j, k);
        const double Sx = dz[k] * dy[j], Sy = dz[k] * dx[i], Sz = dy[j] * dx[i];
        long long f = fx_idx(d, i, j, k);
        const double fxm = axe[f] * Sx * u[f], fxp = axe[f + 1] * Sx * u[f + 1];
        f = fy_idx(d, i, j, k);
        const double fym = aye[f] * Sy * v[f], fyp = aye[f + d.nx] * Sy * v[f + d.nx];
        f = fz_idx(d, i, j, k);
        const double fzm = aze[f] * Sz * w[f], fzp = aze[f + d.plane] * Sz * w[f + d.plane];
        double s = ((fxp - fxm) + (fyp - fym)) + (fzp - fzm);
        if (body) s += body[c];
        div[c] = s;
    }
}

// max |div| over cells into *out (non-negative doubles order like their bit patterns)
__global__ void k_max_abs(long long n, const double* __restrict__ div, unsigned long long* out) {
    double m = 0.0;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x)
        m = fmax(m, fabs(div[c]));
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(out, (unsigned long long)__double_as_longlong(m));
}

}  // namespace

vofp_status project(vofp_ctx* c, const double* p, const double* u, const double* v, const double* w,
                    const double* body, double* uo, double* vo, double* wo, double* div, double* max_div) {
    const Dims d = c->d;
    cudaStream_t st = c->stream;
    Walls wl{};
    for (int f = 0; f < 6; ++f) {
        wl.kind[f] = c->bc[f];
        wl.g[f] = c->has_nflux[f] ? c->nflux[f] : nullptr;
    }
    const int g = grid_cells(d.n);
    launch(c, k_project, g, kNT, st, d, wl, c->phys.dt, (const double*)c->dx, (const double*)c->dy,
           (const double*)c->dz, (const double*)c->rho, (const double*)c->axe, (const double*)c->aye,
           (const double*)c->aze, (const double*)c->kx, (const double*)c->ky, (const double*)c->kz, p, u, v, w, uo, vo,
           wo);
    if (div || max_div) {
        double* dv = div ? div : c->work;
        launch(c, k_divergence, g, kNT, st, d, (const double*)c->dx, (const double*)c->dy, (const double*)c->dz,
               (const double*)c->axe, (const double*)c->aye, (const double*)c->aze, (const uint8_t*)c->inactive,
               (const double*)uo, (const double*)vo, (const double*)wo, body, dv);
        launch_group_fold(c, dv, true);
        if (max_div) {
            unsigned long long* m = reinterpret_cast<unsigned long long*>(c->counters + 40);
            VOFP_CUDA_TRY(c, cudaMemsetAsync(m, 0, sizeof(*m), st));
            launch(c, k_max_abs, g, kNT, st, d.n, (const double*)dv, m);
            unsigned long long h = 0;
            VOFP_CUDA_TRY(c, cudaMemcpyAsync(&h, m, sizeof(h), cudaMemcpyDeviceToHost, st));
            VOFP_CUDA_TRY(c, cudaStreamSynchronize(st));
            double r;
            static_assert(sizeof(r) == sizeof(h), "64-bit");
            std::memcpy(&r, &h, sizeof(r));
            *max_div = r;
        }
    }
    VOFP_CUDA_TRY(c, cudaGetLastError());
    return VOFP_OK;
}

}  // namespace vofp
