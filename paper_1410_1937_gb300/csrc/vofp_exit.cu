// Exit flux of the radiation condition (Sec. 2.6): the x-momentum balance at the exit with the
// Orlanski-type condition du/dt + u_c du/dx = 0 (Eq. orlanski) gives the Neumann datum
// (1/rho) dp/dx = u_c du/dx + R (Eq. exit) on the +x domain face.
//
// Per exit face (row j, k of the +x face, index j + ny k):
//   g = u_c (u_nx - u_{nx-1}) / dx_{nx-1} + R - u_nx / dt
// du/dx is the one-sided difference of the x-face velocities across the last cell.  The term
// -u_nx / dt carries the face's own predicted velocity: the library drops normal velocities on
// free-slip faces from the divergence and sets the projected velocity on a + face to -dt g, so
// with this g the projected exit velocity is u_nx - dt (u_c du/dx + R), the discrete Orlanski
// update with the momentum balance of Eq. exit.
//
// Balance (optional): the radiation condition does not conserve mass by itself (Sec. 2.6), and an
// all-Neumann pressure problem needs sum(b_hat) = 0.  The imbalance I = sum over cells of b with
// the exit flux in place is removed by a uniform shift of g over the open exit area
// (g -= I / sum A_f S_f), the smallest change of the exit flux that makes the problem compatible.
#include "vofp_internal.cuh"
#include "vofp_kernels.cuh"

namespace vofp {
namespace {

constexpr int kNT = 256;

__global__ void k_exit_flux(Dims d, double uc, double dt, const double* __restrict__ dx,
                            const double* __restrict__ u, const double* __restrict__ r1, double* __restrict__ g) {
    const long long rows = (long long)d.ny * d.nz;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < rows; t += (long long)gridDim.x * blockDim.x) {
        const long long f = (long long)(d.nx + 1) * t;   // first x-face of row t
        const double ue = u[f + d.nx], uu = u[f + d.nx - 1];
        const double grad = (ue - uu) / dx[d.nx - 1];
        g[t] = fma(uc, grad, r1 ? r1[t] : 0.0) - ue / dt;
    }
}

// sum of b over the cells, and the open exit area sum A_f S_f over the +x face
__global__ void __launch_bounds__(kNT)
k_exit_sums(Dims d, const double* __restrict__ b, const double* __restrict__ axe, const double* __restrict__ dy,
            const double* __restrict__ dz, double* __restrict__ partials, unsigned int* __restrict__ counter,
            double* out2) {
    __shared__ double sh[32];
    double s = 0.0, a = 0.0;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < d.n; c += stride) s += b[c];
    const long long rows = (long long)d.ny * d.nz;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < rows; t += stride) {
        const int j = int(t % d.ny), k = int(t / d.ny);
        a = fma(axe[(long long)(d.nx + 1) * t + d.nx], dy[j] * dz[k], a);
    }
    double tot;
    if (grid_reduce(s, partials, counter, sh, &tot)) out2[0] = tot;
    __syncthreads();
    if (grid_reduce(a, partials + kMaxPartials / 4, counter + 1, sh, &tot)) out2[1] = tot;
}

// g -= I / area on the open exit faces
__global__ void k_exit_shift(Dims d, const double* __restrict__ axe, const double* __restrict__ sums,
                             double* __restrict__ g) {
    const double area = sums[1];
    if (!(area > 0.0)) return;
    const double shift = sums[0] / area;
    const long long rows = (long long)d.ny * d.nz;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < rows; t += (long long)gridDim.x * blockDim.x)
        if (axe[(long long)(d.nx + 1) * t + d.nx] > 0.0) g[t] -= shift;
}

int grid_rows(long long rows) {
    return (int)std::max(1LL, std::min((rows + kNT - 1) / kNT, (long long)num_sms() * 8));
}

}  // namespace

vofp_status exit_flux(vofp_ctx* c, const double* u, const double* v, const double* w, const double* body, double uc,
                      const double* r1, int balance, double* g_out, double* shift_out) {
    const Dims d = c->d;
    cudaStream_t st = c->stream;
    const long long rows = (long long)d.ny * d.nz;
    vofp_status s;
    if (!c->nflux[1] && (s = c->alloc(&c->nflux[1], rows))) return s;
    double* g = c->nflux[1];
    launch(c, k_exit_flux, grid_rows(rows), kNT, st, d, uc, c->phys.dt, (const double*)c->dx, u, r1, g);
    c->has_nflux[1] = true;
    double sums[2] = {0.0, 0.0};
    if (balance) {
        // b with the raw exit flux in place, then the uniform shift over the open exit area
        if ((s = rhs(c, u, v, w, body, c->work))) return s;
        double* d2 = c->partials + kMaxPartials - 16;
        launch(c, k_exit_sums, grid_rows(d.n), kNT, st, d, (const double*)c->work, (const double*)c->axe,
               (const double*)c->dy, (const double*)c->dz, c->partials, c->counters, d2);
        launch(c, k_exit_shift, grid_rows(rows), kNT, st, d, (const double*)c->axe, (const double*)d2, g);
        VOFP_CUDA_TRY(c, cudaMemcpyAsync(sums, d2, sizeof(sums), cudaMemcpyDeviceToHost, st));
    }
    if (g_out) VOFP_CUDA_TRY(c, cudaMemcpyAsync(g_out, g, sizeof(double) * rows, cudaMemcpyDeviceToDevice, st));
    VOFP_CUDA_TRY(c, cudaStreamSynchronize(st));
    if (shift_out) *shift_out = (balance && sums[1] > 0.0) ? sums[0] / sums[1] : 0.0;
    return VOFP_OK;
}

}  // namespace vofp
